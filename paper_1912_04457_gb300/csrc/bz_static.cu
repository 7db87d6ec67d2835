// bz_collision_term_static: the FP64 collision increment without any
// allocation, for callers that cannot call cudaMalloc (for example code
// running inside another runtime's memory pool, or a plug-in that may only
// use the buffers its host hands it).  The scratch the regular path keeps
// in a handle -- f of the state, the mass accumulators and the counters --
// lives here in file-scope device arrays of fixed size, which every GPU that
// loads the library holds until the process exits.  The kernels are the
// same ones bz_collision_term launches, given these arrays' addresses.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/bz.h"
#include "bz_internal.h"

using namespace bz;

namespace {

constexpr int MAX_DEVICES = 64;

// The shared scratch.  Every call reuses it and it keeps the last call's
// contents; the accumulators and counters are cleared at the start of each
// call and f is overwritten completely.  Calls that overlap on the GPU race.
static __device__ __align__(256) double s_f[BZ_STATIC_MAX_CELLS];
static __device__ __align__(256) long long s_acc[BZ_STATIC_MAX_XCELLS * 4];
static __device__ __align__(256) long long s_flags[4];

struct DevScratch {
    bool ready = false;
    double* f = nullptr;
    long long* acc = nullptr;
    long long* flags = nullptr;
    int nsm = 0;
};
DevScratch g_dev[MAX_DEVICES];
std::mutex g_mu;

int err(char* buf, int len, int code, const char* fmt, ...)
{
    if (buf && len > 0) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, (size_t)len, fmt, ap);
        va_end(ap);
    }
    return code;
}

// Host-side names of the arrays are stand-ins, not device addresses; the
// device addresses come from cudaGetSymbolAddress with the device current.
int setup_device(int dev, DevScratch** out, char* eb, int el)
{
    std::lock_guard<std::mutex> lock(g_mu);
    DevScratch& d = g_dev[dev];
    if (!d.ready) {
        cudaError_t e;
        if ((e = cudaGetSymbolAddress(reinterpret_cast<void**>(&d.f), s_f)) != cudaSuccess ||
            (e = cudaGetSymbolAddress(reinterpret_cast<void**>(&d.acc), s_acc)) != cudaSuccess ||
            (e = cudaGetSymbolAddress(reinterpret_cast<void**>(&d.flags), s_flags)) != cudaSuccess)
            return err(eb, el, BZ_ECUDA, "cudaGetSymbolAddress failed on device %d: %s", dev, cudaGetErrorString(e));
        if ((e = cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return err(eb, el, BZ_ECUDA, "cannot query device %d: %s", dev, cudaGetErrorString(e));
        d.ready = true;
    }
    *out = &d;
    return BZ_OK;
}

// Terms of species d's equation (Eqs. C_gluon, C_quark; antiquarks by charge
// conjugation), legs (k1, k2, k3, p) with (k1, k3) the like-species line --
// the same table the handle path builds.
void terms_of(uint32_t mask, const int* slot_of, TermDev (*terms)[MAX_TERMS], int* nterms)
{
    for (int d = 0; d < NSPEC; ++d) {
        int leg[16][4], cls[16], n = 0;
        double sym[16];
        auto add = [&](int a, int b, int c, int dd, double sy, int cl) {
            leg[n][0] = a; leg[n][1] = b; leg[n][2] = c; leg[n][3] = dd;
            sym[n] = sy; cls[n] = cl; ++n;
        };
        if (d == 0) {
            add(0, 0, 0, 0, 0.5, M_GG);
            for (int f = 0; f < 3; ++f) {
                add(1 + f, 0, 1 + f, 0, 1.0, M_QG);
                add(4 + f, 0, 4 + f, 0, 1.0, M_QG);
                add(1 + f, 4 + f, 0, 0, 1.0, M_QQBGG);
            }
        } else {
            const bool anti = d >= 4;
            const int fa = (d - 1) % 3;
            const int me = anti ? 4 + fa : 1 + fa, bar = anti ? 1 + fa : 4 + fa;
            add(me, me, me, me, 0.5, M_QQ);
            add(bar, me, bar, me, 1.0, M_QQB);
            add(0, 0, bar, me, 0.5, M_QQBGG);
            add(0, me, 0, me, 1.0, M_QG);
            for (int fb = 0; fb < 3; ++fb) {
                if (fb == fa) continue;
                const int Qb = anti ? 4 + fb : 1 + fb, QBb = anti ? 1 + fb : 4 + fb;
                add(Qb, me, Qb, me, 1.0, M_QQP);
                add(QBb, me, QBb, me, 1.0, M_QQP);
                add(Qb, QBb, bar, me, 1.0, M_QQB2);
            }
        }
        int m = 0;
        for (int i = 0; i < n; ++i) {
            bool ok = true;
            for (int l = 0; l < 4; ++l) ok = ok && (mask & (1u << leg[i][l]));
            if (!ok) continue;
            TermDev& o = terms[d][m++];
            for (int l = 0; l < 4; ++l) {
                o.slot[l] = (int8_t)slot_of[leg[i][l]];
                o.mslot[l] = (int8_t)mass_slot(leg[i][l]);
                o.quark[l] = (int8_t)(is_quark(leg[i][l]) ? 1 : 0);
            }
            o.cls = (int8_t)cls[i];
            o.sym = sym[i];
        }
        nterms[d] = m;
    }
}

}  // namespace

#define CKS(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return err(errbuf, errbuf_len, BZ_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" int bz_collision_term_static(const bz_grid* g, uint32_t species_mask, double alpha_s, int32_t mass_mode,
                                        const int64_t* state, const double* m2_in, double* m2_out, int64_t* A,
                                        int32_t nsamples, int32_t step, double dt, void* stream, char* errbuf,
                                        int32_t errbuf_len)
{
    if (!g || !state || !A || !m2_out) return err(errbuf, errbuf_len, BZ_EINVAL, "null argument");
    for (int d = 0; d < 3; ++d) {
        if (g->nx[d] <= 0 || g->np[d] <= 0) return err(errbuf, errbuf_len, BZ_EINVAL, "grid sizes must be positive");
        if (g->np[d] > MAX_NP) return err(errbuf, errbuf_len, BZ_EINVAL, "np[%d] = %d exceeds %d", d, g->np[d], MAX_NP);
    }
    if (!(g->L > 0) || !(g->dx > 0)) return err(errbuf, errbuf_len, BZ_EINVAL, "L and dx must be positive");
    if (np_has_zero_cell(g->np))
        return err(errbuf, errbuf_len, BZ_EINVAL, "np odd along all axes puts a cell at p = 0 (E = 0)");
    if ((species_mask & 0x7Fu) == 0 || (species_mask & ~0x7Fu))
        return err(errbuf, errbuf_len, BZ_EINVAL, "bad species mask 0x%x", species_mask);
    if (!(alpha_s > 0)) return err(errbuf, errbuf_len, BZ_EINVAL, "alpha_s must be positive");
    if (mass_mode < 0 || mass_mode > 2) return err(errbuf, errbuf_len, BZ_EINVAL, "bad mass mode %d", mass_mode);
    if (mass_mode == BZ_MASS_FIXED && !m2_in)
        return err(errbuf, errbuf_len, BZ_EINVAL, "mass mode FIXED needs the masses in m2_in");
    if (nsamples <= 0 || nsamples > MAX_SAMPLES)
        return err(errbuf, errbuf_len, BZ_EINVAL, "nsamples must be in [1, 2^20]");
    if (step < 0 || step >= (1 << 29)) return err(errbuf, errbuf_len, BZ_EINVAL, "step must be in [0, 2^29)");
    if (!(dt > 0)) return err(errbuf, errbuf_len, BZ_EINVAL, "dt must be positive");

    int slot_of[NSPEC], slot_species[NSPEC] = {0}, nslots = 0;
    for (int s = 0; s < NSPEC; ++s) {
        slot_of[s] = (species_mask & (1u << s)) ? nslots : -1;
        if (slot_of[s] >= 0) slot_species[nslots++] = s;
    }
    const int64_t nxc = (int64_t)g->nx[0] * g->nx[1] * g->nx[2];
    const int64_t npc = (int64_t)g->np[0] * g->np[1] * g->np[2];
    const int64_t ncell = (int64_t)nslots * nxc * npc;
    if (ncell > BZ_STATIC_MAX_CELLS)
        return err(errbuf, errbuf_len, BZ_EINVAL,
                   "%lld cells (species x x-cells x p-cells) exceed the static scratch of %d cells",
                   (long long)ncell, BZ_STATIC_MAX_CELLS);
    if (nxc > BZ_STATIC_MAX_XCELLS)
        return err(errbuf, errbuf_len, BZ_EINVAL, "%lld x cells exceed the static maximum of %d", (long long)nxc,
                   BZ_STATIC_MAX_XCELLS);

    int dev = 0;
    CKS(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return err(errbuf, errbuf_len, BZ_ENODEV, "device ordinal %d out of range", dev);
    DevScratch* sc = nullptr;
    int rc = setup_device(dev, &sc, errbuf, errbuf_len);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CKS(cudaMemsetAsync(sc->flags, 0, sizeof(long long) * 4, s));

    const double dF = 3.0, CA = 3.0, CF = 4.0 / 3.0, dA = 8.0;
    const double g2 = 4.0 * PI * alpha_s;
    const double g4 = g2 * g2;
    const double twoL = 2.0 * g->L;
    const double twopi = 2.0 * PI;

    // 1. thermal masses, Eqs. (mg), (mq), into m2_out (mass mode FIXED: copy m2_in)
    if (mass_mode == BZ_MASS_FIXED) {
        if (m2_out != m2_in)
            CKS(cudaMemcpyAsync(m2_out, m2_in, sizeof(double) * 4 * nxc, cudaMemcpyDeviceToDevice, s));
    } else {
        MassArgs ma{};
        ma.state = reinterpret_cast<const long long*>(state);
        ma.acc = sc->acc;
        ma.m2_out = m2_out;
        ma.m2_prev = mass_mode == BZ_MASS_MASSLESS ? nullptr : m2_in;
        ma.flags = sc->flags;
        ma.nxc = nxc;
        ma.npc = npc;
        double dpx = 2.0 * g->L / g->np[0], dpy = 2.0 * g->L / g->np[1], dpz = 2.0 * g->L / g->np[2];
        for (int d = 0; d < 3; ++d) ma.np[d] = g->np[d];
        ma.L = g->L;
        ma.dp[0] = dpx;
        ma.dp[1] = dpy;
        ma.dp[2] = dpz;
        for (int q = 0; q < NSPEC; ++q) ma.slot_of[q] = slot_of[q];
        ma.pref_g = 2.0 * g2 / dA;
        ma.pref_q = 2.0 * CF * g2;
        ma.meas = dpx * dpy * dpz / (twopi * twopi * twopi);
        ma.limit = INT64_MAX / npc / 2;
        CKS(launch_masses(ma, s));  // clears the accumulators first
    }

    // 2. f of the state for the lookups (FP64: f = n 2^-40 / N_s)
    double deg[NSPEC];
    for (int sl = 0; sl < NSPEC; ++sl) deg[sl] = slot_species[sl] == 0 ? 16.0 : 6.0;
    CKS(launch_convert(reinterpret_cast<const long long*>(state), sc->f, 1, nxc, npc, nslots, deg, s));

    // 3. collision sampling and symmetric int64 deposition, FP64 integrand
    CKS(cudaMemsetAsync(A, 0, sizeof(int64_t) * ncell, s));
    CollideArgs<double> a{};
    a.f = sc->f;
    a.f_is_float = 0;
    a.ubits = 32;
    a.A = reinterpret_cast<long long*>(A);
    a.m2 = m2_out;
    a.flags = sc->flags;
    a.nxc = nxc;
    a.npc = npc;
    a.ncell = ncell;
    for (int d = 0; d < 3; ++d) {
        a.np[d] = g->np[d];
        a.dp[d] = twoL / g->np[d];
    }
    a.L = g->L;
    a.twoL = twoL;
    a.key0 = (uint32_t)(g->seed & 0xffffffffu) ^ g->box;
    a.key1 = (uint32_t)(g->seed >> 32);
    philox_key_schedule(a.key0, a.key1, a.ks);
    a.nsamples = nsamples;
    a.step = step;
    a.n_sel = ncell;
    a.a_stride = 1;
    a.a_offset = 0;
    a.sampler = BZ_SAMPLER_SYMMETRIC;
    a.mass_mode = mass_mode;
    a.analytic = 0;
    a.p_center = 0;
    a.T = 0.5;
    const double V = twoL * twoL * twoL * twoL * twoL;
    const double Kq = ((V * dt) / (4.0 * (double)nsamples)) / HBARC * TWO_POW_40;
    a.Kq = Kq;
    a.Kown = Kq;
    a.twopi5 = twopi * twopi * twopi * twopi * twopi;
    a.A1 = 8.0 * g4 * dF * dF * CF * CF / dA;
    a.A2 = 16.0 * g4 * dF * CF * (CF - CA / 2.0);
    a.A3 = 8.0 * g4 * dF * CF * CF;
    a.A4 = 8.0 * g4 * dF * CF * CA;
    a.A5 = 16.0 * g4 * dA * CA * CA;
    for (int q = 0; q < NSPEC; ++q) a.slot_species[q] = slot_species[q];
    terms_of(species_mask, slot_of, a.terms, a.nterms);
    const int64_t total = ncell * (int64_t)nsamples;
    int64_t blocks = (total + 255) / 256;
    if (blocks > (int64_t)sc->nsm * 8) blocks = (int64_t)sc->nsm * 8;
    if (blocks < 1) blocks = 1;
    CKS(launch_collide_f64(a, (int)blocks, s));
    return BZ_OK;
}
