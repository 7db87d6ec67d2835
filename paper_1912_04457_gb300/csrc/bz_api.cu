// C ABI of libbz (declared in include/bz.h): handle management, argument
// checks, and the per-step orchestration of the kernels on the caller's
// stream.  Host arithmetic that feeds bit-exact paths (grid spacings,
// weights, |M|^2 prefactors) is written in the same operation order as the
// formula it implements.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/bz.h"
#include "bz_internal.h"

using namespace bz;

struct bz_handle_s {
    bz_grid g{};
    int device = 0;
    int nsm = 0;
    uint32_t mask = 1;
    double alpha_s = 0.3;
    int mass_mode = BZ_MASS_THERMAL;
    int nslots = 1;
    int slot_species[NSPEC] = {0};
    int slot_of[NSPEC] = {0, -1, -1, -1, -1, -1, -1};
    int64_t nxc = 0, npc = 0, ncell = 0;
    double* d_m2[2] = {nullptr, nullptr};
    int cur = 0;
    bool have_masses = false;
    long long* d_acc = nullptr;
    long long* d_flags = nullptr;
    void* d_freal = nullptr;       // f of the state, double-sized
    int* d_jtab = nullptr;         // packed (jx, jy, jz) of every p cell
    double* d_ppu = nullptr;       // thermal masses: the distinct p^2 of the cell centres
    unsigned short* d_pidx = nullptr;  // and each p cell's index into them
    int nu = 0;                    // their count (0: no table)
    float* d_inv_e = nullptr;      // drift scratch: 1/E of every cell (inhomogeneous grids)
    float* d_gforce = nullptr;     // force-term scratch: g_i per (x cell, mass slot, axis)
    float* d_m2f = nullptr;        // drift scratch: FP32 m^2 per (x cell, mass slot)
    unsigned long long* d_counter = nullptr;  // FP32 collision: units handed out
    double* d_m2prev = nullptr;    // energy source: the caller's previous masses [x][4]
    long long* d_mom_part = nullptr;  // moments: exact partial sums of the p-cell chunks
    int64_t mom_part_cap = 0;
    bool force = false;            // the drift includes the force term -div_p[(grad_x E) f]
    int param = 0;                 // FP64 collision: 0 k2 eliminated, 1 k3 eliminated
    UserRow h_urows[MSQ_ROWS] = {};  // user-defined |M|^2 rows (host copy)
    uint32_t umask = 0;
    UserRow* d_urows = nullptr;
    double* d_audit = nullptr;     // bz_collision_audit sums (8)
    long long* d_sflags = nullptr; // state warnings (2): f < 0 cells, fermion f > 1 cells
    int f64_ubits = 32;            // uniform resolution of the FP64 path (32 or 23 bits)
    bool audit_on = false;
    long long* d_state2 = nullptr; // second state buffer for bz_step
    int* d_qcount = nullptr;       // FP32 deferral queue: per-warp counts
    unsigned long long* d_qitems = nullptr;
    int64_t q_warps = 0, q_items = 0;
    // learned proposal: FP32 master parameters, Adam moments, gradient, per-anchor parameters
    float *d_prop = nullptr, *d_prop_g = nullptr, *d_prop_m = nullptr, *d_prop_v = nullptr;
    float* d_anchor_prm = nullptr;
    float* d_loss = nullptr;
    double* d_wsum = nullptr;          // [sum_weights_scratch()]: the sum, then the per-warp partial sums
    float* d_prop_part = nullptr;      // per-block gradients [4 nsm][nparam] and losses [4 nsm]
    float* d_loss_part = nullptr;
    int* d_prop_err = nullptr;         // tensor-core waits that timed out in the network's kernels
    int adam_step = 0;
    bool anchor_prm_ready = false;
    int step_sampler = BZ_SAMPLER_SYMMETRIC;
    unsigned long long* d_rec_count = nullptr;
    // opt-in per-kernel timing: event pairs recorded around each launch
    bool prof = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_pending;
    std::vector<cudaEvent_t> prof_free;
    double prof_ms[BZ_NKERNELS] = {0};
    int64_t prof_n[BZ_NKERNELS] = {0};
    int analytic = 0;
    double T = 0.5;
    double mu[NSPEC] = {0};
    int64_t a_stride = 1, a_offset = 0;
    // replayed step loop (FP32): two steps captured as one CUDA graph, the step
    // index and moments slot in device memory; every setter bumps gen, which
    // retires the graph
    unsigned gen = 0;
    int* d_step_idx = nullptr;     // [2]: step index, moments slot
    cudaStream_t cap_stream = nullptr;
    struct StepGraph {               // one per parity of the current mass buffer
        cudaGraphExec_t exec = nullptr;
        const long long* cur = nullptr;
        const double* mom = nullptr;
        double dt = 0;
        int nsamples = 0, sampler = 0;
        unsigned gen = 0;
    } sg[2];
    std::string err;
};

static std::string g_init_error;

static int fail(bz_handle h, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_init_error = buf;
    return code;
}

#define CK(h, call)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail((h), BZ_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

// Timing scope around one launch (no-op unless profiling is enabled).
struct ProfScope {
    bz_handle h;
    int id;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ProfScope(bz_handle h_, int id_, cudaStream_t s_) : h(h_), id(id_), s(s_)
    {
        if (!h->prof) return;
        e0 = take();
        e1 = take();
        cudaEventRecord(e0, s);
    }
    cudaEvent_t take()
    {
        cudaEvent_t e;
        if (!h->prof_free.empty()) {
            e = h->prof_free.back();
            h->prof_free.pop_back();
        } else {
            cudaEventCreate(&e);
        }
        return e;
    }
    ~ProfScope()
    {
        if (!h->prof) return;
        cudaEventRecord(e1, s);
        h->prof_pending.push_back({id, {e0, e1}});
    }
};

static void prof_drain(bz_handle h)
{
    for (auto& p : h->prof_pending) {
        float ms = 0;
        cudaEventSynchronize(p.second.second);
        cudaEventElapsedTime(&ms, p.second.first, p.second.second);
        h->prof_ms[p.first] += ms;
        h->prof_n[p.first] += 1;
        h->prof_free.push_back(p.second.first);
        h->prof_free.push_back(p.second.second);
    }
    h->prof_pending.clear();
}

template <typename T>
static bool dalloc(T** p, size_t n)
{
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (n ? n : 1)) == cudaSuccess;
}

static void drop_step_graph(bz_handle h, int parity)
{
    if (h->sg[parity].exec) cudaGraphExecDestroy(h->sg[parity].exec);
    h->sg[parity].exec = nullptr;
}

static void free_scratch(bz_handle h)
{
    drop_step_graph(h, 0);
    drop_step_graph(h, 1);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
    cudaFree(h->d_step_idx);
    h->d_step_idx = nullptr;
    cudaFree(h->d_m2[0]);
    cudaFree(h->d_m2[1]);
    cudaFree(h->d_acc);
    cudaFree(h->d_flags);
    cudaFree(h->d_freal);
    cudaFree(h->d_jtab);
    h->d_jtab = nullptr;
    cudaFree(h->d_ppu);
    h->d_ppu = nullptr;
    cudaFree(h->d_pidx);
    h->d_pidx = nullptr;
    h->nu = 0;
    cudaFree(h->d_inv_e);
    h->d_inv_e = nullptr;
    cudaFree(h->d_gforce);
    h->d_gforce = nullptr;
    cudaFree(h->d_m2f);
    h->d_m2f = nullptr;
    cudaFree(h->d_counter);
    h->d_counter = nullptr;
    cudaFree(h->d_m2prev);
    h->d_m2prev = nullptr;
    cudaFree(h->d_mom_part);
    h->d_mom_part = nullptr;
    h->mom_part_cap = 0;
    cudaFree(h->d_urows);
    h->d_urows = nullptr;
    cudaFree(h->d_audit);
    h->d_audit = nullptr;
    cudaFree(h->d_sflags);
    h->d_sflags = nullptr;
    cudaFree(h->d_state2);
    cudaFree(h->d_qcount);
    cudaFree(h->d_qitems);
    cudaFree(h->d_prop);
    cudaFree(h->d_prop_g);
    cudaFree(h->d_prop_m);
    cudaFree(h->d_prop_v);
    cudaFree(h->d_anchor_prm);
    cudaFree(h->d_loss);
    cudaFree(h->d_wsum);
    cudaFree(h->d_prop_part);
    cudaFree(h->d_loss_part);
    cudaFree(h->d_prop_err);
    h->d_prop_part = h->d_loss_part = nullptr;
    h->d_prop_err = nullptr;
    cudaFree(h->d_rec_count);
    h->d_rec_count = nullptr;
    h->d_prop = h->d_prop_g = h->d_prop_m = h->d_prop_v = h->d_anchor_prm = h->d_loss = nullptr;
    h->d_wsum = nullptr;
    h->d_qcount = nullptr;
    h->d_qitems = nullptr;
    h->q_warps = h->q_items = 0;
    h->d_m2[0] = h->d_m2[1] = nullptr;
    h->d_acc = h->d_flags = h->d_state2 = nullptr;
    h->d_freal = nullptr;
}

static int alloc_scratch(bz_handle h)
{
    cudaFree(h->d_freal);
    cudaFree(h->d_state2);
    cudaFree(h->d_inv_e);
    h->d_freal = nullptr;
    h->d_state2 = nullptr;
    h->d_inv_e = nullptr;
    h->ncell = (int64_t)h->nslots * h->nxc * h->npc;
    if (cudaMalloc(&h->d_freal, sizeof(double) * h->ncell) != cudaSuccess)
        return fail(h, BZ_ENOMEM, "cannot allocate %lld bytes for f", (long long)(8 * h->ncell));
    if (h->nxc > 1 && cudaMalloc(&h->d_inv_e, sizeof(float) * h->ncell) != cudaSuccess)
        return fail(h, BZ_ENOMEM, "cannot allocate %lld bytes for the drift", (long long)(4 * h->ncell));
    if (h->nxc > 1 && !h->d_gforce && cudaMalloc(&h->d_gforce, sizeof(float) * 12 * h->nxc) != cudaSuccess)
        return fail(h, BZ_ENOMEM, "cannot allocate the force-term scratch");
    if (h->nxc > 1 && !h->d_m2f && cudaMalloc(&h->d_m2f, sizeof(float) * 4 * h->nxc) != cudaSuccess)
        return fail(h, BZ_ENOMEM, "cannot allocate the drift's mass table");
    return BZ_OK;
}

// The distinct values of p^2 = (px^2 + py^2) + pz^2 over the cell centres
// p = -L + (j + 1/2) dp (FP64, in that order of operations: the same bits as
// the mass kernels' per-cell evaluation) and each cell's index into them,
// for the thermal-mass kernel, which then evaluates 1/(2E) once per distinct
// value and x cell.  Grids with more than MASS_TAB_MAX distinct values get no
// table (nu = 0).  Returns BZ_OK or BZ_ENOMEM / BZ_ECUDA.
static int build_p2_table(bz_handle h)
{
    h->nu = 0;
    if (h->npc > ((int64_t)1 << 24)) return BZ_OK;
    double dp[3];
    std::vector<double> pc[3];
    for (int d = 0; d < 3; ++d) {
        dp[d] = 2.0 * h->g.L / h->g.np[d];
        for (int j = 0; j < h->g.np[d]; ++j) pc[d].push_back(-h->g.L + ((double)j + 0.5) * dp[d]);
    }
    std::vector<double> values;
    std::vector<unsigned short> idx((size_t)h->npc);
    std::vector<std::pair<uint64_t, int>> seen;  // bit pattern -> index, kept sorted
    int64_t k = 0;
    for (int jx = 0; jx < h->g.np[0]; ++jx)
        for (int jy = 0; jy < h->g.np[1]; ++jy)
            for (int jz = 0; jz < h->g.np[2]; ++jz, ++k) {
                const double px = pc[0][jx], py = pc[1][jy], pz = pc[2][jz];
                const double pp = (px * px + py * py) + pz * pz;
                uint64_t bits;
                std::memcpy(&bits, &pp, sizeof bits);
                auto it = std::lower_bound(seen.begin(), seen.end(), std::make_pair(bits, -1));
                int id;
                if (it != seen.end() && it->first == bits) {
                    id = it->second;
                } else {
                    if ((int)values.size() >= MASS_TAB_MAX) return BZ_OK;
                    id = (int)values.size();
                    values.push_back(pp);
                    seen.insert(it, std::make_pair(bits, id));
                }
                idx[(size_t)k] = (unsigned short)id;
            }
    if (cudaMalloc(&h->d_ppu, sizeof(double) * values.size()) != cudaSuccess ||
        cudaMalloc(&h->d_pidx, sizeof(unsigned short) * idx.size()) != cudaSuccess)
        return fail(h, BZ_ENOMEM, "cannot allocate the p^2 table");
    if (cudaMemcpy(h->d_ppu, values.data(), sizeof(double) * values.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_pidx, idx.data(), sizeof(unsigned short) * idx.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(h, BZ_ECUDA, "cannot upload the p^2 table");
    h->nu = (int)values.size();
    return BZ_OK;
}

static void set_slots(bz_handle h)
{
    int n = 0;
    for (int s = 0; s < NSPEC; ++s) {
        if (h->mask & (1u << s)) {
            h->slot_of[s] = n;
            h->slot_species[n] = s;
            ++n;
        } else {
            h->slot_of[s] = -1;
        }
    }
    h->nslots = n;
}

extern "C" const char* bz_version(void) { return "libbz 0.1 (sm_103a)"; }

extern "C" int bz_check_counts(int64_t* count, int64_t* first_bad, int32_t reset)
{
    unsigned long long c[3][2];
    const cudaError_t e[3] = {check_read_collide_f32(c[0], reset != 0), check_read_collide_f64(c[1], reset != 0),
                              check_read_transport(c[2], reset != 0)};
    if (e[0] == cudaErrorNotSupported) return fail(nullptr, BZ_EINVAL, "the library was built without BZ_CHECK");
    long long n = 0, first = -1;
    for (int u = 0; u < 3; ++u) {
        if (e[u] != cudaSuccess) return fail(nullptr, BZ_ECUDA, "reading the check counters: %s", cudaGetErrorString(e[u]));
        n += (long long)c[u][0];
        if (first < 0 && c[u][0]) first = (long long)c[u][1];
    }
    if (count) *count = n;
    if (first_bad) *first_bad = first;
    return BZ_OK;
}

extern "C" const char* bz_last_error(bz_handle h) { return h ? h->err.c_str() : g_init_error.c_str(); }

extern "C" int bz_init_grid(bz_handle* out, const bz_grid* g)
{
    if (!out || !g) return fail(nullptr, BZ_EINVAL, "null argument");
    *out = nullptr;
    for (int d = 0; d < 3; ++d) {
        if (g->nx[d] <= 0 || g->np[d] <= 0) return fail(nullptr, BZ_EINVAL, "grid sizes must be positive");
        if (g->np[d] > MAX_NP) return fail(nullptr, BZ_EINVAL, "np[%d] = %d exceeds %d", d, g->np[d], MAX_NP);
    }
    if (!(g->L > 0) || !(g->dx > 0)) return fail(nullptr, BZ_EINVAL, "L and dx must be positive");
    if (np_has_zero_cell(g->np)) return fail(nullptr, BZ_EINVAL, "np odd along all axes puts a cell at p = 0 (E = 0)");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(nullptr, BZ_ENODEV, "no CUDA device");
    bz_handle h = new (std::nothrow) bz_handle_s();
    if (!h) return fail(nullptr, BZ_ENOMEM, "out of host memory");
    h->g = *g;
    cudaGetDevice(&h->device);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, h->device);
    if (prop.major * 10 + prop.minor < 100) {
        delete h;
        return fail(nullptr, BZ_ENODEV, "device %s (sm_%d%d) is not a Blackwell GPU", prop.name, prop.major,
                    prop.minor);
    }
    h->nsm = prop.multiProcessorCount;
    h->nxc = (int64_t)g->nx[0] * g->nx[1] * g->nx[2];
    h->npc = (int64_t)g->np[0] * g->np[1] * g->np[2];
    set_slots(h);
    int rc;
    if (cudaMalloc(&h->d_m2[0], sizeof(double) * 4 * h->nxc) != cudaSuccess ||
        cudaMalloc(&h->d_m2[1], sizeof(double) * 4 * h->nxc) != cudaSuccess ||
        cudaMalloc(&h->d_acc, sizeof(long long) * 4 * h->nxc) != cudaSuccess ||
        cudaMalloc(&h->d_flags, sizeof(long long) * 4) != cudaSuccess ||
        cudaMalloc(&h->d_sflags, sizeof(long long) * 2) != cudaSuccess ||
        cudaMalloc(&h->d_jtab, sizeof(int) * h->npc) != cudaSuccess) {
        free_scratch(h);
        delete h;
        return fail(nullptr, BZ_ENOMEM, "cannot allocate handle scratch");
    }
    if (launch_fill_jtab(h->d_jtab, g->np, 0) != cudaSuccess) {
        free_scratch(h);
        delete h;
        return fail(nullptr, BZ_ECUDA, "cannot build the p-cell index table");
    }
    if ((rc = build_p2_table(h)) != BZ_OK) {
        g_init_error = h->err;
        free_scratch(h);
        delete h;
        return rc;
    }
    if ((rc = alloc_scratch(h)) != BZ_OK) {
        g_init_error = h->err;
        free_scratch(h);
        delete h;
        return rc;
    }
    cudaMemset(h->d_flags, 0, sizeof(long long) * 4);
    cudaMemset(h->d_sflags, 0, sizeof(long long) * 2);
    cudaMemset(h->d_m2[0], 0, sizeof(double) * 4 * h->nxc);
    cudaMemset(h->d_m2[1], 0, sizeof(double) * 4 * h->nxc);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        free_scratch(h);
        delete h;
        return fail(nullptr, BZ_ECUDA, "device initialisation failed");
    }
    *out = h;
    return BZ_OK;
}

extern "C" int bz_profile(bz_handle h, int enable)
{
    if (!h) return BZ_EINVAL;
    if (enable) {
        prof_drain(h);
        for (int i = 0; i < BZ_NKERNELS; ++i) {
            h->prof_ms[i] = 0;
            h->prof_n[i] = 0;
        }
    }
    h->prof = enable != 0;
    return BZ_OK;
}

extern "C" int bz_profile_read(bz_handle h, double* ms_host, int64_t* launches_host, int32_t n)
{
    if (!h || n < 0) return BZ_EINVAL;
    prof_drain(h);
    for (int i = 0; i < n && i < BZ_NKERNELS; ++i) {
        if (ms_host) ms_host[i] = h->prof_ms[i];
        if (launches_host) launches_host[i] = h->prof_n[i];
    }
    return BZ_OK;
}

extern "C" int bz_destroy(bz_handle h)
{
    if (!h) return BZ_EINVAL;
    cudaDeviceSynchronize();
    prof_drain(h);
    for (cudaEvent_t e : h->prof_free) cudaEventDestroy(e);
    free_scratch(h);
    delete h;
    return BZ_OK;
}

extern "C" int bz_set_species(bz_handle h, uint32_t species_mask, double alpha_s, int mass_mode)
{
    if (!h) return BZ_EINVAL;
    ++h->gen;
    if ((species_mask & 0x7Fu) == 0 || (species_mask & ~0x7Fu)) return fail(h, BZ_EINVAL, "bad species mask 0x%x", species_mask);
    if (!(alpha_s > 0)) return fail(h, BZ_EINVAL, "alpha_s must be positive");
    if (mass_mode < 0 || mass_mode > 2) return fail(h, BZ_EINVAL, "bad mass mode %d", mass_mode);
    int old = h->nslots;
    h->mask = species_mask;
    h->alpha_s = alpha_s;
    h->mass_mode = mass_mode;
    set_slots(h);
    h->have_masses = false;
    h->anchor_prm_ready = false;
    if (h->nslots != old) {
        cudaFree(h->d_anchor_prm);
        h->d_anchor_prm = nullptr;
        return alloc_scratch(h);
    }
    return BZ_OK;
}

extern "C" int bz_query_sizes(bz_handle h, int32_t* nslots, int64_t* nxcells, int64_t* npcells)
{
    if (!h) return BZ_EINVAL;
    if (nslots) *nslots = h->nslots;
    if (nxcells) *nxcells = h->nxc;
    if (npcells) *npcells = h->npc;
    return BZ_OK;
}

extern "C" int bz_set_uniform_bits(bz_handle h, int32_t bits)
{
    if (!h) return BZ_EINVAL;
    ++h->gen;
    if (bits != 32 && bits != 23) return fail(h, BZ_EINVAL, "uniform bits must be 32 or 23");
    h->f64_ubits = bits;
    return BZ_OK;
}

extern "C" int bz_set_matrix_element(bz_handle h, int32_t row, int32_t nterms, const double* coef,
                                     const int32_t* exps)
{
    if (!h) return BZ_EINVAL;
    ++h->gen;
    if (row < 0 || row >= MSQ_ROWS) return fail(h, BZ_EINVAL, "|M|^2 row must be in [0, %d)", MSQ_ROWS);
    if (nterms < 0 || nterms > 8) return fail(h, BZ_EINVAL, "a user row has 0 to 8 terms");
    if (nterms > 0 && (!coef || !exps)) return fail(h, BZ_EINVAL, "null coefficients or exponents");
    UserRow r{};
    r.n = nterms;
    for (int k = 0; k < nterms; ++k) {
        if (!std::isfinite(coef[k])) return fail(h, BZ_EINVAL, "coefficient %d is not finite", k);
        r.t[k].coef = coef[k];
        r.t[k].coef32 = (float)coef[k];
        for (int i = 0; i < 6; ++i) {
            const int e = exps[6 * k + i];
            if (e < 0 || e > 4) return fail(h, BZ_EINVAL, "exponent %d of term %d outside [0, 4]", i, k);
            r.t[k].e[i] = (uint8_t)e;
        }
    }
    if (!h->d_urows && cudaMalloc(&h->d_urows, sizeof(UserRow) * MSQ_ROWS) != cudaSuccess)
        return fail(h, BZ_ENOMEM, "cannot allocate the |M|^2 table");
    h->h_urows[row] = r;
    if (nterms > 0)
        h->umask |= 1u << row;
    else
        h->umask &= ~(1u << row);
    CK(h, cudaMemcpy(h->d_urows, h->h_urows, sizeof(UserRow) * MSQ_ROWS, cudaMemcpyHostToDevice));
    return BZ_OK;
}

extern "C" int bz_set_parameterisation(bz_handle h, int32_t which)
{
    if (!h) return BZ_EINVAL;
    ++h->gen;
    if (which != 0 && which != 1) return fail(h, BZ_EINVAL, "parameterisation must be 0 (k2) or 1 (k3)");
    h->param = which;
    return BZ_OK;
}

extern "C" int bz_set_force_term(bz_handle h, int32_t enable)
{
    if (!h) return BZ_EINVAL;
    ++h->gen;
    if (enable != 0 && enable != 1) return fail(h, BZ_EINVAL, "enable must be 0 or 1");
    h->force = enable == 1;
    return BZ_OK;
}

extern "C" int bz_set_anchor_subset(bz_handle h, int64_t stride, int64_t offset)
{
    if (!h) return BZ_EINVAL;
    ++h->gen;
    if (stride < 1 || offset < 0 || offset >= stride) return fail(h, BZ_EINVAL, "bad anchor subset");
    h->a_stride = stride;
    h->a_offset = offset;
    return BZ_OK;
}

extern "C" int bz_set_equilibrium(bz_handle h, int enable, double T, const double* mu_host)
{
    if (!h) return BZ_EINVAL;
    ++h->gen;
    if (enable && !(T > 0)) return fail(h, BZ_EINVAL, "T must be positive");
    h->analytic = enable ? 1 : 0;
    h->T = T;
    for (int s = 0; s < NSPEC; ++s) h->mu[s] = mu_host ? mu_host[s] : 0.0;
    return BZ_OK;
}

extern "C" int bz_get_masses(bz_handle h, double* m2_host)
{
    if (!h || !m2_host) return BZ_EINVAL;
    CK(h, cudaDeviceSynchronize());
    CK(h, cudaMemcpy(m2_host, h->d_m2[h->cur], sizeof(double) * 4 * h->nxc, cudaMemcpyDeviceToHost));
    return BZ_OK;
}

extern "C" int bz_set_masses(bz_handle h, const double* m2_host)
{
    if (!h || !m2_host) return BZ_EINVAL;
    ++h->gen;
    for (int64_t i = 0; i < 4 * h->nxc; ++i)
        if (!(m2_host[i] >= 0)) return fail(h, BZ_EINVAL, "masses squared must be >= 0");
    CK(h, cudaDeviceSynchronize());
    CK(h, cudaMemcpy(h->d_m2[h->cur], m2_host, sizeof(double) * 4 * h->nxc, cudaMemcpyHostToDevice));
    h->have_masses = true;
    return BZ_OK;
}

extern "C" int bz_reset_masses(bz_handle h)
{
    if (!h) return BZ_EINVAL;
    ++h->gen;
    h->have_masses = false;
    return BZ_OK;
}

extern "C" int bz_get_state_flags(bz_handle h, int64_t* flags_host)
{
    if (!h || !flags_host) return BZ_EINVAL;
    CK(h, cudaDeviceSynchronize());
    CK(h, cudaMemcpy(flags_host, h->d_sflags, sizeof(long long) * 2, cudaMemcpyDeviceToHost));
    return BZ_OK;
}

extern "C" int bz_get_flags(bz_handle h, int64_t* flags_host)
{
    if (!h || !flags_host) return BZ_EINVAL;
    CK(h, cudaDeviceSynchronize());
    CK(h, cudaMemcpy(flags_host, h->d_flags, sizeof(long long) * 4, cudaMemcpyDeviceToHost));
    return BZ_OK;
}

extern "C" int bz_clear_flags(bz_handle h)
{
    if (!h) return BZ_EINVAL;
    CK(h, cudaMemset(h->d_flags, 0, sizeof(long long) * 4));
    CK(h, cudaMemset(h->d_sflags, 0, sizeof(long long) * 2));
    return BZ_OK;
}

// --------------------------------------------------------------------------
// internal steps
// --------------------------------------------------------------------------
static double dp_of(const bz_handle h, int d) { return 2.0 * h->g.L / h->g.np[d]; }

// Thermal masses of `state` (Eqs. mg, mq) into the other mass buffer, then
// make them current.  E from the current masses if there are any (and not
// in massless mode), else |p|.
static void fill_masses(bz_handle h, MassArgs& a, const long long* state, long long* acc, double* m2_out,
                        const double* m2_prev)
{
    const double dA = 8.0, CF = 4.0 / 3.0;
    double g2 = 4.0 * PI * h->alpha_s;
    double dpx = 2.0 * h->g.L / h->g.np[0], dpy = 2.0 * h->g.L / h->g.np[1], dpz = 2.0 * h->g.L / h->g.np[2];
    double twopi = 2.0 * PI;
    a.state = state;
    a.acc = acc;
    a.m2_out = m2_out;
    a.m2_prev = m2_prev;
    a.flags = h->d_flags;
    a.nxc = h->nxc;
    a.npc = h->npc;
    for (int d = 0; d < 3; ++d) a.np[d] = h->g.np[d];
    a.L = h->g.L;
    a.dp[0] = dpx;
    a.dp[1] = dpy;
    a.dp[2] = dpz;
    for (int s2 = 0; s2 < NSPEC; ++s2) a.slot_of[s2] = h->slot_of[s2];
    a.pref_g = 2.0 * g2 / dA;
    a.pref_q = 2.0 * CF * g2;
    a.meas = dpx * dpy * dpz / (twopi * twopi * twopi);
    a.limit = INT64_MAX / (h->npc > 0 ? h->npc : 1) / 2;
    a.ppu = h->d_ppu;
    a.pidx = h->d_pidx;
    a.nu = h->nu;
}

static int compute_masses(bz_handle h, const long long* state, cudaStream_t s)
{
    if (h->mass_mode == BZ_MASS_FIXED) {
        if (!h->have_masses) return fail(h, BZ_EINVAL, "mass mode FIXED needs bz_set_masses first");
        return BZ_OK;
    }
    MassArgs a{};
    fill_masses(h, a, state, h->d_acc, h->d_m2[h->cur ^ 1],
                (h->have_masses && h->mass_mode != BZ_MASS_MASSLESS) ? h->d_m2[h->cur] : nullptr);
    {
        ProfScope ps(h, BZ_K_MASSES, s);
        CK(h, launch_masses(a, s));
    }
    h->cur ^= 1;
    h->have_masses = true;
    return BZ_OK;
}

static void fill_terms(bz_handle h, TermDev (*terms)[MAX_TERMS], int* nterms)
{
    struct T {
        int leg[4];
        double sym;
        int cls;
    };
    for (int d = 0; d < NSPEC; ++d) {
        T t[16];
        int n = 0;
        auto add = [&](int a, int b, int c, int dd, double sym, int cls) {
            t[n].leg[0] = a; t[n].leg[1] = b; t[n].leg[2] = c; t[n].leg[3] = dd;
            t[n].sym = sym; t[n].cls = cls; ++n;
        };
        // Eq. (C_gluon): 1/2 gg<->gg, and per flavour g q, g qbar, q qbar <-> gg
        if (d == 0) {
            add(0, 0, 0, 0, 0.5, M_GG);
            for (int f = 0; f < 3; ++f) {
                int q = 1 + f, qb = 4 + f;
                add(q, 0, q, 0, 1.0, M_QG);
                add(qb, 0, qb, 0, 1.0, M_QG);
                add(q, qb, 0, 0, 1.0, M_QQBGG);
            }
        } else {
            // Eq. (C_quark); the antiquark equation is its charge conjugate.
            // Legs are labelled so that (k1, k3) is the like-species line.
            bool anti = d >= 4;
            int fa = (d - 1) % 3;
            int me = anti ? 4 + fa : 1 + fa, bar = anti ? 1 + fa : 4 + fa;
            add(me, me, me, me, 0.5, M_QQ);
            add(bar, me, bar, me, 1.0, M_QQB);
            add(0, 0, bar, me, 0.5, M_QQBGG);
            add(0, me, 0, me, 1.0, M_QG);
            for (int fb = 0; fb < 3; ++fb) {
                if (fb == fa) continue;
                int Qb = anti ? 4 + fb : 1 + fb, QBb = anti ? 1 + fb : 4 + fb;
                add(Qb, me, Qb, me, 1.0, M_QQP);
                add(QBb, me, QBb, me, 1.0, M_QQP);
                add(Qb, QBb, bar, me, 1.0, M_QQB2);
            }
        }
        int m = 0;
        for (int i = 0; i < n; ++i) {
            bool ok = true;
            for (int l = 0; l < 4; ++l)
                if (!(h->mask & (1u << t[i].leg[l]))) ok = false;
            if (!ok) continue;
            TermDev& o = terms[d][m++];
            for (int l = 0; l < 4; ++l) {
                o.slot[l] = (int8_t)h->slot_of[t[i].leg[l]];
                o.mslot[l] = (int8_t)mass_slot(t[i].leg[l]);
                o.quark[l] = (int8_t)(is_quark(t[i].leg[l]) ? 1 : 0);
            }
            o.cls = (int8_t)t[i].cls;
            o.sym = t[i].sym;
        }
        // Kinematic groups: terms whose legs k1, k2, k3 carry the same masses have
        // the same roots (only |M|^2 and the legs' species differ), so they are
        // made adjacent, in order of first appearance, and the FP32 kernel solves
        // the roots once per group.  With the massless dispersion every term has
        // zero masses in the kinematics: one group.
        // The groups are then ordered by the |M|^2 row of their first term, so
        // that the 32 roots evaluated together mostly share one row.
        TermDev grouped[MAX_TERMS];
        int gstart[MAX_TERMS], glen[MAX_TERMS], ng = 0;
        bool used[MAX_TERMS] = {false};
        int k = 0;
        for (int i = 0; i < m; ++i) {
            if (used[i]) continue;
            gstart[ng] = k;
            for (int j = i; j < m; ++j) {
                const bool same = h->mass_mode == BZ_MASS_MASSLESS ||
                                  (terms[d][j].mslot[0] == terms[d][i].mslot[0] &&
                                   terms[d][j].mslot[1] == terms[d][i].mslot[1] &&
                                   terms[d][j].mslot[2] == terms[d][i].mslot[2]);
                if (used[j] || !same) continue;
                grouped[k] = terms[d][j];
                grouped[k].gfirst = (int8_t)(j == i);
                used[j] = true;
                ++k;
            }
            glen[ng] = k - gstart[ng];
            ++ng;
        }
        int order[MAX_TERMS];
        for (int g = 0; g < ng; ++g) order[g] = g;
        std::stable_sort(order, order + ng, [&](int x, int y) { return grouped[gstart[x]].cls < grouped[gstart[y]].cls; });
        k = 0;
        for (int g = 0; g < ng; ++g)
            for (int i = 0; i < glen[order[g]]; ++i) terms[d][k++] = grouped[gstart[order[g]] + i];
        nterms[d] = m;
    }
}

template <typename R>
static void fill_collide(bz_handle h, CollideArgs<R>& a, long long* A, int nsamples, int step, double dt,
                         int sampler)
{
    const double dF = 3.0, CA = 3.0, CF = 4.0 / 3.0, dA = 8.0;
    double g2 = 4.0 * PI * h->alpha_s;
    double g4 = g2 * g2;
    double twoL = 2.0 * h->g.L;
    double V = twoL * twoL * twoL * twoL * twoL;
    double Kq = ((V * dt) / (4.0 * (double)nsamples)) / HBARC * TWO_POW_40;
    double twopi = 2.0 * PI;
    double twopi5 = twopi * twopi * twopi * twopi * twopi;
    a.f = h->d_freal;
    a.f_is_float = sizeof(R) == 4 ? 1 : 0;
    a.ubits = sizeof(R) == 4 ? 23 : h->f64_ubits;
    a.tau = 0;
    a.prop = h->d_anchor_prm;
    a.rec = nullptr;
    a.rec_count = nullptr;
    a.rec_cap = 0;
    a.rec_stride = 0;
    a.audit = h->audit_on ? h->d_audit : nullptr;
    a.qcount = nullptr;
    a.qitems = nullptr;
    a.qcap = 0;
    a.A = A;
    a.m2 = h->d_m2[h->cur];
    a.flags = h->d_flags;
    a.nxc = h->nxc;
    a.npc = h->npc;
    a.ncell = h->ncell;
    for (int d = 0; d < 3; ++d) {
        a.np[d] = h->g.np[d];
        a.dp[d] = (R)(twoL / h->g.np[d]);
    }
    a.L = (R)h->g.L;
    a.twoL = (R)twoL;
    a.L64 = h->g.L;
    for (int d = 0; d < 3; ++d) a.dp64[d] = twoL / h->g.np[d];
    {
        const int64_t nchunk = (nsamples + 31) / 32;
        a.dv_group = div_magic((uint32_t)((nchunk + F32_GROUP - 1) / F32_GROUP));
        a.dv_slot = div_magic((uint32_t)std::min<int64_t>(h->nxc * h->npc, 0x7fffffff));
        a.dv_npc = div_magic((uint32_t)h->npc);
        a.dv_yz = div_magic((uint32_t)(h->g.np[1] * h->g.np[2]));
        a.dv_z = div_magic((uint32_t)h->g.np[2]);
    }
    a.key0 = (uint32_t)(h->g.seed & 0xffffffffu) ^ h->g.box;
    a.key1 = (uint32_t)(h->g.seed >> 32);
    philox_key_schedule(a.key0, a.key1, a.ks);
    a.nsamples = nsamples;
    a.step = step;
    a.a_stride = h->a_stride;
    a.a_offset = h->a_offset;
    a.n_sel = h->a_offset < h->ncell ? (h->ncell - h->a_offset + h->a_stride - 1) / h->a_stride : 0;
    a.sampler = sampler;
    a.mass_mode = h->mass_mode;
    a.analytic = h->analytic;
    a.p_center = 0;
    a.param = sizeof(R) == sizeof(double) ? h->param : 0;
    a.urows = h->d_urows;
    a.umask = h->d_urows ? h->umask : 0u;
    a.T = (R)h->T;
    for (int s = 0; s < NSPEC; ++s) a.mu[s] = (R)h->mu[s];
    a.Kq = (R)Kq;
    a.Kown = (R)(sampler == BZ_SAMPLER_PLAIN ? Kq * 4.0 : Kq);
    a.twopi5 = (R)twopi5;
    a.A1 = (R)(8.0 * g4 * dF * dF * CF * CF / dA);
    a.A2 = (R)(16.0 * g4 * dF * CF * (CF - CA / 2.0));
    a.A3 = (R)(8.0 * g4 * dF * CF * CF);
    a.A4 = (R)(8.0 * g4 * dF * CF * CA);
    a.A5 = (R)(16.0 * g4 * dA * CA * CA);
    for (int s = 0; s < NSPEC; ++s) a.slot_species[s] = s < h->nslots ? h->slot_species[s] : 0;
    // terms indexed by species d
    TermDev terms[NSPEC][MAX_TERMS];
    int nterms[NSPEC];
    std::memset(terms, 0, sizeof terms);
    fill_terms(h, terms, nterms);
    std::memcpy(a.terms, terms, sizeof terms);
    std::memcpy(a.nterms, nterms, sizeof nterms);
}

static int run_collide(bz_handle h, long long* A, int nsamples, int step, double dt, int prec, int sampler,
                       cudaStream_t s, const int* step_dev = nullptr)
{
    const int64_t n_sel = h->a_offset < h->ncell ? (h->ncell - h->a_offset + h->a_stride - 1) / h->a_stride : 0;
    const int64_t total = n_sel * (int64_t)nsamples;
    int64_t blocks = (total + 255) / 256;
    int64_t cap = (int64_t)h->nsm * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (prec == BZ_PREC_F64) {
        CollideArgs<double> a{};
        fill_collide(h, a, A, nsamples, step, dt, sampler);
        ProfScope ps(h, BZ_K_COLLIDE, s);
        CK(h, launch_collide_f64(a, (int)blocks, s));
        return BZ_OK;
    }
    // FP32 integrand, one warp per unit (an anchor and up to 256 of its samples);
    // ill-conditioned terms queued per warp for the float-float re-evaluation.
    // Cell indices are 32-bit there.
    if (h->ncell >= (int64_t)1 << 31)
        return fail(h, BZ_EINVAL, "the FP32 path needs fewer than 2^31 cells (has %lld)", (long long)h->ncell);
    const int64_t units = f32_units(n_sel, nsamples);
    if (units >= ((int64_t)1 << 31))
        return fail(h, BZ_EINVAL, "anchors x samples too large for one FP32 call (%lld work units); use an anchor subset",
                    (long long)units);
    CollideArgs<float> a{};
    fill_collide(h, a, A, nsamples, step, dt, sampler);
    a.step_dev = step_dev;
    // a resident grid whose warps take one unit at a time from a counter; a
    // problem of at most two units per resident warp keeps one warp per unit
    // (no counter to reset, no atomics).  BZ_F32_SCHEDULE=counter|static
    // forces either form, so tests can check that they give the same bits.
    blocks = (units + F32_WARPS - 1) / F32_WARPS;
    const int64_t resident = (int64_t)h->nsm * collide_f32_resident_blocks(a);
    bool dyn = blocks > 2 * resident;
    if (const char* sched = std::getenv("BZ_F32_SCHEDULE")) {
        if (!std::strcmp(sched, "counter")) dyn = true;
        else if (!std::strcmp(sched, "static")) dyn = false;
    }
    if (dyn) blocks = resident;
    if (blocks < 1) blocks = 1;
    if (dyn && !h->d_counter && cudaMalloc(&h->d_counter, sizeof(unsigned long long)) != cudaSuccess)
        return fail(h, BZ_ENOMEM, "cannot allocate the unit counter");
    const int64_t warps = blocks * F32_WARPS;
    const int64_t samples_per_warp = ((units + warps - 1) / warps) * 32 * F32_GROUP;
    const int64_t qcap = samples_per_warp * MAX_TERMS / DEFER_CAP_DIV + 64;
    if (warps > h->q_warps || warps * qcap > h->q_items) {
        cudaFree(h->d_qcount);
        cudaFree(h->d_qitems);
        h->d_qcount = nullptr;
        h->d_qitems = nullptr;
        h->q_warps = h->q_items = 0;
        if (cudaMalloc(&h->d_qcount, sizeof(int) * warps) != cudaSuccess ||
            cudaMalloc(&h->d_qitems, sizeof(unsigned long long) * warps * qcap) != cudaSuccess)
            return fail(h, BZ_ENOMEM, "cannot allocate the FP32 deferral queue (%lld items)",
                        (long long)(warps * qcap));
        h->q_warps = warps;
        h->q_items = warps * qcap;
    }
    a.tau = (float)DEFER_TAU;
    a.qcount = h->d_qcount;
    a.qitems = h->d_qitems;
    a.qcap = qcap;
    if (dyn) CK(h, cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned long long), s));
    {
        ProfScope ps(h, BZ_K_COLLIDE, s);
        CK(h, launch_collide_f32(a, (int)blocks, dyn ? h->d_counter : nullptr, s));
    }
    {  // float-float sample point and root solve, FP32 integrand
        ProfScope ps(h, BZ_K_FIXUP, s);
        CK(h, launch_fixup_f32(a, (int)warps, s));
    }
    return BZ_OK;
}

static const double kDeg[NSPEC] = {16.0, 6.0, 6.0, 6.0, 6.0, 6.0, 6.0};

static int fill_drift(bz_handle h, DriftArgs& a, const long long* in, long long* out, double dt, void* freal,
                      int freal_double)
{
    a.in = in;
    a.out = out;
    a.freal = freal;
    a.freal_double = freal_double;
    a.m2 = h->d_m2[h->cur];
    a.nxc = h->nxc;
    a.npc = h->npc;
    a.ncell = h->ncell;
    for (int d = 0; d < 3; ++d) {
        a.nx[d] = h->g.nx[d];
        a.np[d] = h->g.np[d];
    }
    a.mass_mode = h->mass_mode;
    a.dtdxf = (float)(dt / h->g.dx);
    for (int sl = 0; sl < NSPEC; ++sl) {
        int sp = sl < h->nslots ? h->slot_species[sl] : 0;
        a.slot_mslot[sl] = mass_slot(sp);
        a.deg[sl] = kDeg[sp];
        a.inv_deg[sl] = 1.0 / kDeg[sp];
        a.fscale[sl] = (float)(TWO_POW_M40 * a.inv_deg[sl]);
    }
    for (int d = 0; d < 3; ++d) {
        double dp = dp_of(h, d);
        for (int j = 0; j < h->g.np[d]; ++j) a.pf[d][j] = (float)(-h->g.L + ((double)j + 0.5) * dp);
    }
    a.jtab = h->d_jtab;
    a.inv_e = h->d_inv_e;
    a.m2f = h->d_m2f;
    // the force needs a mass gradient: none with one x cell or the massless dispersion
    a.force = h->force && h->nxc > 1 && h->mass_mode != BZ_MASS_MASSLESS;
    a.gforce = h->d_gforce;
    a.inv4dx = 1.0 / (4.0 * h->g.dx);
    for (int d = 0; d < 3; ++d) a.Kp[d] = (float)(dt / dp_of(h, d)) * 1073741824.0f;
    return BZ_OK;
}

static int fill_moments(bz_handle h, MomentArgs& a, const long long* state, double* out, bool chunked = true)
{
    a.state = state;
    a.out = out;
    a.m2 = h->d_m2[h->cur];
    a.nxc = h->nxc;
    a.npc = h->npc;
    a.nslots = h->nslots;
    a.mass_mode = h->mass_mode;
    double dp[3];
    for (int d = 0; d < 3; ++d) {
        a.np[d] = h->g.np[d];
        dp[d] = dp_of(h, d);
        a.half_dp[d] = 0.5 * dp[d];
        for (int j = 0; j < h->g.np[d]; ++j) a.pf[d][j] = (float)(-h->g.L + ((double)j + 0.5) * dp[d]);
    }
    for (int sl = 0; sl < NSPEC; ++sl) a.slot_mslot[sl] = mass_slot(sl < h->nslots ? h->slot_species[sl] : 0);
    double twopi = 2.0 * PI;
    a.pref = dp[0] * dp[1] * dp[2] / (twopi * twopi * twopi) * TWO_POW_M40;
    a.jtab = h->d_jtab;  // null for the boxes of a batch
    a.sflags = h->d_sflags;
    for (int sl = 0; sl < NSPEC; ++sl) {
        const int sp = sl < h->nslots ? h->slot_species[sl] : 0;
        a.pauli[sl] = is_quark(sp) ? (long long)(kDeg[sp] * TWO_POW_40) : 0x7fffffffffffffffLL;
    }
    // few (x cell, slot) rows: split each over blocks of >= 1024 p cells so that every SM works
    const int64_t rows = h->nxc * h->nslots;
    int64_t nch = 1;
    if (chunked && rows < 2 * (int64_t)h->nsm)
        nch = std::min<int64_t>((2 * (int64_t)h->nsm + rows - 1) / rows, std::max<int64_t>(1, h->npc / 1024));
    if (nch > 1) {
        const int64_t need = rows * nch * 10;
        if (need > h->mom_part_cap) {
            cudaFree(h->d_mom_part);
            h->d_mom_part = nullptr;
            h->mom_part_cap = 0;
            if (cudaMalloc(&h->d_mom_part, sizeof(long long) * need) != cudaSuccess)
                return fail(h, BZ_ENOMEM, "cannot allocate the moments scratch");
            h->mom_part_cap = need;
        }
        a.part = h->d_mom_part;
    }
    a.nchunk = (int)nch;
    return BZ_OK;
}

static int check_common(bz_handle h, int nsamples, int step, double dt, int prec, int sampler)
{
    if (nsamples <= 0 || nsamples > MAX_SAMPLES) return fail(h, BZ_EINVAL, "nsamples must be in [1, 2^20]");
    if (step < 0 || step >= (1 << 29)) return fail(h, BZ_EINVAL, "step must be in [0, 2^29)");
    if (!(dt > 0)) return fail(h, BZ_EINVAL, "dt must be positive");
    if (prec != BZ_PREC_F64 && prec != BZ_PREC_F32) return fail(h, BZ_EINVAL, "bad precision %d", prec);
    if (sampler != BZ_SAMPLER_SYMMETRIC && sampler != BZ_SAMPLER_PLAIN && sampler != BZ_SAMPLER_LEARNED)
        return fail(h, BZ_EINVAL, "bad sampler %d", sampler);
    if (sampler == BZ_SAMPLER_LEARNED && !h->anchor_prm_ready)
        return fail(h, BZ_EINVAL, "the learned sampler needs per-anchor proposal parameters (bz_proposal_infer)");
    if (h->param == 1 && (prec != BZ_PREC_F64 || sampler == BZ_SAMPLER_LEARNED))
        return fail(h, BZ_EINVAL, "the k3-eliminating parameterisation runs on the FP64 path with uniform samples");
    return BZ_OK;
}

// --------------------------------------------------------------------------
// public entry points
// --------------------------------------------------------------------------
extern "C" int bz_collision_term(bz_handle h, const int64_t* state, int64_t* A, int32_t nsamples, int32_t step,
                                 double dt, int32_t prec, int32_t sampler, void* stream)
{
    if (!h || !state || !A) return BZ_EINVAL;
    int rc = check_common(h, nsamples, step, dt, prec, sampler);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long* st = reinterpret_cast<const long long*>(state);
    if ((rc = compute_masses(h, st, s))) return rc;
    if (!h->analytic) {
        double deg[NSPEC];
        for (int sl = 0; sl < NSPEC; ++sl) deg[sl] = kDeg[sl < h->nslots ? h->slot_species[sl] : 0];
        ProfScope ps(h, BZ_K_CONVERT, s);
        CK(h, launch_convert(st, h->d_freal, prec == BZ_PREC_F64, h->nxc, h->npc, h->nslots, deg, s));
    }
    CK(h, cudaMemsetAsync(A, 0, sizeof(int64_t) * h->ncell, s));
    return run_collide(h, reinterpret_cast<long long*>(A), nsamples, step, dt, prec, sampler, s);
}

extern "C" int bz_collision_audit(bz_handle h, const int64_t* state, int64_t* A, int32_t nsamples, int32_t step,
                                  double dt, int32_t sampler, double* audit_host, void* stream)
{
    if (!h || !state || !A || !audit_host) return BZ_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!h->d_audit && !dalloc(&h->d_audit, 8)) return fail(h, BZ_ENOMEM, "scratch");
    CK(h, cudaMemsetAsync(h->d_audit, 0, 8 * sizeof(double), s));
    h->audit_on = true;
    const int rc = bz_collision_term(h, state, A, nsamples, step, dt, BZ_PREC_F64, sampler, stream);
    h->audit_on = false;
    if (rc) return rc;
    // slot 7 (zeroed above, as an int64) receives the exact sum of A
    long long* sum = reinterpret_cast<long long*>(h->d_audit + 7);
    CK(h, launch_sum_ll(reinterpret_cast<const long long*>(A), h->ncell, sum, s));
    double host[8];
    CK(h, cudaMemcpyAsync(host, h->d_audit, sizeof host, cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    long long sa;
    std::memcpy(&sa, &host[7], sizeof sa);
    host[7] = (double)sa;
    std::memcpy(audit_host, host, sizeof host);
    return BZ_OK;
}

namespace {
// Checkpoint file: this header, then the current masses (double [nx][4]) if
// have_masses, then the state (int64 [ncell]), all little-endian.
struct CkptHeader {
    char magic[8];  // "BZCKPT1"
    int32_t nx[3], np[3];
    double dx, L;
    uint64_t seed;
    uint32_t box, species_mask;
    double alpha_s;
    int32_t mass_mode, have_masses;
    int64_t step, ncell;
};
const char kCkptMagic[8] = {'B', 'Z', 'C', 'K', 'P', 'T', '1', 0};
}  // namespace

extern "C" int bz_save(bz_handle h, const int64_t* state, int64_t step, const char* path)
{
    if (!h || !state || !path) return BZ_EINVAL;
    CkptHeader hd{};
    std::memcpy(hd.magic, kCkptMagic, 8);
    for (int d = 0; d < 3; ++d) {
        hd.nx[d] = h->g.nx[d];
        hd.np[d] = h->g.np[d];
    }
    hd.dx = h->g.dx;
    hd.L = h->g.L;
    hd.seed = h->g.seed;
    hd.box = h->g.box;
    hd.species_mask = h->mask;
    hd.alpha_s = h->alpha_s;
    hd.mass_mode = h->mass_mode;
    hd.have_masses = h->have_masses ? 1 : 0;
    hd.step = step;
    hd.ncell = h->ncell;
    std::vector<double> m2(h->have_masses ? 4 * h->nxc : 0);
    std::vector<int64_t> st(h->ncell);
    CK(h, cudaDeviceSynchronize());
    if (h->have_masses)
        CK(h, cudaMemcpy(m2.data(), h->d_m2[h->cur], sizeof(double) * m2.size(), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(st.data(), state, sizeof(int64_t) * st.size(), cudaMemcpyDeviceToHost));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(h, BZ_EINVAL, "cannot open %s for writing", path);
    bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1 &&
              (m2.empty() || std::fwrite(m2.data(), sizeof(double), m2.size(), f) == m2.size()) &&
              std::fwrite(st.data(), sizeof(int64_t), st.size(), f) == st.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(h, BZ_EINVAL, "cannot write %s", path);
    return BZ_OK;
}

extern "C" int bz_load(bz_handle h, int64_t* state, int64_t* step, const char* path)
{
    if (!h || !state || !step || !path) return BZ_EINVAL;
    ++h->gen;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(h, BZ_EINVAL, "cannot open %s", path);
    CkptHeader hd{};
    bool ok = std::fread(&hd, sizeof hd, 1, f) == 1 && std::memcmp(hd.magic, kCkptMagic, 8) == 0;
    if (ok) {
        for (int d = 0; d < 3; ++d) ok = ok && hd.nx[d] == h->g.nx[d] && hd.np[d] == h->g.np[d];
        ok = ok && hd.dx == h->g.dx && hd.L == h->g.L && hd.seed == h->g.seed && hd.box == h->g.box &&
             hd.species_mask == h->mask && hd.alpha_s == h->alpha_s && hd.mass_mode == h->mass_mode &&
             hd.ncell == h->ncell;
        if (!ok) {
            std::fclose(f);
            return fail(h, BZ_EINVAL, "checkpoint %s was written for another grid, species set or mass mode", path);
        }
    }
    std::vector<double> m2(ok && hd.have_masses ? 4 * h->nxc : 0);
    std::vector<int64_t> st(h->ncell);
    ok = ok && (m2.empty() || std::fread(m2.data(), sizeof(double), m2.size(), f) == m2.size()) &&
         std::fread(st.data(), sizeof(int64_t), st.size(), f) == st.size();
    std::fclose(f);
    if (!ok) return fail(h, BZ_EINVAL, "%s is not a complete checkpoint", path);
    CK(h, cudaMemcpy(state, st.data(), sizeof(int64_t) * st.size(), cudaMemcpyHostToDevice));
    if (!m2.empty()) {
        CK(h, cudaMemcpy(h->d_m2[h->cur], m2.data(), sizeof(double) * m2.size(), cudaMemcpyHostToDevice));
        h->have_masses = true;
    } else {
        h->have_masses = false;
    }
    *step = hd.step;
    return BZ_OK;
}

extern "C" int bz_drift(bz_handle h, const int64_t* in, int64_t* out, double dt, void* stream)
{
    if (!h || !in || !out) return BZ_EINVAL;
    if (!(dt > 0)) return fail(h, BZ_EINVAL, "dt must be positive");
    if (in == out) return fail(h, BZ_EINVAL, "in and out must not overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    if (!h->have_masses && h->mass_mode == BZ_MASS_THERMAL)
        if ((rc = compute_masses(h, reinterpret_cast<const long long*>(in), s))) return rc;
    DriftArgs a{};
    fill_drift(h, a, reinterpret_cast<const long long*>(in), reinterpret_cast<long long*>(out), dt, nullptr, 0);
    {
        ProfScope ps(h, BZ_K_DRIFT, s);
        CK(h, launch_drift(a, s));
    }
    return BZ_OK;
}

extern "C" int bz_moments(bz_handle h, const int64_t* state, double* out, void* stream)
{
    if (!h || !state || !out) return BZ_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    if (!h->have_masses && h->mass_mode == BZ_MASS_THERMAL)
        if ((rc = compute_masses(h, reinterpret_cast<const long long*>(state), s))) return rc;
    MomentArgs a{};
    if ((rc = fill_moments(h, a, reinterpret_cast<const long long*>(state), out))) return rc;
    {
        ProfScope ps(h, BZ_K_MOMENTS, s);
        CK(h, launch_moments(a, s));
    }
    return BZ_OK;
}

extern "C" int bz_energy_source(bz_handle h, const int64_t* state, const double* m2_prev_host, double dt, double* out,
                                void* stream)
{
    if (!h || !state || !out) return BZ_EINVAL;
    if (!(dt > 0)) return fail(h, BZ_EINVAL, "dt must be positive");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    if (!h->have_masses && h->mass_mode == BZ_MASS_THERMAL)
        if ((rc = compute_masses(h, reinterpret_cast<const long long*>(state), s))) return rc;
    if (!h->have_masses && h->mass_mode == BZ_MASS_FIXED)
        return fail(h, BZ_EINVAL, "mass mode FIXED needs bz_set_masses first");
    MomentArgs a{};  // with the massless dispersion the masses are not read
    fill_moments(h, a, reinterpret_cast<const long long*>(state), out, false);
    a.sflags = nullptr;
    a.dt = dt;
    if (m2_prev_host) {
        if (!h->d_m2prev && cudaMalloc(&h->d_m2prev, sizeof(double) * 4 * h->nxc) != cudaSuccess)
            return fail(h, BZ_ENOMEM, "cannot allocate the previous masses");
        CK(h, cudaMemcpyAsync(h->d_m2prev, m2_prev_host, sizeof(double) * 4 * h->nxc, cudaMemcpyHostToDevice, s));
        a.m2_prev = h->d_m2prev;
    } else {
        a.m2_prev = h->d_m2[h->cur];  // no previous masses given: no source
    }
    {
        ProfScope ps(h, BZ_K_MOMENTS, s);
        CK(h, launch_energy_source(a, s));
    }
    return BZ_OK;
}

// One Euler step from cur into nxt (Sec. III): masses of cur, drift into nxt
// (with f of cur for the lookups), collision deposits into nxt, moments of
// nxt.  Eager (step_dev null): step index `step`, moments at mom; inside a
// captured graph: the step index and the moments slot of mom are read from
// the device words step_dev[0], step_dev[1], advanced after the step.
static int one_step(bz_handle h, long long* cur, long long* nxt, double dt, int nsamples, int prec, int step,
                    double* mom, const int* step_dev, cudaStream_t s)
{
    int rc;
    if ((rc = compute_masses(h, cur, s))) return rc;
    DriftArgs d{};
    fill_drift(h, d, cur, nxt, dt, h->analytic ? nullptr : h->d_freal, prec == BZ_PREC_F64);
    {
        ProfScope ps(h, BZ_K_DRIFT, s);
        CK(h, launch_drift(d, s));
    }
    if ((rc = run_collide(h, nxt, nsamples, step, dt, prec, h->step_sampler, s, step_dev))) return rc;
    if (mom) {
        MomentArgs m{};
        if ((rc = fill_moments(h, m, nxt, mom))) return rc;
        if (step_dev) {
            m.kidx = step_dev + 1;
            m.kstride = h->nxc * h->nslots * 5;
        }
        ProfScope ps(h, BZ_K_MOMENTS, s);
        CK(h, launch_moments(m, s));
    }
    if (step_dev) CK(h, launch_step_advance(const_cast<int*>(step_dev), const_cast<int*>(step_dev) + 1, s));
    return BZ_OK;
}

extern "C" int bz_step(bz_handle h, int64_t* state, double dt, int32_t nsteps, int32_t nsamples, int32_t prec,
                       int32_t step0, double* moments_out, void* stream)
{
    if (!h || !state) return BZ_EINVAL;
    if (nsteps < 0) return fail(h, BZ_EINVAL, "nsteps must be >= 0");
    int rc = check_common(h, nsamples, step0, dt, prec, h->step_sampler);
    if (rc) return rc;
    if ((int64_t)step0 + nsteps > (1 << 29)) return fail(h, BZ_EINVAL, "step index overflows 2^29");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!h->d_state2 && cudaMalloc(&h->d_state2, sizeof(long long) * h->ncell) != cudaSuccess)
        return fail(h, BZ_ENOMEM, "cannot allocate the second state buffer");
    long long* cur = reinterpret_cast<long long*>(state);
    long long* nxt = h->d_state2;
    const int64_t mstride = h->nxc * h->nslots * 5;
    int k = 0;
    auto eager = [&]() -> int {
        int r = one_step(h, cur, nxt, dt, nsamples, prec, step0 + k, moments_out ? moments_out + k * mstride : nullptr,
                         nullptr, s);
        if (r) return r;
        std::swap(cur, nxt);
        ++k;
        return BZ_OK;
    };
    // FP32 runs of several steps replay a captured pair of steps (cur -> nxt ->
    // cur, the mass buffers back in their roles): the same launches with the
    // same arguments, so the same bits, at one launch per two steps.  The first
    // step runs eagerly (it sizes the scratch, and a fresh handle's first
    // masses take E = |p|); per-kernel profiling, and BZ_STEP_GRAPH=0 in the
    // environment, keep every step eager.
    const char* env = std::getenv("BZ_STEP_GRAPH");
    const bool graphs = prec == BZ_PREC_F32 && !h->prof && !(env && !std::strcmp(env, "0"));
    if (graphs && nsteps >= 3) {
        if ((rc = eager())) return rc;
        if (!h->d_step_idx && cudaMalloc(&h->d_step_idx, 2 * sizeof(int)) != cudaSuccess)
            return fail(h, BZ_ENOMEM, "cannot allocate the step index");
        if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(h, BZ_ECUDA, "cannot create the capture stream");
        bz_handle_s::StepGraph& G = h->sg[h->cur];
        if (!G.exec || G.cur != cur || G.mom != moments_out || G.dt != dt || G.nsamples != nsamples ||
            G.sampler != h->step_sampler || G.gen != h->gen) {
            drop_step_graph(h, h->cur);
            CK(h, cudaStreamSynchronize(s));
            cudaGraph_t graph = nullptr;
            CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
            rc = one_step(h, cur, nxt, dt, nsamples, prec, step0 + k, moments_out, h->d_step_idx, h->cap_stream);
            if (!rc) rc = one_step(h, nxt, cur, dt, nsamples, prec, step0 + k + 1, moments_out, h->d_step_idx,
                                   h->cap_stream);
            const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (ce != cudaSuccess) return fail(h, BZ_ECUDA, "step graph capture failed: %s", cudaGetErrorString(ce));
            const cudaError_t ie = cudaGraphInstantiate(&G.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                G.exec = nullptr;
                return fail(h, BZ_ECUDA, "step graph instantiation failed: %s", cudaGetErrorString(ie));
            }
            G.cur = cur;
            G.mom = moments_out;
            G.dt = dt;
            G.nsamples = nsamples;
            G.sampler = h->step_sampler;
            G.gen = h->gen;
        }
        CK(h, launch_set_step(h->d_step_idx, step0 + k, h->d_step_idx + 1, k, s));
        for (; nsteps - k >= 2; k += 2) CK(h, cudaGraphLaunch(G.exec, s));
    }
    while (k < nsteps)
        if ((rc = eager())) return rc;
    if (cur != reinterpret_cast<long long*>(state))
        CK(h, cudaMemcpyAsync(state, cur, sizeof(long long) * h->ncell, cudaMemcpyDeviceToDevice, s));
    return BZ_OK;
}

// --------------------------------------------------------------------------
// Batched ensemble: independent homogeneous boxes of any grid size, species
// set, coupling and sample count, stepped together.  Per step: thermal
// masses of every box (one launch), f of the concatenated state (one
// launch), collision of every (box, anchor, 32 samples) unit in one
// persistent launch with dynamic work distribution, float-float fixup of queued
// terms, moments, and the end-of-step bookkeeping; the step is captured
// once as a CUDA graph and replayed, the step index living in device memory.
// The collision increment is deposited into the state in place: the kernels
// read f, the FP32 snapshot of the state taken at the start of the step.
// --------------------------------------------------------------------------
struct bz_batch_s {
    int nboxes = 0;
    int device = 0, nsm = 0;
    std::vector<bz_box> desc;
    std::vector<bz_handle_s> hb;  // per-box descriptors; their device pointers alias the batch buffers
    std::vector<int64_t> cell_prefix, unit_prefix, mchunk_prefix, cchunk_prefix;
    std::vector<int> slot_prefix;
    int64_t ncell = 0, nunits = 0, nmchunks = 0, ncchunks = 0;
    int total_slots = 0;
    float* d_f = nullptr;
    double *d_m2_cur = nullptr, *d_m2_prev = nullptr;
    long long *d_acc = nullptr, *d_flags = nullptr;
    int *d_have_prev = nullptr, *d_step = nullptr, *d_kidx = nullptr;
    unsigned long long* d_counter = nullptr;
    int64_t *d_cell_prefix = nullptr, *d_unit_prefix = nullptr, *d_mchunk_prefix = nullptr, *d_cchunk_prefix = nullptr;
    int* d_slot_prefix = nullptr;
    float* d_scale = nullptr;
    int* d_slot_cells = nullptr;
    CollideArgs<float>* d_a32 = nullptr;
    MassArgs* d_mass = nullptr;
    MomentArgs* d_mom = nullptr;
    std::vector<CollideArgs<float>> a32;
    std::vector<MassArgs> mass;
    std::vector<MomentArgs> mom;
    int* d_qcount = nullptr;
    unsigned long long* d_qitems = nullptr;
    int64_t qcap = 0, qwarps = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    const long long* g_state = nullptr;
    const double* g_mom = nullptr;
    double g_dt = 0;
    bool tuned = false;
    int chunk = 4, bps = 24 / F32_WARPS;
    double tuned_ms = 0;
    std::string err;
};

static int bfail(bz_batch b, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b)
        b->err = buf;
    else
        g_init_error = buf;
    return code;
}

#define CKB(b, call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return bfail((b), BZ_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static void batch_free(bz_batch b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    void* ptrs[] = {b->d_f, b->d_m2_cur, b->d_m2_prev, b->d_acc, b->d_flags, b->d_have_prev, b->d_step, b->d_kidx,
                    b->d_counter, b->d_cell_prefix, b->d_unit_prefix, b->d_mchunk_prefix, b->d_cchunk_prefix,
                    b->d_slot_prefix, b->d_scale, b->d_slot_cells, b->d_a32, b->d_mass, b->d_mom,
                    b->d_qcount, b->d_qitems};
    for (void* p : ptrs) cudaFree(p);
    for (auto& h : b->hb) {
        h.d_m2[0] = h.d_m2[1] = nullptr;  // aliases, owned by the batch
        h.d_freal = nullptr;
        h.d_flags = h.d_acc = nullptr;
    }
}


extern "C" int bz_batch_create(bz_batch* out, int32_t nboxes, const bz_box* boxes)
{
    if (!out || !boxes || nboxes <= 0 || nboxes > 65535) return bfail(nullptr, BZ_EINVAL, "need 1..65535 boxes");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return bfail(nullptr, BZ_ENODEV, "no CUDA device");
    bz_batch b = new (std::nothrow) bz_batch_s();
    if (!b) return bfail(nullptr, BZ_ENOMEM, "out of host memory");
    b->nboxes = nboxes;
    b->desc.assign(boxes, boxes + nboxes);
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
    b->hb.resize(nboxes);
    b->cell_prefix.assign(nboxes + 1, 0);
    b->unit_prefix.assign(nboxes + 1, 0);
    b->mchunk_prefix.assign(nboxes + 1, 0);
    b->cchunk_prefix.assign(nboxes + 1, 0);
    b->slot_prefix.assign(nboxes + 1, 0);
    for (int i = 0; i < nboxes; ++i) {
        const bz_box& d = boxes[i];
        for (int k = 0; k < 3; ++k)
            if (d.np[k] <= 0 || d.np[k] > MAX_NP) {
                delete b;
                return bfail(nullptr, BZ_EINVAL, "box %d: np out of range", i);
            }
        if (np_has_zero_cell(d.np)) {
            delete b;
            return bfail(nullptr, BZ_EINVAL, "box %d: np odd along all axes puts a cell at p = 0", i);
        }
        if (!(d.L > 0) || !(d.alpha_s > 0) || (d.species_mask & 0x7Fu) == 0 || (d.species_mask & ~0x7Fu) ||
            d.nsamples <= 0 || d.nsamples > MAX_SAMPLES ||
            (d.mass_mode != BZ_MASS_THERMAL && d.mass_mode != BZ_MASS_MASSLESS)) {
            delete b;
            return bfail(nullptr, BZ_EINVAL, "box %d: bad L, alpha_s, species, nsamples or mass mode", i);
        }
        bz_handle_s& h = b->hb[i];
        h.g.nx[0] = h.g.nx[1] = h.g.nx[2] = 1;
        h.g.dx = 1.0;
        for (int k = 0; k < 3; ++k) h.g.np[k] = d.np[k];
        h.g.L = d.L;
        h.g.seed = d.seed;
        h.g.box = d.box_id;
        h.mask = d.species_mask;
        h.alpha_s = d.alpha_s;
        h.mass_mode = d.mass_mode;
        set_slots(&h);
        h.nxc = 1;
        h.npc = (int64_t)d.np[0] * d.np[1] * d.np[2];
        h.ncell = h.nslots * h.npc;
        h.nsm = b->nsm;
        b->cell_prefix[i + 1] = b->cell_prefix[i] + h.ncell;
        b->unit_prefix[i + 1] = b->unit_prefix[i] + f32_units(h.ncell, d.nsamples);
        b->mchunk_prefix[i + 1] = b->mchunk_prefix[i] + (h.npc + 2047) / 2048;
        b->cchunk_prefix[i + 1] = b->cchunk_prefix[i] + (h.ncell + 2047) / 2048;
        b->slot_prefix[i + 1] = b->slot_prefix[i] + h.nslots;
    }
    b->ncell = b->cell_prefix[nboxes];
    b->nunits = b->unit_prefix[nboxes];
    b->nmchunks = b->mchunk_prefix[nboxes];
    b->ncchunks = b->cchunk_prefix[nboxes];
    b->total_slots = b->slot_prefix[nboxes];
    if (b->ncell >= ((int64_t)1 << 31) || b->nunits >= ((int64_t)1 << 31)) {
        delete b;
        return bfail(nullptr, BZ_EINVAL, "the batch needs fewer than 2^31 cells and work units");
    }
    // persistent grid of up to 32 warps per SM; per-warp queue room for 4% of an
    // even share at 24 warps per SM (2.7% at 16, 5.3% at 32)
    b->qwarps = (int64_t)b->nsm * 32;
    b->qcap = (b->nunits * 32 * F32_GROUP * MAX_TERMS) / ((int64_t)b->nsm * 24) / 25 + 64;
    bool ok = dalloc(&b->d_f, b->ncell) && dalloc(&b->d_m2_cur, 4 * nboxes) && dalloc(&b->d_m2_prev, 4 * nboxes) &&
              dalloc(&b->d_acc, 4 * nboxes) && dalloc(&b->d_flags, 4) && dalloc(&b->d_have_prev, 1) &&
              dalloc(&b->d_step, 1) && dalloc(&b->d_kidx, 1) && dalloc(&b->d_counter, 1) &&
              dalloc(&b->d_cell_prefix, nboxes + 1) && dalloc(&b->d_unit_prefix, nboxes + 1) &&
              dalloc(&b->d_mchunk_prefix, nboxes + 1) && dalloc(&b->d_cchunk_prefix, nboxes + 1) &&
              dalloc(&b->d_slot_prefix, nboxes + 1) && dalloc(&b->d_scale, 2 * nboxes) &&
              dalloc(&b->d_slot_cells, nboxes) && dalloc(&b->d_a32, nboxes) &&
              dalloc(&b->d_mass, nboxes) && dalloc(&b->d_mom, nboxes) && dalloc(&b->d_qcount, b->qwarps) &&
              dalloc(&b->d_qitems, b->qwarps * b->qcap);
    if (!ok) {
        batch_free(b);
        delete b;
        return bfail(nullptr, BZ_ENOMEM, "cannot allocate the batch buffers");
    }
    std::vector<float> scale(2 * nboxes);
    std::vector<int> slot_cells(nboxes);
    for (int i = 0; i < nboxes; ++i) {
        bz_handle_s& h = b->hb[i];
        h.d_freal = b->d_f + b->cell_prefix[i];
        h.d_m2[0] = b->d_m2_cur + 4 * i;
        h.cur = 0;
        h.have_masses = true;
        h.d_flags = b->d_flags;
        h.d_acc = b->d_acc + 4 * i;
        const bool has_g = (h.mask & 1u) != 0;
        scale[2 * i] = (float)(TWO_POW_M40 / 16.0);
        scale[2 * i + 1] = (float)(TWO_POW_M40 / 6.0);
        slot_cells[i] = has_g ? (int)h.npc : 0;
    }
    cudaMemcpy(b->d_cell_prefix, b->cell_prefix.data(), sizeof(int64_t) * (nboxes + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_unit_prefix, b->unit_prefix.data(), sizeof(int64_t) * (nboxes + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_mchunk_prefix, b->mchunk_prefix.data(), sizeof(int64_t) * (nboxes + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_cchunk_prefix, b->cchunk_prefix.data(), sizeof(int64_t) * (nboxes + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_slot_prefix, b->slot_prefix.data(), sizeof(int) * (nboxes + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_scale, scale.data(), sizeof(float) * 2 * nboxes, cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_slot_cells, slot_cells.data(), sizeof(int) * nboxes, cudaMemcpyHostToDevice);
    cudaMemset(b->d_have_prev, 0, sizeof(int));
    cudaMemset(b->d_flags, 0, sizeof(long long) * 4);
    cudaMemset(b->d_m2_prev, 0, sizeof(double) * 4 * nboxes);
    cudaMemset(b->d_m2_cur, 0, sizeof(double) * 4 * nboxes);
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        batch_free(b);
        delete b;
        return bfail(nullptr, BZ_ECUDA, "batch initialisation failed");
    }
    *out = b;
    return BZ_OK;
}

extern "C" int bz_batch_destroy(bz_batch b)
{
    if (!b) return BZ_EINVAL;
    cudaDeviceSynchronize();
    batch_free(b);
    delete b;
    return BZ_OK;
}

extern "C" const char* bz_batch_last_error(bz_batch b) { return b ? b->err.c_str() : g_init_error.c_str(); }

extern "C" int bz_batch_layout(bz_batch b, int64_t* cell_offsets, int32_t* slot_offsets)
{
    if (!b) return BZ_EINVAL;
    for (int i = 0; i <= b->nboxes; ++i) {
        if (cell_offsets) cell_offsets[i] = b->cell_prefix[i];
        if (slot_offsets) slot_offsets[i] = b->slot_prefix[i];
    }
    return BZ_OK;
}

extern "C" int bz_batch_get_masses(bz_batch b, double* m2_host)
{
    if (!b || !m2_host) return BZ_EINVAL;
    CKB(b, cudaDeviceSynchronize());
    CKB(b, cudaMemcpy(m2_host, b->d_m2_cur, sizeof(double) * 4 * b->nboxes, cudaMemcpyDeviceToHost));
    return BZ_OK;
}

extern "C" int bz_batch_get_flags(bz_batch b, int64_t* flags_host)
{
    if (!b || !flags_host) return BZ_EINVAL;
    CKB(b, cudaDeviceSynchronize());
    CKB(b, cudaMemcpy(flags_host, b->d_flags, sizeof(long long) * 4, cudaMemcpyDeviceToHost));
    return BZ_OK;
}

extern "C" int bz_batch_tuning(bz_batch b, int32_t* chunk, int32_t* blocks_per_sm, double* ms_collide)
{
    if (!b) return BZ_EINVAL;
    if (chunk) *chunk = b->chunk;
    if (blocks_per_sm) *blocks_per_sm = b->bps;
    if (ms_collide) *ms_collide = b->tuned_ms;
    return b->tuned ? BZ_OK : BZ_EINVAL;
}

// Per-box argument blocks for the state buffer `state` and time step dt.
static int batch_fill_args(bz_batch b, long long* state, double dt, cudaStream_t s)
{
    const int n = b->nboxes;
    b->a32.assign(n, CollideArgs<float>{});
    b->mass.assign(n, MassArgs{});
    b->mom.assign(n, MomentArgs{});
    for (int i = 0; i < n; ++i) {
        bz_handle_s* h = &b->hb[i];
        long long* st = state + b->cell_prefix[i];
        fill_collide(h, b->a32[i], st, b->desc[i].nsamples, 0, dt, BZ_SAMPLER_SYMMETRIC);
        b->a32[i].tau = (float)DEFER_TAU;
        fill_masses(h, b->mass[i], st, b->d_acc + 4 * i, b->d_m2_cur + 4 * i,
                    h->mass_mode == BZ_MASS_MASSLESS ? nullptr : b->d_m2_prev + 4 * i);
        fill_moments(h, b->mom[i], st, nullptr, false);
    }
    CKB(b, cudaMemcpyAsync(b->d_a32, b->a32.data(), sizeof(CollideArgs<float>) * n, cudaMemcpyHostToDevice, s));
    CKB(b, cudaMemcpyAsync(b->d_mass, b->mass.data(), sizeof(MassArgs) * n, cudaMemcpyHostToDevice, s));
    CKB(b, cudaMemcpyAsync(b->d_mom, b->mom.data(), sizeof(MomentArgs) * n, cudaMemcpyHostToDevice, s));
    return BZ_OK;
}

static int batch_collide(bz_batch b, int chunk, int bps, cudaStream_t s)
{
    const int grid = b->nsm * bps;
    CKB(b, cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), s));
    CKB(b, launch_collide_f32_batch(b->d_a32, b->d_unit_prefix, b->nboxes, b->d_counter, b->d_step, chunk, grid,
                                    b->d_qcount, b->d_qitems, b->qcap, s));
    CKB(b, launch_fixup_f32_batch(b->d_a32, b->d_qcount, b->d_qitems, b->qcap, b->d_step, grid * F32_WARPS, s));
    return BZ_OK;
}

static int batch_record_step(bz_batch b, long long* state, double* moments_out, cudaStream_t s)
{
    int rc;
    CKB(b, launch_masses_batch(b->d_mass, b->d_mchunk_prefix, b->nboxes, b->nmchunks, b->d_have_prev, b->d_acc, s));
    CKB(b, launch_convert_batch(state, b->d_f, b->d_cell_prefix, b->d_cchunk_prefix, b->d_scale, b->d_slot_cells,
                                b->nboxes, b->ncchunks, s));
    if ((rc = batch_collide(b, b->chunk, b->bps, s))) return rc;
    if (moments_out)
        CKB(b, launch_moments_batch(b->d_mom, b->d_slot_prefix, b->nboxes, b->total_slots, moments_out, b->d_kidx,
                                    5 * b->total_slots, s));
    CKB(b, launch_batch_end_step(b->d_m2_prev, b->d_m2_cur, 4 * b->nboxes, b->d_have_prev, b->d_step, b->d_kidx, s));
    return BZ_OK;
}

// Autotuner: times the persistent collision launch for each (chunk, blocks
// per SM) candidate on a copy of the state and keeps the fastest.
static int batch_autotune(bz_batch b, long long* state, double dt, cudaStream_t s)
{
    long long* scratch = nullptr;
    if (!dalloc(&scratch, b->ncell)) return bfail(b, BZ_ENOMEM, "cannot allocate the tuning copy");
    int rc = BZ_OK;
    const int chunks[] = {1, 2, 4, 8, 16};
    const int bpss[] = {16 / F32_WARPS, 20 / F32_WARPS, 24 / F32_WARPS};  // 16, 20, 24 warps per SM (24 resident at most)
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    int zero = 0;
    do {
        if (cudaMemcpyAsync(scratch, state, sizeof(long long) * b->ncell, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            rc = bfail(b, BZ_ECUDA, "tuning copy failed");
            break;
        }
        if ((rc = batch_fill_args(b, scratch, dt, s))) break;
        if (cudaMemcpyAsync(b->d_step, &zero, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) {
            rc = bfail(b, BZ_ECUDA, "tuning set-up failed");
            break;
        }
        if (launch_masses_batch(b->d_mass, b->d_mchunk_prefix, b->nboxes, b->nmchunks, b->d_have_prev, b->d_acc, s) !=
                cudaSuccess ||
            launch_convert_batch(scratch, b->d_f, b->d_cell_prefix, b->d_cchunk_prefix, b->d_scale, b->d_slot_cells,
                                 b->nboxes, b->ncchunks, s) != cudaSuccess) {
            rc = bfail(b, BZ_ECUDA, "tuning set-up launch failed");
            break;
        }
        for (int bps : bpss) {
            for (int ch : chunks) {
                if ((rc = batch_collide(b, ch, bps, s))) break;  // warm-up
                cudaEventRecord(e0, s);
                for (int r = 0; r < 2; ++r)
                    if ((rc = batch_collide(b, ch, bps, s))) break;
                cudaEventRecord(e1, s);
                if (rc) break;
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms / 2 < best) {
                    best = ms / 2;
                    b->chunk = ch;
                    b->bps = bps;
                }
            }
            if (rc) break;
        }
    } while (0);
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    cudaMemsetAsync(b->d_flags, 0, sizeof(long long) * 4, s);
    if (rc) return rc;
    b->tuned = true;
    b->tuned_ms = best;
    b->g_state = nullptr;  // argument blocks now point at the copy: rebuild
    return BZ_OK;
}

extern "C" int bz_batch_step(bz_batch b, int64_t* state, double dt, int32_t nsteps, int32_t step0, double* moments_out,
                             void* stream)
{
    if (!b || !state) return BZ_EINVAL;
    if (nsteps < 0 || step0 < 0 || (int64_t)step0 + nsteps > (1 << 29))
        return bfail(b, BZ_EINVAL, "steps must stay in [0, 2^29)");
    if (!(dt > 0)) return bfail(b, BZ_EINVAL, "dt must be positive");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    long long* st = reinterpret_cast<long long*>(state);
    int rc;
    if (!b->tuned && (rc = batch_autotune(b, st, dt, s))) return rc;
    if (b->g_state != st || b->g_mom != moments_out || b->g_dt != dt || !b->exec) {
        if ((rc = batch_fill_args(b, st, dt, s))) return rc;
        CKB(b, cudaStreamSynchronize(s));
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        CKB(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = batch_record_step(b, st, moments_out, b->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (ce != cudaSuccess) return bfail(b, BZ_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return bfail(b, BZ_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
        b->g_state = st;
        b->g_mom = moments_out;
        b->g_dt = dt;
    }
    int zero = 0;
    CKB(b, cudaMemcpyAsync(b->d_step, &step0, sizeof(int), cudaMemcpyHostToDevice, s));
    CKB(b, cudaMemcpyAsync(b->d_kidx, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
    for (int k = 0; k < nsteps; ++k) CKB(b, cudaGraphLaunch(b->exec, s));
    return BZ_OK;
}


// --------------------------------------------------------------------------
// Learned proposal (network, training, inference)
// --------------------------------------------------------------------------
static int prop_alloc(bz_handle h)
{
    const int n = mlp_nparam();
    if (h->d_prop) return BZ_OK;
    if (!dalloc(&h->d_prop, n) || !dalloc(&h->d_prop_g, n) || !dalloc(&h->d_prop_m, n) ||
        !dalloc(&h->d_prop_v, n) || !dalloc(&h->d_loss, 1) || !dalloc(&h->d_wsum, sum_weights_scratch()) ||
        !dalloc(&h->d_prop_part, (size_t)4 * h->nsm * n) || !dalloc(&h->d_loss_part, (size_t)4 * h->nsm) ||
        !dalloc(&h->d_prop_err, 1))
        return fail(h, BZ_ENOMEM, "cannot allocate the proposal network");
    CK(h, cudaMemset(h->d_prop_g, 0, sizeof(float) * n));
    CK(h, cudaMemset(h->d_prop_m, 0, sizeof(float) * n));
    CK(h, cudaMemset(h->d_prop_v, 0, sizeof(float) * n));
    return BZ_OK;
}

static ProposalArgs prop_args(bz_handle h)
{
    ProposalArgs A{};
    A.nxc = h->nxc;
    A.npc = h->npc;
    for (int d = 0; d < 3; ++d) A.np[d] = h->g.np[d];
    A.L = (float)h->g.L;
    for (int q = 0; q < NSPEC; ++q) A.slot_species[q] = q < h->nslots ? h->slot_species[q] : 0;
    return A;
}

extern "C" int bz_proposal_nparams(void) { return mlp_nparam(); }

extern "C" int bz_proposal_init(bz_handle h, uint64_t seed)
{
    if (!h) return BZ_EINVAL;
    ++h->gen;
    int rc = prop_alloc(h);
    if (rc) return rc;
    const int H = 128, NIN = 16, NOUT = 8;
    std::vector<float> p(mlp_nparam(), 0.0f);
    // uniform(-a, a) with a = sqrt(6 / (fan_in + fan_out)), from a splitmix64 stream
    uint64_t st = seed * 0x9E3779B97F4A7C15ull + 1;
    auto uni = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    float* W1 = p.data();
    float* W2 = W1 + NIN * H + H;
    float* W3 = W2 + H * H + H;
    const double a1 = std::sqrt(6.0 / (9 + H)), a2 = std::sqrt(6.0 / (2 * H)), a3 = 0.1 * std::sqrt(6.0 / (H + 6));
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < H; ++j) W1[i * H + j] = (float)((2 * uni() - 1) * a1);
    for (int i = 0; i < H * H; ++i) W2[i] = (float)((2 * uni() - 1) * a2);
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < 6; ++j) W3[i * NOUT + j] = (float)((2 * uni() - 1) * a3);
    CK(h, cudaMemcpy(h->d_prop, p.data(), sizeof(float) * p.size(), cudaMemcpyHostToDevice));
    CK(h, cudaMemset(h->d_prop_m, 0, sizeof(float) * p.size()));
    CK(h, cudaMemset(h->d_prop_v, 0, sizeof(float) * p.size()));
    h->adam_step = 0;
    h->anchor_prm_ready = false;
    return BZ_OK;
}

extern "C" int bz_proposal_get_params(bz_handle h, float* host)
{
    if (!h || !host || !h->d_prop) return h ? fail(h, BZ_EINVAL, "no proposal network (bz_proposal_init)") : BZ_EINVAL;
    CK(h, cudaDeviceSynchronize());
    CK(h, cudaMemcpy(host, h->d_prop, sizeof(float) * mlp_nparam(), cudaMemcpyDeviceToHost));
    return BZ_OK;
}

extern "C" int bz_proposal_set_params(bz_handle h, const float* host)
{
    if (!h || !host) return BZ_EINVAL;
    int rc = prop_alloc(h);
    if (rc) return rc;
    CK(h, cudaDeviceSynchronize());
    CK(h, cudaMemcpy(h->d_prop, host, sizeof(float) * mlp_nparam(), cudaMemcpyHostToDevice));
    h->anchor_prm_ready = false;
    return BZ_OK;
}

extern "C" int bz_proposal_grad(bz_handle h, const void* records, int64_t n, float* grad, float* loss, void* stream)
{
    if (!h || !records || !grad || !loss || n <= 0) return BZ_EINVAL;
    if (!h->d_prop) return fail(h, BZ_EINVAL, "no proposal network (bz_proposal_init)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const ProposalRecord* rec = static_cast<const ProposalRecord*>(records);
    CK(h, launch_sum_weights(rec, n, h->d_wsum, s));
    double wsum = 0;
    CK(h, cudaMemcpyAsync(&wsum, h->d_wsum, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    if (!(wsum > 0)) return fail(h, BZ_EINVAL, "records carry no weight");
    CK(h, cudaMemsetAsync(grad, 0, sizeof(float) * mlp_nparam(), s));
    CK(h, cudaMemsetAsync(loss, 0, sizeof(float), s));
    CK(h, cudaMemsetAsync(h->d_prop_err, 0, sizeof(int), s));
    CK(h, launch_mlp_grad(h->d_prop, prop_args(h), rec, n, (float)(1.0 / wsum), grad, loss, h->nsm, h->d_prop_part,
                          h->d_loss_part, h->d_prop_err, s));
    int herr = 0;
    CK(h, cudaMemcpyAsync(&herr, h->d_prop_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    if (herr) return fail(h, BZ_ECUDA, "proposal gradient: %d tensor-core waits timed out", herr);
    return BZ_OK;
}

extern "C" int bz_proposal_train(bz_handle h, const void* records, int64_t n, int32_t steps, int32_t batch,
                                 double lr, float* losses_host, void* stream)
{
    if (!h || !records || n <= 0 || steps < 0 || batch <= 0 || !(lr > 0)) return BZ_EINVAL;
    if (!h->d_prop) return fail(h, BZ_EINVAL, "no proposal network (bz_proposal_init)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const ProposalRecord* rec = static_cast<const ProposalRecord*>(records);
    CK(h, launch_sum_weights(rec, n, h->d_wsum, s));
    double wsum = 0;
    CK(h, cudaMemcpyAsync(&wsum, h->d_wsum, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    if (!(wsum > 0)) return fail(h, BZ_EINVAL, "records carry no weight");
    const double wbar = wsum / (double)n;
    const ProposalArgs A = prop_args(h);
    const int np = mlp_nparam();
    CK(h, cudaMemsetAsync(h->d_prop_g, 0, sizeof(float) * np, s));
    // each step's minibatch: b records drawn independently and uniformly from all n
    // (the record buffer is in arrival order, i.e. clustered by anchor)
    CK(h, cudaMemsetAsync(h->d_prop_err, 0, sizeof(int), s));
    for (int k = 0; k < steps; ++k) {
        const int64_t b = batch;
        const uint64_t key = ((uint64_t)(h->adam_step + 1) << 32) * 0x9E3779B97F4A7C15ull;
        CK(h, launch_mlp_grad(h->d_prop, A, rec, b, (float)(1.0 / (wbar * (double)b)), h->d_prop_g, h->d_loss, h->nsm,
                              h->d_prop_part, h->d_loss_part, h->d_prop_err, s, n, key));
        CK(h, launch_adam(h->d_prop, h->d_prop_g, h->d_prop_m, h->d_prop_v, np, (float)lr, ++h->adam_step, s));
        if (losses_host) CK(h, cudaMemcpyAsync(&losses_host[k], h->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    int herr = 0;
    CK(h, cudaMemcpyAsync(&herr, h->d_prop_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    if (herr) return fail(h, BZ_ECUDA, "proposal training: %d tensor-core waits timed out", herr);
    h->anchor_prm_ready = false;
    return BZ_OK;
}

static int anchor_prm_alloc(bz_handle h)
{
    if (!h->d_anchor_prm && !dalloc(&h->d_anchor_prm, 8 * h->ncell))
        return fail(h, BZ_ENOMEM, "cannot allocate the per-anchor proposal parameters");
    return BZ_OK;
}

extern "C" int bz_proposal_infer(bz_handle h, void* stream)
{
    if (!h) return BZ_EINVAL;
    ++h->gen;
    if (!h->d_prop) return fail(h, BZ_EINVAL, "no proposal network (bz_proposal_init)");
    int rc = anchor_prm_alloc(h);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* err = h->d_prop_err;
    CK(h, cudaMemsetAsync(err, 0, sizeof(int), s));
    CK(h, launch_mlp_infer(h->d_prop, prop_args(h), h->ncell, h->d_anchor_prm, h->nsm * 2, err, s));
    int herr = 0;
    CK(h, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    if (herr) return fail(h, BZ_ECUDA, "proposal inference: %d tensor-core waits timed out", herr);
    h->anchor_prm_ready = true;
    return BZ_OK;
}

extern "C" int bz_proposal_anchor_params(bz_handle h, float* out_host, const float* in_host)
{
    if (!h || (!out_host && !in_host)) return BZ_EINVAL;
    ++h->gen;
    int rc = anchor_prm_alloc(h);
    if (rc) return rc;
    CK(h, cudaDeviceSynchronize());
    if (in_host) {
        CK(h, cudaMemcpy(h->d_anchor_prm, in_host, sizeof(float) * 8 * h->ncell, cudaMemcpyHostToDevice));
        h->anchor_prm_ready = true;
    }
    if (out_host) {
        if (!h->anchor_prm_ready) return fail(h, BZ_EINVAL, "no per-anchor proposal parameters yet");
        CK(h, cudaMemcpy(out_host, h->d_anchor_prm, sizeof(float) * 8 * h->ncell, cudaMemcpyDeviceToHost));
    }
    return BZ_OK;
}

extern "C" int bz_set_step_sampler(bz_handle h, int32_t sampler)
{
    if (!h) return BZ_EINVAL;
    ++h->gen;
    if (sampler != BZ_SAMPLER_SYMMETRIC && sampler != BZ_SAMPLER_LEARNED)
        return fail(h, BZ_EINVAL, "bz_step supports the symmetric and learned samplers");
    h->step_sampler = sampler;
    return BZ_OK;
}

extern "C" int bz_record(bz_handle h, const int64_t* state, int32_t nsamples, int32_t step, double dt,
                         int32_t unit_stride, void* records, int64_t max_records, int64_t* n_written, void* stream)
{
    if (!h || !state || !records || max_records <= 0 || unit_stride <= 0) return BZ_EINVAL;
    int rc = check_common(h, nsamples, step, dt, BZ_PREC_F32, BZ_SAMPLER_SYMMETRIC);
    if (rc) return rc;
    if (h->ncell >= (int64_t)1 << 31) return fail(h, BZ_EINVAL, "record mode needs fewer than 2^31 cells");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long* st = reinterpret_cast<const long long*>(state);
    if ((rc = compute_masses(h, st, s))) return rc;
    double deg[NSPEC];
    for (int sl = 0; sl < NSPEC; ++sl) deg[sl] = kDeg[sl < h->nslots ? h->slot_species[sl] : 0];
    CK(h, launch_convert(st, h->d_freal, 0, h->nxc, h->npc, h->nslots, deg, s));
    if (!h->d_qcount && !dalloc(&h->d_qcount, 1)) return fail(h, BZ_ENOMEM, "scratch");
    if (!h->d_rec_count && !dalloc(&h->d_rec_count, 1)) return fail(h, BZ_ENOMEM, "scratch");
    unsigned long long* cnt = h->d_rec_count;
    CK(h, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    const int64_t n_sel = h->a_offset < h->ncell ? (h->ncell - h->a_offset + h->a_stride - 1) / h->a_stride : 0;
    const int64_t units = f32_units(n_sel, nsamples);
    if (units >= ((int64_t)1 << 31)) return fail(h, BZ_EINVAL, "anchors x samples too large for one record call");
    int64_t blocks = (units + F32_WARPS - 1) / F32_WARPS;
    if (blocks > (int64_t)h->nsm * 48) blocks = (int64_t)h->nsm * 48;
    if (blocks < 1) blocks = 1;
    CollideArgs<float> a{};
    fill_collide(h, a, nullptr, nsamples, step, dt, BZ_SAMPLER_SYMMETRIC);
    a.tau = 0.0f;
    a.rec = static_cast<ProposalRecord*>(records);
    a.rec_count = cnt;
    a.rec_cap = max_records;
    a.rec_stride = unit_stride;
    // the kernel writes its per-warp queue counts even with no deferral: give it room
    if ((int64_t)blocks * F32_WARPS > h->q_warps) {
        cudaFree(h->d_qcount);
        h->d_qcount = nullptr;
        if (!dalloc(&h->d_qcount, blocks * F32_WARPS)) return fail(h, BZ_ENOMEM, "scratch");
        h->q_warps = blocks * F32_WARPS;
        if (!h->d_qitems && !dalloc(&h->d_qitems, 1)) return fail(h, BZ_ENOMEM, "scratch");
    }
    a.qcount = h->d_qcount;
    a.qitems = h->d_qitems;
    a.qcap = 0;
    CK(h, launch_collide_f32(a, (int)blocks, nullptr, s));
    unsigned long long n = 0;
    CK(h, cudaMemcpyAsync(&n, cnt, sizeof(n), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    const int64_t nw = (int64_t)(n < (unsigned long long)max_records ? n : (unsigned long long)max_records);
    // a fixed order (warps append in arrival order); when the buffer overflowed
    // the set of kept records itself depends on that order
    CK(h, launch_sort_records(static_cast<ProposalRecord*>(records), nw, s));
    if (n_written) *n_written = nw;
    return BZ_OK;
}
