// Collision kernels, templated on the integrand precision R (double: the
// FP64 path, compiled without FMA contraction so every operation matches
// the written formula order; float: the FP32 path).
//
// One thread evaluates one (anchor, sample): anchor = (species d, x cell,
// p cell).  Eqs. (MC C_gg), (ca): the sample draws the jitter of p inside
// its cell and (k1x, k1y, k3) uniformly in [-L, L)^5 from Philox4x32-10;
// for every term of d's equation, Eqs. (C_gluon)/(C_quark), the k1z roots
// of E1 + E2 = E3 + Ep (Eqs. work out delta E, delta replace) give k1 and
// k2 = p + k3 - k1; each valid root inside the box contributes
//   c~ = sym W |M|^2 / (|J| (2 pi)^5 16 E1 E2 E3 Ep)
// and, with symmetrical sampling (Eq. small c relation), the integer
// q = rint(c~ K) goes +q to (d, p) and (c, k3) and -q to (a, k1), (b, k2).
// The +q of the anchor cell is summed in registers and over the warp
// (exact int64), the other legs use 64-bit global reductions.
//
// FP32 conditioning: near the tangency of the k1_perp line to the energy
// ellipsoid the discriminant H = kappa^2 - a^2 D is a small difference of
// O(E^4) numbers and the integrand goes like 1/sqrt(H), so FP32 rounding
// of the inputs alone gives O(eps kappa^2 / H) relative error.  The FP32
// kernel therefore queues every term with |H| < tau kappa^2 (about 0.3% of
// the in-box terms at tau = 2e-3) and k_fixup_f32 redoes their sample point
// and root solve in float-float arithmetic (about 48 bits) from the same
// Philox counter; deposits are still exact integers.
#pragma once
#include <cstdint>
#include "bz_internal.h"

namespace bz {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same rounds with the keys taken from a schedule (philox_key_schedule).
__device__ __forceinline__ uint4 philox4x32_10_ks(uint4 c, const uint32_t* ks)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ ks[2 * r], lo1, hi0 ^ c.w ^ ks[2 * r + 1], lo0);
    }
    return c;
}

// Philox4x32-10 over a family of counters (c0, cy, cz, cw) that share
// (cy, cz, cw) -- the samples of one anchor: in the first round the product
// of cz, and in the second the product of the first round's x word
// mulhi(M1, cz) ^ cy ^ k0, do not depend on c0.  philox_head computes them
// once for the family, folded with the key words they meet; philox_tail_*
// finishes one counter.  The rounds and the words are those of
// philox4x32_10.  Head words: (cw ^ k1 of round 1, lo(M1 cz) ^ k0 of round 2,
// hi(M0 x1) ^ k1 of round 2, lo(M0 x1)).
__device__ __forceinline__ uint4 philox_head(uint32_t cy, uint32_t cz, uint32_t cw, uint32_t k0a, uint32_t k1a,
                                             uint32_t k0b, uint32_t k1b)
{
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, cz), lo1 = 0xCD9E8D57u * cz;
    const uint32_t x1 = hi1 ^ cy ^ k0a;
    return make_uint4(cw ^ k1a, lo1 ^ k0b, __umulhi(0xD2511F53u, x1) ^ k1b, 0xD2511F53u * x1);
}

// Rounds 1 and 2 of counter c0 from the head, rounds 3..10 in full.
__device__ __forceinline__ uint4 philox_tail_first2(uint32_t c0, uint4 h)
{
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t z1 = hi0 ^ h.x;
    return make_uint4(__umulhi(0xCD9E8D57u, z1) ^ h.y, 0xCD9E8D57u * z1, h.z ^ lo0, h.w);
}

// The key words of every round from a schedule (philox_key_schedule).
__device__ __forceinline__ uint4 philox_tail_ks(uint32_t c0, uint4 h, const uint32_t* ks)
{
    uint4 c = philox_tail_first2(c0, h);
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ ks[2 * r], lo1, hi0 ^ c.w ^ ks[2 * r + 1], lo0);
    }
    return c;
}

// The key words bumped round by round from the key (k0, k1) of round 1.
__device__ __forceinline__ uint4 philox_tail(uint32_t c0, uint4 h, uint32_t k0, uint32_t k1)
{
    uint4 c = philox_tail_first2(c0, h);
    k0 += 2u * 0x9E3779B9u;
    k1 += 2u * 0xBB67AE85u;
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

template <typename R> struct Ops;
template <> struct Ops<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double floor_(double x) { return floor(x); }
    static __device__ __forceinline__ double fabs_(double x) { return fabs(x); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ long long rint_(double x) { return __double2ll_rn(x); }
    // u = (x + 1/2) 2^-32, or ((x >> 9) + 1/2) 2^-23 when re-evaluating FP32 samples
    static __device__ __forceinline__ double unif(uint32_t x, int ubits)
    {
        return ubits == 23 ? ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0) : ((double)x + 0.5) * (1.0 / 4294967296.0);
    }
    static constexpr double LIM = 4611686018427387904.0;  // 2^62
};
template <> struct Ops<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
    static __device__ __forceinline__ float fabs_(float x) { return fabsf(x); }
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    static __device__ __forceinline__ long long rint_(float x) { return __float2ll_rn(x); }
    // u = ((x >> 9) + 1/2) 2^-23, exact in FP32
    static __device__ __forceinline__ float unif(uint32_t x, int) { return ((float)(x >> 9) + 0.5f) * (1.0f / 8388608.0f); }
    static constexpr float LIM = 4611686018427387904.0f;
};

template <typename R>
__device__ __forceinline__ int bin_of(R k, R L, R dp, int n)
{
    int j = (int)Ops<R>::floor_((k + L) / dp);
    j = j < 0 ? 0 : j;
    return j >= n ? n - 1 : j;
}

template <typename R>
__device__ __forceinline__ bool in_box(R k, R L) { return k >= -L && k < L; }

// A user-defined row: terms in order, each power a product of its factors
// from 1 left to right.
template <typename R>
__device__ __forceinline__ R upow(R x, int n)
{
    R r = R(1);
    for (int i = 0; i < n; ++i) r = r * x;
    return r;
}

template <typename R>
__device__ __forceinline__ R msq_user(const UserRow* row, R s, R t, R u, R mg2)
{
    const R tm = t - mg2, um = u - mg2;
    R acc = R(0);
    const int n = row->n;
    for (int k = 0; k < n; ++k) {
        const UserTerm& T = row->t[k];
        const R num = (upow(s, T.e[0]) * upow(t, T.e[1])) * upow(u, T.e[2]);
        const R den = (upow(s, T.e[3]) * upow(tm, T.e[4])) * upow(um, T.e[5]);
        const R c = sizeof(R) == sizeof(double) ? (R)T.coef : (R)T.coef32;
        acc = acc + c * (num / den);
    }
    return acc;
}

template <typename R>
__device__ __forceinline__ R msq(int cls, const CollideArgs<R>& P, R s, R t, R u, R mg2)
{
    if ((P.umask >> cls) & 1u) return msq_user<R>(P.urows + cls, s, t, u, mg2);
    R tm = t - mg2, um = u - mg2;
    switch (cls) {
    case M_QQP:
        return P.A1 * ((s * s + u * u) / (tm * tm));
    case M_QQ:
        return P.A1 * ((s * s + u * u) / (tm * tm) + (s * s + t * t) / (um * um))
               + P.A2 * ((s * s) / (tm * um));
    case M_QQB:
        return P.A1 * ((s * s + u * u) / (tm * tm) + (u * u + t * t) / (s * s))
               + P.A2 * ((u * u) / (tm * s));
    case M_QQB2:
        return P.A1 * ((t * t + u * u) / (s * s));
    case M_QQBGG:
        return P.A3 * (u / tm + t / um) - P.A4 * ((t * t + u * u) / (s * s));
    case M_QG:
        return P.A4 * ((s * s + u * u) / (tm * tm)) - P.A3 * (u / s + s / um);
    default:  // M_GG
        return P.A5 * (R(3) - (s * u) / (tm * tm) - (s * t) / (um * um) - (t * u) / (s * s));
    }
}

template <typename R>
__device__ __forceinline__ R f_equilibrium(const CollideArgs<R>& P, int s, R E)
{
    R x = (E - P.mu[s]) / P.T;
    return is_quark(s) ? R(1) / (Ops<R>::exp_(x) + R(1)) : R(1) / (Ops<R>::exp_(x) - R(1));
}

template <typename R>
__device__ __forceinline__ R load_f(const CollideArgs<R>& P, int64_t i)
{
    return P.f_is_float ? (R)__ldg(static_cast<const float*>(P.f) + i)
                        : (R)__ldg(static_cast<const double*>(P.f) + i);
}

__device__ __forceinline__ void red_add(long long* addr, long long v)
{
    atomicAdd(reinterpret_cast<unsigned long long*>(addr), static_cast<unsigned long long>(v));
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Everything of one sample that does not depend on the term.
template <typename R>
struct Geom {
    int64_t x, xoff, lin3;
    int d;
    R p[3], k3[3], k1x, k1y, pp, kk3, Pz, PP, bx, by, a2m, b2m;
    bool k2xy_in;
    R mdisp[4], mg2;
R wfac;  // learned sampler: 1/(32 q(y)), else 1
};

template <typename R>
__device__ __forceinline__ void make_geom(const CollideArgs<R>& P, int64_t a, int smp, Geom<R>& G, int step)
{
    using O = Ops<R>;
    const R L = P.L, twoL = P.twoL;
    const int64_t nxc = P.nxc, npc = P.npc;
    const int sl = (int)(a / (nxc * npc));
    const int64_t x = (a / npc) % nxc;
    const int64_t j = a % npc;
    G.x = x;
    G.xoff = x * npc;
    G.d = P.slot_species[sl];
    const int jv[3] = {(int)(j / ((int64_t)P.np[1] * P.np[2])), (int)((j / P.np[2]) % P.np[1]), (int)(j % P.np[2])};
    const uint32_t ctr3 = ((uint32_t)step << 3) | (uint32_t)G.d;
    const uint4 r0 = philox4x32_10(make_uint4(2u * smp, (uint32_t)j, (uint32_t)x, ctr3), P.key0, P.key1);
    const uint4 r1 = philox4x32_10(make_uint4(2u * smp + 1u, (uint32_t)j, (uint32_t)x, ctr3), P.key0, P.key1);
    const R u[8] = {O::unif(r0.x, P.ubits), O::unif(r0.y, P.ubits), O::unif(r0.z, P.ubits), O::unif(r0.w, P.ubits),
                    O::unif(r1.x, P.ubits), O::unif(r1.y, P.ubits), O::unif(r1.z, P.ubits), O::unif(r1.w, P.ubits)};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const R pc = -L + ((R)jv[i] + R(0.5)) * P.dp[i];
        G.p[i] = P.p_center ? pc : pc + P.dp[i] * (u[i] - R(0.5));
    }
    G.wfac = R(1);
    if (P.sampler == SAMPLER_LEARNED) {
        // defensive mixture of the uniform density and truncated Student-t densities with two
        // degrees of freedom (per-anchor parameters): F(z) = 1/2 + z / (2 sqrt(2 + z^2)), so the
        // inverse CDF and the density need square roots only
        const uint4 r2 = philox4x32_10(make_uint4(0x80000000u | (uint32_t)smp, (uint32_t)j, (uint32_t)x, ctr3), P.key0,
                                       P.key1);
        R prm[6];
        for (int i = 0; i < 6; ++i) prm[i] = (R)P.prop[a * 8 + i];
        const bool uni = O::unif(r2.x, P.ubits) < prm[5];
        R y[5], Gd = R(1);
        auto tail = [](R z) {  // F(-|z|)
            const R r = O::sqrt_(R(2) + z * z);
            return R(1) / (r * (r + O::fabs_(z)));
        };
        for (int i = 0; i < 5; ++i) {
            const R mu = i < 2 ? R(0) : prm[i - 2];
            const R sg = i < 2 ? prm[4] : prm[3];
            const R Fa = tail((R(-1) - mu) / sg), cFb = tail((R(1) - mu) / sg);
            const R D = (R(1) - cFb) - Fa;
            if (uni) {
                y[i] = R(2) * u[3 + i] - R(1);
                const R z = (y[i] - mu) / sg;
                const R r = O::sqrt_(R(2) + z * z);
                Gd *= R(1) / (r * r * r * sg * D);
            } else {
                const R v = Fa + u[3 + i] * D, cv = cFb + (R(1) - u[3 + i]) * D;
                const R t = R(2) * v * cv;
                y[i] = mu + sg * ((v - cv) / O::sqrt_(t));
                y[i] = y[i] < R(-1) ? R(-1) : (y[i] >= R(1) ? R(0.99999994) : y[i]);
                Gd *= t * O::sqrt_(t) / (sg * D);
            }
        }
        G.wfac = R(1) / (R(32) * (prm[5] * (R(1) / R(32)) + (R(1) - prm[5]) * Gd));
        G.k1x = L * y[0];
        G.k1y = L * y[1];
        for (int i = 0; i < 3; ++i) G.k3[i] = L * y[2 + i];
    } else {
        G.k1x = -L + twoL * u[3];
        G.k1y = -L + twoL * u[4];
#pragma unroll
        for (int i = 0; i < 3; ++i) G.k3[i] = -L + twoL * u[5 + i];
    }
    G.pp = (G.p[0] * G.p[0] + G.p[1] * G.p[1]) + G.p[2] * G.p[2];
    G.kk3 = (G.k3[0] * G.k3[0] + G.k3[1] * G.k3[1]) + G.k3[2] * G.k3[2];
    G.lin3 = ((int64_t)bin_of(G.k3[0], L, P.dp[0], P.np[0]) * P.np[1] + bin_of(G.k3[1], L, P.dp[1], P.np[1])) * P.np[2]
             + bin_of(G.k3[2], L, P.dp[2], P.np[2]);
    const R Px = G.p[0] + G.k3[0], Py = G.p[1] + G.k3[1];
    G.Pz = G.p[2] + G.k3[2];
    G.PP = (Px * Px + Py * Py) + G.Pz * G.Pz;
    G.bx = Px - G.k1x;
    G.by = Py - G.k1y;
    G.a2m = G.k1x * G.k1x + G.k1y * G.k1y;
    G.b2m = G.bx * G.bx + G.by * G.by;
    G.k2xy_in = in_box(G.bx, L) && in_box(G.by, L);
#pragma unroll
    for (int i = 0; i < 4; ++i) G.mdisp[i] = P.mass_mode == 1 ? R(0) : (R)P.m2[x * 4 + i];
    G.mg2 = (R)P.m2[x * 4 + 0];
}

// Per-warp queue of deferred (anchor, sample, term) items (FP32 path).
struct DeferCtx {
    int* s_count;          // this warp's counter in shared memory
    unsigned long long* seg;
    int cap;
};

// Evaluates term ti of sample (a, smp); deposits the k1, k2, k3 legs and
// returns the anchor cell's +q.
template <typename R>
__device__ __forceinline__ long long eval_term(const CollideArgs<R>& P, const Geom<R>& G, int64_t a, int smp, int ti)
{
    using O = Ops<R>;
    const R L = P.L;
    const int64_t nxc = P.nxc, npc = P.npc;
    const TermDev& T = P.terms[G.d][ti];
    const R ma2 = G.mdisp[T.mslot[0]], mb2 = G.mdisp[T.mslot[1]];
    const R mc2 = G.mdisp[T.mslot[2]], md2 = G.mdisp[T.mslot[3]];
    const R Ep = O::sqrt_(G.pp + md2);
    const R E3 = O::sqrt_(G.kk3 + mc2);
    // k1z roots, stable quadratic
    const R E = Ep + E3;
    const R Pz = G.Pz;
    const R a2 = G.a2m + ma2;
    const R b2 = G.b2m + mb2;
    const R D = E * E - Pz * Pz;
    const R kap = (E * E + a2 - b2 - Pz * Pz) * R(0.5);
    const R H = kap * kap - a2 * D;
    if (H < R(0) || D <= R(0)) return 0;
    if (!G.k2xy_in) return 0;
    const R kp = kap * Pz;
    const R sq = E * O::sqrt_(H);
    const R Q = kp >= R(0) ? kp + sq : kp - sq;
    if (Q == R(0)) return 0;
    R zc[2];
    zc[0] = Q / D;
    zc[1] = (E * E * a2 - kap * kap) / Q;
    long long own = 0;
#pragma unroll
    for (int ri = 0; ri < 2; ++ri) {
        const R z = zc[ri];
        const R e1 = (kap + Pz * z) / E;
        if (!(e1 > R(0) && e1 < E)) continue;
        const R E1 = O::sqrt_(a2 + z * z);
        const R dz = Pz - z;
        const R E2 = O::sqrt_(b2 + dz * dz);
        const R J = z / E1 - dz / E2;
        if (J == R(0)) continue;
        if (!in_box(z, L) || !in_box(dz, L)) continue;
        const R s = E * E - G.PP;
        const R k1k3 = (G.k1x * G.k3[0] + G.k1y * G.k3[1]) + z * G.k3[2];
        const R k1p = (G.k1x * G.p[0] + G.k1y * G.p[1]) + z * G.p[2];
        const R t = (ma2 + mc2) - R(2) * (E1 * E3 - k1k3);
        const R uu = (ma2 + md2) - R(2) * (E1 * Ep - k1p);
        const R mg2 = G.mg2;
        if (s <= R(0) || t - mg2 >= R(0) || uu - mg2 >= R(0)) {
            red_add(&P.flags[0], 1);
            continue;
        }
        const R M2 = msq<R>(T.cls, P, s, t, uu, mg2);
        const int64_t lin1 = ((int64_t)bin_of(G.k1x, L, P.dp[0], P.np[0]) * P.np[1] + bin_of(G.k1y, L, P.dp[1], P.np[1]))
                                 * P.np[2]
                             + bin_of(z, L, P.dp[2], P.np[2]);
        const int64_t lin2 = ((int64_t)bin_of(G.bx, L, P.dp[0], P.np[0]) * P.np[1] + bin_of(G.by, L, P.dp[1], P.np[1]))
                                 * P.np[2]
                             + bin_of(dz, L, P.dp[2], P.np[2]);
        const int64_t i1 = (int64_t)T.slot[0] * nxc * npc + G.xoff + lin1;
        const int64_t i2 = (int64_t)T.slot[1] * nxc * npc + G.xoff + lin2;
        const int64_t i3 = (int64_t)T.slot[2] * nxc * npc + G.xoff + G.lin3;
        if (!(bz_in(i1, P.ncell) & bz_in(i2, P.ncell) & bz_in(i3, P.ncell) & bz_in(a, P.ncell))) continue;
        R f1, f2, f3, fp;
        if (P.analytic) {
            f1 = f_equilibrium(P, P.slot_species[T.slot[0]], E1);
            f2 = f_equilibrium(P, P.slot_species[T.slot[1]], E2);
            f3 = f_equilibrium(P, P.slot_species[T.slot[2]], E3);
            fp = f_equilibrium(P, P.slot_species[T.slot[3]], Ep);
        } else {
            f1 = load_f(P, i1);
            f2 = load_f(P, i2);
            f3 = load_f(P, i3);
            fp = load_f(P, a);
        }
        const R F1 = T.quark[0] ? R(1) - f1 : R(1) + f1;
        const R F2 = T.quark[1] ? R(1) - f2 : R(1) + f2;
        const R F3 = T.quark[2] ? R(1) - f3 : R(1) + f3;
        const R Fp = T.quark[3] ? R(1) - fp : R(1) + fp;
        const R gain = f1 * f2 * F3 * Fp;
        const R W = gain - F1 * F2 * f3 * fp;
        const R den = O::fabs_(J) * P.twopi5 * R(16) * E1 * E2 * E3 * Ep;
        const R ct = (R)T.sym * W * M2 / den;
        const R wq = P.sampler == SAMPLER_LEARNED ? ct * P.Kown * G.wfac : ct * P.Kown;
        if (!(O::fabs_(wq) < O::LIM)) {
            red_add(&P.flags[1], 1);
            continue;
        }
        if (P.audit) {  // continuous-leg energy / momentum balance of this deposit set
            const double w = (double)(ct * P.Kq * (P.sampler == SAMPLER_LEARNED ? G.wfac : R(1)));
            atomicAdd(&P.audit[0], w * (double)((Ep + E3) - (E1 + E2)));
            atomicAdd(&P.audit[1], w * (double)((G.p[0] + G.k3[0]) - (G.k1x + G.bx)));
            atomicAdd(&P.audit[2], w * (double)((G.p[1] + G.k3[1]) - (G.k1y + G.by)));
            atomicAdd(&P.audit[3], w * (double)((G.p[2] + G.k3[2]) - (z + dz)));
            atomicAdd(&P.audit[4], fabs(w) * (double)(Ep + E3 + E1 + E2));
            atomicAdd(&P.audit[5], 1.0);
            atomicAdd(&P.audit[6], fabs(w));
        }
        const long long q = O::rint_(wq);
        if (q == 0) continue;
        own += q;
        if (P.sampler != 1) {
            red_add(&P.A[i3], q);
            red_add(&P.A[i1], -q);
            red_add(&P.A[i2], -q);
        }
    }
    return own;
}

// The second parameterisation of Sec. III.A (param 1): k3 = k1 + k2 - p
// eliminated, (k1_perp, k2) sampled (G.k3 and G.kk3 hold k2 and |k2|^2).
// E1 - E3 = Ep - E2 = dl squared twice gives (K^2 - dl^2) z^2
// - K (A0 + 2 dl^2) z + A0^2/4 - dl^2 (c2 + K^2) = 0, K = k2z - pz,
// A0 = a2 - c2 - K^2 - dl^2; a root is one of the original equation iff
// A0 - 2 K z has the sign of dl and E3 + dl > 0; |J| = |z/E1 - (z + K)/E3|.
// Deposits, weights and flags as eval_term.  FP64 only.
template <typename R>
__device__ __forceinline__ long long eval_term_k3(const CollideArgs<R>& P, const Geom<R>& G, int64_t a, int ti)
{
    using O = Ops<R>;
    const R L = P.L;
    const int64_t nxc = P.nxc, npc = P.npc;
    const TermDev& T = P.terms[G.d][ti];
    const R ma2 = G.mdisp[T.mslot[0]], mb2 = G.mdisp[T.mslot[1]];
    const R mc2 = G.mdisp[T.mslot[2]], md2 = G.mdisp[T.mslot[3]];
    const R* k2 = G.k3;
    const R Ep = O::sqrt_(G.pp + md2);
    const R E2 = O::sqrt_(G.kk3 + mb2);
    const R k1x = G.k1x, k1y = G.k1y;
    const R cx = (k1x + k2[0]) - G.p[0], cy = (k1y + k2[1]) - G.p[1], K = k2[2] - G.p[2];
    const R a2 = G.a2m + ma2;
    const R c2 = (cx * cx + cy * cy) + mc2;
    const R dl = Ep - E2;
    const R A0 = ((a2 - c2) - K * K) - dl * dl;
    const R qa = K * K - dl * dl;
    const R qb = -K * (A0 + R(2) * dl * dl);
    const R qc = R(0.25) * A0 * A0 - dl * dl * (c2 + K * K);
    if (qa == R(0) || dl == R(0)) return 0;
    const R disc = qb * qb - R(4) * qa * qc;
    if (disc < R(0)) return 0;
    const R sq = O::sqrt_(disc);
    const R Q = R(-0.5) * (qb >= R(0) ? qb + sq : qb - sq);
    if (Q == R(0)) return 0;
    R zc[2];
    zc[0] = Q / qa;
    zc[1] = qc / Q;
    const int64_t lin2 = ((int64_t)bin_of(k2[0], L, P.dp[0], P.np[0]) * P.np[1] + bin_of(k2[1], L, P.dp[1], P.np[1]))
                             * P.np[2]
                         + bin_of(k2[2], L, P.dp[2], P.np[2]);
    long long own = 0;
#pragma unroll
    for (int ri = 0; ri < 2; ++ri) {
        const R z = zc[ri];
        const R w = A0 - R(2) * K * z;
        if (!(dl > R(0) ? w > R(0) : w < R(0))) continue;
        const R zk = z + K;
        const R E3 = O::sqrt_(c2 + zk * zk);
        if (!(E3 + dl > R(0))) continue;
        const R E1 = O::sqrt_(a2 + z * z);
        const R J = z / E1 - zk / E3;
        if (J == R(0)) continue;
        const R k3[3] = {cx, cy, z + (k2[2] - G.p[2])};
        if (!in_box(z, L) || !in_box(k3[0], L) || !in_box(k3[1], L) || !in_box(k3[2], L)) continue;
        const R E = Ep + E3;
        const R PP = ((G.p[0] + k3[0]) * (G.p[0] + k3[0]) + (G.p[1] + k3[1]) * (G.p[1] + k3[1]))
                     + (G.p[2] + k3[2]) * (G.p[2] + k3[2]);
        const R s = E * E - PP;
        const R k1k3 = (k1x * k3[0] + k1y * k3[1]) + z * k3[2];
        const R k1p = (k1x * G.p[0] + k1y * G.p[1]) + z * G.p[2];
        const R t = (ma2 + mc2) - R(2) * (E1 * E3 - k1k3);
        const R uu = (ma2 + md2) - R(2) * (E1 * Ep - k1p);
        const R mg2 = G.mg2;
        if (s <= R(0) || t - mg2 >= R(0) || uu - mg2 >= R(0)) {
            red_add(&P.flags[0], 1);
            continue;
        }
        const R M2 = msq<R>(T.cls, P, s, t, uu, mg2);
        const int64_t lin1 = ((int64_t)bin_of(k1x, L, P.dp[0], P.np[0]) * P.np[1] + bin_of(k1y, L, P.dp[1], P.np[1]))
                                 * P.np[2]
                             + bin_of(z, L, P.dp[2], P.np[2]);
        const int64_t lin3 = ((int64_t)bin_of(k3[0], L, P.dp[0], P.np[0]) * P.np[1] + bin_of(k3[1], L, P.dp[1], P.np[1]))
                                 * P.np[2]
                             + bin_of(k3[2], L, P.dp[2], P.np[2]);
        const int64_t i1 = (int64_t)T.slot[0] * nxc * npc + G.xoff + lin1;
        const int64_t i2 = (int64_t)T.slot[1] * nxc * npc + G.xoff + lin2;
        const int64_t i3 = (int64_t)T.slot[2] * nxc * npc + G.xoff + lin3;
        if (!(bz_in(i1, P.ncell) & bz_in(i2, P.ncell) & bz_in(i3, P.ncell) & bz_in(a, P.ncell))) continue;
        R f1, f2, f3, fp;
        if (P.analytic) {
            f1 = f_equilibrium(P, P.slot_species[T.slot[0]], E1);
            f2 = f_equilibrium(P, P.slot_species[T.slot[1]], E2);
            f3 = f_equilibrium(P, P.slot_species[T.slot[2]], E3);
            fp = f_equilibrium(P, P.slot_species[T.slot[3]], Ep);
        } else {
            f1 = load_f(P, i1);
            f2 = load_f(P, i2);
            f3 = load_f(P, i3);
            fp = load_f(P, a);
        }
        const R F1 = T.quark[0] ? R(1) - f1 : R(1) + f1;
        const R F2 = T.quark[1] ? R(1) - f2 : R(1) + f2;
        const R F3 = T.quark[2] ? R(1) - f3 : R(1) + f3;
        const R Fp = T.quark[3] ? R(1) - fp : R(1) + fp;
        const R gain = f1 * f2 * F3 * Fp;
        const R W = gain - F1 * F2 * f3 * fp;
        const R den = O::fabs_(J) * P.twopi5 * R(16) * E1 * E2 * E3 * Ep;
        const R ct = (R)T.sym * W * M2 / den;
        const R wq = ct * P.Kown;
        if (!(O::fabs_(wq) < O::LIM)) {
            red_add(&P.flags[1], 1);
            continue;
        }
        if (P.audit) {
            const double wa = (double)(ct * P.Kq);
            atomicAdd(&P.audit[0], wa * (double)((Ep + E3) - (E1 + E2)));
            atomicAdd(&P.audit[1], wa * (double)((G.p[0] + k3[0]) - (k1x + k2[0])));
            atomicAdd(&P.audit[2], wa * (double)((G.p[1] + k3[1]) - (k1y + k2[1])));
            atomicAdd(&P.audit[3], wa * (double)((G.p[2] + k3[2]) - (z + k2[2])));
            atomicAdd(&P.audit[4], fabs(wa) * (double)(Ep + E3 + E1 + E2));
            atomicAdd(&P.audit[5], 1.0);
            atomicAdd(&P.audit[6], fabs(wa));
        }
        const long long q = O::rint_(wq);
        if (q == 0) continue;
        own += q;
        if (P.sampler != 1) {
            red_add(&P.A[i3], q);
            red_add(&P.A[i1], -q);
            red_add(&P.A[i2], -q);
        }
    }
    return own;
}

// FP64 kernel: grid-stride over (anchor, sample) items, 32 consecutive items
// per warp.
template <typename R>
__global__ void __launch_bounds__(256) k_collide(const __grid_constant__ CollideArgs<R> P)
{
    const int64_t total = P.n_sel * (int64_t)P.nsamples;
    const int lane = threadIdx.x & 31;
    const bool warp_anchor = (P.nsamples & 31) == 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
        const int64_t item = base + lane;
        long long own = 0;
        int64_t a = 0;
        if (item < total) {
            const int64_t al = item / P.nsamples;
            const int smp = (int)(item - al * P.nsamples);
            a = P.a_offset + al * P.a_stride;
            Geom<R> G;
            make_geom(P, a, smp, G, P.step);
            const int nt = P.nterms[G.d];
            if (P.param == 1)
                for (int ti = 0; ti < nt; ++ti) own += eval_term_k3<R>(P, G, a, ti);
            else
                for (int ti = 0; ti < nt; ++ti) own += eval_term<R>(P, G, a, smp, ti);
        }
        if (warp_anchor) {
            own = warp_sum_ll(own);
            if (lane == 0 && own != 0 && bz_in(a, P.ncell)) red_add(&P.A[a], own);
        } else if (own != 0 && bz_in(a, P.ncell)) {
            red_add(&P.A[a], own);
        }
    }
}



}  // namespace bz
