// Collision kernel, templated on the integrand precision R (double: the
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

template <typename R> struct Ops;
template <> struct Ops<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double floor_(double x) { return floor(x); }
    static __device__ __forceinline__ double fabs_(double x) { return fabs(x); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ long long rint_(double x) { return __double2ll_rn(x); }
    // u = (x + 1/2) 2^-32
    static __device__ __forceinline__ double unif(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }
    static constexpr double LIM = 4611686018427387904.0;  // 2^62
};
template <> struct Ops<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
    static __device__ __forceinline__ float fabs_(float x) { return fabsf(x); }
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    static __device__ __forceinline__ long long rint_(float x) { return __float2ll_rn(x); }
    // u = ((x >> 9) + 1/2) 2^-23, exact in FP32
    static __device__ __forceinline__ float unif(uint32_t x) { return ((float)(x >> 9) + 0.5f) * (1.0f / 8388608.0f); }
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

template <typename R>
__device__ __forceinline__ R msq(int cls, const CollideArgs<R>& P, R s, R t, R u, R mg2)
{
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

template <typename R>
__global__ void __launch_bounds__(256) k_collide(const __grid_constant__ CollideArgs<R> P)
{
    using O = Ops<R>;
    const int64_t total = P.n_sel * (int64_t)P.nsamples;
    const int lane = threadIdx.x & 31;
    const bool warp_anchor = (P.nsamples & 31) == 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const R L = P.L, twoL = P.twoL;
    const int64_t nxc = P.nxc, npc = P.npc;

    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total;
         base += stride) {
        const int64_t item = base + lane;
        long long own = 0;
        int64_t own_idx = 0;
        if (item < total) {
            const int64_t al = item / P.nsamples;
            const int smp = (int)(item - al * P.nsamples);
            const int64_t a = P.a_offset + al * P.a_stride;
            const int sl = (int)(a / (nxc * npc));
            const int64_t x = (a / npc) % nxc;
            const int64_t j = a % npc;
            const int d = P.slot_species[sl];
            const int jv[3] = {(int)(j / ((int64_t)P.np[1] * P.np[2])), (int)((j / P.np[2]) % P.np[1]),
                               (int)(j % P.np[2])};
            own_idx = a;

            uint32_t ctr3 = ((uint32_t)P.step << 3) | (uint32_t)d;
            uint4 r0 = philox4x32_10(make_uint4(2u * smp, (uint32_t)j, (uint32_t)x, ctr3), P.key0, P.key1);
            uint4 r1 = philox4x32_10(make_uint4(2u * smp + 1u, (uint32_t)j, (uint32_t)x, ctr3), P.key0, P.key1);
            R u[8] = {O::unif(r0.x), O::unif(r0.y), O::unif(r0.z), O::unif(r0.w),
                      O::unif(r1.x), O::unif(r1.y), O::unif(r1.z), O::unif(r1.w)};
            R p[3], k3[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                R pc = -L + ((R)jv[i] + R(0.5)) * P.dp[i];
                p[i] = P.p_center ? pc : pc + P.dp[i] * (u[i] - R(0.5));
            }
            const R k1x = -L + twoL * u[3];
            const R k1y = -L + twoL * u[4];
#pragma unroll
            for (int i = 0; i < 3; ++i) k3[i] = -L + twoL * u[5 + i];
            const R pp = (p[0] * p[0] + p[1] * p[1]) + p[2] * p[2];
            const R kk3 = (k3[0] * k3[0] + k3[1] * k3[1]) + k3[2] * k3[2];
            const int64_t lin3 = ((int64_t)bin_of(k3[0], L, P.dp[0], P.np[0]) * P.np[1]
                                  + bin_of(k3[1], L, P.dp[1], P.np[1])) * P.np[2]
                                 + bin_of(k3[2], L, P.dp[2], P.np[2]);
            const R Px = p[0] + k3[0], Py = p[1] + k3[1], Pz = p[2] + k3[2];
            const R PP = (Px * Px + Py * Py) + Pz * Pz;
            const R bx = Px - k1x, by = Py - k1y;
            const R a2m = k1x * k1x + k1y * k1y;
            const R b2m = bx * bx + by * by;
            const bool k2xy_in = in_box(bx, L) && in_box(by, L);

            R mdisp[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) mdisp[i] = P.mass_mode == 1 ? R(0) : (R)P.m2[x * 4 + i];
            const R mg2 = (R)P.m2[x * 4 + 0];
            const int64_t xoff = x * npc;

            const int nt = P.nterms[d];
            for (int ti = 0; ti < nt; ++ti) {
                const TermDev& T = P.terms[d][ti];
                const R ma2 = mdisp[T.mslot[0]], mb2 = mdisp[T.mslot[1]];
                const R mc2 = mdisp[T.mslot[2]], md2 = mdisp[T.mslot[3]];
                const R Ep = O::sqrt_(pp + md2);
                const R E3 = O::sqrt_(kk3 + mc2);
                // k1z roots, stable quadratic
                const R E = Ep + E3;
                const R a2 = a2m + ma2;
                const R b2 = b2m + mb2;
                const R D = E * E - Pz * Pz;
                const R kap = (E * E + a2 - b2 - Pz * Pz) * R(0.5);
                const R H = kap * kap - a2 * D;
                if (H < R(0) || D <= R(0)) continue;
                if (!k2xy_in) continue;
                const R kp = kap * Pz;
                const R sq = E * O::sqrt_(H);
                const R Q = kp >= R(0) ? kp + sq : kp - sq;
                if (Q == R(0)) continue;
                R zc[2];
                zc[0] = Q / D;
                zc[1] = (E * E * a2 - kap * kap) / Q;
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
                    const R s = E * E - PP;
                    const R k1k3 = (k1x * k3[0] + k1y * k3[1]) + z * k3[2];
                    const R k1p = (k1x * p[0] + k1y * p[1]) + z * p[2];
                    const R t = (ma2 + mc2) - R(2) * (E1 * E3 - k1k3);
                    const R uu = (ma2 + md2) - R(2) * (E1 * Ep - k1p);
                    if (s <= R(0) || t - mg2 >= R(0) || uu - mg2 >= R(0)) {
                        red_add(&P.flags[0], 1);
                        continue;
                    }
                    const R M2 = msq<R>(T.cls, P, s, t, uu, mg2);
                    const int64_t lin1 = ((int64_t)bin_of(k1x, L, P.dp[0], P.np[0]) * P.np[1]
                                          + bin_of(k1y, L, P.dp[1], P.np[1])) * P.np[2]
                                         + bin_of(z, L, P.dp[2], P.np[2]);
                    const int64_t lin2 = ((int64_t)bin_of(bx, L, P.dp[0], P.np[0]) * P.np[1]
                                          + bin_of(by, L, P.dp[1], P.np[1])) * P.np[2]
                                         + bin_of(dz, L, P.dp[2], P.np[2]);
                    const int64_t i1 = (int64_t)T.slot[0] * nxc * npc + xoff + lin1;
                    const int64_t i2 = (int64_t)T.slot[1] * nxc * npc + xoff + lin2;
                    const int64_t i3 = (int64_t)T.slot[2] * nxc * npc + xoff + lin3;
                    R f1, f2, f3, fp;
                    if (P.analytic) {
                        const int d0 = P.slot_species[T.slot[0]], d1 = P.slot_species[T.slot[1]];
                        const int d2 = P.slot_species[T.slot[2]], d3 = P.slot_species[T.slot[3]];
                        f1 = f_equilibrium(P, d0, E1);
                        f2 = f_equilibrium(P, d1, E2);
                        f3 = f_equilibrium(P, d2, E3);
                        fp = f_equilibrium(P, d3, Ep);
                    } else {
                        f1 = __ldg(&P.f[i1]);
                        f2 = __ldg(&P.f[i2]);
                        f3 = __ldg(&P.f[i3]);
                        fp = __ldg(&P.f[a]);
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
                    const long long q = O::rint_(wq);
                    if (q == 0) continue;
                    own += q;
                    if (P.sampler == 0) {
                        red_add(&P.A[i3], q);
                        red_add(&P.A[i1], -q);
                        red_add(&P.A[i2], -q);
                    }
                }
            }
        }
        if (warp_anchor) {
            own = warp_sum_ll(own);
            if (lane == 0 && own != 0) red_add(&P.A[own_idx], own);
        } else if (own != 0) {
            red_add(&P.A[own_idx], own);
        }
    }
}

}  // namespace bz
