// Thermal masses, drift and moments.  Compiled with -fmad=false so the FP64
// mass integrand and the FP32 Courant numbers round exactly as written; all
// sums are exact integer sums, so results do not depend on the order in
// which threads accumulate.
#include <cstdint>
#include "bz_internal.h"
#include "exact64.cuh"
#include "intconv.cuh"

namespace bz {

__device__ __forceinline__ void red_add_ll(long long* addr, long long v)
{
    atomicAdd(reinterpret_cast<unsigned long long*>(addr), static_cast<unsigned long long>(v));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ __int128 warp_sum_i128(__int128 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long lo = (unsigned long long)v;
        long long hi = (long long)(v >> 64);
        unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, lo, o);
        long long hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
        v += ((__int128)hi2 << 64) | (__int128)lo2;
    }
    return v;
}

// ---------------------------------------------------------------------------
// Thermal masses, Eqs. (mg), (mq).  Per bin, in FP64 with r_a = 1/(2E_a):
// 3x the Eq. (mg) integrand N_g C_A f_g r_g + sum_i N_q C_F (f_qi + f_qbi) r_qi
// and 24x the Eq. (mq) integrand 2 f_g r_g + (f_qi + f_qbi) r_qi, written in
// the state n = N_s f 2^40 (integer coefficients), each rounded to 2^-30 of
// f and summed exactly.  Grid: one block per (x cell, chunk of 2048 bins).
// ---------------------------------------------------------------------------
constexpr int MASS_CHUNK = 2048;
#ifndef BZ_MASS_MINB
#define BZ_MASS_MINB 3  // resident blocks of 256 threads per SM the masses' register budget is cut for (85 registers)
#endif

static int device_sms();

// Fixed-point partial sums of one (x cell, chunk of `chunk` bins) block; the
// block sums add into exact integers, so the chunking does not change them.
__device__ __forceinline__ void masses_block(const MassArgs& P, int64_t x, int64_t c0, int64_t chunk, bool use_prev)
{
    __shared__ double s_p[3][MAX_NP];  // cell-centre momenta, -L + (j + 1/2) dp
    for (int d = 0; d < 3; ++d)
        for (int i = threadIdx.x; i < P.np[d]; i += blockDim.x) s_p[d][i] = -P.L + ((double)i + 0.5) * P.dp[d];
    __syncthreads();
    double m2p[4] = {0.0, 0.0, 0.0, 0.0};
    if (use_prev && P.m2_prev)
        for (int i = 0; i < 4; ++i) m2p[i] = P.m2_prev[x * 4 + i];
    // A species pair with no state (no active slot) contributes the product
    // 0 r = +0 to every sum as long as r is finite, i.e. E^2 = p^2 + m^2 > 0:
    // its 1/(2E) is then not evaluated (set to 0, the same +0 product).
    const bool skip_g = P.slot_of[0] < 0 && m2p[0] >= 0.0;
    bool skip_q[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) skip_q[i] = P.slot_of[1 + i] < 0 && P.slot_of[4 + i] < 0 && m2p[1 + i] >= 0.0;
    const int np1 = P.np[1], np2 = P.np[2], np12 = np1 * np2;
    long long sg = 0, sq[3] = {0, 0, 0};
    bool ovf = false;
    for (int64_t j = c0 + threadIdx.x; j < c0 + chunk && j < P.npc; j += blockDim.x) {
        const int jj = (int)j;  // npc < 2^31
        const double px = s_p[0][jj / np12], py = s_p[1][(jj / np2) % np1], pz = s_p[2][jj % np2];
        const double pp = (px * px + py * py) + pz * pz;
        // N_s f_s = n_s 2^-40 and r_a = 1/(2 E_a): 3x the Eq. (mg) bin integrand
        // is 2^-40 (9 n_g r_g + 4 sum_i q_i r_qi), 24x the Eq. (mq) one is
        // 2^-40 (3 n_g r_g + 4 q_i r_qi), q_i = n_qi + n_qbi
        long long nsp[NSPEC];
#pragma unroll
        for (int s = 0; s < NSPEC; ++s) {
            const int sl = P.slot_of[s];
            nsp[s] = sl < 0 ? 0 : P.state[((int64_t)sl * P.nxc + x) * P.npc + j];
        }
        const double ng = skip_g ? 0.0 : (double)nsp[0];
        const double rg = skip_g ? 0.0 : 0.5 / sqrt(pp + m2p[0]);
        double q[3], rq[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            q[i] = skip_q[i] ? 0.0 : (double)(nsp[1 + i] + nsp[4 + i]);
            rq[i] = skip_q[i] ? 0.0 : 0.5 / sqrt(pp + m2p[1 + i]);
        }
        const double g3 = 9.0 * ng * rg + 4.0 * ((q[0] * rq[0] + q[1] * rq[1]) + q[2] * rq[2]);
        const long long qg = __double2ll_rn(g3 * MASS_FX);
        ovf |= qg > P.limit || qg < -P.limit;
        sg += qg;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double q24 = 3.0 * ng * rg + 4.0 * q[i] * rq[i];
            const long long qq = __double2ll_rn(q24 * MASS_FX);
            ovf |= qq > P.limit || qq < -P.limit;
            sq[i] += qq;
        }
    }
    __shared__ long long red[4][8];
    long long v[4] = {sg, sq[0], sq[1], sq[2]};
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[i] = warp_sum(v[i]);
        if (lane == 0) red[i][warp] = v[i];
    }
    if (ovf) red_add_ll(&P.flags[2], 1);
    __syncthreads();
    if (threadIdx.x < 4) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
        red_add_ll(&P.acc[x * 4 + threadIdx.x], t);
    }
}

// One bin of the Eq. (mg), (mq) sums in FP64 with the factors r = 1/(2E)
// given (0 for a skipped species pair): the integer parts of 3x and 24x the
// bin integrands in 2^-30 of f, exactly as in masses_block.
__device__ __forceinline__ void mass_bin_fp64(const long long nsp[NSPEC], const double r[4], const bool skip[4],
                                              long long* qg, long long qq[3])
{
    const double ng = skip[0] ? 0.0 : (double)nsp[0];
    double q[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) q[i] = skip[1 + i] ? 0.0 : (double)(nsp[1 + i] + nsp[4 + i]);
    const double g3 = 9.0 * ng * r[0] + 4.0 * ((q[0] * r[1] + q[1] * r[2]) + q[2] * r[3]);
    *qg = __double2ll_rn(g3 * MASS_FX);
#pragma unroll
    for (int i = 0; i < 3; ++i) qq[i] = __double2ll_rn((3.0 * ng * r[0] + 4.0 * q[i] * r[1 + i]) * MASS_FX);
}

// Thermal masses with the table of distinct p^2 values: the same sums as
// masses_block, bit for bit.  A block (x cell, chunk of bins) first evaluates
// r_a = 1/(2 E_a) = 0.5 / sqrt(p^2 + m_a^2) once per distinct p^2 (496 values
// for the 20^3 grid instead of 8000 cells), in shared memory; every bin then
// reads its r.  GLUON_ONLY (no quark slot): with the quark pairs skipped, the
// bin integrands reduce to 3x: rint(2^-10 RN(RN(9 n) r_g)) and 24x:
// rint(2^-10 RN(RN(3 n) r_g)) (the quark terms add +0), and for |n| < 2^49
// 9n and 3n are exact integers, so each is one integer-times-double product
// and one conversion, evaluated with integer instructions (exact64.cuh: the
// same IEEE round-to-nearest-even results) instead of FP64 ones.  Bins outside
// that range, and blocks whose r is not a normal double in [2^-900, 2^900],
// take the FP64 instructions.
// Species pairs whose 1/(2E) the mass sums skip: no state of the pair and
// E^2 = p^2 + m^2 > 0 for every p (a skipped pair adds +0, see masses_block).
__device__ __forceinline__ void mass_skips(const MassArgs& P, const double m2p[4], bool skip[4])
{
    skip[0] = P.slot_of[0] < 0 && m2p[0] >= 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) skip[1 + i] = P.slot_of[1 + i] < 0 && P.slot_of[4 + i] < 0 && m2p[1 + i] >= 0.0;
}

__device__ __forceinline__ void mass_prev(const MassArgs& P, int64_t x, double m2p[4])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) m2p[i] = P.m2_prev ? P.m2_prev[x * 4 + i] : 0.0;
}

template <bool GLUON_ONLY>
__global__ void __launch_bounds__(256, 4) k_masses_tab(const __grid_constant__ MassArgs P)
{
    extern __shared__ double s_r[];  // [4][nu]
    const int nu = P.nu;
    const int64_t nchunk = (P.npc + P.chunk - 1) / P.chunk;
    const int64_t x = blockIdx.x / nchunk, c0 = (blockIdx.x % nchunk) * P.chunk;
    double m2p[4];
    bool skip[4];
    mass_prev(P, x, m2p);
    mass_skips(P, m2p, skip);
    int ok = 1;
    for (int u = threadIdx.x; u < nu; u += blockDim.x) {
        const double pp = P.ppu[u];
#pragma unroll
        for (int s = 0; s < 4; ++s) s_r[s * nu + u] = skip[s] ? 0.0 : 0.5 / sqrt(pp + m2p[s]);
        const double rg = s_r[u];
        ok &= (rg >= 0x1p-900 && rg <= 0x1p+900) ? 1 : 0;
    }
    ok = __syncthreads_and(ok);
    const bool fast = GLUON_ONLY && ok && skip[1] && skip[2] && skip[3];
    long long sg = 0, sq[3] = {0, 0, 0};
    bool ovf = false;
    const long long* st0 = P.state + x * P.npc;  // slot 0 (the gluons when GLUON_ONLY)
    const int64_t jend = c0 + P.chunk < P.npc ? c0 + P.chunk : P.npc;
    constexpr int AHEAD = 4;  // bins whose loads are in flight together
    for (int64_t jb = c0 + threadIdx.x; jb < jend; jb += AHEAD * (int64_t)blockDim.x) {
        long long nb[AHEAD];
        int ub[AHEAD];
#pragma unroll
        for (int k = 0; k < AHEAD; ++k) {
            const int64_t j = jb + k * (int64_t)blockDim.x;
            nb[k] = (fast && j < jend) ? st0[j] : 0;
            ub[k] = j < jend ? P.pidx[j] : 0;
        }
#pragma unroll
        for (int k = 0; k < AHEAD; ++k) {
        const int64_t j = jb + k * (int64_t)blockDim.x;
        if (j >= jend) break;
        const int u = ub[k];
        long long qg, qq[3];
        bool done = false;
        if (fast) {
            const long long n = nb[k];
            const uint64_t a = n < 0 ? 0ull - (uint64_t)n : (uint64_t)n;
            if (a == 0) {
                qg = qq[0] = 0;
                done = true;
            } else if (a < (1ull << 49)) {
                Exact64 rg = x64_from_double(s_r[u]);
                rg.neg = n < 0;  // r > 0: the sign of n
                done = x64_rint_scaled(x64_mul_u(9ull * a, rg), -10, &qg) &
                       x64_rint_scaled(x64_mul_u(3ull * a, rg), -10, &qq[0]);
            }
            qq[1] = qq[2] = qq[0];
        }
        if (!done) {
            long long nsp[NSPEC];
#pragma unroll
            for (int s = 0; s < NSPEC; ++s) {
                const int sl = P.slot_of[s];
                nsp[s] = sl < 0 ? 0 : P.state[((int64_t)sl * P.nxc + x) * P.npc + j];
            }
            const double r[4] = {s_r[u], s_r[nu + u], s_r[2 * nu + u], s_r[3 * nu + u]};
            mass_bin_fp64(nsp, r, skip, &qg, qq);
        }
        ovf |= qg > P.limit || qg < -P.limit;
        sg += qg;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (fast && i > 0) break;  // the three quark-flavour sums are equal: added once, copied below
            ovf |= qq[i] > P.limit || qq[i] < -P.limit;
            sq[i] += qq[i];
        }
        }
    }
    if (fast) sq[1] = sq[2] = sq[0];
    __shared__ long long red[4][8];
    long long v[4] = {sg, sq[0], sq[1], sq[2]};
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[i] = warp_sum(v[i]);
        if (lane == 0) red[i][warp] = v[i];
    }
    if (ovf) red_add_ll(&P.flags[2], 1);
    __syncthreads();
    if (threadIdx.x < 4) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
        red_add_ll(&P.acc[x * 4 + threadIdx.x], t);
    }
}

__global__ void __launch_bounds__(256, BZ_MASS_MINB) k_masses(const __grid_constant__ MassArgs P)
{
    const int64_t nchunk = (P.npc + P.chunk - 1) / P.chunk;
    masses_block(P, blockIdx.x / nchunk, (blockIdx.x % nchunk) * P.chunk, P.chunk, true);
}

__device__ __forceinline__ int find_box(const int64_t* prefix, int nboxes, int64_t v)
{
    int lo = 0, hi = nboxes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Batch of homogeneous boxes: block -> (box, chunk) through chunk_prefix.
__global__ void __launch_bounds__(256, BZ_MASS_MINB) k_masses_batch(const MassArgs* __restrict__ boxes,
                                                      const int64_t* __restrict__ chunk_prefix, int nboxes,
                                                      const int* have_prev)
{
    const int b = find_box(chunk_prefix, nboxes, blockIdx.x);
    masses_block(boxes[b], 0, (blockIdx.x - chunk_prefix[b]) * MASS_CHUNK, MASS_CHUNK, *have_prev != 0);
}

__global__ void k_masses_finish_batch(const MassArgs* __restrict__ boxes, int nboxes)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nboxes) return;
    const MassArgs& P = boxes[b];
    const double inv = 1.0 / (double)(1LL << MASS_SHIFT);
    P.m2_out[0] = P.pref_g * P.meas * ((double)P.acc[0] * inv) / 3.0;
    for (int i = 0; i < 3; ++i) P.m2_out[1 + i] = P.pref_q * P.meas * ((double)P.acc[1 + i] * inv) / 24.0;
}

__global__ void k_masses_finish(const __grid_constant__ MassArgs P)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= P.nxc) return;
    const double inv = 1.0 / (double)(1LL << MASS_SHIFT);
    P.m2_out[x * 4 + 0] = P.pref_g * P.meas * ((double)P.acc[x * 4 + 0] * inv) / 3.0;
    for (int i = 0; i < 3; ++i)
        P.m2_out[x * 4 + 1 + i] = P.pref_q * P.meas * ((double)P.acc[x * 4 + 1 + i] * inv) / 24.0;
}

cudaError_t launch_masses(const MassArgs& a, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(a.acc, 0, sizeof(long long) * 4 * a.nxc, s);
    if (e != cudaSuccess) return e;
    // chunks of 256 to 2048 bins, enough blocks for every SM on small grids;
    // with the p^2 table a block of many x cells' grid takes a whole x cell,
    // so that each x cell's table is evaluated once
    MassArgs b = a;
    const int64_t per_x = ((int64_t)4 * device_sms() + a.nxc - 1) / a.nxc;
    int64_t chunk = ((a.npc + per_x - 1) / per_x + 255) / 256 * 256;
    b.chunk = chunk < 256 ? 256 : (chunk > MASS_CHUNK ? MASS_CHUNK : chunk);
    if (a.nu > 0 && per_x == 1) b.chunk = a.npc;
    const int64_t nchunk = (a.npc + b.chunk - 1) / b.chunk;
    if (a.nu > 0 && a.nu <= MASS_TAB_MAX) {
        bool gluon_only = a.slot_of[0] == 0;
        for (int s = 1; s < NSPEC; ++s) gluon_only = gluon_only && a.slot_of[s] < 0;
        const size_t smem = sizeof(double) * 4 * (size_t)a.nu;
        if (gluon_only) {
            if (smem > 48 * 1024) cudaFuncSetAttribute(k_masses_tab<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_masses_tab<true><<<(unsigned)(nchunk * a.nxc), 256, smem, s>>>(b);
        } else {
            if (smem > 48 * 1024) cudaFuncSetAttribute(k_masses_tab<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_masses_tab<false><<<(unsigned)(nchunk * a.nxc), 256, smem, s>>>(b);
        }
    } else {
        k_masses<<<(unsigned)(nchunk * a.nxc), 256, 0, s>>>(b);
    }
    k_masses_finish<<<(unsigned)((a.nxc + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Drift, Eq. (left handside) in flux form: first-order upwind, periodic in
// x.  Courant number c_d = (p_d (1/sqrt(p^2 + m^2(x)))) dt/dx in IEEE FP32,
// held as C = rint(c 2^30); face flux = floor((n C + 2^29) / 2^30) exactly,
// taken at the upwind cell with the upwind cell's mass, so both cells of a
// face apply the same integer.
// Grid: block (row, tile), row = (slot, x cell), tile = DRIFT_TILE p cells;
// rows vary fastest, so the upwind neighbour rows (x +- 1 along each axis)
// of a tile are read while they are still in L2.  Per-row masses and
// neighbour offsets are set up once per block; per-cell index arithmetic is
// 32-bit.
// ---------------------------------------------------------------------------
constexpr int DRIFT_THREADS = 256;
constexpr int DRIFT_PER_THREAD = 4;
constexpr int DRIFT_TILE = DRIFT_THREADS * DRIFT_PER_THREAD;


// floor((n C + 2^29) / 2^30) as an int64 (two's complement, like the exact
// 128-bit product truncated to 64 bits).  For |C| < 2^31 the product splits
// exactly: n = nh 2^32 + nl with 0 <= nl < 2^32, so the result is
// 4 nh C + floor((nl C + 2^29) / 2^30) with both products inside int64.
__device__ __forceinline__ long long flux_fx(long long n, long long C)
{
    if (C > -2147483648LL && C < 2147483648LL) {
        const long long nh = n >> 32;
        const long long nl = (long long)((unsigned long long)n & 0xffffffffull);
        const long long lo = (nl * C + (1LL << 29)) >> 30;
        return (long long)((unsigned long long)(nh * C) * 4ull + (unsigned long long)lo);
    }
    const __int128 prod = (__int128)n * (__int128)C + ((__int128)1 << 29);
    return (long long)(prod >> 30);
}

// Inverse energy 1/sqrt(p^2 + m^2(x)) (IEEE FP32, the factor of every
// Courant number) of each cell, once per step, so that the drift reads the
// upwind neighbours' values instead of recomputing them per face.
__global__ void __launch_bounds__(DRIFT_THREADS) k_inv_energy(const __grid_constant__ DriftArgs P)
{
    __shared__ float s_pf[3][MAX_NP];
    for (int d = 0; d < 3; ++d)
        for (int i = threadIdx.x; i < P.np[d]; i += blockDim.x) s_pf[d][i] = P.pf[d][i];
    __syncthreads();
    const int64_t row = blockIdx.x;
    const int sl = (int)(row / P.nxc);
    const int64_t x = row - (int64_t)sl * P.nxc;
    __shared__ float s_m;  // the row's mass, converted once
    if (threadIdx.x == 0) s_m = P.mass_mode == 1 ? 0.0f : (float)P.m2[x * 4 + P.slot_mslot[sl]];
    __syncthreads();
    const float m = s_m;
    const int npc = (int)P.npc;
    float* out = P.inv_e + row * P.npc;
    for (int j = blockIdx.y * DRIFT_TILE + threadIdx.x, k = 0; k < DRIFT_PER_THREAD && j < npc;
         ++k, j += DRIFT_THREADS) {
        const int jp = __ldg(P.jtab + j);
        const float p0 = s_pf[0][jp & 0xff], p1 = s_pf[1][(jp >> 8) & 0xff], p2 = s_pf[2][jp >> 16];
        out[j] = 1.0f / sqrtf((p0 * p0 + p1 * p1) + p2 * p2 + m);
    }
}

// Narrow form for |C| < 2^31 (every stable step: |c| <= dt/dx < 2): n C split
// exactly into a signed 32 x 32 and an unsigned 32 x 32 product,
// n = nh 2^32 + nl.
__device__ __forceinline__ long long flux32(int nh, unsigned nl, int C)
{
    const long long hi = (long long)nh * C;
    long long lo = (long long)((unsigned long long)nl * (unsigned)C);
    if (C < 0) lo -= (long long)((unsigned long long)nl << 32);  // nl (C + 2^32) - nl 2^32
    return (long long)(((unsigned long long)hi << 2) + (unsigned long long)((lo + (1LL << 29)) >> 30));
}

// rint(w), round half even, for |w| < 2^31, branch-free with FP32 and
// integer instructions: w = h 2^16 + l exactly, where h = rint(w 2^-16) and
// |l| <= 2^15, and each half is rounded with the 1.5 2^23 shifter (h 2^16 is
// even, so rint(w) = h 2^16 + rint(l), ties included).
__device__ __forceinline__ int rint_split(float w)
{
    const float hs = fmaf(w, 1.0f / 65536.0f, 12582912.0f);  // exact product, one rounding: rint(w / 2^16) + 1.5 2^23
    const float h = hs - 12582912.0f;
    const float l = fmaf(-h, 65536.0f, w);                    // exact
    const float ls = l + 12582912.0f;
    return (int)(((unsigned)(__float_as_int(hs) - 0x4B400000) << 16) + (unsigned)(__float_as_int(ls) - 0x4B400000));
}


__device__ __forceinline__ long long flux_n(long long n, int C)
{
    return flux32((int)(n >> 32), (unsigned)n, C);
}

// Courant integer of the narrow form, rint((p_d inv) K) with K = dt/dx 2^30,
// round half even by the hardware conversion (|w| < 2^31 in the narrow form):
// the exact power-of-two factor folded into K gives the same float as
// ((p_d inv) dt/dx) 2^30 wherever the rounded value can be nonzero.
__device__ __forceinline__ int courant_cvt(float pd, float inv, float K)
{
    return __float2int_rn((pd * inv) * K);
}

// Force term of Eq. (left handside), -div_p[(grad_x E) f]: along p_i the p
// cells of an x cell all move with dp_i/dt = -dE/dx_i = -g_i / E, where
// g_i = (m^2(x + e_i) - m^2(x - e_i)) / (4 dx) is half the central difference
// of the species' m^2 (written per x cell and mass slot by k_force_grad, FP64
// then FP32).  Courant number ((-g_i) (1/E)) dt/dp_i in FP32, in 2^-30 fixed
// point; upwind in p; no flux through the faces of the momentum box, so the
// sum of the state is exact.
__global__ void k_force_grad(const __grid_constant__ DriftArgs P)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.nxc * 4) return;
    const int64_t x = t >> 2;
    const int ms = (int)(t & 3);
    const int ny = P.nx[1], nz = P.nx[2];
    const int xi[3] = {(int)(x / ((int64_t)ny * nz)), (int)((x / nz) % ny), (int)(x % nz)};
    const int64_t xs[3] = {(int64_t)ny * nz, nz, 1};
    for (int i = 0; i < 3; ++i) {
        float g = 0.0f;
        if (P.nx[i] > 1 && P.mass_mode != 1) {
            const int64_t xl = x + (int64_t)(xi[i] == 0 ? P.nx[i] - 1 : -1) * xs[i];
            const int64_t xh = x + (int64_t)(xi[i] == P.nx[i] - 1 ? 1 - P.nx[i] : 1) * xs[i];
            g = (float)((P.m2[xh * 4 + ms] - P.m2[xl * 4 + ms]) * P.inv4dx);
        }
        P.gforce[t * 3 + i] = g;
    }
}

// one face flux of the force term: narrow integer form for |w| < 2^31
__device__ __forceinline__ long long force_flux(long long n, float g, float inv, float K)
{
    const float w = ((-g) * inv) * K;
    if (fabsf(w) < 2147483648.0f) return flux32((int)(n >> 32), (unsigned)n, __float2int_rn(w));
    return flux_fx(n, rint_ll(w));
}

// Force-term part of the update of cell j (p indices jv) of one (slot, x)
// row: the cell's own outflow through the face it moves towards and the
// inflow from the cell behind it, each only if that face is inside the box.
__device__ __forceinline__ long long force_acc(const DriftArgs& P, const float* g3, int jp, int j,
                                               const long long* in_row, const float* ie_row, long long n, float inv)
{
    const int jv[3] = {jp & 0xff, (jp >> 8) & 0xff, jp >> 16};
    const int stride[3] = {P.np[1] * P.np[2], P.np[2], 1};
    long long acc = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (P.nx[i] == 1) continue;
        const float g = g3[i];
        const bool up = (-g) > 0.0f;  // towards larger p_i
        const int jo = jv[i] + (up ? 1 : -1), jb = jv[i] + (up ? -1 : 1);
        long long own = 0, behind = 0;
        if (jo >= 0 && jo < P.np[i]) own = force_flux(n, g, inv, P.Kp[i]);
        if (jb >= 0 && jb < P.np[i] && bz_in(j + (up ? -stride[i] : stride[i]), P.npc)) {
            const int jj = j + (up ? -stride[i] : stride[i]);
            behind = force_flux(__ldg(in_row + jj), g, __ldg(ie_row + jj), P.Kp[i]);
        }
        acc += up ? own - behind : behind - own;
    }
    return acc;
}

template <bool NARROW>
__global__ void __launch_bounds__(DRIFT_THREADS) k_drift(const __grid_constant__ DriftArgs P)
{
    __shared__ long long s_off[6];    // cell offsets of the (lower, upper) neighbour rows per axis
    __shared__ float s_pf[3][MAX_NP]; // cell-centre momenta (lanes index them at different cells)
    for (int d = 0; d < 3; ++d)
        for (int i = threadIdx.x; i < P.np[d]; i += blockDim.x) s_pf[d][i] = P.pf[d][i];
    const int64_t row = blockIdx.x;
    const int sl = (int)(row / P.nxc);
    const int64_t x = row - (int64_t)sl * P.nxc;
    const int ms = P.slot_mslot[sl];
    if (threadIdx.x < 6) {
        const int d = threadIdx.x >> 1, up = threadIdx.x & 1;
        const int64_t xs = d == 0 ? (int64_t)P.nx[1] * P.nx[2] : (d == 1 ? (int64_t)P.nx[2] : 1);
        const int xi = (int)((x / xs) % P.nx[d]);
        const int64_t step = up ? (xi == P.nx[d] - 1 ? 1 - P.nx[d] : 1) : (xi == 0 ? P.nx[d] - 1 : -1);
        s_off[threadIdx.x] = step * xs * P.npc;
    }
    __syncthreads();
    const long long* in_row = P.in + row * P.npc;
    long long* out_row = P.out + row * P.npc;
    const int npc = (int)P.npc;
    const int j0 = blockIdx.y * DRIFT_TILE + threadIdx.x;
#pragma unroll 1
    for (int k = 0; k < DRIFT_PER_THREAD; ++k) {
        const int j = j0 + k * DRIFT_THREADS;
        if (j >= npc) break;
        const long long ncj = __ldg(in_row + j);
        const int jp = __ldg(P.jtab + j);
        const float pf[3] = {s_pf[0][jp & 0xff], s_pf[1][(jp >> 8) & 0xff], s_pf[2][jp >> 16]};
        long long acc = 0;
        if (NARROW && P.inv_e) {
            const float* ie_row = P.inv_e + row * P.npc;
            const float inv = __ldg(ie_row + j);
            const int nh = (int)(ncj >> 32);
            const unsigned nl = (unsigned)ncj;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (P.nx[d] == 1) continue;
                const int own_C = rint_split(((pf[d] * inv) * P.dtdxf) * 1073741824.0f);
                const long long off = s_off[2 * d + (pf[d] > 0.0f ? 0 : 1)];  // the upwind neighbour
                if (!bz_in(row * P.npc + off + j, P.ncell)) continue;
                const long long nn = __ldg(in_row + off + j);
                const int nb_C = rint_split(((pf[d] * __ldg(ie_row + off + j)) * P.dtdxf) * 1073741824.0f);
                const long long f_own = flux32(nh, nl, own_C), f_nb = flux32((int)(nn >> 32), (unsigned)nn, nb_C);
                // p_d > 0: outflow up, inflow from below; p_d < 0: inflow from above, outflow down
                acc += pf[d] > 0.0f ? f_own - f_nb : f_nb - f_own;
            }
            if (P.force) acc += force_acc(P, P.gforce + (x * 4 + ms) * 3, jp, j, in_row, ie_row, ncj, inv);
        } else if (P.inv_e) {  // inverse energies of every cell precomputed by k_inv_energy
            const float* ie_row = P.inv_e + row * P.npc;
            const float inv = __ldg(ie_row + j);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (P.nx[d] == 1) continue;
                const long long own_C = rint_ll(((pf[d] * inv) * P.dtdxf) * 1073741824.0f);
                const long long off = s_off[2 * d + (pf[d] > 0.0f ? 0 : 1)];  // the upwind neighbour
                if (!bz_in(row * P.npc + off + j, P.ncell)) continue;
                const long long nn = __ldg(in_row + off + j);
                const long long nb_C = rint_ll(((pf[d] * __ldg(ie_row + off + j)) * P.dtdxf) * 1073741824.0f);
                // p_d > 0: outflow up, inflow from below; p_d < 0: inflow from above, outflow down
                acc += pf[d] > 0.0f ? flux_fx(ncj, own_C) - flux_fx(nn, nb_C) : flux_fx(nn, nb_C) - flux_fx(ncj, own_C);
            }
            if (P.force) acc += force_acc(P, P.gforce + (x * 4 + ms) * 3, jp, j, in_row, ie_row, ncj, inv);
        }  // without inverse energies (one x cell) nothing moves: n^{n+1} = n^n
        out_row[j] = ncj - acc;
        if (P.freal) {
            const int64_t cell = row * P.npc + j;
            if (P.freal_double)
                static_cast<double*>(P.freal)[cell] = (double)ncj * TWO_POW_M40 / P.deg[sl];
            else
                static_cast<float*>(P.freal)[cell] = ll2float_rn(ncj) * P.fscale[sl];
        }
    }
}

constexpr int PLANE_THREADS = 128;
constexpr int PLANE_MAX_NZ = 40;  // y-face buffer: n_z x PLANE_THREADS int64 of dynamic shared memory
#ifndef BZ_PLANE_THREADS_PER_SM
#define BZ_PLANE_THREADS_PER_SM 2048
#endif
#ifndef BZ_PLANE_XFAST
#define BZ_PLANE_XFAST 1  // 1: blocks of all (slot, x index, segment) of a p tile run together (x neighbours in L2)
#endif
#ifndef BZ_HW_CVT
#define BZ_HW_CVT 0       // 1: f conversion with the hardware int64 -> float instruction (slower here)
#endif

// Asynchronous global -> shared copies (cp.async): the streaming drift keeps
// its state loads BZ_DPIPE cells ahead of their use without holding registers.
// Each thread copies and later reads only its own words, so completion of its
// own groups (wait_group) is the only ordering needed.
__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

#ifndef BZ_DPIPE
#define BZ_DPIPE 2  // cells in flight per thread (cp.async groups)
#endif

// FP32 m^2 of every (x cell, mass slot) for the streaming drift, the same
// rounding as k_inv_energy's per-row value.
__global__ void k_mass_table(const __grid_constant__ DriftArgs P)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < P.nxc * 4) P.m2f[t] = P.mass_mode == 1 ? 0.0f : (float)P.m2[t];
}

// Force-term part of the update of cell j of one (slot, x) row, as
// force_acc, with the inverse energy of the cell behind computed in place:
// it differs from cell j only in its p_i, and shares the x cell's m^2.
__device__ __forceinline__ long long force_acc_inline(const DriftArgs& P, const float* g3, int jp, int j,
                                                      const long long* in_row, long long n, float inv,
                                                      const float (*pf)[MAX_NP], float m)
{
    const int jv[3] = {jp & 0xff, (jp >> 8) & 0xff, jp >> 16};
    const int stride[3] = {P.np[1] * P.np[2], P.np[2], 1};
    long long acc = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (P.nx[i] == 1) continue;
        const float g = __ldg(g3 + i);
        const bool up = (-g) > 0.0f;  // towards larger p_i
        const int jo = jv[i] + (up ? 1 : -1), jb = jv[i] + (up ? -1 : 1);
        long long own = 0, behind = 0;
        if (jo >= 0 && jo < P.np[i]) own = force_flux(n, g, inv, P.Kp[i]);
        if (jb >= 0 && jb < P.np[i] && bz_in(j + (up ? -stride[i] : stride[i]), P.npc)) {
            const int jj = j + (up ? -stride[i] : stride[i]);
            const float q0 = pf[0][i == 0 ? jb : jv[0]], q1 = pf[1][i == 1 ? jb : jv[1]], q2 = pf[2][i == 2 ? jb : jv[2]];
            const float invb = 1.0f / sqrtf((q0 * q0 + q1 * q1) + q2 * q2 + m);
            behind = force_flux(__ldg(in_row + jj), g, invb, P.Kp[i]);
        }
        acc += up ? own - behind : behind - own;
    }
    return acc;
}

// Drift by (y, z) planes, streaming: the integer fluxes of k_drift with every
// face flux of the two inner x axes computed once per step.  A thread owns
// one p cell of one (slot, x index ix) and walks a segment of y rows and each
// row's z cells in the upwind order of its own p_y and p_z, so the flux into
// the current cell is the one it computed for the previous cell (z, in a
// register) or for the previous row (y, per z cell in shared memory); each
// row starts with its periodic wrap cell.  The x axis reads the upwind
// neighbour.  1/E = 1/sqrt(p^2 + m^2(x)) is computed in place (IEEE FP32, as
// k_inv_energy) from the p cell's p^2 and the x cell's FP32 m^2, and the
// state is streamed through a cp.async ring BZ_DPIPE cells ahead, so a step
// reads the state once (the x neighbours from L2) and writes it and f once.
// Face fluxes per cell: 4 + 1/n_z + 1/(rows per segment), against 6 in
// k_drift.  Integer sums do not depend on their order: the result is the
// bits of k_drift.
template <bool FORCE>
__global__ void __launch_bounds__(PLANE_THREADS) k_drift_stream(const __grid_constant__ DriftArgs P, int nseg, float K)
{
    constexpr int D = BZ_DPIPE;
    __shared__ float s_pf[3][MAX_NP];
    extern __shared__ long long s_dyn[];  // y-face buffer [n_z][PLANE_THREADS], then the ring [D][2][PLANE_THREADS]
    for (int d = 0; d < 3; ++d)
        for (int i = threadIdx.x; i < P.np[d]; i += blockDim.x) s_pf[d][i] = P.pf[d][i];
    __syncthreads();
    const int npc = (int)P.npc;
    const unsigned bj = BZ_PLANE_XFAST ? blockIdx.y : blockIdx.x, bs = BZ_PLANE_XFAST ? blockIdx.x : blockIdx.y;
    const int j = bj * PLANE_THREADS + threadIdx.x;
    if (j >= npc) return;
    const int nx0 = P.nx[0], ny = P.nx[1], nz = P.nx[2];
    const int seg = (int)(bs % (unsigned)nseg);
    const int rest = (int)(bs / (unsigned)nseg);
    const int ix = rest % nx0, sl = rest / nx0;
    const int jp = __ldg(P.jtab + j);
    const float p0 = s_pf[0][jp & 0xff], p1 = s_pf[1][(jp >> 8) & 0xff], p2 = s_pf[2][jp >> 16];
    const float pp = (p0 * p0 + p1 * p1) + p2 * p2;
    const bool sx = p0 > 0.0f, sy = p1 > 0.0f, sz = p2 > 0.0f;  // p_d > 0: the upwind neighbour is the lower one
    const int ixu = sx ? (ix == 0 ? nx0 - 1 : ix - 1) : (ix == nx0 - 1 ? 0 : ix + 1);
    const int64_t plane = (int64_t)ny * nz * P.npc;  // cells of one x index
    const int64_t zs = P.npc;                         // cells between z neighbours
    const int64_t b_own = (int64_t)sl * P.nxc * P.npc + (int64_t)ix * plane + j;
    const int64_t dup = (int64_t)(ixu - ix) * plane;  // to the x-upwind cell
    const int ms = P.slot_mslot[sl];
    const float* m2f = P.m2f + ms;                    // [x * 4]
    const int xo = ix * ny * nz, xuo = ixu * ny * nz;   // x cell = (ix n_y + iy) n_z + iz
    const long long* in = P.in;
    long long* fy = s_dyn + threadIdx.x;
    long long* ring = s_dyn + (size_t)nz * PLANE_THREADS + threadIdx.x;
    const bool mx = nx0 > 1, my = ny > 1, mz = nz > 1;
    const int t0 = (int)((int64_t)seg * ny / nseg), t1 = (int)((int64_t)(seg + 1) * ny / nseg);
    const int W = mz ? 1 : 0, per_row = nz + W, nr = t1 - t0;
    if (my) {  // y-face fluxes of the row upwind of the segment's first row
        const int tw = t0 == 0 ? ny - 1 : t0 - 1;
        const int iy = sy ? tw : ny - 1 - tw;
        const int64_t rw = b_own + (int64_t)iy * nz * zs;
        for (int iz = 0; iz < nz; ++iz) {
            const int xw = xo + iy * nz + iz;
            const int64_t ow = rw + iz * zs;
            if (!(bz_in(xw, P.nxc) & bz_in(ow, P.ncell))) continue;
            const float inv = 1.0f / sqrtf(pp + __ldg(m2f + xw * 4));
            fy[iz * PLANE_THREADS] = flux_n(__ldg(in + ow), courant_cvt(p1, inv, K));
        }
    }
    // item i of a row: i < W the wrap cell, else the (i - W)-th cell in upwind order
    int pr = 0, pi = 0, ps = 0;  // next item to copy and its ring slot
    auto issue = [&]() {
        if (pr < nr) {
            const int iy = sy ? t0 + pr : ny - 1 - t0 - pr;
            int k = pi - W;
            const bool wrap = k < 0;
            if (wrap) k = nz - 1;
            const int iz = sz ? k : nz - 1 - k;
            const int64_t o = b_own + ((int64_t)iy * nz + iz) * zs;
            if (bz_in(o, P.ncell)) cp_async8(ring + (2 * ps) * PLANE_THREADS, in + o);
            if (mx && !wrap && bz_in(o + dup, P.ncell)) cp_async8(ring + (2 * ps + 1) * PLANE_THREADS, in + o + dup);
            if (++pi == per_row) {
                pi = 0;
                ++pr;
            }
        }
        cp_async_commit();
        ps = ps + 1 == D ? 0 : ps + 1;
    };
#pragma unroll
    for (int q = 0; q < D - 1; ++q) issue();
    long long fz_up = 0;  // z flux of the previous cell of the walk (the upwind one)
    int cr = 0, ci = 0, cs = 0;
#pragma unroll 1
    for (int g = 0, G = nr * per_row; g < G; ++g) {
        issue();
        cp_async_wait<D - 1>();
        const long long n = ring[(2 * cs) * PLANE_THREADS];
        const int iy = sy ? t0 + cr : ny - 1 - t0 - cr;
        int k = ci - W;
        const bool wrap = k < 0;
        if (wrap) k = nz - 1;
        const int iz = sz ? k : nz - 1 - k;
        const int xr = iy * nz + iz;
        const float m = bz_in(xo + xr, P.nxc) ? __ldg(m2f + (xo + xr) * 4) : 0.0f;
        const float inv = 1.0f / sqrtf(pp + m);
        if (wrap) {
            fz_up = flux_n(n, courant_cvt(p2, inv, K));
        } else {
            long long acc = 0;
            // p_d > 0: outflow through the upper face, inflow from below; else the mirror
            if (mz) {
                const long long f2 = flux_n(n, courant_cvt(p2, inv, K));
                acc += sz ? f2 - fz_up : fz_up - f2;
                fz_up = f2;
            }
            if (my) {
                const long long f1 = flux_n(n, courant_cvt(p1, inv, K));
                const long long fu = fy[iz * PLANE_THREADS];
                acc += sy ? f1 - fu : fu - f1;
                fy[iz * PLANE_THREADS] = f1;
            }
            if (mx) {
                const long long nu = ring[(2 * cs + 1) * PLANE_THREADS];
                const float invu = 1.0f / sqrtf(pp + (bz_in(xuo + xr, P.nxc) ? __ldg(m2f + (xuo + xr) * 4) : 0.0f));
                const long long f0 = flux_n(n, courant_cvt(p0, inv, K));
                const long long fu = flux_n(nu, courant_cvt(p0, invu, K));
                acc += sx ? f0 - fu : fu - f0;
            }
            const int64_t oc = b_own + (int64_t)xr * zs;
            if (bz_in(oc, P.ncell) & bz_in(xo + xr, P.nxc)) {
                if (FORCE)
                    acc += force_acc_inline(P, P.gforce + ((int64_t)(xo + xr) * 4 + ms) * 3, jp, j, in + (oc - j), n,
                                            inv, s_pf, m);
                P.out[oc] = n - acc;
                if (P.freal) {
                    if (P.freal_double)
                        static_cast<double*>(P.freal)[oc] = (double)n * TWO_POW_M40 / P.deg[sl];
                    else
                        static_cast<float*>(P.freal)[oc] =
                            (BZ_HW_CVT ? __ll2float_rn(n) : ll2float_rn(n)) * P.fscale[sl];
                }
            }
        }
        if (++ci == per_row) {
            ci = 0;
            ++cr;
        }
        cs = cs + 1 == D ? 0 : cs + 1;
    }
    cp_async_wait<0>();
}

static int device_sms()
{
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            nsm < 1)
            nsm = 1;
    }
    return nsm;
}

cudaError_t check_read_transport(unsigned long long out[2], bool reset)
{
#if BZ_CHECK
    cudaError_t e = cudaMemcpyFromSymbol(out, g_bz_check, 2 * sizeof(unsigned long long));
    const unsigned long long zero[2] = {0ull, 0ull};
    if (e == cudaSuccess && reset) e = cudaMemcpyToSymbol(g_bz_check, zero, sizeof(zero));
    return e;
#else
    out[0] = out[1] = 0ull;
    (void)reset;
    return cudaErrorNotSupported;
#endif
}

cudaError_t launch_drift(const DriftArgs& a, cudaStream_t s)
{
    const int64_t rows = a.ncell / a.npc;
    const int64_t tiles = (a.npc + DRIFT_TILE - 1) / DRIFT_TILE;
    if (rows < 1 || rows > 2147483647LL || tiles > 65535) return cudaErrorInvalidConfiguration;
    const bool moving = a.nx[0] > 1 || a.nx[1] > 1 || a.nx[2] > 1;
    if (moving && !(a.inv_e && a.m2f)) return cudaErrorInvalidValue;  // scratch of the moving forms
    if (a.force && !(a.gforce && moving)) return cudaErrorInvalidValue;
    if (a.force) k_force_grad<<<(unsigned)((a.nxc * 4 + 127) / 128), 128, 0, s>>>(a);
    const int64_t nslots = rows / a.nxc;
    if (moving && a.dtdxf < 1.99f && a.nx[2] <= PLANE_MAX_NZ) {
        // y segments: enough threads for every SM at full occupancy
        const int64_t base = nslots * a.nx[0] * a.npc;
        int64_t nseg = ((int64_t)device_sms() * BZ_PLANE_THREADS_PER_SM + base - 1) / base;
        nseg = nseg < 1 ? 1 : (nseg > a.nx[1] ? a.nx[1] : nseg);
        const int64_t gs = nslots * a.nx[0] * nseg, gj = (a.npc + PLANE_THREADS - 1) / PLANE_THREADS;
        const int64_t gx = BZ_PLANE_XFAST ? gs : gj, gy = BZ_PLANE_XFAST ? gj : gs;
        if (gy <= 65535 && gx <= 2147483647LL) {
            const size_t smem = sizeof(long long) * PLANE_THREADS * ((size_t)a.nx[2] + 2 * BZ_DPIPE);
            if (smem > 48 * 1024) {
                const cudaError_t e =
                    a.force ? cudaFuncSetAttribute(k_drift_stream<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                            : cudaFuncSetAttribute(k_drift_stream<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
            }
            const dim3 grid((unsigned)gx, (unsigned)gy);
            const float K = a.dtdxf * 1073741824.0f;
            k_mass_table<<<(unsigned)((a.nxc * 4 + 255) / 256), 256, 0, s>>>(a);
            if (a.force)
                k_drift_stream<true><<<grid, PLANE_THREADS, smem, s>>>(a, (int)nseg, K);
            else
                k_drift_stream<false><<<grid, PLANE_THREADS, smem, s>>>(a, (int)nseg, K);
            return cudaGetLastError();
        }
    }
    DriftArgs b = a;
    if (!moving) b.inv_e = nullptr;
    if (moving) k_inv_energy<<<dim3((unsigned)rows, (unsigned)tiles), DRIFT_THREADS, 0, s>>>(a);
    if (a.dtdxf < 1.99f)  // |C| <= 2^30 dt/dx < 2^31
        k_drift<true><<<dim3((unsigned)rows, (unsigned)tiles), DRIFT_THREADS, 0, s>>>(b);
    else
        k_drift<false><<<dim3((unsigned)rows, (unsigned)tiles), DRIFT_THREADS, 0, s>>>(b);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// f of the state for the collision lookups: f = n 2^-40 / N_s (FP64) or its
// FP32 rounding.
// ---------------------------------------------------------------------------
__global__ void k_convert(const long long* state, void* freal, int as_double, int64_t nxc, int64_t npc,
                          int nslots, ConvScale sc)
{
    const int64_t n = (int64_t)nslots * nxc * npc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int sl = (int)(i / (nxc * npc));
        const long long v = state[i];
        if (as_double)
            static_cast<double*>(freal)[i] = (double)v * TWO_POW_M40 / sc.deg[sl];
        else
            static_cast<float*>(freal)[i] = ll2float_rn(v) * sc.f32[sl];
    }
}

cudaError_t launch_convert(const long long* state, void* freal, int as_double, int64_t nxc, int64_t npc,
                           int nslots, const double* deg, cudaStream_t s)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t n = (int64_t)nslots * nxc * npc;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)nsm * 8) blocks = (int64_t)nsm * 8;
    if (blocks < 1) blocks = 1;
    ConvScale sc;
    for (int sl = 0; sl < NSPEC; ++sl) {
        sc.deg[sl] = deg[sl];
        sc.f32[sl] = (float)(TWO_POW_M40 * (1.0 / deg[sl]));  // as the drift's fscale
    }
    k_convert<<<(unsigned)blocks, 256, 0, s>>>(state, freal, as_double, nxc, npc, nslots, sc);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_sum_ll(const long long* __restrict__ a, int64_t n, long long* out)
{
    long long v = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v += a[i];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0 && v != 0) red_add_ll(out, v);
}

cudaError_t launch_sum_ll(const long long* a, int64_t n, long long* out, cudaStream_t s)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_sum_ll<<<(unsigned)blocks, 256, 0, s>>>(a, n, out);
    return cudaGetLastError();
}

// Packed momentum-cell indices jx | jy << 8 | jz << 16 of the linear p index
// (np <= 256 per axis), built once per grid so the streaming kernels need no
// integer division.
__global__ void k_fill_jtab(int* jtab, int np0, int np1, int np2)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np0 * np1 * np2) return;
    const int jz = j % np2, jxy = j / np2;
    jtab[j] = (jxy / np1) | ((jxy % np1) << 8) | (jz << 16);
}

cudaError_t launch_fill_jtab(int* jtab, const int* np, cudaStream_t s)
{
    const int n = np[0] * np[1] * np[2];
    k_fill_jtab<<<(n + 255) / 256, 256, 0, s>>>(jtab, np[0], np[1], np[2]);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Moments, Eqs. (particle numbers), (energy momentum tensor): one block per
// (x cell, slot); exact 128-bit integer sums of n, E_fx n and (2j+1-n) n.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double i128_to_double(__int128 v)
{
    return (double)(long long)(v >> 64) * 18446744073709551616.0 + (double)(unsigned long long)v;
}

#ifndef BZ_MOM_UNROLL
#define BZ_MOM_UNROLL 2  // cells in flight per thread
#endif
#ifndef BZ_MOM_MINB
#define BZ_MOM_MINB 4    // resident blocks per SM (register budget)
#endif

// The 5 doubles of one (x cell, slot) from its exact sums.
__device__ __forceinline__ void moments_out(const MomentArgs& P, const __int128* t, double* o)
{
    o[0] = i128_to_double(t[0]) * P.pref;
    o[1] = i128_to_double(t[1]) * P.pref * (1.0 / 16777216.0);
    for (int d = 0; d < 3; ++d) o[2 + d] = i128_to_double(t[2 + d]) * P.pref * P.half_dp[d];
}

// Exact sums of the cells [jlo, jhi) of one (x cell, slot): 5 doubles at o,
// or, with part set, the 5 exact 128-bit sums (lo, hi words) at part.
__device__ __forceinline__ void moments_block(const MomentArgs& P, int64_t x, int sl, int jlo, int jhi, double* o,
                                              long long* part)
{
    __shared__ float s_pf[3][MAX_NP];  // cell-centre momenta (lanes index them at different cells)
    for (int d = 0; d < 3; ++d)
        for (int i = threadIdx.x; i < P.np[d]; i += blockDim.x) s_pf[d][i] = P.pf[d][i];
    __syncthreads();
    const float m = P.mass_mode == 1 ? 0.0f : (float)P.m2[x * 4 + P.slot_mslot[sl]];
    const long long* st = P.state + ((int64_t)sl * P.nxc + x) * P.npc;
    const int np1 = P.np[1], np2 = P.np[2];
    const long long pauli = P.pauli[sl];
    int neg = 0, over = 0;  // state warnings: f < 0 anywhere, f > 1 for fermions (Pauli)
    // n = nh 2^32 + nl (nl unsigned): every product below is 32 x 32 bits and
    // every partial sum is exact, for at most 2^16 cells per thread
    // (npc <= 2^24, 256 threads): sum nl < 2^48, sum (k_d + 256) nl < 2^57,
    // sum k_d nh < 2^55 with |k_d| = |2 j_d + 1 - n_d| < 2^8.  E_fx n is
    // accumulated in 128 bits (lo word and carries).
    unsigned long long s_nl = 0;
    long long s_nh = 0;
    unsigned long long el_lo = 0, el_hi = 0;  // sum E_fx nl (unsigned, 128 bits)
    unsigned long long eh_lo = 0;             // sum E_fx nh (signed, 128 bits: lo word ...
    long long eh_hi = 0;                      // ... and high word)
    unsigned long long kl[3] = {0, 0, 0};     // sum (k_d + 256) nl
    long long kh[3] = {0, 0, 0};              // sum k_d nh
    __int128 e_wide = 0;                      // sum E_fx n of cells with E_fx >= 2^31 (exact, rare)
    constexpr int U = BZ_MOM_UNROLL;          // cells in flight per thread
    for (int j0 = jlo + (int)threadIdx.x; j0 < jhi; j0 += U * (int)blockDim.x) {
        long long nv[U];
        int jpv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + u * (int)blockDim.x;
            nv[u] = j < jhi ? __ldg(&st[j]) : 0;
            if (P.jtab) {
                jpv[u] = j < jhi ? __ldg(P.jtab + j) : 0;
            } else {
                const int jj = j < jhi ? j : 0, jxy = jj / np2;
                jpv[u] = (jxy / np1) | ((jxy % np1) << 8) | ((jj % np2) << 16);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + u * (int)blockDim.x;
            if (j >= jhi) break;
            const long long n = nv[u];
            const int jv[3] = {jpv[u] & 0xff, (jpv[u] >> 8) & 0xff, jpv[u] >> 16};
            const float pf0 = s_pf[0][jv[0]], pf1 = s_pf[1][jv[1]], pf2 = s_pf[2][jv[2]];
            const float ppf = (pf0 * pf0 + pf1 * pf1) + pf2 * pf2;
            const float ew = sqrtf(ppf + m) * 16777216.0f;
            neg += n < 0;
            over += n > pauli;
            const unsigned nl = (unsigned)n;
            const int nh = (int)(n >> 32);
            s_nl += nl;
            s_nh += nh;
            if (ew < 2147483648.0f) {  // E_fx < 2^31 (ew is >= 0 or NaN)
                const unsigned Efx = (unsigned)__float2int_rn(ew);  // round half even
                const unsigned long long tl = (unsigned long long)Efx * nl;
                el_lo += tl;
                el_hi += el_lo < tl;
                const long long th = (long long)(int)Efx * nh;
                const unsigned long long o = eh_lo;
                eh_lo += (unsigned long long)th;
                eh_hi += (th >> 63) + (eh_lo < o);
            } else {
                e_wide += (__int128)rint_ll(ew) * n;
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int k = 2 * jv[d] + 1 - P.np[d];
                kl[d] += (unsigned long long)(unsigned)(k + 256) * nl;
                kh[d] += (long long)k * nh;
            }
        }
    }
    __int128 v[5];
    const __int128 snl = (__int128)s_nl;
    const __int128 two32 = (__int128)1 << 32;
    v[0] = (__int128)s_nh * two32 + snl;
    const __int128 eh = (__int128)(((unsigned __int128)(unsigned long long)eh_hi << 64) | eh_lo);
    v[1] = (__int128)(((unsigned __int128)el_hi << 64) | el_lo) + eh * two32 + e_wide;
#pragma unroll
    for (int d = 0; d < 3; ++d) v[2 + d] = (__int128)kh[d] * two32 + ((__int128)kl[d] - 256 * snl);
    __shared__ __int128 red[5][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (P.sflags) {
        neg = warp_sum(neg);
        over = warp_sum(over);
        if (lane == 0 && neg) red_add_ll(&P.sflags[0], neg);
        if (lane == 0 && over) red_add_ll(&P.sflags[1], over);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        v[i] = warp_sum_i128(v[i]);
        if (lane == 0) red[i][warp] = v[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __int128 t[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int i = 0; i < 5; ++i) t[i] += red[i][w];
        if (part) {  // exact partial sums of this chunk, combined by k_moments_finish
            for (int i = 0; i < 5; ++i) {
                part[2 * i] = (long long)(unsigned long long)t[i];
                part[2 * i + 1] = (long long)(t[i] >> 64);
            }
        } else {
            moments_out(P, t, o);
        }
    }
}

// Block = (x cell, slot, chunk of the p cells); with one chunk the block
// writes the moments, else its exact partial sums for k_moments_finish.
__global__ void __launch_bounds__(256, BZ_MOM_MINB) k_moments(const __grid_constant__ MomentArgs P)
{
    const int nch = P.nchunk > 1 ? P.nchunk : 1;
    const int64_t row = blockIdx.x / nch;
    const int c = (int)(blockIdx.x % nch);
    const int64_t x = row / P.nslots;
    const int sl = (int)(row % P.nslots);
    const int jlo = (int)((int64_t)c * P.npc / nch), jhi = (int)((int64_t)(c + 1) * P.npc / nch);
    double* out = P.out + (P.kidx ? (int64_t)*P.kidx * P.kstride : 0);
    moments_block(P, x, sl, jlo, jhi, out + (x * P.nslots + sl) * 5, nch > 1 ? P.part + (int64_t)blockIdx.x * 10 : nullptr);
}

// Adds the chunks' partial sums of each (x cell, slot) in chunk order.
__global__ void k_moments_finish(const __grid_constant__ MomentArgs P)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= P.nxc * P.nslots) return;
    __int128 t[5] = {0, 0, 0, 0, 0};
    for (int c = 0; c < P.nchunk; ++c) {
        const long long* q = P.part + (row * P.nchunk + c) * 10;
        for (int i = 0; i < 5; ++i)
            t[i] += (__int128)(((unsigned __int128)(unsigned long long)q[2 * i + 1] << 64) | (unsigned long long)q[2 * i]);
    }
    moments_out(P, t, P.out + (P.kidx ? (int64_t)*P.kidx * P.kstride : 0) + row * 5);
}

cudaError_t launch_moments(const MomentArgs& a, cudaStream_t s)
{
    const int nch = a.nchunk > 1 && a.part ? a.nchunk : 1;
    MomentArgs b = a;
    b.nchunk = nch;
    k_moments<<<(unsigned)(a.nxc * a.nslots * nch), 256, 0, s>>>(b);
    if (nch > 1) k_moments_finish<<<(unsigned)((a.nxc * a.nslots + 127) / 128), 128, 0, s>>>(b);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Energy source, Eq. (current conservation): per (x cell, slot) the integral
// I = int d^3p/(2pi)^3 N f / E as an exact integer sum of n round(2^24 / E)
// (1/E in IEEE FP32 at the bin centre, as the drift), then
// S_ex^0 part (1/2)((m^2 - m^2_prev)/dt) I and the T_total term -(1/4) m^2 I
// in FP64.  With the massless dispersion both m^2 terms are zero.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_energy_source(const __grid_constant__ MomentArgs P)
{
    __shared__ float s_pf[3][MAX_NP];
    for (int d = 0; d < 3; ++d)
        for (int i = threadIdx.x; i < P.np[d]; i += blockDim.x) s_pf[d][i] = P.pf[d][i];
    __syncthreads();
    const int64_t x = blockIdx.x / P.nslots;
    const int sl = blockIdx.x % P.nslots;
    const int ms = P.slot_mslot[sl];
    const float m = P.mass_mode == 1 ? 0.0f : (float)P.m2[x * 4 + ms];
    const long long* st = P.state + ((int64_t)sl * P.nxc + x) * P.npc;
    const int npc = (int)P.npc;
    // n = nh 2^32 + nl: sum R nl (unsigned) and sum R nh (signed), each in 128 bits by carries
    unsigned long long l_lo = 0, l_hi = 0, h_lo = 0;
    long long h_hi = 0;
    __int128 wide = 0;  // cells with 2^24 / E >= 2^31 (E < 2^-7 GeV)
    for (int j = threadIdx.x; j < npc; j += blockDim.x) {
        const int jp = __ldg(P.jtab + j);
        const float pf0 = s_pf[0][jp & 0xff], pf1 = s_pf[1][(jp >> 8) & 0xff], pf2 = s_pf[2][jp >> 16];
        const float ppf = (pf0 * pf0 + pf1 * pf1) + pf2 * pf2;
        const float w = (1.0f / sqrtf(ppf + m)) * 16777216.0f;
        const long long n = __ldg(st + j);
        if (w < 2147483648.0f) {
            const unsigned R = (unsigned)rint_split(w);
            const unsigned long long tl = (unsigned long long)R * (unsigned)n;
            l_lo += tl;
            l_hi += l_lo < tl;
            const long long th = (long long)(int)R * (int)(n >> 32);
            const unsigned long long o = h_lo;
            h_lo += (unsigned long long)th;
            h_hi += (th >> 63) + (h_lo < o);
        } else {
            wide += (__int128)rint_ll(w) * n;
        }
    }
    const __int128 hpart = (__int128)(((unsigned __int128)(unsigned long long)h_hi << 64) | h_lo);
    __int128 v = (__int128)(((unsigned __int128)l_hi << 64) | l_lo) + hpart * ((__int128)1 << 32) + wide;
    __shared__ __int128 red[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    v = warp_sum_i128(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        __int128 t = 0;
        for (int w8 = 0; w8 < (int)(blockDim.x >> 5); ++w8) t += red[w8];
        const double I = i128_to_double(t) * P.pref * (1.0 / 16777216.0);
        const double mc = P.mass_mode == 1 ? 0.0 : P.m2[x * 4 + ms];
        const double mp = P.mass_mode == 1 ? 0.0 : P.m2_prev[x * 4 + ms];
        double* o = P.out + (x * P.nslots + sl) * 3;
        o[0] = I;
        o[1] = 0.5 * ((mc - mp) / P.dt) * I;
        o[2] = -0.25 * mc * I;
    }
}

cudaError_t launch_energy_source(const MomentArgs& a, cudaStream_t s)
{
    if (!a.jtab || !a.m2_prev) return cudaErrorInvalidValue;
    k_energy_source<<<(unsigned)(a.nxc * a.nslots), 256, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void k_zero_ll(long long* p, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0;
}

cudaError_t launch_masses_batch(const MassArgs* boxes, const int64_t* chunk_prefix, int nboxes, int64_t nchunks,
                                const int* have_prev, long long* acc_all, cudaStream_t s)
{
    k_zero_ll<<<(unsigned)((4 * nboxes + 255) / 256), 256, 0, s>>>(acc_all, 4 * (int64_t)nboxes);
    k_masses_batch<<<(unsigned)nchunks, 256, 0, s>>>(boxes, chunk_prefix, nboxes, have_prev);
    k_masses_finish_batch<<<(unsigned)((nboxes + 127) / 128), 128, 0, s>>>(boxes, nboxes);
    return cudaGetLastError();
}

// f of the concatenated batch state (FP32): f = n 2^-40 / N_s, block -> (box, chunk of 2048 cells)
__global__ void __launch_bounds__(256) k_convert_batch(const long long* __restrict__ state, float* __restrict__ f,
                                                       const int64_t* __restrict__ cell_prefix,
                                                       const int64_t* __restrict__ chunk_prefix,
                                                       const float* __restrict__ gluon_first_scale,
                                                       const int* __restrict__ slot_cells, int nboxes)
{
    const int b = find_box(chunk_prefix, nboxes, blockIdx.x);
    const int64_t base = cell_prefix[b];
    const int64_t ncell = cell_prefix[b + 1] - base;
    const int64_t c0 = (blockIdx.x - chunk_prefix[b]) * MASS_CHUNK;
    const float s0 = gluon_first_scale[2 * b], s1 = gluon_first_scale[2 * b + 1];
    const int per_slot = slot_cells[b];
    for (int64_t i = c0 + threadIdx.x; i < c0 + MASS_CHUNK && i < ncell; i += blockDim.x)
        f[base + i] = ll2float_rn(state[base + i]) * (i < per_slot ? s0 : s1);
}

cudaError_t launch_convert_batch(const long long* state, float* f, const int64_t* cell_prefix,
                                 const int64_t* chunk_prefix, const float* scale, const int* slot_cells, int nboxes,
                                 int64_t nchunks, cudaStream_t s)
{
    k_convert_batch<<<(unsigned)nchunks, 256, 0, s>>>(state, f, cell_prefix, chunk_prefix, scale, slot_cells, nboxes);
    return cudaGetLastError();
}

// Moments of every (box, slot): one block each, through slot_prefix; out
// advances by one step's worth per call index (*kidx).
__global__ void __launch_bounds__(256, BZ_MOM_MINB) k_moments_batch(const MomentArgs* __restrict__ boxes,
                                                       const int* __restrict__ slot_prefix, int nboxes,
                                                       double* out, const int* kidx, int per_step)
{
    int lo = 0, hi = nboxes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (slot_prefix[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    moments_block(boxes[lo], 0, (int)blockIdx.x - slot_prefix[lo], 0, (int)boxes[lo].npc,
                  out + (int64_t)(*kidx) * per_step + 5 * (int64_t)blockIdx.x, nullptr);
}

cudaError_t launch_moments_batch(const MomentArgs* boxes, const int* slot_prefix, int nboxes, int nblocks,
                                 double* out, const int* kidx, int per_step, cudaStream_t s)
{
    k_moments_batch<<<nblocks, 256, 0, s>>>(boxes, slot_prefix, nboxes, out, kidx, per_step);
    return cudaGetLastError();
}

// End of a batch step: current masses become the previous ones, step and
// call-local step index advance.
__global__ void k_batch_end_step(double* m2_prev, const double* m2_cur, int n, int* have_prev, int* step_dev,
                                 int* kidx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) m2_prev[i] = m2_cur[i];
    if (i == 0) {
        *have_prev = 1;
        *step_dev += 1;
        *kidx += 1;
    }
}

cudaError_t launch_batch_end_step(double* m2_prev, const double* m2_cur, int n, int* have_prev, int* step_dev,
                                  int* kidx, cudaStream_t s)
{
    k_batch_end_step<<<(n + 127) / 128, 128, 0, s>>>(m2_prev, m2_cur, n, have_prev, step_dev, kidx);
    return cudaGetLastError();
}

__global__ void k_set_step(int* step_dev, int step, int* kidx, int k)
{
    *step_dev = step;
    *kidx = k;
}

__global__ void k_step_advance(int* step_dev, int* kidx)
{
    *step_dev += 1;
    *kidx += 1;
}

cudaError_t launch_set_step(int* step_dev, int step, int* kidx, int k, cudaStream_t s)
{
    k_set_step<<<1, 1, 0, s>>>(step_dev, step, kidx, k);
    return cudaGetLastError();
}

cudaError_t launch_step_advance(int* step_dev, int* kidx, cudaStream_t s)
{
    k_step_advance<<<1, 1, 0, s>>>(step_dev, kidx);
    return cudaGetLastError();
}

}  // namespace bz
