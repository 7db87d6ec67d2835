// FP32 collision path (warp-cooperative).
//
// Work unit: one anchor (species d, x cell, p cell) and 32 of its samples,
// one sample per lane, so the anchor's index decode, masses and f_p are
// warp-uniform.  Per kinematic group of d's equation (Eqs. C_gluon /
// C_quark: consecutive terms whose legs k1, k2, k3 carry equal masses):
//   phase A (every lane): E3, D, kappa, H and the two k1z candidates of
//     Eq. (work out delta E); ill-conditioned terms (|H| < tau kappa^2) go to
//     the float-float re-evaluation queue; each valid root inside the box is
//     appended once, as (lane, the group's terms, z, E3, sqrt H), to a
//     per-warp ring in shared memory;
//   phase B (whenever 32 roots are pending, and at the end): all 32 lanes
//     take one root each and evaluate E1, s, t, u and the solved legs' bins,
//     then for each term of the group |M|^2, W and c~ (Eq. ca), using
//     |J| E1 E2 = sqrt(H) at a root, and deposit the int64 weight to the
//     k1, k2, k3 legs; the anchor's own +q is summed in registers and over
//     the warp, one reduction per unit.
// The per-lane sample geometry lives in shared memory so phase B can read
// any lane's sample.  Uniforms: u = ((x >> 9) + 1/2) 2^-23 built from the
// mantissa bits; weights are rounded to int64 with integer operations only,
// so the FP64 pipe is never used.
#include "collide.cuh"
#include "ff.cuh"
#include "intconv.cuh"

namespace bz {

namespace {

constexpr int RING = 128;         // pending roots per warp (power of 2)
constexpr int SBUF = 64;          // buffered live samples per warp (power of 2)
constexpr int WARPS = F32_WARPS;  // warps per block
#ifndef BZ_FIX_SPLIT_MAX
#define BZ_FIX_SPLIT_MAX 8  // most warps sharing one queue segment
#endif
#ifndef BZ_FIX_MINB
#define BZ_FIX_MINB 4  // resident blocks of 256 threads per SM the fixup's register budget is cut for (64 registers)
#endif
#ifndef BZ_F32_MIN_BLOCKS
#define BZ_F32_MIN_BLOCKS (24 / WARPS)  // resident blocks per SM the register budget is cut for (80 registers)
#endif
#ifndef BZ_F32_MIN_BLOCKS_GROUPED
#define BZ_F32_MIN_BLOCKS_GROUPED 7  // the same for single boxes whose equations have groups of several terms
#endif

struct WarpSmemBase {
    // live samples (k2 inside the box in x and y, or on its edge), [field][slot];
    // fields read together are paired into 8-byte words
    float2 EpPz[SBUF];            // Ep, Pz
    float2 ab2m[SBUF];            // a^2 - m_a^2 = |k1perp|^2, b^2 - m_b^2 = |k2perp|^2
    float2 PPkk3[SBUF];           // P^2, |k3|^2
    float2 k13k3z[SBUF];          // k1perp.k3perp, k3z
    float2 k1ppz[SBUF];           // k1perp.pperp, pz
    int2 lin3meta[SBUF];          // bin of k3 or its Philox word (see below); sample index | k2perp inside << 24 | on an edge << 25
    float wfac[SBUF];             // learned: 1/(32 q(y)); record mode: sum of |c~| of the sample
    float3 tlc[4];                // learned: t2_consts of k1 (centre 0, sigma1) and of k3x, k3y, k3z
    // pending roots: (z, E3, sqrt H, tag as bits), one 16-byte entry per root;
    // tag = live-sample sequence number | first term << 24 | (terms - 1) << 28
    float4 ring[RING];
    // this unit's terms: masses of the legs and sym, packed leg slots / flags / row
    float4 tm[MAX_TERMS];         // (ma2, mb2, mc2, sym)
    int tinfo[MAX_TERMS];         // slot0 | slot1 << 3 | slot2 << 6 | quark0..3 << 9..12 | cls << 13
    int tgn[MAX_TERMS];           // terms of the kinematic group the term opens (0: not a group's first)
};

// The sampled legs' bins.  Equations whose groups have several terms (several
// roots per sample) take them at the draw: bxy = (bin of k1perp, bin of
// k2perp), lin3meta.x = bin of k3.  Equations of one-term groups in uniform and
// record modes (about a third of their samples have a root) take them when a
// root is evaluated, from the kept Philox words of k1perp and k3 (w4 = k1x,
// k1y, k3x, k3y words; lin3meta.x = the k3z word) and k2perp (bxyf).
template <bool BINS_AT_ROOT> struct WarpSmem;
template <> struct WarpSmem<false> : WarpSmemBase {
    int2 bxy[SBUF];
};
template <> struct WarpSmem<true> : WarpSmemBase {
    uint4 w4[SBUF];
    float2 bxyf[SBUF];
};

__device__ __forceinline__ float unif23(uint32_t x)
{
    // ((x >> 9) + 1/2) 2^-23 = 1.m - (1 - 2^-24), exact in one subtraction:
    // (2m + 1) 2^-24 has at most 24 significant bits
    return __uint_as_float(0x3F800000u | (x >> 9)) - 0.99999994f;
}

// unif23(x) - 1/2, exactly: 1.m - 3/2 is exact (operands within a factor of
// two), and adding 2^-24 to it is too ((2m + 1 - 2^23) 2^-24, |.| < 2^23 units)
__device__ __forceinline__ float jit23(uint32_t x)
{
    return (__uint_as_float(0x3F800000u | (x >> 9)) - 1.5f) + 5.9604644775390625e-8f;
}

__device__ __forceinline__ float sel4(int k, float a, float b, float c, float d)
{
    return k == 0 ? a : (k == 1 ? b : (k == 2 ? c : d));
}

// Bin of a solved coordinate, clamped to [0, n).  floor(t) for 0 <= t < 2^23
// is read from the mantissa of t + 2^23 added with rounding down (no
// float-to-int conversion instruction; those issue on the FP64 pipe here).
// t is clamped to [0, n - 1/2] first (a NaN to 0), so floor(t) <= n - 1.
__device__ __forceinline__ int binf(float k, float L, float inv_dp, int n)
{
    const float nf = __uint_as_float(0x4B000000u | (unsigned)n) - 8388608.0f;  // (float)n exactly, n < 2^23
    const float t = fminf(fmaxf((k + L) * inv_dp, 0.0f), nf - 0.5f);
    return __float_as_int(__fadd_rd(t, 8388608.0f)) - 0x4B000000;
}

// Bin of a sampled coordinate k = -L + 2L u, u = ((x >> 9) + 1/2) 2^-23:
// floor(u n) = ((2 (x >> 9) + 1) n) >> 24 exactly (u n is never within 2^-24
// of an integer, so the FP64 definition floor((k + L)/dp) gives the same bin),
// evaluated as the high word of ((x >> 9) 2^9 + 2^8) n (n < 2^23).
__device__ __forceinline__ int bin_word(uint32_t x, int n)
{
    return (int)__umulhi((x & 0xFFFFFE00u) | 0x100u, (uint32_t)n);
}

// A solved coordinate within nu bin widths of a bin (or box) edge: FP32
// rounding could put it on the other side, so the term is re-evaluated in float-float.  k2x,
// k2y carry a few ulps (EDGE_XY); a root's error grows with the
// conditioning |kappa|/sqrt(H) of the quadratic (EDGE_Z per unit of it).
constexpr float EDGE_XY = 1e-5f;
constexpr float EDGE_Z = 1e-5f;
__device__ __forceinline__ bool near_edge(float v, float L, float inv_dp, float nu)
{
    // r = frac(t) within nu of 0 or 1: |r - 1/2| > 1/2 - nu (r - 1/2 is exact)
    const float t = (v + L) * inv_dp;
    return fabsf((t - floorf(t)) - 0.5f) > 0.5f - nu;
}

// Student-t with two degrees of freedom, truncated to [-1, 1), centre mu and
// scale s (|mu| < 1): Fa = F(-1), cFb = 1 - F(1) and D = F(1) - F(-1), the
// tails F(-|z|) = 1 / (r (r + |z|)), r = sqrt(2 + z^2), without cancellation.
__device__ __forceinline__ float t2_tail(float z)
{
    const float r = sqrtf(2.0f + z * z);
    return 1.0f / (r * (r + fabsf(z)));
}

__device__ __forceinline__ float3 t2_consts(float mu, float s)
{
    const float Fa = t2_tail((-1.0f - mu) / s);
    const float cFb = t2_tail((1.0f - mu) / s);
    return make_float3(Fa, cFb, (1.0f - cFb) - Fa);
}

}  // namespace

// Sampling modes, resolved at compile time so that the uniform kernel carries
// none of the learned-proposal or record-mode state (registers set occupancy).
enum { M_UNIFORM = 0, M_LEARNED = 1, M_RECORD = 2 };

// One unit: the anchor of unit / ngroup and its samples of the chunks
// [F32_GROUP g, F32_GROUP (g + 1)) of 32.  Samples whose k2perp falls outside
// the box (they contribute nothing to any term) are dropped, the others are
// compacted into the live-sample buffer, and the roots are solved on full
// warps of live samples.  box_tag is or-ed into queued items (the box index
// << 48 in a batch).
// SINGLE: P is the kernel's own argument block (constant bank), so the Philox
// key schedule is read from it as instruction operands; a batch box's block
// lives in global memory and the keys are bumped round by round instead.
// The samples of a unit share the counter words (p cell, x cell, step and
// species), so the parts of the first two Philox rounds that depend only on
// them are computed once per unit (head) and each draw finishes its counter.
template <bool SINGLE>
__device__ __forceinline__ uint4 draw_head(const CollideArgs<float>& P, uint32_t cy, uint32_t cz, uint32_t cw)
{
    return SINGLE ? philox_head(cy, cz, cw, P.ks[0], P.ks[1], P.ks[2], P.ks[3])
                  : philox_head(cy, cz, cw, P.key0, P.key1, P.key0 + 0x9E3779B9u, P.key1 + 0xBB67AE85u);
}
template <bool SINGLE>
__device__ __forceinline__ uint4 draw(const CollideArgs<float>& P, uint32_t c0, uint4 head, uint32_t cy, uint32_t cz,
                                      uint32_t cw)
{
    return SINGLE ? philox_tail_ks(c0, head, P.ks) : philox4x32_10(make_uint4(c0, cy, cz, cw), P.key0, P.key1);
}

template <int MODE, bool GROUPS, bool SINGLE>
__device__ __forceinline__ void collide_unit(const CollideArgs<float>& P, int64_t unit, int step,
                                             WarpSmem<(!GROUPS && MODE != M_LEARNED)>& S,
                                             DeferCtx& dq, unsigned long long box_tag)
{
    // the sampled legs' bins when a root is evaluated (one-term groups, sampled words)
    constexpr bool BINS_AT_ROOT = !GROUPS && MODE != M_LEARNED;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const float L = P.L, twoL = P.twoL;
    const float inv_dp0 = 1.0f / P.dp[0], inv_dp1 = 1.0f / P.dp[1], inv_dp2 = 1.0f / P.dp[2];
    const int64_t nxc = P.nxc, npc = P.npc;
    const int nchunk = (P.nsamples + 31) >> 5;
    const int ngroup = (nchunk + F32_GROUP - 1) / F32_GROUP;
    // index decode with exact multiply-shift division (all indices < 2^31)
    const uint32_t al = udiv((uint32_t)unit, P.dv_group);
    const int grp = (int)((uint32_t)unit - al * (uint32_t)ngroup);
    const int c0 = grp * F32_GROUP, c1 = min(c0 + F32_GROUP, nchunk);
    const int64_t a = P.a_offset + (int64_t)al * P.a_stride;
    const uint32_t sl_u = udiv((uint32_t)a, P.dv_slot);
    const uint32_t rem = (uint32_t)a - sl_u * (uint32_t)(nxc * npc);
    const uint32_t x_u = udiv(rem, P.dv_npc);
    const int sl = (int)sl_u;
    const int64_t x = x_u;
    const int j = (int)(rem - x_u * (uint32_t)npc);
    const int d = P.slot_species[sl];
    const uint32_t jx_u = udiv((uint32_t)j, P.dv_yz);
    const uint32_t ryz = (uint32_t)j - jx_u * (uint32_t)(P.np[1] * P.np[2]);
    const uint32_t jy_u = udiv(ryz, P.dv_z);
    const int jx = (int)jx_u, jy = (int)jy_u, jz = (int)(ryz - jy_u * (uint32_t)P.np[2]);
    const unsigned xoff = (unsigned)(x * npc);
    const unsigned slot_stride = (unsigned)(nxc * npc);
    // warp-uniform masses: lanes 0..4 convert one double each, then broadcast
    float mv = 0.0f;
    if (lane < 5) mv = (float)P.m2[x * 4 + (lane < 4 ? lane : 0)];
    const float mg2 = __shfl_sync(0xffffffffu, mv, 4);
    float m0 = __shfl_sync(0xffffffffu, mv, 0), m1 = __shfl_sync(0xffffffffu, mv, 1);
    float m2v = __shfl_sync(0xffffffffu, mv, 2), m3 = __shfl_sync(0xffffffffu, mv, 3);
    if (P.mass_mode == 1) m0 = m1 = m2v = m3 = 0.0f;
    const float fp = P.analytic ? 0.0f : __ldg(static_cast<const float*>(P.f) + a);

    const int nt = P.nterms[d];
    // kinematic groups: consecutive terms with equal leg masses (the first
    // term of each is flagged); a group's size is the distance to the next first
    const bool gfirst = lane < nt && P.terms[d][lane].gfirst;
    const unsigned firsts = __ballot_sync(0xffffffffu, gfirst);
    if (lane < nt) {
        const TermDev& T = P.terms[d][lane];
        S.tm[lane] = make_float4(sel4(T.mslot[0], m0, m1, m2v, m3), sel4(T.mslot[1], m0, m1, m2v, m3),
                                 sel4(T.mslot[2], m0, m1, m2v, m3), (float)T.sym);
        S.tinfo[lane] = T.slot[0] | (T.slot[1] << 3) | (T.slot[2] << 6) | (T.quark[0] << 9) | (T.quark[1] << 10)
                        | (T.quark[2] << 11) | (T.quark[3] << 12) | (T.cls << 13);
        const unsigned after = firsts & ~((2u << lane) - 1u);
        S.tgn[lane] = gfirst ? (after ? __ffs(after) - 1 : nt) - lane : 0;
    }
    const float md2 = sel4(P.terms[d][0].mslot[3], m0, m1, m2v, m3);
    float pm0 = 0.0f, pm1 = 0.0f, pm2 = 0.0f, ps3 = 1.0f, ps1 = 1.0f, pa = 1.0f;
    if (MODE == M_LEARNED) {  // this anchor's proposal parameters (mu3, sigma3, sigma1, alpha)
        const float v = lane < 6 ? __ldg(&P.prop[a * 8 + lane]) : 0.0f;
        pm0 = __shfl_sync(0xffffffffu, v, 0);
        pm1 = __shfl_sync(0xffffffffu, v, 1);
        pm2 = __shfl_sync(0xffffffffu, v, 2);
        ps3 = __shfl_sync(0xffffffffu, v, 3);
        ps1 = __shfl_sync(0xffffffffu, v, 4);
        pa = __shfl_sync(0xffffffffu, v, 5);
        if (lane < 4) S.tlc[lane] = t2_consts(lane == 0 ? 0.0f : (lane == 1 ? pm0 : (lane == 2 ? pm1 : pm2)),
                                             lane == 0 ? ps1 : ps3);
    }
    const uint32_t ctr3 = ((uint32_t)step << 3) | (uint32_t)d;
    // single boxes: the unit's Philox head; the batch kernel (whose registers
    // are spoken for) runs every round of each counter
    const uint4 phead = SINGLE ? draw_head<SINGLE>(P, (uint32_t)j, (uint32_t)x, ctr3) : make_uint4(0u, 0u, 0u, 0u);
    const float pc0 = -L + ((float)jx + 0.5f) * P.dp[0];
    const float pc1 = -L + ((float)jy + 0.5f) * P.dp[1];
    const float pc2 = -L + ((float)jz + 0.5f) * P.dp[2];
    const bool may_defer = P.tau > 0.0f;
    __syncwarp();

    int c = c0;               // next chunk of 32 samples to draw
    int nlive = 0, cons = 0;  // live samples buffered / taken by phase A (sequence numbers)
    int head = 0, tail = 0;   // ring indices (warp-uniform)
    long long own = 0;

    // phase B on n pending roots starting at head
    auto process = [&](int n) {
        float w_root = 0.0f;  // record mode: sum of |c~| over this root's terms
        int src_rec = -1 - lane;
        if (lane < n) {
            const int ri = (head + lane) & (RING - 1);
            const float4 rv = S.ring[ri];
            const unsigned tg = __float_as_uint(rv.w);
            const int src = tg & (SBUF - 1), t0 = (tg >> 24) & 15, tn = GROUPS ? (int)(tg >> 28) + 1 : 1;
            src_rec = src;
            const float z = rv.x, E3 = rv.y, sqH = rv.z;
            const float4 tmv0 = S.tm[t0];  // leg masses shared by the group's terms
            const float ma2 = tmv0.x, mc2 = tmv0.z;
            const float2 epz = S.EpPz[src];
            const float Ep = epz.x;
            const float E = Ep + E3;
            const float a2 = S.ab2m[src].x + ma2;
            const float E1 = sqrtf(a2 + z * z);
            const float dz = epz.y - z;
            const float s = E * E - S.PPkk3[src].x;
            const float2 k13 = S.k13k3z[src], k1p_ = S.k1ppz[src];
            const float k1k3 = k13.x + z * k13.y;
            const float k1p = k1p_.x + z * k1p_.y;
            const float t = (ma2 + mc2) - 2.0f * (E1 * E3 - k1k3);
            const float uu = (ma2 + md2) - 2.0f * (E1 * Ep - k1p);
            if (s <= 0.0f || t - mg2 >= 0.0f || uu - mg2 >= 0.0f) {
                red_add(&P.flags[0], tn);
            } else {
                int b1xy, b2xy, lin3;
                if constexpr (!BINS_AT_ROOT) {
                    const int2 bxy = S.bxy[src];
                    b1xy = bxy.x;
                    b2xy = bxy.y;
                    lin3 = S.lin3meta[src].x;
                } else {
                    const uint4 w4 = S.w4[src];
                    const float2 bb = S.bxyf[src];
                    b1xy = bin_word(w4.x, P.np[0]) * P.np[1] + bin_word(w4.y, P.np[1]);
                    lin3 = (bin_word(w4.z, P.np[0]) * P.np[1] + bin_word(w4.w, P.np[1])) * P.np[2]
                           + bin_word((uint32_t)S.lin3meta[src].x, P.np[2]);
                    b2xy = binf(bb.x, L, inv_dp0, P.np[0]) * P.np[1] + binf(bb.y, L, inv_dp1, P.np[1]);
                }
                const int lin1 = b1xy * P.np[2] + binf(z, L, inv_dp2, P.np[2]);
                const int lin2 = b2xy * P.np[2] + binf(dz, L, inv_dp2, P.np[2]);
                // |J| E1 E2 = sqrt(H) at a root of Eq. (work out delta E)
                const float den = P.twopi5 * 16.0f * sqH * E3 * Ep;
                for (int k = 0; k < tn; ++k) {  // the group's terms: |M|^2, leg species, statistics
                    const int ti = t0 + k;
                    const float sym = S.tm[ti].w;
                    const int info = S.tinfo[ti];
                    const float M2 = msq<float>(info >> 13, P, s, t, uu, mg2);
                    const unsigned i1 = (unsigned)(info & 7) * slot_stride + xoff + lin1;
                    const unsigned i2 = (unsigned)((info >> 3) & 7) * slot_stride + xoff + lin2;
                    const unsigned i3 = (unsigned)((info >> 6) & 7) * slot_stride + xoff + lin3;
                    if (!(bz_in(i1, P.ncell) & bz_in(i2, P.ncell) & bz_in(i3, P.ncell))) continue;
                    float f1, f2, f3, fpp;
                    if (P.analytic) {
                        const float E2 = E - E1;
                        f1 = f_equilibrium(P, P.slot_species[info & 7], E1);
                        f2 = f_equilibrium(P, P.slot_species[(info >> 3) & 7], E2);
                        f3 = f_equilibrium(P, P.slot_species[(info >> 6) & 7], E3);
                        fpp = f_equilibrium(P, d, Ep);
                    } else {
                        const float* F = static_cast<const float*>(P.f);
                        f1 = __ldg(F + i1);
                        f2 = __ldg(F + i2);
                        f3 = __ldg(F + i3);
                        fpp = fp;
                    }
                    const float F1 = (info & (1 << 9)) ? 1.0f - f1 : 1.0f + f1;
                    const float F2 = (info & (1 << 10)) ? 1.0f - f2 : 1.0f + f2;
                    const float F3 = (info & (1 << 11)) ? 1.0f - f3 : 1.0f + f3;
                    const float Fp = (info & (1 << 12)) ? 1.0f - fpp : 1.0f + fpp;
                    const float W = f1 * f2 * F3 * Fp - F1 * F2 * f3 * fpp;
                    const float ct = sym * W * M2 / den;
                    const float wq = ct * P.Kown * (MODE == M_LEARNED ? S.wfac[src] : 1.0f);
                    if (MODE == M_RECORD) {  // record mode: sum |c~| per sample, no deposits
                        w_root += fabsf(ct);
                    } else if (!(fabsf(wq) < 4611686018427387904.0f)) {
                        red_add(&P.flags[1], 1);
                    } else {
                        const long long q = rint_ll(wq);
                        if (q != 0) {
                            own += q;
                            if (P.sampler != 1) {
                                red_add(&P.A[i3], q);
                                red_add(&P.A[i1], -q);
                                red_add(&P.A[i2], -q);
                            }
                        }
                    }
                }
            }
        }
        if (MODE == M_RECORD) {
            // add each root's |c~| to its sample in lane order (two roots of one
            // sample can share this pass), so the record weights do not depend on
            // the order of shared-memory atomics
            const unsigned same = __match_any_sync(0xffffffffu, src_rec);
            float acc = 0.0f;
            for (int l = 0; l < 32; ++l) {
                const float v = __shfl_sync(0xffffffffu, w_root, l);
                if ((same >> l) & 1u) acc += v;
            }
            if (src_rec >= 0 && lane == __ffs(same) - 1) S.wfac[src_rec] += acc;
        }
        head += n;
        __syncwarp();
    };

    // One loop with a single site per phase, so the code stays small enough
    // for the instruction cache.  In order of priority: evaluate 32 pending
    // roots (or all of them during a flush); solve the next kinematic group
    // of the running batch of <= 32 live samples; otherwise draw the next
    // chunk of 32 samples into the live-sample buffer and, once 32 live
    // samples are buffered (or the unit's chunks are drawn), start a batch
    // and solve its first group in the same pass: each pass through the loop
    // costs issue slots of its own (the dispatch and the register moves at
    // its joins), so the common path draw -> batch -> group takes one pass.
    int bstart = 0, bcnt = 0, ti = -1;  // running batch: first sequence number, size, next term (-1: none)
    bool flush = false, rec_due = false;
    float bEp = 0.0f, bPz = 0.0f, ba2m = 0.0f, bb2m = 0.0f, bkk3 = 0.0f;
    int bmeta = 0;
    for (;;) {
        int pend = tail - head;
        if (pend >= 32 || (flush && pend > 0)) {
            process(min(pend, 32));
            pend = tail - head;
            if (pend >= 32 || (flush && pend > 0)) continue;
        }
        flush = false;
        if (ti < 0) {  // no running batch
            if (MODE == M_RECORD && rec_due) {
                // one record per sample with at least one accepted root (a zero
                // weight teaches nothing); the sample's coordinates are drawn again
                rec_due = false;
                if (unit % P.rec_stride == 0) {
                    const int sb = (bstart + lane) & (SBUF - 1);
                    const bool keep = lane < bcnt && S.wfac[sb] > 0.0f;
                    const unsigned keep_mask = __ballot_sync(0xffffffffu, keep);
                    unsigned long long base = 0;
                    if (lane == 0 && keep_mask) base = atomicAdd(P.rec_count, (unsigned long long)__popc(keep_mask));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    const unsigned pos = __popc(keep_mask & lt_mask);
                    if (keep && (long long)(base + pos) < P.rec_cap) {
                        const int smp = bmeta & 0xFFFFFF;
                        const uint4 r0 = draw<SINGLE>(P, 2u * smp, phead, (uint32_t)j, (uint32_t)x, ctr3);
                        const uint4 r1 = draw<SINGLE>(P, 2u * smp + 1u, phead, (uint32_t)j, (uint32_t)x, ctr3);
                        ProposalRecord R;
                        R.a = a;
                        R.w = S.wfac[sb];
                        R.y[0] = (-L + twoL * unif23(r0.w)) / L;
                        R.y[1] = (-L + twoL * unif23(r1.x)) / L;
                        R.y[2] = (-L + twoL * unif23(r1.y)) / L;
                        R.y[3] = (-L + twoL * unif23(r1.z)) / L;
                        R.y[4] = (-L + twoL * unif23(r1.w)) / L;
                        P.rec[base + pos] = R;
                    }
                }
                __syncwarp();
                continue;
            }
            if (!(nlive - cons >= 32 || (c >= c1 && nlive > cons))) {
                if (c >= c1) {  // every chunk drawn and every live sample taken: finish the pending roots
                    if (tail > head) {
                        flush = true;
                        continue;
                    }
                    break;
                }
                // draw chunks until 32 live samples are buffered (the buffer then holds
                // fewer than 64 not yet taken) or the unit's chunks are drawn
                bool redo = false;
                do {
                    // ---- sample geometry (one sample per lane) ----
                    const int smp = c * 32 + lane;
                    const bool live = smp < P.nsamples;
                    const uint4 r0 = draw<SINGLE>(P, 2u * smp, phead, (uint32_t)j, (uint32_t)x, ctr3);
                    const uint4 r1 = draw<SINGLE>(P, 2u * smp + 1u, phead, (uint32_t)j, (uint32_t)x, ctr3);
                    const float p0 = pc0 + P.dp[0] * jit23(r0.x);
                    const float p1 = pc1 + P.dp[1] * jit23(r0.y);
                    const float p2 = pc2 + P.dp[2] * jit23(r0.z);
                    float k1x, k1y, k30, k31, k32, wfac = 1.0f;
                    bool margk = false;
                    if (MODE == M_LEARNED) {
                        // defensive mixture alpha U + (1 - alpha) prod g_i, selector from a third block
                        const uint4 r2 = draw<SINGLE>(P, 0x80000000u | (uint32_t)smp, phead, (uint32_t)j, (uint32_t)x, ctr3);
                        // Component i: with v = Fa + u D and cv = cFb + (1 - u) D = 1 - v,
                        // y = mu + s (v - cv) / sqrt(2 v cv), where the density is
                        // (2 v cv)^(3/2) / (s D); a uniform draw y = 2u - 1 has density
                        // (2 + z^2)^(-3/2) / (s D).  Square roots only.
                        const float uv[5] = {unif23(r0.w), unif23(r1.x), unif23(r1.y), unif23(r1.z), unif23(r1.w)};
                        float y[5];
                        const bool uni = unif23(r2.x) < pa;
                        float G = 1.0f;
#pragma unroll
                        for (int i = 0; i < 5; ++i) {
                            const float mu = i < 2 ? 0.0f : (i == 2 ? pm0 : (i == 3 ? pm1 : pm2));
                            const float sg = i < 2 ? ps1 : ps3;
                            const float3 tc = S.tlc[i < 2 ? 0 : i - 1];
                            if (uni) {
                                y[i] = 2.0f * uv[i] - 1.0f;
                                const float zz = (y[i] - mu) / sg;
                                const float r = rsqrtf(2.0f + zz * zz);
                                G *= r * r * r / (sg * tc.z);
                            } else {
                                const float v = tc.x + uv[i] * tc.z;
                                const float cv = tc.y + (1.0f - uv[i]) * tc.z;
                                const float t = 2.0f * v * cv;
                                const float rt = rsqrtf(t);
                                y[i] = fminf(fmaxf(mu + sg * ((v - cv) * rt), -1.0f), 0.99999994f);
                                G *= t * t * rt / (sg * tc.z);
                            }
                        }
                        wfac = 1.0f / (32.0f * (pa * (1.0f / 32.0f) + (1.0f - pa) * G));
                        k1x = L * y[0];
                        k1y = L * y[1];
                        k30 = L * y[2];
                        k31 = L * y[3];
                        k32 = L * y[4];
                        margk = near_edge(k1x, L, inv_dp0, EDGE_XY) || near_edge(k1y, L, inv_dp1, EDGE_XY) ||
                                near_edge(k30, L, inv_dp0, EDGE_XY) || near_edge(k31, L, inv_dp1, EDGE_XY) ||
                                near_edge(k32, L, inv_dp2, EDGE_XY);
                    } else {
                        k1x = -L + twoL * unif23(r0.w);
                        k1y = -L + twoL * unif23(r1.x);
                        k30 = -L + twoL * unif23(r1.y);
                        k31 = -L + twoL * unif23(r1.z);
                        k32 = -L + twoL * unif23(r1.w);
                    }
                    const float Px = p0 + k30, Py = p1 + k31, Pz = p2 + k32;
                    const float bx = Px - k1x, by = Py - k1y;
                    const bool k2xy_in = in_box(bx, L) && in_box(by, L);
                    const bool marg_xy = near_edge(bx, L, inv_dp0, EDGE_XY) || near_edge(by, L, inv_dp1, EDGE_XY) || margk;
                    const bool keep = live && (k2xy_in || marg_xy);
                    const unsigned kb = __ballot_sync(0xffffffffu, keep);
                    const int cnt = __popc(kb);
                    // the new samples take the slots of sequence numbers nlive - SBUF ..:
                    // finish the pending roots that may still refer to those first.  The
                    // oldest pending root belongs to the batch of the head root, which
                    // starts at a multiple of 32 (only the last batch of a unit is short).
                    if (pend > 0 && ((__float_as_uint(S.ring[head & (RING - 1)].w) & 0xFFFFFF) & ~31) + SBUF < nlive + cnt) {
                        redo = true;  // draw this chunk again after the flush
                        break;
                    }
                    if (keep) {
                        const int sb = (nlive + __popc(kb & lt_mask)) & (SBUF - 1);
                        S.EpPz[sb] = make_float2(sqrtf((p0 * p0 + p1 * p1) + p2 * p2 + md2), Pz);
                        S.PPkk3[sb] = make_float2((Px * Px + Py * Py) + Pz * Pz, (k30 * k30 + k31 * k31) + k32 * k32);
                        S.ab2m[sb] = make_float2(k1x * k1x + k1y * k1y, bx * bx + by * by);
                        S.k13k3z[sb] = make_float2(k1x * k30 + k1y * k31, k32);
                        S.k1ppz[sb] = make_float2(k1x * p0 + k1y * p1, p2);
                        const int meta = smp | ((int)k2xy_in << 24) | ((int)marg_xy << 25);
                        if constexpr (!BINS_AT_ROOT) {
                            int lin3, b1xy;
                            if (MODE == M_LEARNED) {
                                lin3 = (binf(k30, L, inv_dp0, P.np[0]) * P.np[1] + binf(k31, L, inv_dp1, P.np[1])) * P.np[2]
                                       + binf(k32, L, inv_dp2, P.np[2]);
                                b1xy = binf(k1x, L, inv_dp0, P.np[0]) * P.np[1] + binf(k1y, L, inv_dp1, P.np[1]);
                            } else {
                                lin3 = (bin_word(r1.y, P.np[0]) * P.np[1] + bin_word(r1.z, P.np[1])) * P.np[2]
                                       + bin_word(r1.w, P.np[2]);
                                b1xy = bin_word(r0.w, P.np[0]) * P.np[1] + bin_word(r1.x, P.np[1]);
                            }
                            S.bxy[sb] = make_int2(b1xy, binf(bx, L, inv_dp0, P.np[0]) * P.np[1] + binf(by, L, inv_dp1, P.np[1]));
                            S.lin3meta[sb] = make_int2(lin3, meta);
                        } else {
                            S.w4[sb] = make_uint4(r0.w, r1.x, r1.y, r1.z);
                            S.bxyf[sb] = make_float2(bx, by);
                            S.lin3meta[sb] = make_int2((int)r1.w, meta);
                        }
                        S.wfac[sb] = MODE == M_RECORD ? 0.0f : wfac;
                    }
                    nlive += cnt;
                    ++c;
                    __syncwarp();
                } while (c < c1 && nlive - cons < 32);
                if (redo) {
                    flush = true;
                    continue;
                }
                if (!(nlive - cons >= 32 || (c >= c1 && nlive > cons))) continue;
            }
            // start a batch: the next <= 32 live samples, one per lane
            bstart = cons;
            bcnt = min(nlive - cons, 32);
            const int sb = (bstart + lane) & (SBUF - 1);
            if (lane < bcnt) {
                const float2 epz = S.EpPz[sb], ab = S.ab2m[sb];
                bEp = epz.x; bPz = epz.y; ba2m = ab.x; bb2m = ab.y; bkk3 = S.PPkk3[sb].y;
                bmeta = S.lin3meta[sb].y;
            } else {
                bmeta = 0;
            }
            ti = 0;
        }
        if (ti < nt) {
            // the batch's further groups in the same pass while the ring has room
            do {
                // ---- phase A: the kinematic group opened by term ti, for this lane's
                // live sample.  Its terms (equal leg masses) share E3, D, kappa, H, the
                // roots and the re-evaluation decision; each valid root goes to the
                // ring once, tagged with the group's terms. ----
                const int seq = bstart + lane;
                const int gn = GROUPS ? S.tgn[ti] : 1;  // without GROUPS every group has one term
                const bool act = lane < bcnt;
                const bool k2xy_in = (bmeta >> 24) & 1, marg_xy = (bmeta >> 25) & 1;
                const float4 tmv = S.tm[ti];
                const float ma2 = tmv.x, mb2 = tmv.y, mc2 = tmv.z;
                const float E3 = sqrtf(bkk3 + mc2);
                const float E = bEp + E3;
                const float Pz = bPz;
                const float a2 = ba2m + ma2;
                const float b2 = bb2m + mb2;
                const float D = E * E - Pz * Pz;
                const float kap = (E * E + a2 - b2 - Pz * Pz) * 0.5f;
                const float H = kap * kap - a2 * D;
                // straight-line form (no divergent branches): every lane evaluates the
                // roots, and the flags select; float-float re-evaluation when the term is
                // ill-conditioned (|H| < tau kappa^2) or a solved coordinate sits on an edge
                const bool ok = act & (D > 0.0f);
                const bool hp = ok & (H > 0.0f);
                bool defer = ok & may_defer & (fabsf(H) < P.tau * (kap * kap));
                const float sqH = sqrtf(H);
                const float kp = kap * Pz;
                const float sq = E * sqH;
                const float Q = kp >= 0.0f ? kp + sq : kp - sq;
                const bool qv = hp & (Q != 0.0f);
                const float z0 = Q / D;
                const float z1 = (E * E * a2 - kap * kap) / Q;
                const float w0 = kap + Pz * z0, w1 = kap + Pz * z1, EE = E * E;
                const bool e0 = qv & (w0 > 0.0f) & (w0 < EE), e1v = qv & (w1 > 0.0f) & (w1 < EE);
                const float nu = EDGE_Z * (1.0f + fabsf(kap) / sqH);
                const bool edge = (marg_xy & (e0 | e1v))
                                  | (e0 & (near_edge(z0, L, inv_dp2, nu) | near_edge(Pz - z0, L, inv_dp2, nu)))
                                  | (e1v & (near_edge(z1, L, inv_dp2, nu) | near_edge(Pz - z1, L, inv_dp2, nu)));
                defer = defer | (may_defer & edge);
                bool v0 = k2xy_in & e0 & in_box(z0, L) & in_box(Pz - z0, L);
                bool v1 = k2xy_in & e1v & in_box(z1, L) & in_box(Pz - z1, L);
                int t0 = ti, tn = gn;  // terms whose roots phase B evaluates
                if (defer) {  // queued for re-evaluation; when the queue is full the FP32 roots stand
                    const int qs = atomicAdd(dq.s_count, gn);
                    const int nq = min(gn, max(0, dq.cap - qs));
                    for (int k = 0; k < nq; ++k)
                        dq.seg[qs + k] = box_tag | ((unsigned long long)a << 24)
                                         | ((unsigned long long)(bmeta & 0xFFFFFF) << 4) | (unsigned long long)(ti + k);
                    if (nq < gn) red_add(&P.flags[3], gn - nq);
                    t0 = ti + nq;
                    tn = gn - nq;
                    if (tn == 0) v0 = v1 = false;
                }
                // append the valid roots to the ring
                const unsigned tag = (unsigned)seq | ((unsigned)t0 << 24) | ((unsigned)(tn - 1) << 28);
                const unsigned b0 = __ballot_sync(0xffffffffu, v0);
                const unsigned b1 = __ballot_sync(0xffffffffu, v1);
                const int n0 = __popc(b0);
                if (v0) {
                    const int r = (tail + __popc(b0 & lt_mask)) & (RING - 1);
                    S.ring[r] = make_float4(z0, E3, sqH, __uint_as_float(tag));
                }
                if (v1) {
                    const int r = (tail + n0 + __popc(b1 & lt_mask)) & (RING - 1);
                    S.ring[r] = make_float4(z1, E3, sqH, __uint_as_float(tag));
                }
                tail += n0 + __popc(b1);
                ti += gn;
                __syncwarp();
            } while (GROUPS && ti < nt && tail - head < 32);
        }
        if (ti >= nt) {  // batch done; record mode first finishes its roots, then writes records
            cons = bstart + bcnt;
            ti = -1;
            if (MODE == M_RECORD) {
                flush = true;
                rec_due = true;
            }
        }
    }
    if (MODE != M_RECORD) {
        own = warp_sum_ll(own);
        if (lane == 0 && own != 0 && bz_in(a, P.ncell)) red_add(&P.A[a], own);
    }
    __syncwarp();
}

// FP32 collision, one warp per unit (an anchor and up to 32 F32_GROUP of its samples).
// Single box (BATCH false): a grid of resident blocks whose warps take
// `chunk` units at a time from `counter` (zeroed by the caller), so every
// warp works until the units run out; without a counter, warps stride over
// the units of `one`.
// Batch of independent boxes (BATCH true): warps take chunks of `chunk`
// units from a global counter over the concatenated unit space (prefix[b] =
// first unit of box b), so ragged boxes share the GPU evenly; the step index
// is read from device memory, so a captured graph replays with the same
// parameters.
// Both run the same collide_unit source (the single box with its argument
// block in the constant bank, the batch with each box's block in global
// memory): a box gives the same bits alone or inside a batch.
template <int MODE, bool GROUPS, bool BATCH>
__global__ void __launch_bounds__(32 * WARPS, (GROUPS && !BATCH) ? BZ_F32_MIN_BLOCKS_GROUPED : BZ_F32_MIN_BLOCKS)
    k_collide_f32(const __grid_constant__ CollideArgs<float> one, const CollideArgs<float>* __restrict__ boxes,
                  const int64_t* __restrict__ prefix, int nboxes, unsigned long long* counter, const int* step_dev,
                  int chunk, int* qcount, unsigned long long* qitems, long long qcap)
{
    __shared__ WarpSmem<(!GROUPS && MODE != M_LEARNED)> smem[WARPS];
    __shared__ int s_qcount[WARPS];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * WARPS + warp;
    const int64_t nwarps = (int64_t)gridDim.x * WARPS;
    if (lane == 0) s_qcount[warp] = 0;
    __syncwarp();
    DeferCtx dq;
    dq.s_count = &s_qcount[warp];
    dq.seg = qitems + gw * qcap;
    dq.cap = (int)qcap;
    const bool batch = BATCH;
    const bool dyn = counter != nullptr;  // chunks of units from the counter (a batch always)
    const int64_t total = batch ? prefix[nboxes] : f32_units(one.n_sel, one.nsamples);
    const int step = batch ? *step_dev : (one.step_dev ? *one.step_dev : one.step);
    int b = 0;
    int64_t u = dyn ? 0 : gw, stop = 0;  // next unit; end of the current chunk
    for (;;) {
        if (dyn) {
            if (u >= stop) {
                unsigned long long start = 0;
                if (lane == 0) start = atomicAdd(counter, (unsigned long long)chunk);
                start = __shfl_sync(0xffffffffu, start, 0);
                if ((int64_t)start >= total) break;
                u = (int64_t)start;
                stop = min(u + chunk, total);
            }
            if (batch && (u < prefix[b] || u >= prefix[b + 1])) {  // binary search for the box of u
                int lo = 0, hi = nboxes - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (prefix[mid] <= u) lo = mid; else hi = mid - 1;
                }
                b = lo;
            }
        } else if (u >= total) {
            break;
        }
        // one call site per instantiation: a single box reads its arguments
        // from the constant bank, a batch box from global memory; the
        // arithmetic is the same source, so a box gives the same bits either way
        if (BATCH)
            collide_unit<MODE, GROUPS, false>(boxes[b], u - prefix[b], step, smem[warp], dq,
                                              (unsigned long long)b << 48);
        else
            collide_unit<MODE, GROUPS, true>(one, u, step, smem[warp], dq, 0ull);
        u += dyn ? 1 : nwarps;
    }
    __syncwarp();
    if (lane == 0) {
        const int c = s_qcount[warp];
        qcount[gw] = c < qcap ? c : (int)qcap;
    }
}

// Some equation has a kinematic group of several terms (else every ring
// entry carries one term and phase B needs no loop over a group).
static bool has_groups(const CollideArgs<float>& a)
{
    for (int d = 0; d < NSPEC; ++d)
        for (int t = 1; t < a.nterms[d]; ++t)
            if (!a.terms[d][t].gfirst) return true;
    return false;
}

cudaError_t check_read_collide_f32(unsigned long long out[2], bool reset)
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

// The instantiation a single-box launch runs, and its resident blocks per SM.
template <int MODE, bool GROUPS>
static int resident_blocks()
{
    static int n = 0;
    if (!n && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_collide_f32<MODE, GROUPS, false>, 32 * WARPS, 0) !=
                   cudaSuccess || n < 1))
        n = 1;
    return n;
}

int collide_f32_resident_blocks(const CollideArgs<float>& a)
{
    if (a.rec_stride) return resident_blocks<M_RECORD, true>();
    if (a.sampler == SAMPLER_LEARNED) return resident_blocks<M_LEARNED, true>();
    return has_groups(a) ? resident_blocks<M_UNIFORM, true>() : resident_blocks<M_UNIFORM, false>();
}

cudaError_t launch_collide_f32(const CollideArgs<float>& a, int grid, unsigned long long* counter, cudaStream_t s)
{
    if (a.rec_stride)
        k_collide_f32<M_RECORD, true, false><<<grid, 32 * WARPS, 0, s>>>(a, nullptr, nullptr, 0, counter, nullptr, 1, a.qcount,
                                                                   a.qitems, a.qcap);
    else if (a.sampler == SAMPLER_LEARNED)
        k_collide_f32<M_LEARNED, true, false><<<grid, 32 * WARPS, 0, s>>>(a, nullptr, nullptr, 0, counter, nullptr, 1, a.qcount,
                                                                    a.qitems, a.qcap);
    else if (has_groups(a))
        k_collide_f32<M_UNIFORM, true, false><<<grid, 32 * WARPS, 0, s>>>(a, nullptr, nullptr, 0, counter, nullptr, 1, a.qcount,
                                                                    a.qitems, a.qcap);
    else
        k_collide_f32<M_UNIFORM, false, false><<<grid, 32 * WARPS, 0, s>>>(a, nullptr, nullptr, 0, counter, nullptr, 1,
                                                                     a.qcount, a.qitems, a.qcap);
    return cudaGetLastError();
}

cudaError_t launch_collide_f32_batch(const CollideArgs<float>* boxes, const int64_t* prefix, int nboxes,
                                     unsigned long long* counter, const int* step_dev, int chunk, int grid,
                                     int* qcount, unsigned long long* qitems, long long qcap, cudaStream_t s)
{
    const CollideArgs<float> none{};
    k_collide_f32<M_UNIFORM, true, true><<<grid, 32 * WARPS, 0, s>>>(none, boxes, prefix, nboxes, counter, step_dev, chunk, qcount,
                                                          qitems, qcap);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Re-evaluation of a queued (anchor, sample, term).  What made the term
// ill-conditioned, or put a solved coordinate on a bin edge, is redone in
// float-float arithmetic (about 48 bits, FP32 instructions only; FP64 issues
// at 1/64 of the FP32 rate here): the sample point from the same Philox
// words (the uniform sampler's exactly, the learned one's Student-t inverse
// CDF too; its weight in FP32), E, D, kappa, H, the roots and
// their validity, box and bin decisions (the uniform sampler's sampled legs
// take the exact integer bins), E1, s, t and u.  From the accepted roots on
// (|M|^2, W and c~ in FP32) it is an ordinary term of the FP32 path.
// Returns the anchor's +q.  Not inlined: the single-box and the batch fixup
// kernels call one compiled body, so a queued term gives the same bits in
// both.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int bin_ff(ff k, ff L, ff dp, int n)
{
    int j = ff_floor(ff_div(ff_add(k, L), dp));
    j = j < 0 ? 0 : j;
    return j >= n ? n - 1 : j;
}

// Learned sampler: FP64 truncation constants of the last anchor a thread saw
// (consecutive queue items mostly come from one anchor).
struct PropCache {
    int64_t a = -1;
    float mu[3], s1, s3, alpha;
    ff Fa[4], cFb[4], D[4];  // components: k1 (centre 0, sigma1), k3x, k3y, k3z
    // float-float constants of the last box and x cell a thread saw, so that an item
    // converts no doubles (FP64 instructions issue at 1/64 of the FP32 rate)
    const void* box = nullptr;
    int64_t x = -1;
    ff L, nL, twoL, dp[3];
    ff m2[4], mg2;
};

template <bool LEARNED>
__device__ __noinline__ long long fixup_term_ff(const CollideArgs<float>& P, int64_t a, int smp, int ti, int step,
                                                PropCache& pc)
{
    const int64_t nxc = P.nxc, npc = P.npc;
    const uint32_t sl_u = udiv((uint32_t)a, P.dv_slot);
    const uint32_t rem = (uint32_t)a - sl_u * (uint32_t)(nxc * npc);
    const uint32_t x_u = udiv(rem, P.dv_npc);
    const int sl = (int)sl_u;
    const int64_t x = x_u;
    const int j = (int)(rem - x_u * (uint32_t)npc);
    const int d = P.slot_species[sl];
    const uint32_t jx_u = udiv((uint32_t)j, P.dv_yz);
    const uint32_t ryz = (uint32_t)j - jx_u * (uint32_t)(P.np[1] * P.np[2]);
    const uint32_t jy_u = udiv(ryz, P.dv_z);
    const int jx = (int)jx_u, jy = (int)jy_u, jz = (int)(ryz - jy_u * (uint32_t)P.np[2]);
    const uint32_t ctr3 = ((uint32_t)step << 3) | (uint32_t)d;
    const uint4 r0 = philox4x32_10(make_uint4(2u * smp, (uint32_t)j, (uint32_t)x, ctr3), P.key0, P.key1);
    const uint4 r1 = philox4x32_10(make_uint4(2u * smp + 1u, (uint32_t)j, (uint32_t)x, ctr3), P.key0, P.key1);
    // 23-bit uniforms (x + 1/2) 2^-23 are exact in FP32, and so is u - 1/2
    auto u23 = [](uint32_t w) { return unif23(w); };  // exact, without a conversion instruction
    if (pc.box != (const void*)&P) {
        pc.box = &P;
        pc.x = -1;
        pc.L = ff_from_double(P.L64);
        pc.nL = ff_neg(pc.L);
        pc.twoL = ff_from_double(2.0 * P.L64);
        for (int i = 0; i < 3; ++i) pc.dp[i] = ff_from_double(P.dp64[i]);
    }
    if (pc.x != x) {
        pc.x = x;
        for (int i = 0; i < 4; ++i) pc.m2[i] = P.mass_mode == 1 ? ff{0.0f, 0.0f} : ff_from_double(P.m2[x * 4 + i]);
        pc.mg2 = ff_from_double(P.m2[x * 4]);
    }
    const ff L = pc.L, nL = pc.nL, twoL = pc.twoL;
    const ff dp[3] = {pc.dp[0], pc.dp[1], pc.dp[2]};
    const int jv[3] = {jx, jy, jz};
    const float uj[3] = {u23(r0.x), u23(r0.y), u23(r0.z)};
    ff p[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        p[i] = ff_add(ff_add(nL, ff_mul_f(dp[i], (__uint_as_float(0x4B000000u | (unsigned)jv[i]) - 8388608.0f) + 0.5f)),
                      ff_mul_f(dp[i], uj[i] - 0.5f));  // the bin index as a float, exactly (< 2^23)
    ff k1x, k1y, k30, k31, k32;
    int b1xy, lin3;
    float wfac = 1.0f;
    if (LEARNED) {
        // the learned sample point in float-float (the integrand of a queued term is
        // sensitive to it): v = Fa + u D, cv = cFb + (1 - u) D, y = mu + s (v - cv) /
        // sqrt(2 v cv) on Student-t draws, y = 2u - 1 on uniform ones; its weight 1/(32 q)
        // in FP32 from the same values
        if (pc.a != a) {
            const float* pr = P.prop + a * 8;
            for (int i = 0; i < 3; ++i) pc.mu[i] = pr[i];
            pc.s3 = pr[3];
            pc.s1 = pr[4];
            pc.alpha = pr[5];
            for (int c = 0; c < 4; ++c) {
                const ff mu = ff_from(c == 0 ? 0.0f : pc.mu[c - 1]), sg = ff_from(c == 0 ? pc.s1 : pc.s3);
                pc.Fa[c] = ff_t2_tail(ff_div(ff_sub(ff_from(-1.0f), mu), sg));
                pc.cFb[c] = ff_t2_tail(ff_div(ff_sub(ff_from(1.0f), mu), sg));
                pc.D[c] = ff_sub(ff_sub(ff_from(1.0f), pc.cFb[c]), pc.Fa[c]);
            }
            pc.a = a;
        }
        const uint4 r2 = philox4x32_10(make_uint4(0x80000000u | (uint32_t)smp, (uint32_t)j, (uint32_t)x, ctr3),
                                       P.key0, P.key1);
        const float uv[5] = {u23(r0.w), u23(r1.x), u23(r1.y), u23(r1.z), u23(r1.w)};
        const bool uni = u23(r2.x) < pc.alpha;
        ff y[5];
        float G = 1.0f;
        for (int i = 0; i < 5; ++i) {
            const int c = i < 2 ? 0 : i - 1;
            const float mu = i < 2 ? 0.0f : pc.mu[i - 2], sg = i < 2 ? pc.s1 : pc.s3;
            const float Dh = ff_to_float(pc.D[c]);
            if (uni) {
                y[i] = ff_from(2.0f * uv[i] - 1.0f);  // exact
                const float zz = (y[i].hi - mu) / sg;
                const float r = rsqrtf(2.0f + zz * zz);
                G *= r * r * r / (sg * Dh);
            } else {
                const ff v = ff_add(pc.Fa[c], ff_mul_f(pc.D[c], uv[i]));
                const ff cv = ff_add(pc.cFb[c], ff_mul_f(pc.D[c], 1.0f - uv[i]));  // 1 - u exact
                const ff t = ff_mul_f(ff_mul(v, cv), 2.0f);
                y[i] = ff_add(ff_from(mu), ff_mul_f(ff_div(ff_sub(v, cv), ff_sqrt(t)), sg));
                if (ff_lt(y[i], ff_from(-1.0f))) y[i] = ff_from(-1.0f);
                if (ff_ge(y[i], ff_from(1.0f))) y[i] = ff_from(0.99999994f);
                const float th = ff_to_float(t);
                G *= th * sqrtf(th) / (sg * Dh);
            }
        }
        wfac = 1.0f / (32.0f * (pc.alpha * (1.0f / 32.0f) + (1.0f - pc.alpha) * G));
        k1x = ff_mul(L, y[0]);
        k1y = ff_mul(L, y[1]);
        k30 = ff_mul(L, y[2]);
        k31 = ff_mul(L, y[3]);
        k32 = ff_mul(L, y[4]);
        b1xy = bin_ff(k1x, L, dp[0], P.np[0]) * P.np[1] + bin_ff(k1y, L, dp[1], P.np[1]);
        lin3 = (bin_ff(k30, L, dp[0], P.np[0]) * P.np[1] + bin_ff(k31, L, dp[1], P.np[1])) * P.np[2]
               + bin_ff(k32, L, dp[2], P.np[2]);
    } else {
        k1x = ff_add(nL, ff_mul_f(twoL, u23(r0.w)));
        k1y = ff_add(nL, ff_mul_f(twoL, u23(r1.x)));
        k30 = ff_add(nL, ff_mul_f(twoL, u23(r1.y)));
        k31 = ff_add(nL, ff_mul_f(twoL, u23(r1.z)));
        k32 = ff_add(nL, ff_mul_f(twoL, u23(r1.w)));
        b1xy = bin_word(r0.w, P.np[0]) * P.np[1] + bin_word(r1.x, P.np[1]);
        lin3 = (bin_word(r1.y, P.np[0]) * P.np[1] + bin_word(r1.z, P.np[1])) * P.np[2] + bin_word(r1.w, P.np[2]);
    }
    const ff Px = ff_add(p[0], k30), Py = ff_add(p[1], k31), Pz = ff_add(p[2], k32);
    const ff bx = ff_sub(Px, k1x), by = ff_sub(Py, k1y);
    if (!(ff_ge(bx, nL) && ff_lt(bx, L) && ff_ge(by, nL) && ff_lt(by, L))) return 0;
    const TermDev& T = P.terms[d][ti];
    const ff mg2 = pc.mg2;
    const ff ma2 = pc.m2[T.mslot[0]], mb2 = pc.m2[T.mslot[1]], mc2 = pc.m2[T.mslot[2]], md2 = pc.m2[T.mslot[3]];
    const ff Ep = ff_sqrt(ff_add(ff_add(ff_add(ff_sqr(p[0]), ff_sqr(p[1])), ff_sqr(p[2])), md2));
    const ff E3 = ff_sqrt(ff_add(ff_add(ff_add(ff_sqr(k30), ff_sqr(k31)), ff_sqr(k32)), mc2));
    const ff E = ff_add(Ep, E3), EE = ff_sqr(E);
    const ff a2 = ff_add(ff_add(ff_sqr(k1x), ff_sqr(k1y)), ma2);
    const ff b2 = ff_add(ff_add(ff_sqr(bx), ff_sqr(by)), mb2);
    const ff Pz2 = ff_sqr(Pz);
    const ff D = ff_sub(EE, Pz2);
    ff kap = ff_sub(ff_sub(ff_add(EE, a2), b2), Pz2);
    kap = {kap.hi * 0.5f, kap.lo * 0.5f};
    const ff H = ff_sub(ff_sqr(kap), ff_mul(a2, D));
    if (!ff_gt0(D) || !ff_gt0(H)) return 0;
    const ff sqH = ff_sqrt(H);
    const ff kp = ff_mul(kap, Pz), sq = ff_mul(E, sqH);
    const ff Q = ff_ge0(kp) ? ff_add(kp, sq) : ff_sub(kp, sq);
    if (Q.hi == 0.0f) return 0;
    const ff zr[2] = {ff_div(Q, D), ff_div(ff_sub(ff_mul(EE, a2), ff_sqr(kap)), Q)};
    const float s = ff_to_float(ff_sub(EE, ff_add(ff_add(ff_sqr(Px), ff_sqr(Py)), Pz2)));
    const ff k13 = ff_add(ff_mul(k1x, k30), ff_mul(k1y, k31)), k1p = ff_add(ff_mul(k1x, p[0]), ff_mul(k1y, p[1]));
    const ff mac = ff_add(ma2, mc2), mad = ff_add(ma2, md2);
    const unsigned slot_stride = (unsigned)(nxc * npc), xoff = (unsigned)(x * npc);
    const int b2xy = bin_ff(bx, L, dp[0], P.np[0]) * P.np[1] + bin_ff(by, L, dp[1], P.np[1]);
    const float fp = P.analytic ? 0.0f : __ldg(static_cast<const float*>(P.f) + a);
    const float den0 = __fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(P.twopi5, 16.0f), ff_to_float(sqH)), ff_to_float(E3)),
                                 ff_to_float(Ep));
    long long own = 0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const ff z = zr[r], dz = ff_sub(Pz, z);
        const ff e2E = ff_add(kap, ff_mul(Pz, z));  // E2 E at a root: valid iff 0 < E2 < E
        if (!(ff_gt0(e2E) && ff_lt(e2E, EE))) continue;
        if (!(ff_ge(z, nL) && ff_lt(z, L) && ff_ge(dz, nL) && ff_lt(dz, L))) continue;
        const ff E1 = ff_sqrt(ff_add(a2, ff_sqr(z)));
        const ff tt = ff_sub(mac, ff_mul_f(ff_sub(ff_mul(E1, E3), ff_add(k13, ff_mul(z, k32))), 2.0f));
        const ff uf = ff_sub(mad, ff_mul_f(ff_sub(ff_mul(E1, Ep), ff_add(k1p, ff_mul(z, p[2]))), 2.0f));
        if (!(s > 0.0f) || ff_ge0(ff_sub(tt, mg2)) || ff_ge0(ff_sub(uf, mg2))) {
            red_add(&P.flags[0], 1);
            continue;
        }
        const float M2 = msq<float>(T.cls, P, s, ff_to_float(tt), ff_to_float(uf), ff_to_float(mg2));
        const int lin1 = b1xy * P.np[2] + bin_ff(z, L, dp[2], P.np[2]);
        const int lin2 = b2xy * P.np[2] + bin_ff(dz, L, dp[2], P.np[2]);
        const unsigned i1 = (unsigned)T.slot[0] * slot_stride + xoff + lin1;
        const unsigned i2 = (unsigned)T.slot[1] * slot_stride + xoff + lin2;
        const unsigned i3 = (unsigned)T.slot[2] * slot_stride + xoff + lin3;
        if (!(bz_in(i1, P.ncell) & bz_in(i2, P.ncell) & bz_in(i3, P.ncell))) continue;
        float f1, f2, f3, fpp;
        if (P.analytic) {
            f1 = f_equilibrium(P, P.slot_species[T.slot[0]], ff_to_float(E1));
            f2 = f_equilibrium(P, P.slot_species[T.slot[1]], ff_to_float(ff_sub(E, E1)));
            f3 = f_equilibrium(P, P.slot_species[T.slot[2]], ff_to_float(E3));
            fpp = f_equilibrium(P, d, ff_to_float(Ep));
        } else {
            const float* F = static_cast<const float*>(P.f);
            f1 = __ldg(F + i1);
            f2 = __ldg(F + i2);
            f3 = __ldg(F + i3);
            fpp = fp;
        }
        const float F1 = T.quark[0] ? 1.0f - f1 : 1.0f + f1;
        const float F2 = T.quark[1] ? 1.0f - f2 : 1.0f + f2;
        const float F3 = T.quark[2] ? 1.0f - f3 : 1.0f + f3;
        const float Fp = T.quark[3] ? 1.0f - fpp : 1.0f + fpp;
        // W and c~ rounded as written (no contraction), like the float-float part
        const float W = __fsub_rn(__fmul_rn(__fmul_rn(__fmul_rn(f1, f2), F3), Fp),
                                  __fmul_rn(__fmul_rn(__fmul_rn(F1, F2), f3), fpp));
        // |J| E1 E2 = sqrt(H) at a root of Eq. (work out delta E)
        const float ct = __fdiv_rn(__fmul_rn(__fmul_rn((float)T.sym, W), M2), den0);
        const float wq = LEARNED ? __fmul_rn(__fmul_rn(ct, P.Kown), wfac) : __fmul_rn(ct, P.Kown);
        if (!(fabsf(wq) < 4611686018427387904.0f)) {
            red_add(&P.flags[1], 1);
            continue;
        }
        const long long q = rint_ll(wq);
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

// `split` warps per queue segment (the items of a segment are dealt over
// their 32 split lanes).  The learned form gives each lane a contiguous run
// of items, so that its cached per-anchor constants are reused.
template <bool LEARNED>
__global__ void __launch_bounds__(256, BZ_FIX_MINB) k_fixup_f32(const __grid_constant__ CollideArgs<float> P, const int* qcount,
                                                   const unsigned long long* qitems, int64_t qcap, int nseg, int split)
{
    const int64_t gw = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int64_t seg = gw / split;
    if (seg >= nseg) return;
    const int n = qcount[seg];
    const int slots = 32 * split, slot = (int)(gw - seg * split) * 32 + (threadIdx.x & 31);
    const int run = LEARNED ? (n + slots - 1) / slots : 1;
    const int i0 = LEARNED ? slot * run : slot, i1 = LEARNED ? min(n, i0 + run) : n, di = LEARNED ? 1 : slots;
    PropCache pc;
    const int step = P.step_dev ? *P.step_dev : P.step;
    for (int i = i0; i < i1; i += di) {
        const unsigned long long it = qitems[seg * qcap + i];
        const int64_t a = (int64_t)(it >> 24);
        const int smp = (int)((it >> 4) & 0xFFFFFu), ti = (int)(it & 0xFu);
        const long long own = fixup_term_ff<LEARNED>(P, a, smp, ti, step, pc);
        if (own != 0 && bz_in(a, P.ncell)) red_add(&P.A[a], own);
    }
}

// Batch form: the item carries its box (bits 48..63); the step is read from
// device memory.
__global__ void __launch_bounds__(256, BZ_FIX_MINB) k_fixup_f32_batch(const CollideArgs<float>* __restrict__ boxes,
                                                         const int* qcount, const unsigned long long* qitems,
                                                         int64_t qcap, const int* step_dev, int nseg, int split)
{
    const int64_t gw = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int64_t seg = gw / split;
    if (seg >= nseg) return;
    const int n = qcount[seg];
    const int slots = 32 * split, slot = (int)(gw - seg * split) * 32 + (threadIdx.x & 31);
    const int step = *step_dev;
    PropCache pc;
    for (int i = slot; i < n; i += slots) {
        const unsigned long long it = qitems[seg * qcap + i];
        const CollideArgs<float>& P = boxes[(int)(it >> 48)];
        const int64_t a = (int64_t)((it >> 24) & 0xFFFFFFull);
        const long long own = fixup_term_ff<false>(P, a, (int)((it >> 4) & 0xFFFFFu), (int)(it & 0xFu), step, pc);
        if (own != 0 && bz_in(a, P.ncell)) red_add(&P.A[a], own);
    }
}

// Warps per queue segment: enough warps for about two full waves of the
// fixup's resident warps (BZ_FIX_MINB blocks of 8 warps per SM).
static int fixup_split(int nseg)
{
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || nsm < 1)
            nsm = 1;
    }
    const int64_t want = 2ll * nsm * BZ_FIX_MINB * 8;
    const int64_t sp = (want + nseg - 1) / (nseg > 0 ? nseg : 1);
    return (int)(sp < 1 ? 1 : (sp > BZ_FIX_SPLIT_MAX ? BZ_FIX_SPLIT_MAX : sp));
}

cudaError_t launch_fixup_f32(const CollideArgs<float>& a, int nseg, cudaStream_t s)
{
    // the learned form keeps one warp per segment: longer runs per lane reuse
    // its cached per-anchor constants more (measured: split 3 was 3% slower)
    const int split = a.sampler == SAMPLER_LEARNED ? 1 : fixup_split(nseg);
    const unsigned grid = (unsigned)(((int64_t)nseg * split + 7) / 8);
    if (a.sampler == SAMPLER_LEARNED)
        k_fixup_f32<true><<<grid, 256, 0, s>>>(a, a.qcount, a.qitems, a.qcap, nseg, split);
    else
        k_fixup_f32<false><<<grid, 256, 0, s>>>(a, a.qcount, a.qitems, a.qcap, nseg, split);
    return cudaGetLastError();
}

cudaError_t launch_fixup_f32_batch(const CollideArgs<float>* boxes, const int* qcount, const unsigned long long* qitems,
                                   int64_t qcap, const int* step_dev, int nseg, cudaStream_t s)
{
    const int split = fixup_split(nseg);
    k_fixup_f32_batch<<<(unsigned)(((int64_t)nseg * split + 7) / 8), 256, 0, s>>>(boxes, qcount, qitems, qcap, step_dev,
                                                                                 nseg, split);
    return cudaGetLastError();
}


}  // namespace bz
