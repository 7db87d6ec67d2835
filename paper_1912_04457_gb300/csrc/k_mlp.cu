// Learned proposal network: a 9 -> 128 -> 128 -> 6 MLP (SiLU) on BF16 tensor
// cores with FP32 accumulation (mma.sync.m16n8k16), its training forward and
// backward pass, the Adam update, and per-anchor inference.
//
// Precision contract (the CPU oracle rounds at the same points): every GEMM
// operand is BF16 (inputs, weights, activations, output gradients), every
// accumulation FP32; pre-activations Z are kept in BF16 and SiLU / SiLU' are
// evaluated in FP32 from them; bias gradients are sums of the BF16 dZ.
//
// Parameter vector (FP32 master copy, flat): W1[16][128] (input rows 9..15
// zero), b1[128], W2[128][128], b2[128], W3[128][8] (output columns 6, 7
// zero), b3[8] -- W[in][out], y = x W + b.
//
// Proposal from the 6 outputs o (normalised box y = (k1x, k1y, k3)/L in
// [-1, 1)^5): mu3 = tanh(o0..2), sigma3 = 0.02 + 0.5 sigmoid(o3), sigma1 =
// 0.02 + 0.5 sigmoid(o4), alpha = 0.1 + 0.9 sigmoid(o5);
//   q(y) = alpha / 32 + (1 - alpha) prod_i g_i(y_i),
// g_i the Student-t density with two degrees of freedom, f(z) = (2 + z^2)^(-3/2),
// truncated to [-1, 1), with centre 0 (k1 components, scale sigma1) or mu3
// (k3 components, scale sigma3); its CDF is 1/2 + z / (2 sqrt(2 + z^2)).
// Training loss over records (y, w = sum over terms and roots of |c~|, taken
// with the uniform sampler): L = -sum w log q(y) / sum w  (q -> |c~| / int|c~|).
#include <cuda_bf16.h>
#include <cstdint>
#include "bz_internal.h"

namespace bz {

namespace {

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// C[16x8 tile at (m0, n0)] += A[m0.., 0..K) B[0..K, n0..], A(m, k) = A[m ars + k acs],
// B(k, n) = B[k bks + n bns], K a multiple of 16.  Fragment layout of
// mma.m16n8k16 .row.col (PTX ISA): g = lane >> 2, t = lane & 3;
// A regs {(g, 2t..2t+1), (g+8, 2t..), (g, 2t+8..), (g+8, 2t+8..)},
// B regs {(2t..2t+1, g), (2t+8.., g)}, C {(g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)}.
__device__ __forceinline__ void mma_tile(float c[4], const __nv_bfloat16* A, int ars, int acs, const __nv_bfloat16* B,
                                         int bks, int bns, int m0, int n0, int K)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const __nv_bfloat16* a0 = A + (m0 + g) * ars;
    const __nv_bfloat16* a1 = A + (m0 + g + 8) * ars;
    const __nv_bfloat16* bb = B + (n0 + g) * bns;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int ka = k0 + 2 * t, kb = k0 + 2 * t + 8;
        uint32_t ra[4], rb[2];
        ra[0] = pack2(a0[ka * acs], a0[(ka + 1) * acs]);
        ra[1] = pack2(a1[ka * acs], a1[(ka + 1) * acs]);
        ra[2] = pack2(a0[kb * acs], a0[(kb + 1) * acs]);
        ra[3] = pack2(a1[kb * acs], a1[(kb + 1) * acs]);
        rb[0] = pack2(bb[ka * bks], bb[(ka + 1) * bks]);
        rb[1] = pack2(bb[kb * bks], bb[(kb + 1) * bks]);
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(ra[0]), "r"(ra[1]), "r"(ra[2]), "r"(ra[3]), "r"(rb[0]), "r"(rb[1]));
    }
}

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu(float z) { return z * sigm(z); }
__device__ __forceinline__ float dsilu(float z)
{
    const float s = sigm(z);
    return s * (1.0f + z * (1.0f - s));
}

constexpr int H = 128;        // hidden width
constexpr int NIN = 16;       // padded input width (9 used)
constexpr int NOUT = 8;       // padded output width (6 used)
constexpr int CH = 64;        // samples per training chunk
constexpr int NPARAM = NIN * H + H + H * H + H + H * NOUT + NOUT;

struct MlpSmem {
    __nv_bfloat16 W1[NIN * H], W2[H * H], W3[H * 16];  // W3 padded to 16 output columns (zero)
    float b1[H], b2[H], b3[NOUT];
};

__device__ void load_weights(MlpSmem& S, const float* __restrict__ P)
{
    const float* W1 = P;
    const float* b1 = W1 + NIN * H;
    const float* W2 = b1 + H;
    const float* b2 = W2 + H * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + H * NOUT;
    for (int i = threadIdx.x; i < NIN * H; i += blockDim.x) S.W1[i] = __float2bfloat16_rn(W1[i]);
    for (int i = threadIdx.x; i < H * H; i += blockDim.x) S.W2[i] = __float2bfloat16_rn(W2[i]);
    for (int i = threadIdx.x; i < H * 16; i += blockDim.x) {
        const int r = i >> 4, c = i & 15;
        S.W3[i] = __float2bfloat16_rn(c < NOUT ? W3[r * NOUT + c] : 0.0f);
    }
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        S.b1[i] = b1[i];
        S.b2[i] = b2[i];
    }
    if (threadIdx.x < NOUT) S.b3[threadIdx.x] = b3[threadIdx.x];
}

// features of an anchor: p at its cell centre / L, |p|/L, |p|^2/L^2, species one-hot, 1
__device__ __forceinline__ void anchor_features(const ProposalArgs& A, int64_t a, float f[NIN])
{
    const int64_t npc = A.npc;
    const int sl = (int)(a / (A.nxc * npc));
    const int j = (int)(a % npc);
    const int d = A.slot_species[sl];
    const int jv[3] = {j / (A.np[1] * A.np[2]), (j / A.np[2]) % A.np[1], j % A.np[2]};
    float p[3];
    for (int i = 0; i < 3; ++i) p[i] = (-A.L + ((float)jv[i] + 0.5f) * (2.0f * A.L / A.np[i])) / A.L;
    const float pp = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    f[0] = p[0];
    f[1] = p[1];
    f[2] = p[2];
    f[3] = sqrtf(pp);
    f[4] = pp;
    f[5] = d == 0 ? 1.0f : 0.0f;
    f[6] = (d >= 1 && d <= 3) ? 1.0f : 0.0f;
    f[7] = d >= 4 ? 1.0f : 0.0f;
    f[8] = 1.0f;
    for (int i = 9; i < NIN; ++i) f[i] = 0.0f;
}

// proposal parameters from the outputs
__device__ __forceinline__ void head(const float o[6], float prm[8])
{
    prm[0] = tanhf(o[0]);
    prm[1] = tanhf(o[1]);
    prm[2] = tanhf(o[2]);
    prm[3] = 0.02f + 0.5f * sigm(o[3]);
    prm[4] = 0.02f + 0.5f * sigm(o[4]);
    prm[5] = 0.1f + 0.9f * sigm(o[5]);
    prm[6] = 0.0f;
    prm[7] = 0.0f;
}

// truncated Student-t (two degrees of freedom): density and the tail F(-|z|)
__device__ __forceinline__ float t2_pdf(float z)
{
    const float r = rsqrtf(2.0f + z * z);
    return r * r * r;
}
__device__ __forceinline__ float t2_tail(float z)
{
    const float s = sqrtf(2.0f + z * z);
    return 1.0f / (s * (s + fabsf(z)));
}

// log q(y) and d log q / d o (6) for one record
__device__ void logq_grad(const float o[6], const float y[5], float& logq, float g[6])
{
    float prm[8];
    head(o, prm);
    float G = 1.0f;
    float dmu[3], dsig3 = 0.0f, dsig1 = 0.0f;
    for (int i = 0; i < 5; ++i) {
        const bool k3 = i >= 2;
        const float mu = k3 ? prm[i - 2] : 0.0f;
        const float s = k3 ? prm[3] : prm[4];
        const float z = (y[i] - mu) / s, za = (-1.0f - mu) / s, zb = (1.0f - mu) / s;
        // za < 0 < zb: Z = F(zb) - F(za) = 1 - tail(zb) - tail(za)
        const float Z = (1.0f - t2_tail(zb)) - t2_tail(za);
        const float pa = t2_pdf(za), pb = t2_pdf(zb);
        G *= t2_pdf(z) / (s * Z);
        // d log g / d mu and d log g / d s, with d log f / dz = -3 z / (2 + z^2)
        const float dlf = -3.0f * z / (2.0f + z * z);
        const float dm = -dlf / s + (pb - pa) / (s * Z);
        const float ds = -dlf * z / s - 1.0f / s + (pb * zb - pa * za) / (s * Z);
        if (k3) {
            dmu[i - 2] = dm;
            dsig3 += ds;
        } else {
            dsig1 += ds;
        }
    }
    const float al = prm[5];
    const float q = al * (1.0f / 32.0f) + (1.0f - al) * G;
    logq = logf(q);
    const float r = (1.0f - al) * G / q;  // d log q / d log G
    for (int i = 0; i < 3; ++i) g[i] = r * dmu[i] * (1.0f - prm[i] * prm[i]);
    const float s3 = (prm[3] - 0.02f) / 0.5f, s1 = (prm[4] - 0.02f) / 0.5f;
    g[3] = r * dsig3 * 0.5f * s3 * (1.0f - s3);
    g[4] = r * dsig1 * 0.5f * s1 * (1.0f - s1);
    const float sa = (al - 0.1f) / 0.9f;
    g[5] = ((1.0f / 32.0f) - G) / q * 0.9f * sa * (1.0f - sa);
}

struct TrainSmem {
    MlpSmem w;
    __nv_bfloat16 X[CH * NIN];
    __nv_bfloat16 Z1[CH * H], H1[CH * H], Z2[CH * H], H2[CH * H];
    __nv_bfloat16 dO[CH * 16], dZ2[CH * H], dZ1[CH * H];
    float O[CH * NOUT];
    float yv[CH * 5], wv[CH];
    float db[H + H + NOUT];
};

}  // namespace

// One gradient evaluation over records [0, n): grad (FP32, NPARAM) += dL/dtheta
// with L = -sum w log q / wsum, and loss_sum += L.  Each block walks chunks of
// CH records and keeps its weight-gradient tiles in registers.
// SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): a bijective 64-bit mix.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Each block writes its own gradient and loss (part[block][NPARAM],
// part_loss[block]); k_grad_reduce adds the blocks in block order, so the
// result does not depend on which block finishes first.
__global__ void __launch_bounds__(256, 1) k_mlp_grad(const float* __restrict__ params, const ProposalArgs A,
                                                     const ProposalRecord* __restrict__ rec, int64_t n, float inv_wsum,
                                                     float* __restrict__ part, float* __restrict__ part_loss,
                                                     int64_t ntot, uint64_t key)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    load_weights(S.w, params);
    for (int i = threadIdx.x; i < 2 * H + NOUT; i += blockDim.x) S.db[i] = 0.0f;
    // register tiles of the weight gradients owned by this warp
    float gW2[16][4], gW1[2][4], gW3[4];
#pragma unroll
    for (int i = 0; i < 16; ++i) gW2[i][0] = gW2[i][1] = gW2[i][2] = gW2[i][3] = 0.0f;
#pragma unroll
    for (int i = 0; i < 2; ++i) gW1[i][0] = gW1[i][1] = gW1[i][2] = gW1[i][3] = 0.0f;
    gW3[0] = gW3[1] = gW3[2] = gW3[3] = 0.0f;
    float loss_blk = 0.0f;
    __syncthreads();
    const int64_t nchunks = (n + CH - 1) / CH;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        // ---- inputs ----
        if (threadIdx.x < CH) {
            const int64_t r = c * CH + threadIdx.x;
            float f[NIN];
            if (r < n) {
                const int64_t ri = ntot > 0 ? (int64_t)(splitmix64(key + (uint64_t)r) % (uint64_t)ntot) : r;
                const ProposalRecord R = rec[ri];
                anchor_features(A, R.a, f);
                for (int i = 0; i < 5; ++i) S.yv[threadIdx.x * 5 + i] = R.y[i];
                S.wv[threadIdx.x] = R.w * inv_wsum;
            } else {
                for (int i = 0; i < NIN; ++i) f[i] = 0.0f;
                for (int i = 0; i < 5; ++i) S.yv[threadIdx.x * 5 + i] = 0.0f;
                S.wv[threadIdx.x] = 0.0f;
            }
            for (int i = 0; i < NIN; ++i) S.X[threadIdx.x * NIN + i] = __float2bfloat16_rn(f[i]);
        }
        __syncthreads();
        // ---- Z1 = X W1 + b1 (64 x 128): 32 tiles of 16x8 per ... 4 m x 16 n = 64 tiles, 8 per warp ----
        for (int tt = warp; tt < 64; tt += 8) {
            const int m0 = (tt >> 4) * 16, n0 = (tt & 15) * 8;
            float acc[4] = {0, 0, 0, 0};
            mma_tile(acc, S.X, NIN, 1, S.w.W1, H, 1, m0, n0, NIN);
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + g + (e >> 1) * 8, nn = n0 + 2 * t + (e & 1);
                const __nv_bfloat16 z = __float2bfloat16_rn(acc[e] + S.w.b1[nn]);
                S.Z1[m * H + nn] = z;
                S.H1[m * H + nn] = __float2bfloat16_rn(silu(__bfloat162float(z)));
            }
        }
        __syncthreads();
        // ---- Z2 = H1 W2 + b2 ----
        for (int tt = warp; tt < 64; tt += 8) {
            const int m0 = (tt >> 4) * 16, n0 = (tt & 15) * 8;
            float acc[4] = {0, 0, 0, 0};
            mma_tile(acc, S.H1, H, 1, S.w.W2, H, 1, m0, n0, H);
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + g + (e >> 1) * 8, nn = n0 + 2 * t + (e & 1);
                const __nv_bfloat16 z = __float2bfloat16_rn(acc[e] + S.w.b2[nn]);
                S.Z2[m * H + nn] = z;
                S.H2[m * H + nn] = __float2bfloat16_rn(silu(__bfloat162float(z)));
            }
        }
        __syncthreads();
        // ---- O = H2 W3 + b3 (64 x 8): 4 tiles ----
        if (warp < 4) {
            const int m0 = warp * 16;
            float acc[4] = {0, 0, 0, 0};
            mma_tile(acc, S.H2, H, 1, S.w.W3, 16, 1, m0, 0, H);
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + g + (e >> 1) * 8, nn = 2 * t + (e & 1);
                S.O[m * NOUT + nn] = acc[e] + S.w.b3[nn];
            }
        }
        __syncthreads();
        // ---- loss and dL/dO per record ----
        if (threadIdx.x < CH) {
            const int r = threadIdx.x;
            const float w = S.wv[r];
            float gq[6] = {0, 0, 0, 0, 0, 0}, lq = 0.0f;
            if (w != 0.0f) {
                logq_grad(&S.O[r * NOUT], &S.yv[r * 5], lq, gq);
                loss_blk += -w * lq;
            }
            for (int i = 0; i < 16; ++i) S.dO[r * 16 + i] = __float2bfloat16_rn(i < 6 ? -w * gq[i] : 0.0f);
        }
        __syncthreads();
        // ---- dW3 += H2^T dO (128 x 8): 8 row tiles, one per warp ----
        mma_tile(gW3, S.H2, 1, H, S.dO, 16, 1, warp * 16, 0, CH);
        // ---- dZ2 = (dO W3^T) * silu'(Z2) (64 x 128), K = 16 ----
        for (int tt = warp; tt < 64; tt += 8) {
            const int m0 = (tt >> 4) * 16, n0 = (tt & 15) * 8;
            float acc[4] = {0, 0, 0, 0};
            mma_tile(acc, S.dO, 16, 1, S.w.W3, 1, 16, m0, n0, 16);
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + g + (e >> 1) * 8, nn = n0 + 2 * t + (e & 1);
                S.dZ2[m * H + nn] = __float2bfloat16_rn(acc[e] * dsilu(__bfloat162float(S.Z2[m * H + nn])));
            }
        }
        __syncthreads();
        // ---- dW2 += H1^T dZ2 (128 x 128): 128 tiles, 16 per warp ----
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int tt = warp * 16 + i;
            const int m0 = (tt >> 4) * 16, n0 = (tt & 15) * 8;
            mma_tile(gW2[i], S.H1, 1, H, S.dZ2, H, 1, m0, n0, CH);
        }
        // ---- dZ1 = (dZ2 W2^T) * silu'(Z1), K = 128 ----
        for (int tt = warp; tt < 64; tt += 8) {
            const int m0 = (tt >> 4) * 16, n0 = (tt & 15) * 8;
            float acc[4] = {0, 0, 0, 0};
            mma_tile(acc, S.dZ2, H, 1, S.w.W2, 1, H, m0, n0, H);
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + g + (e >> 1) * 8, nn = n0 + 2 * t + (e & 1);
                S.dZ1[m * H + nn] = __float2bfloat16_rn(acc[e] * dsilu(__bfloat162float(S.Z1[m * H + nn])));
            }
        }
        __syncthreads();
        // ---- dW1 += X^T dZ1 (16 x 128): 16 tiles, 2 per warp ----
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int n0 = (warp * 2 + i) * 8;
            mma_tile(gW1[i], S.X, 1, NIN, S.dZ1, H, 1, 0, n0, CH);
        }
        // ---- bias gradients: column sums of dZ1, dZ2, dO ----
        for (int col = threadIdx.x; col < 2 * H + NOUT; col += blockDim.x) {
            float s = 0.0f;
            if (col < H) {
                for (int m = 0; m < CH; ++m) s += __bfloat162float(S.dZ1[m * H + col]);
            } else if (col < 2 * H) {
                for (int m = 0; m < CH; ++m) s += __bfloat162float(S.dZ2[m * H + col - H]);
            } else {
                for (int m = 0; m < CH; ++m) s += __bfloat162float(S.dO[m * 16 + col - 2 * H]);
            }
            S.db[col] += s;
        }
        __syncthreads();
    }
    // ---- this block's gradient, every parameter written once ----
    float* gW1g = part + (int64_t)blockIdx.x * NPARAM;
    float* gb1g = gW1g + NIN * H;
    float* gW2g = gb1g + H;
    float* gb2g = gW2g + H * H;
    float* gW3g = gb2g + H;
    float* gb3g = gW3g + H * NOUT;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int tt = warp * 16 + i;
        const int m0 = (tt >> 4) * 16, n0 = (tt & 15) * 8;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int m = m0 + g + (e >> 1) * 8, nn = n0 + 2 * t + (e & 1);
            gW2g[m * H + nn] = gW2[i][e];
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int n0 = (warp * 2 + i) * 8;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int m = g + (e >> 1) * 8, nn = n0 + 2 * t + (e & 1);
            gW1g[m * H + nn] = gW1[i][e];
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int m = warp * 16 + g + (e >> 1) * 8, nn = 2 * t + (e & 1);
        gW3g[m * NOUT + nn] = gW3[e];
    }
    for (int col = threadIdx.x; col < 2 * H + NOUT; col += blockDim.x) {
        const float s = S.db[col];
        if (col < H)
            gb1g[col] = s;
        else if (col < 2 * H)
            gb2g[col - H] = s;
        else
            gb3g[col - 2 * H] = s;
    }
    // loss: the two warps of record threads, in warp order
    loss_blk += __shfl_xor_sync(0xffffffffu, loss_blk, 16);
    loss_blk += __shfl_xor_sync(0xffffffffu, loss_blk, 8);
    loss_blk += __shfl_xor_sync(0xffffffffu, loss_blk, 4);
    loss_blk += __shfl_xor_sync(0xffffffffu, loss_blk, 2);
    loss_blk += __shfl_xor_sync(0xffffffffu, loss_blk, 1);
    __shared__ float s_loss[2];
    if (lane == 0 && warp < 2) s_loss[warp] = loss_blk;
    __syncthreads();
    if (threadIdx.x == 0) part_loss[blockIdx.x] = s_loss[0] + s_loss[1];
}

// grad[i] += sum over blocks b = 0, 1, ... of part[b][i]; loss = sum of the
// blocks' losses in block order.
__global__ void k_grad_reduce(const float* __restrict__ part, const float* __restrict__ part_loss, int nblk,
                              float* __restrict__ grad, float* loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NPARAM) {
        float s = 0.0f;
        for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * NPARAM + i];
        grad[i] += s;
    }
    if (i == 0) {
        float l = 0.0f;
        for (int b = 0; b < nblk; ++b) l += part_loss[b];
        *loss = l;
    }
}

// Adam on the FP32 master parameters; zeroes the gradient.
__global__ void k_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g[i] = 0.0f;
}

// Per-anchor proposal parameters (8 floats: mu3 x3, sigma3, sigma1, alpha, 0, 0)
// for anchors [0, nanchor): each warp runs 16 anchors through the network.
__global__ void __launch_bounds__(256) k_mlp_infer(const float* __restrict__ params, const ProposalArgs A,
                                                   int64_t nanchor, float* __restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem& W = *reinterpret_cast<MlpSmem*>(smem_raw);
    __nv_bfloat16* act = reinterpret_cast<__nv_bfloat16*>(smem_raw + sizeof(MlpSmem));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    __nv_bfloat16* X = act + warp * (16 * NIN + 2 * 16 * H);
    __nv_bfloat16* H1 = X + 16 * NIN;
    __nv_bfloat16* H2 = H1 + 16 * H;
    load_weights(W, params);
    __syncthreads();
    const int64_t ngroups = (nanchor + 15) / 16;
    for (int64_t grp = (int64_t)blockIdx.x * 8 + warp; grp < ngroups; grp += (int64_t)gridDim.x * 8) {
        if (lane < 16) {
            const int64_t a = grp * 16 + lane;
            float f[NIN];
            if (a < nanchor)
                anchor_features(A, a, f);
            else
                for (int i = 0; i < NIN; ++i) f[i] = 0.0f;
            for (int i = 0; i < NIN; ++i) X[lane * NIN + i] = __float2bfloat16_rn(f[i]);
        }
        __syncwarp();
        for (int n0 = 0; n0 < H; n0 += 8) {
            float acc[4] = {0, 0, 0, 0};
            mma_tile(acc, X, NIN, 1, W.W1, H, 1, 0, n0, NIN);
            for (int e = 0; e < 4; ++e) {
                const int m = g + (e >> 1) * 8, nn = n0 + 2 * t + (e & 1);
                const __nv_bfloat16 z = __float2bfloat16_rn(acc[e] + W.b1[nn]);
                H1[m * H + nn] = __float2bfloat16_rn(silu(__bfloat162float(z)));
            }
        }
        __syncwarp();
        for (int n0 = 0; n0 < H; n0 += 8) {
            float acc[4] = {0, 0, 0, 0};
            mma_tile(acc, H1, H, 1, W.W2, H, 1, 0, n0, H);
            for (int e = 0; e < 4; ++e) {
                const int m = g + (e >> 1) * 8, nn = n0 + 2 * t + (e & 1);
                const __nv_bfloat16 z = __float2bfloat16_rn(acc[e] + W.b2[nn]);
                H2[m * H + nn] = __float2bfloat16_rn(silu(__bfloat162float(z)));
            }
        }
        __syncwarp();
        float acc[4] = {0, 0, 0, 0};
        mma_tile(acc, H2, H, 1, W.W3, 16, 1, 0, 0, H);
        // gather the 6 outputs of each anchor row through shared memory (reuse X)
        float* o = reinterpret_cast<float*>(X);
        for (int e = 0; e < 4; ++e) {
            const int m = g + (e >> 1) * 8, nn = 2 * t + (e & 1);
            o[m * NOUT + nn] = acc[e] + W.b3[nn];
        }
        __syncwarp();
        if (lane < 16) {
            const int64_t a = grp * 16 + lane;
            if (a < nanchor) {
                float prm[8];
                head(&o[lane * NOUT], prm);
                for (int i = 0; i < 8; ++i) out[a * 8 + i] = prm[i];
            }
        }
        __syncwarp();
    }
}

// Sum of the record weights in a fixed order: per warp of a fixed grid, then
// the warps' sums in warp order (out[1..] holds the partial sums).
constexpr int SUMW_BLOCKS = 256, SUMW_WARPS = SUMW_BLOCKS * 8;
__global__ void k_sum_weights(const ProposalRecord* __restrict__ rec, int64_t n, double* out)
{
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)rec[i].w;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) out[1 + blockIdx.x * 8 + (threadIdx.x >> 5)] = s;
}

__global__ void k_sum_weights_final(double* out)
{
    double s = 0.0;
    for (int w = 0; w < SUMW_WARPS; ++w) s += out[1 + w];
    out[0] = s;
}

cudaError_t launch_sum_weights(const ProposalRecord* rec, int64_t n, double* out, cudaStream_t s)
{
    k_sum_weights<<<SUMW_BLOCKS, 256, 0, s>>>(rec, n, out);
    k_sum_weights_final<<<1, 1, 0, s>>>(out);
    return cudaGetLastError();
}

int sum_weights_scratch() { return 1 + SUMW_WARPS; }

// Records in a fixed order: ascending by (anchor, the bits of y[0..4], of w),
// so that the training data and its minibatches do not depend on the order
// in which warps appended them.  Bitonic network for any n, in place: per
// block size k the mirror step (i, i ^ (k - 1)), then (i, i ^ j) for j =
// k/4 ... 1, each putting the smaller record at the lower index; a partner
// at or beyond n counts as larger than every record.
__device__ __forceinline__ bool rec_less(const ProposalRecord& x, const ProposalRecord& y)
{
    if (x.a != y.a) return x.a < y.a;
    for (int i = 0; i < 5; ++i) {
        const unsigned bx = __float_as_uint(x.y[i]), by = __float_as_uint(y.y[i]);
        if (bx != by) return bx < by;
    }
    return __float_as_uint(x.w) < __float_as_uint(y.w);
}

__global__ void k_sort_records(ProposalRecord* rec, int64_t n, int64_t k, int64_t j, int mirror)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t p = mirror ? (i ^ (k - 1)) : (i ^ j);
    if (p <= i || p >= n) return;
    if (mirror && (i & (k >> 1))) return;
    const ProposalRecord a = rec[i], b = rec[p];
    if (rec_less(b, a)) {
        rec[i] = b;
        rec[p] = a;
    }
}

cudaError_t launch_sort_records(ProposalRecord* rec, int64_t n, cudaStream_t s)
{
    int64_t P = 1;
    while (P < n) P <<= 1;
    const unsigned grid = (unsigned)((n + 255) / 256);
    for (int64_t k = 2; k <= P; k <<= 1) {
        k_sort_records<<<grid, 256, 0, s>>>(rec, n, k, 0, 1);
        for (int64_t j = k >> 2; j >= 1; j >>= 1) k_sort_records<<<grid, 256, 0, s>>>(rec, n, k, j, 0);
    }
    return cudaGetLastError();
}

int mlp_nparam() { return NPARAM; }

cudaError_t launch_mlp_grad(const float* params, const ProposalArgs& A, const ProposalRecord* rec, int64_t n,
                            float inv_wsum, float* grad, float* loss, int grid, float* part, float* part_loss,
                            cudaStream_t s, int64_t ntot, uint64_t key)
{
    const size_t smem = sizeof(TrainSmem);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_mlp_grad<<<grid, 256, smem, s>>>(params, A, rec, n, inv_wsum, part, part_loss, ntot, key);
    k_grad_reduce<<<(NPARAM + 255) / 256, 256, 0, s>>>(part, part_loss, grid, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, float* g, float* m, float* v, int n, float lr, int step, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_mlp_infer(const float* params, const ProposalArgs& A, int64_t nanchor, float* out, int grid,
                             cudaStream_t s)
{
    const size_t smem = sizeof(MlpSmem) + 8 * (16 * NIN + 2 * 16 * H) * sizeof(__nv_bfloat16);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_mlp_infer<<<grid, 256, smem, s>>>(params, A, nanchor, out);
    return cudaGetLastError();
}

}  // namespace bz
