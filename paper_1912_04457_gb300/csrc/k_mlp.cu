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
constexpr int NPARAM = NIN * H + H + H * H + H + H * NOUT + NOUT;

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

}  // namespace

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// instruction descriptor of tcgen05.mma .kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 =
// 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// shared-memory matrix descriptor, no swizzle: start >> 4 (bits 0-13), leading-dimension byte offset
// >> 4 (bits 16-29, here the K-direction core stride), stride-dimension byte offset >> 4 (bits 32-45, the
// row-direction core stride), descriptor version 1 (bits 46-47), layout type 0 (no swizzle, bits 61-63)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ int op_off(int r, int k, int K)  // element offset of (r, k) in an R x K operand
{
    return (((r >> 3) * (K >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        :: "r"(dt), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void commit(uint64_t* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(smem_u32(mbar))
                 : "memory");
}

// waits for the mbarrier phase `parity` to complete; false after ~2^22 polls
__device__ __forceinline__ bool wait_parity(uint64_t* mbar, uint32_t parity)
{
    const uint32_t a = smem_u32(mbar);
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void ld32(uint32_t taddr, float v[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int TM = 128;    // anchors per tile (the MMA's M)
constexpr int TCOLS = 128; // tensor-memory columns held by a CTA

struct InferSmem {
    __nv_bfloat16 B1[H * NIN];   // W1^T: 128 x 16
    __nv_bfloat16 B3[16 * H];    // W3^T: 16 x 128 (output rows 6..15 zero)
    __nv_bfloat16 X[TM * NIN];   // 128 x 16
    __nv_bfloat16 B2[H * H];     // W2^T: 128 x 128
    __nv_bfloat16 H1[TM * H];
    __nv_bfloat16 H2[TM * H];
    float b1[H], b2[H], b3[16];
    uint64_t mbar;
    uint32_t taddr;
};

}  // namespace tc

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

// Training pass on the tensor cores (tcgen05), chunks of 128 records (the
// MMA's M).  Weights stay in shared memory in their [in][out] orientation
// (op_off(in, out, OUT)), activations as [record][unit]; a descriptor reads a
// buffer either K-major (rows = the operand's M or N) or MN-major (rows = K):
// no-swizzle core matrices, the K-direction stride as the leading byte
// offset and the M/N-direction stride as the stride byte offset.  Per chunk:
//   Z1 = X W1 + b1, H1 = silu(Z1); Z2 = H1 W2 + b2, H2; O = H2 W3 + b3;
//   dO = -w dlogq/dO per record;  dW3 += H2^T dO;  dZ2 = (dO W3^T) silu'(Z2);
//   dW2 += H1^T dZ2;  dZ1 = (dZ2 W2^T) silu'(Z1);  dW1^T += dZ1^T X,
// with Z, H, dO and dZ rounded to BF16 where the CPU reference rounds, FP32
// accumulation in tensor memory; the weight gradients accumulate there over
// all of the block's chunks in a fixed order.  Each block then writes its own
// gradient and loss (part[block][NPARAM], part_loss[block]); k_grad_reduce
// adds the blocks in block order, so the result does not depend on which
// block finishes first.  Waits are bounded (err counts timeouts).
namespace tc {
constexpr int RB = 128;          // records per chunk
constexpr int TRAIN_COLS = 512;  // tensor memory: temp [0,128), O [128,144), dW2 [256,384), dW3 [384,400), dW1^T [400,416)
constexpr uint32_t C_T = 0, C_O = 128, C_W2 = 256, C_W3 = 384, C_W1 = 400;

struct TrainSmem {
    __nv_bfloat16 W1[NIN * H];  // op_off(f, i, H)
    __nv_bfloat16 W3[H * 16];   // op_off(i, j, 16), outputs 8..15 zero
    __nv_bfloat16 X[RB * NIN];  // op_off(r, f, NIN)
    __nv_bfloat16 dO[RB * 16];  // op_off(r, j, 16)
    __nv_bfloat16 W2[H * H];    // op_off(i, n, H)
    __nv_bfloat16 H1[RB * H], H2[RB * H], Z1[RB * H], Z2[RB * H];  // op_off(r, i, H); Z1, Z2 later hold dZ1, dZ2
    float b1[H], b2[H], b3[16];
    float yv[RB * 5], wv[RB];
    float db[H + H + NOUT];
    float wloss[4];
    uint64_t mbar;
    uint32_t taddr;
};

__host__ __device__ constexpr uint32_t idesc_major(int M, int N, int a_mn, int b_mn)
{
    return idesc_bf16(M, N) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16);
}
// K-slice kk (16 deep) of a buffer read K-major (rows = M or N, K columns)
__device__ __forceinline__ uint64_t dk(uint32_t base, int K, int kk) { return sdesc(base + kk * 256, 128, (K / 8) * 128); }
// K-slice kk of a buffer read MN-major (rows = K, C columns = M or N)
__device__ __forceinline__ uint64_t dmn(uint32_t base, int C, int kk)
{
    return sdesc(base + kk * 2 * (C / 8) * 128, (C / 8) * 128, 128);
}
}  // namespace tc

__global__ void __launch_bounds__(128, 1) k_mlp_grad(const float* __restrict__ params, const ProposalArgs A,
                                                     const ProposalRecord* __restrict__ rec, int64_t n, float inv_wsum,
                                                     float* __restrict__ part, float* __restrict__ part_loss,
                                                     int64_t ntot, uint64_t key, int* err)
{
    using namespace tc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        const float* W1 = params;
        const float* b1 = W1 + NIN * H;
        const float* W2 = b1 + H;
        const float* b2 = W2 + H * H;
        const float* W3 = b2 + H;
        const float* b3 = W3 + H * NOUT;
        for (int i = tid; i < NIN * H; i += blockDim.x) S.W1[op_off(i / H, i % H, H)] = __float2bfloat16_rn(W1[i]);
        for (int i = tid; i < H * H; i += blockDim.x) S.W2[op_off(i / H, i % H, H)] = __float2bfloat16_rn(W2[i]);
        for (int i = tid; i < H * 16; i += blockDim.x) {
            const int r = i / 16, c = i % 16;
            S.W3[op_off(r, c, 16)] = __float2bfloat16_rn(c < NOUT ? W3[r * NOUT + c] : 0.0f);
        }
        for (int i = tid; i < H; i += blockDim.x) {
            S.b1[i] = b1[i];
            S.b2[i] = b2[i];
        }
        if (tid < 16) S.b3[tid] = tid < NOUT ? b3[tid] : 0.0f;
        for (int i = tid; i < 2 * H + NOUT; i += blockDim.x) S.db[i] = 0.0f;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&S.taddr)),
                     "r"(TRAIN_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.taddr, lq = (uint32_t)(warp * 32) << 16;
    const uint32_t aX = smem_u32(S.X), adO = smem_u32(S.dO), aH1 = smem_u32(S.H1), aH2 = smem_u32(S.H2);
    const uint32_t aZ1 = smem_u32(S.Z1), aZ2 = smem_u32(S.Z2);
    const uint32_t aW1 = smem_u32(S.W1), aW2 = smem_u32(S.W2), aW3 = smem_u32(S.W3);
    uint32_t phase = 0;
    bool ok = true;
    float loss_me = 0.0f;
    auto wait_all = [&]() -> bool {
        const bool done = wait_parity(&S.mbar, phase);
        phase ^= 1;
        fence_after();
        return __syncthreads_and(done) != 0;
    };
    auto sync_operands = [&]() {  // activations written by the threads become MMA operands; TMEM reads done
        fence_before();
        fence_async_smem();
        __syncthreads();
    };
    const int64_t nchunks = (n + RB - 1) / RB;
    bool first = true;
    for (int64_t c = blockIdx.x; c < nchunks && ok; c += gridDim.x, first = false) {
        // ---- inputs: one record per thread ----
        {
            const int64_t r = c * RB + tid;
            float f[NIN];
            if (r < n) {
                const int64_t ri = ntot > 0 ? (int64_t)(splitmix64(key + (uint64_t)r) % (uint64_t)ntot) : r;
                const ProposalRecord R = rec[ri];
                anchor_features(A, R.a, f);
                for (int i = 0; i < 5; ++i) S.yv[tid * 5 + i] = R.y[i];
                S.wv[tid] = R.w * inv_wsum;
            } else {
                for (int i = 0; i < NIN; ++i) f[i] = 0.0f;
                for (int i = 0; i < 5; ++i) S.yv[tid * 5 + i] = 0.0f;
                S.wv[tid] = 0.0f;
            }
            for (int i = 0; i < NIN; ++i) S.X[op_off(tid, i, NIN)] = __float2bfloat16_rn(f[i]);
        }
        sync_operands();
        // ---- hidden layers ----
        for (int l = 0; l < 2 && ok; ++l) {
            if (tid == 0) {
                fence_after();
                if (l == 0) {
                    mma(tmem + C_T, dk(aX, NIN, 0), dmn(aW1, H, 0), idesc_major(RB, H, 0, 1), 0);
                } else {
                    for (int kk = 0; kk < H / 16; ++kk)
                        mma(tmem + C_T, dk(aH1, H, kk), dmn(aW2, H, kk), idesc_major(RB, H, 0, 1), kk > 0);
                }
                commit(&S.mbar);
            }
            if (!(ok = wait_all())) break;
            __nv_bfloat16* Zb = l == 0 ? S.Z1 : S.Z2;
            __nv_bfloat16* Hb = l == 0 ? S.H1 : S.H2;
            const float* bias = l == 0 ? S.b1 : S.b2;
            for (int c0 = 0; c0 < H; c0 += 32) {
                float v[32];
                ld32(tmem + lq + C_T + c0, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const __nv_bfloat16 z = __float2bfloat16_rn(v[i] + bias[c0 + i]);
                    Zb[op_off(tid, c0 + i, H)] = z;
                    Hb[op_off(tid, c0 + i, H)] = __float2bfloat16_rn(silu(__bfloat162float(z)));
                }
            }
            sync_operands();
        }
        if (!ok) break;
        // ---- outputs, loss and dO (one record per thread) ----
        if (tid == 0) {
            fence_after();
            for (int kk = 0; kk < H / 16; ++kk)
                mma(tmem + C_O, dk(aH2, H, kk), dmn(aW3, 16, kk), idesc_major(RB, 16, 0, 1), kk > 0);
            commit(&S.mbar);
        }
        if (!(ok = wait_all())) break;
        {
            float v[32];
            ld32(tmem + lq + C_O, v);
            float o[NOUT];
            for (int i = 0; i < NOUT; ++i) o[i] = v[i] + S.b3[i];
            const float w = S.wv[tid];
            float gq[6] = {0, 0, 0, 0, 0, 0}, lg = 0.0f;
            if (w != 0.0f) {
                logq_grad(o, &S.yv[tid * 5], lg, gq);
                loss_me += -w * lg;
            }
            for (int j = 0; j < 16; ++j) S.dO[op_off(tid, j, 16)] = __float2bfloat16_rn(j < 6 ? -w * gq[j] : 0.0f);
        }
        sync_operands();
        // ---- dW3 += H2^T dO;  T = dO W3^T ----
        if (tid == 0) {
            fence_after();
            for (int kk = 0; kk < RB / 16; ++kk)
                mma(tmem + C_W3, dmn(aH2, H, kk), dmn(adO, 16, kk), idesc_major(H, 16, 1, 1), !(first && kk == 0));
            mma(tmem + C_T, dk(adO, 16, 0), dk(aW3, 16, 0), idesc_major(RB, H, 0, 0), 0);
            commit(&S.mbar);
        }
        if (!(ok = wait_all())) break;
        for (int c0 = 0; c0 < H; c0 += 32) {  // dZ2 = T silu'(Z2), in place of Z2
            float v[32];
            ld32(tmem + lq + C_T + c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int o2 = op_off(tid, c0 + i, H);
                S.Z2[o2] = __float2bfloat16_rn(v[i] * dsilu(__bfloat162float(S.Z2[o2])));
            }
        }
        sync_operands();
        // ---- dW2 += H1^T dZ2;  T = dZ2 W2^T ----
        if (tid == 0) {
            fence_after();
            for (int kk = 0; kk < RB / 16; ++kk)
                mma(tmem + C_W2, dmn(aH1, H, kk), dmn(aZ2, H, kk), idesc_major(H, H, 1, 1), !(first && kk == 0));
            for (int kk = 0; kk < H / 16; ++kk)
                mma(tmem + C_T, dk(aZ2, H, kk), dk(aW2, H, kk), idesc_major(RB, H, 0, 0), kk > 0);
            commit(&S.mbar);
        }
        if (!(ok = wait_all())) break;
        for (int c0 = 0; c0 < H; c0 += 32) {  // dZ1 = T silu'(Z1), in place of Z1
            float v[32];
            ld32(tmem + lq + C_T + c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int o1 = op_off(tid, c0 + i, H);
                S.Z1[o1] = __float2bfloat16_rn(v[i] * dsilu(__bfloat162float(S.Z1[o1])));
            }
        }
        sync_operands();
        // ---- dW1^T += dZ1^T X; meanwhile the bias gradients (column sums of dZ1, dZ2, dO) ----
        if (tid == 0) {
            fence_after();
            for (int kk = 0; kk < RB / 16; ++kk)
                mma(tmem + C_W1, dmn(aZ1, H, kk), dmn(aX, NIN, kk), idesc_major(H, 16, 1, 1), !(first && kk == 0));
            commit(&S.mbar);
        }
        for (int col = tid; col < 2 * H + NOUT; col += blockDim.x) {
            float s = 0.0f;
            if (col < H) {
                for (int r = 0; r < RB; ++r) s += __bfloat162float(S.Z1[op_off(r, col, H)]);
            } else if (col < 2 * H) {
                for (int r = 0; r < RB; ++r) s += __bfloat162float(S.Z2[op_off(r, col - H, H)]);
            } else {
                for (int r = 0; r < RB; ++r) s += __bfloat162float(S.dO[op_off(r, col - 2 * H, 16)]);
            }
            S.db[col] += s;
        }
        if (!(ok = wait_all())) break;  // X and Z1 may be overwritten by the next chunk
    }
    // ---- this block's gradient, every parameter written once ----
    float* gW1 = part + (int64_t)blockIdx.x * NPARAM;
    float* gb1 = gW1 + NIN * H;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + H * NOUT;
    if (ok) {
        const int i = tid;  // tensor-memory lane = hidden unit i of the weight-gradient accumulators
        for (int c0 = 0; c0 < H; c0 += 32) {
            float v[32];
            ld32(tmem + lq + C_W2 + c0, v);
            for (int k = 0; k < 32; ++k) gW2[i * H + c0 + k] = v[k];
        }
        float v[32];
        ld32(tmem + lq + C_W3, v);  // columns 384..415: dW3 (16), then dW1^T (16)
        for (int j = 0; j < NOUT; ++j) gW3[i * NOUT + j] = v[j];
        for (int f = 0; f < NIN; ++f) gW1[f * H + i] = v[16 + f];
    }
    __syncthreads();
    for (int col = tid; col < 2 * H + NOUT; col += blockDim.x) {
        const float s = S.db[col];
        if (col < H)
            gb1[col] = s;
        else if (col < 2 * H)
            gb2[col - H] = s;
        else
            gb3[col - 2 * H] = s;
    }
    // loss: warps in order
    for (int o = 16; o > 0; o >>= 1) loss_me += __shfl_xor_sync(0xffffffffu, loss_me, o);
    if (lane == 0) S.wloss[warp] = loss_me;
    __syncthreads();
    if (tid == 0) part_loss[blockIdx.x] = ((S.wloss[0] + S.wloss[1]) + S.wloss[2]) + S.wloss[3];
    if (!ok && tid == 0) atomicAdd(err, 1);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TRAIN_COLS) : "memory");
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

// ---------------------------------------------------------------------------
// Per-anchor inference on the 5th-generation tensor cores (tcgen05).  A CTA of
// four warps takes tiles of 128 anchors: the activations of a tile (A, 128
// rows) and the transposed weights (B) sit in shared memory in the
// no-swizzle K-major layout of 8-row x 16-byte core matrices (element (r, k)
// of an R x K operand at byte ((r/8)(K/8) + k/8) 128 + (r%8) 16 + (k%8) 2, so
// core matrices adjacent along K are 128 bytes apart and along the rows
// (K/8) 128 bytes); one thread issues tcgen05.mma (M = 128, K = 16 per
// instruction, BF16 operands, FP32 accumulation in tensor memory) and
// commits to an mbarrier; each warp then reads its 32 rows of the
// accumulator (tcgen05.ld, lane quarter = warp) for the epilogue: bias, BF16
// rounding of Z, SiLU in FP32, BF16 activation written back as the next
// layer's A.  Every wait on the mbarrier is bounded: on a timeout the CTA
// records it in err and stops issuing work, then releases its tensor memory.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(128) k_mlp_infer(const float* __restrict__ params, const ProposalArgs A,
                                                   int64_t nanchor, float* __restrict__ out, int* err)
{
    using namespace tc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    InferSmem& S = *reinterpret_cast<InferSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    // weights, transposed into the B operands (K-major rows = output units)
    {
        const float* W1 = params;
        const float* b1 = W1 + NIN * H;
        const float* W2 = b1 + H;
        const float* b2 = W2 + H * H;
        const float* W3 = b2 + H;
        const float* b3 = W3 + H * NOUT;
        for (int i = tid; i < H * NIN; i += blockDim.x) {
            const int n = i / NIN, k = i % NIN;
            S.B1[op_off(n, k, NIN)] = __float2bfloat16_rn(W1[k * H + n]);
        }
        for (int i = tid; i < H * H; i += blockDim.x) {
            const int n = i / H, k = i % H;
            S.B2[op_off(n, k, H)] = __float2bfloat16_rn(W2[k * H + n]);
        }
        for (int i = tid; i < 16 * H; i += blockDim.x) {
            const int n = i / H, k = i % H;
            S.B3[op_off(n, k, H)] = __float2bfloat16_rn(n < NOUT ? W3[k * NOUT + n] : 0.0f);
        }
        for (int i = tid; i < H; i += blockDim.x) {
            S.b1[i] = b1[i];
            S.b2[i] = b2[i];
        }
        if (tid < 16) S.b3[tid] = tid < NOUT ? b3[tid] : 0.0f;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&S.taddr)),
                     "r"(TCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.taddr;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;  // this warp's lane quarter
    const uint32_t aX = smem_u32(S.X), aH1 = smem_u32(S.H1), aH2 = smem_u32(S.H2);
    const uint32_t aB1 = smem_u32(S.B1), aB2 = smem_u32(S.B2), aB3 = smem_u32(S.B3);
    uint32_t phase = 0;
    bool ok = true;
    const int64_t ntiles = (nanchor + TM - 1) / TM;
    // one layer: MMAs over K (K/16 instructions), then all threads wait for the accumulator
    auto layer = [&](uint32_t a_base, uint32_t b_base, int K, int N) -> bool {
        if (tid == 0) {
            fence_after();
            for (int kk = 0; kk < K / 16; ++kk)
                mma(tmem, sdesc(a_base + kk * 256, 128, (K / 8) * 128), sdesc(b_base + kk * 256, 128, (K / 8) * 128),
                    idesc_bf16(TM, N), kk > 0);
            commit(&S.mbar);
        }
        const bool done = wait_parity(&S.mbar, phase);
        phase ^= 1;
        fence_after();
        return __syncthreads_and(done) != 0;  // the same answer in every thread
    };
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t a = tile * TM + tid;
        {
            float f[NIN];
            if (a < nanchor)
                anchor_features(A, a, f);
            else
                for (int i = 0; i < NIN; ++i) f[i] = 0.0f;
            for (int i = 0; i < NIN; ++i) S.X[op_off(tid, i, NIN)] = __float2bfloat16_rn(f[i]);
        }
        fence_async_smem();
        __syncthreads();
        // hidden layers: Z = bf16(acc + b), activation bf16(silu(Z)) as the next A operand
        for (int l = 0; l < 2 && ok; ++l) {
            ok = layer(l == 0 ? aX : aH1, l == 0 ? aB1 : aB2, l == 0 ? NIN : H, H);
            if (!ok) break;
            __nv_bfloat16* act = l == 0 ? S.H1 : S.H2;
            const float* bias = l == 0 ? S.b1 : S.b2;
            for (int c0 = 0; c0 < H; c0 += 32) {
                float v[32];
                ld32(tmem + lane_base + c0, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const __nv_bfloat16 z = __float2bfloat16_rn(v[i] + bias[c0 + i]);
                    act[op_off(tid, c0 + i, H)] = __float2bfloat16_rn(silu(__bfloat162float(z)));
                }
            }
            fence_before();
            fence_async_smem();
            __syncthreads();
        }
        if (!ok) break;
        ok = layer(aH2, aB3, H, 16);
        if (!ok) break;
        float v[32];
        ld32(tmem + lane_base, v);  // columns 0..31: the 16 outputs (and whatever follows)
        if (a < nanchor) {
            float o[NOUT], prm[8];
            for (int i = 0; i < NOUT; ++i) o[i] = v[i] + S.b3[i];
            head(o, prm);
            for (int i = 0; i < 8; ++i) out[a * 8 + i] = prm[i];
        }
        fence_before();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicAdd(err, 1);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TCOLS) : "memory");
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
                            float inv_wsum, float* grad, float* loss, int grid, float* part, float* part_loss, int* err,
                            cudaStream_t s, int64_t ntot, uint64_t key)
{
    // room beyond the buffers: a descriptor read of the last activation buffer stays inside the
    // allocation for either assignment of the two core-matrix strides
    const size_t smem = sizeof(tc::TrainSmem) > 212 * 1024 ? sizeof(tc::TrainSmem) : 212 * 1024;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t nch = (n + tc::RB - 1) / tc::RB;
    const int g = (int)(nch < grid ? nch : grid);
    k_mlp_grad<<<g > 0 ? g : 1, 128, smem, s>>>(params, A, rec, n, inv_wsum, part, part_loss, ntot, key, err);
    k_grad_reduce<<<(NPARAM + 255) / 256, 256, 0, s>>>(part, part_loss, g > 0 ? g : 1, grad, loss);
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
                             int* err, cudaStream_t s)
{
    const size_t smem = sizeof(tc::InferSmem) + 128;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t ntiles = (nanchor + tc::TM - 1) / tc::TM;
    const int g = (int)(ntiles < grid ? ntiles : grid);
    k_mlp_infer<<<g > 0 ? g : 1, 128, smem, s>>>(params, A, nanchor, out, err);
    return cudaGetLastError();
}

}  // namespace bz
