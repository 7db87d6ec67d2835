// Internal host/device interface of libbz: argument blocks passed by value
// to the kernels and the launchers each translation unit exports.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace bz {

// Bounds-checked build (compile with -DBZ_CHECK=1): every index that the
// collision and drift kernels compute into a global buffer is tested before
// the access; an index outside its buffer is counted, with the first one
// seen, in the translation unit's counters and the access is skipped, so a
// wrong index shows up as a count (bz_check_counts) instead of a fault.  The
// default build compiles the tests away.
#ifndef BZ_CHECK
#define BZ_CHECK 0
#endif
#ifdef __CUDACC__
#if BZ_CHECK
static __device__ unsigned long long g_bz_check[2];  // count, first index outside its buffer
__device__ __forceinline__ bool bz_in(long long i, long long n)
{
    if (i >= 0 && i < n) return true;
    if (atomicAdd(&g_bz_check[0], 1ull) == 0ull) g_bz_check[1] = (unsigned long long)i;
    return false;
}
#else
__device__ __forceinline__ bool bz_in(long long, long long) { return true; }
#endif
#endif
// Counters of each translation unit of a checked build (count, first index);
// reset clears them.  cudaErrorNotSupported without BZ_CHECK.
cudaError_t check_read_collide_f32(unsigned long long out[2], bool reset);
cudaError_t check_read_collide_f64(unsigned long long out[2], bool reset);
cudaError_t check_read_transport(unsigned long long out[2], bool reset);

constexpr int NSPEC = 7;
constexpr int MAX_TERMS = 10;
constexpr int MAX_NP = 256;     // momentum cells per axis
constexpr double HBARC = 0.1973269804;
constexpr double PI = 3.14159265358979323846;
constexpr double TWO_POW_40 = 1099511627776.0;
constexpr double TWO_POW_M40 = 1.0 / 1099511627776.0;
constexpr int MASS_SHIFT = 30;
// A grid odd along all three axes has a cell centred at p = 0, where the
// massless dispersion E = |p| (first mass evaluation, mass mode MASSLESS)
// is zero and 1/(2E) in Eqs. (mg), (mq) diverges; such grids are rejected.
inline bool np_has_zero_cell(const int* np) { return (np[0] & 1) && (np[1] & 1) && (np[2] & 1); }
constexpr double MASS_FX = 1.0 / 1024.0;  // state units (2^-40 of N f) to 2^-30 of f: 2^(MASS_SHIFT - 40)

enum { M_QQP = 0, M_QQ, M_QQB, M_QQB2, M_QQBGG, M_QG, M_GG };

inline __host__ __device__ int mass_slot(int s) { return s == 0 ? 0 : 1 + (s - 1) % 3; }
inline __host__ __device__ bool is_quark(int s) { return s != 0; }

// One term of a species' equation: legs (k1, k2, k3, p).
struct TermDev {
    int8_t slot[4];   // state slot of each leg's species
    int8_t mslot[4];  // mass slot (0 g, 1..3 flavour) of each leg
    int8_t quark[4];  // 1 if the leg is a (anti)quark: F = 1 - f, else F = 1 + f
    int8_t cls;       // |M|^2 row
    int8_t gfirst;    // 1 if the term opens a kinematic group (consecutive terms with equal leg masses)
    int8_t pad[2];
    double sym;       // 1/2 for identical initial particles
};

// Learned proposal: anchor description for the network's features, and one
// training record (anchor, weight sum |c~|, normalised sample y = (k1x, k1y, k3)/L).
struct ProposalArgs {
    int64_t nxc, npc;
    int np[3];
    float L;
    int slot_species[NSPEC];
};
struct ProposalRecord {
    int64_t a;
    float w;
    float y[5];
};
constexpr int SAMPLER_LEARNED = 2;

// Exact division of 0 <= n < 2^31 by a fixed d >= 1 (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994): with
// l = ceil(log2 d) and m = ceil(2^(31+l) / d) < 2^32, n / d = (n m) >> (31 + l).
struct DivMagic {
    uint32_t m;
    int s;
};
inline DivMagic div_magic(uint32_t d)
{
    int l = 0;
    while (l < 32 && (1ull << l) < (unsigned long long)d) ++l;
    const unsigned long long num = 1ull << (31 + l);
    return DivMagic{(uint32_t)((num + d - 1) / d), 31 + l};
}
__host__ __device__ __forceinline__ uint32_t udiv(uint32_t n, DivMagic dm)
{
    return (uint32_t)(((unsigned long long)n * dm.m) >> dm.s);
}

// User-defined |M|^2 row: sum over n <= 8 terms of coef s^a t^b u^c /
// (s^d (t - m_g^2)^e (u - m_g^2)^f), e = (a, b, c, d, e, f) in [0, 4]
// (coef32: its FP32 rounding, used by the FP32 path).
struct UserTerm {
    double coef;
    float coef32;
    uint8_t e[6];
    uint8_t pad[2];
};
struct UserRow {
    int n, pad;
    UserTerm t[8];
};
constexpr int MSQ_ROWS = 7;

// Philox4x32-10 keys of rounds 0..9: the key is bumped by the Weyl
// constants 0x9E3779B9 and 0xBB67AE85 after every round (Salmon et al., SC'11).
inline void philox_key_schedule(uint32_t k0, uint32_t k1, uint32_t ks[20])
{
    for (int r = 0; r < 10; ++r) {
        ks[2 * r] = k0;
        ks[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

template <typename R>
struct CollideArgs {
    const void* f;          // f per cell [slot][x][p] (unused in equilibrium mode)
    int f_is_float;         // f holds float (1) or double (0)
    int ubits;              // uniforms: 32-bit (FP64 path) or 23-bit (FP32 path and its fixup)
    long long* A;           // deposit target, int64 [slot][x][p]
    const double* m2;       // [x][4]
    long long* flags;       // [4]
    int64_t nxc, npc;
    int64_t ncell;          // cells of f and A (slots x nxc x npc)
    int np[3];
    R L, twoL, dp[3];
    double L64, dp64[3];    // L and 2L/n in FP64 (the FP32 path's fixup works in FP64 geometry)
    // FP32 path index decode without hardware division (all indices < 2^31):
    // units per anchor, cells per slot, p cells, np[1] np[2], np[2]
    DivMagic dv_group, dv_slot, dv_npc, dv_yz, dv_z;
    uint32_t key0, key1;
    uint32_t ks[20];        // Philox key schedule: (k0, k1) of rounds 0..9, so a kernel whose
                            // arguments sit in the constant bank reads them as operands
    int nsamples, step;
    const int* step_dev;    // FP32 path: the step index in device memory (a replayed step graph), or null: step
    int64_t n_sel, a_stride, a_offset;
    int sampler, mass_mode, analytic, p_center;
    int param;              // FP64 path: 0 k2 eliminated (the paper's choice), 1 k3 eliminated
    const UserRow* urows;   // [MSQ_ROWS] device table of user-defined |M|^2 rows, or null
    uint32_t umask;         // bit r: row r of the |M|^2 table is user-defined
    R T, mu[NSPEC];
    R Kq, Kown, twopi5;
    R A1, A2, A3, A4, A5;
    int slot_species[NSPEC];
    int nterms[NSPEC];
    TermDev terms[NSPEC][MAX_TERMS];
    // learned sampler: per-anchor proposal (mu3 x3, sigma3, sigma1, alpha, -, -)
    const float* prop;
    // record mode (FP32 uniform sampler): per-sample sum of |c~| written to rec
    ProposalRecord* rec;
    unsigned long long* rec_count;
    long long rec_cap;
    int rec_stride;  // 0: off; else units with index % rec_stride == 0 are recorded
    // FP32 path: terms with |H| < tau kappa^2 are queued per warp for re-evaluation
    // FP64 path: continuous-leg audit sums per accepted root, or null:
    // [0] sum w (Ep + E3 - E1 - E2), [1..3] sum w (p + k3 - k1 - k2), [4] sum |w| (Ep + E3 + E1 + E2),
    // [5] roots, [6] sum |w|; w = c~ Kq (unquantised)
    double* audit;
    R tau;                          // 0: never defer
    int* qcount;                    // [warps] items queued by each warp
    unsigned long long* qitems;     // [warps][qcap] packed (anchor << 24 | sample << 4 | term)
    long long qcap;
};

struct MassArgs {
    const long long* state;
    long long* acc;         // [x][4] fixed-point sums (zeroed by the caller)
    double* m2_out;         // [x][4]
    const double* m2_prev;  // [x][4] or null (E = |p|)
    long long* flags;
    int64_t nxc, npc;
    int np[3];
    double L, dp[3];
    int slot_of[NSPEC];     // -1 if inactive
    double pref_g, pref_q, meas;
    long long limit;
    int64_t chunk;          // bins per block (set by launch_masses)
    // the distinct values of p^2 = (px^2 + py^2) + pz^2 over the cell centres
    // (FP64, in the order of the formula) and the index of each cell's value,
    // or nu = 0 (no table: grids with more than MASS_TAB_MAX distinct values)
    const double* ppu;
    const unsigned short* pidx;  // [npc]
    int nu;
};
constexpr int MASS_TAB_MAX = 6144;  // 4 x 6144 doubles of 1/(2E) per block in shared memory

struct DriftArgs {
    const long long* in;
    long long* out;
    void* freal;            // optional f of `in` (float or double) written alongside
    int freal_double;
    const double* m2;
    int64_t nxc, npc, ncell;
    int nx[3], np[3];
    int mass_mode;
    float dtdxf;
    int slot_mslot[NSPEC];
    double inv_deg[NSPEC];  // per slot: 1 / N_s (f = n 2^-40 / N_s in the FP64 conversion)
    double deg[NSPEC];
    float fscale[NSPEC];    // per slot: FP32 rounding of 2^-40 / N_s (the FP32 f is n_fp32 * fscale)
    const int* jtab;        // [npc] jx | jy << 8 | jz << 16
    float* inv_e;           // [ncell] scratch: 1/sqrt(p^2 + m^2) of every cell, written by k_inv_energy
    float* m2f;             // [nxc][4] scratch: FP32 rounding of m^2 per x cell and mass slot (0: massless)
    // force term -div_p[(grad_x E) f] (off: force = 0): per (x cell, mass slot, axis) the FP32
    // g_i = (m^2(x + e_i) - m^2(x - e_i)) / (4 dx), written by k_force_grad into gforce
    int force;
    float* gforce;          // [nxc][4][3] scratch
    double inv4dx;          // 1 / (4 dx)
    float Kp[3];            // FP32 rounding of dt/dp_i, times 2^30
    float pf[3][MAX_NP];    // FP32 cell-centre momenta per axis
};

struct MomentArgs {
    const long long* state;
    double* out;            // [x][slot][5]
    const double* m2;
    int64_t nxc, npc;
    int nslots;
    int np[3];
    int mass_mode;
    int slot_mslot[NSPEC];
    double pref, half_dp[3];
    float pf[3][MAX_NP];
    const int* jtab;        // [npc] jx | jy << 8 | jz << 16, or null (decoded by division)
    long long* sflags;      // [2] cells with n < 0, fermion cells with f > 1 (added), or null
    long long pauli[NSPEC]; // per slot: N_s 2^40 (f = 1) for (anti)quarks, LLONG_MAX for gluons
    // energy source (k_energy_source): out is [x][slot][3], masses of the previous evaluation, dt
    const double* m2_prev;
    double dt;
    // k_moments: p-cell chunks per (x cell, slot), and their exact partial sums
    // ([x][slot][chunk][5] 128-bit as (lo, hi) int64 pairs) when nchunk > 1
    int nchunk;
    long long* part;
    // a replayed step graph writes the moments of step *kidx at out + *kidx kstride (kidx null: out)
    const int* kidx;
    int64_t kstride;
};

// Per-slot scales of the f conversion: FP64 degeneracy, and the FP32
// rounding of 2^-40 / N_s
struct ConvScale {
    double deg[NSPEC];
    float f32[NSPEC];
};

// launchers (return cudaGetLastError())
cudaError_t launch_collide_f64(const CollideArgs<double>& a, int grid, cudaStream_t s);
cudaError_t launch_fill_jtab(int* jtab, const int* np, cudaStream_t s);
// exact int64 sum of a[0, n) added into *out
cudaError_t launch_sum_ll(const long long* a, int64_t n, long long* out, cudaStream_t s);
// counter: zeroed device word for the dynamic distribution of units over a
// resident grid (see collide_f32_resident_blocks), or null for a static stride
cudaError_t launch_collide_f32(const CollideArgs<float>& a, int grid, unsigned long long* counter, cudaStream_t s);
int collide_f32_resident_blocks(const CollideArgs<float>& a);  // per SM, for the instantiation `a` runs
// FP32 path, uniform sampler: re-evaluation of the queued terms with an FP64
// root solve (one warp per queue segment)
cudaError_t launch_fixup_f32(const CollideArgs<float>& a, int nseg, cudaStream_t s);
cudaError_t launch_fixup_f32_batch(const CollideArgs<float>* boxes, const int* qcount, const unsigned long long* qitems,
                                   int64_t qcap, const int* step_dev, int nseg, cudaStream_t s);
cudaError_t launch_collide_f32_batch(const CollideArgs<float>* boxes, const int64_t* prefix, int nboxes,
                                     unsigned long long* counter, const int* step_dev, int chunk, int grid,
                                     int* qcount, unsigned long long* qitems, long long qcap, cudaStream_t s);
// batched transport kernels over independent homogeneous boxes
cudaError_t launch_masses_batch(const MassArgs* boxes, const int64_t* chunk_prefix, int nboxes, int64_t nchunks,
                                const int* have_prev, long long* acc_all, cudaStream_t s);
cudaError_t launch_convert_batch(const long long* state, float* f, const int64_t* cell_prefix,
                                 const int64_t* chunk_prefix, const float* scale, const int* slot_cells, int nboxes,
                                 int64_t nchunks, cudaStream_t s);
cudaError_t launch_moments_batch(const MomentArgs* boxes, const int* slot_prefix, int nboxes, int nblocks,
                                 double* out, const int* kidx, int per_step, cudaStream_t s);
cudaError_t launch_batch_end_step(double* m2_prev, const double* m2_cur, int n, int* have_prev, int* step_dev,
                                  int* kidx, cudaStream_t s);
// a replayed single-box step: set, then advance, the device step index and moments slot
cudaError_t launch_set_step(int* step_dev, int step, int* kidx, int k, cudaStream_t s);
cudaError_t launch_step_advance(int* step_dev, int* kidx, cudaStream_t s);
#ifndef BZ_DEFER_TAU
#define BZ_DEFER_TAU 2e-3
#endif
constexpr double DEFER_TAU = BZ_DEFER_TAU;  // FP32 terms with |H| < tau kappa^2 are re-evaluated (float-float)
#ifndef BZ_DEFER_CAP_DIV
#define BZ_DEFER_CAP_DIV 50
#endif
constexpr int DEFER_CAP_DIV = BZ_DEFER_CAP_DIV;  // queue room: 1/DIV of a warp's term evaluations
constexpr int MAX_SAMPLES = 1 << 20;
// FP32 collision kernel: warps per block, and 32-sample chunks per work unit
// (an anchor and up to 256 of its samples; the live ones are compacted).
constexpr int F32_WARPS = 4;
constexpr int F32_GROUP = 8;
__host__ __device__ inline int64_t f32_units(int64_t n_sel, int nsamples)
{
    const int64_t nchunk = (nsamples + 31) / 32;
    return n_sel * ((nchunk + F32_GROUP - 1) / F32_GROUP);
}
int mlp_nparam();
// ntot > 0: minibatch position r reads record splitmix64(key + r) mod ntot of rec
// (i.i.d. draws from all ntot records); ntot = 0: records [0, n) in order
// part [grid][nparam], part_loss [grid]: per-block scratch, added in block order into grad (+=) and loss (=);
// err (device int): incremented by a block whose tensor-core wait timed out.  At most `grid` blocks, one
// per SM (each holds 512 columns of tensor memory).
cudaError_t launch_mlp_grad(const float* params, const ProposalArgs& A, const ProposalRecord* rec, int64_t n,
                            float inv_wsum, float* grad, float* loss, int grid, float* part, float* part_loss, int* err,
                            cudaStream_t s, int64_t ntot = 0, uint64_t key = 0);
cudaError_t launch_adam(float* p, float* g, float* m, float* v, int n, float lr, int step, cudaStream_t s);
// err (device int, zeroed by the caller): incremented by a CTA whose tensor-core wait timed out
cudaError_t launch_mlp_infer(const float* params, const ProposalArgs& A, int64_t nanchor, float* out, int grid,
                             int* err, cudaStream_t s);
// out[0] = sum of the weights in a fixed order; out needs sum_weights_scratch() doubles
cudaError_t launch_sum_weights(const ProposalRecord* rec, int64_t n, double* out, cudaStream_t s);
int sum_weights_scratch();
// records sorted ascending by (anchor, y bits, w bits), in place
cudaError_t launch_sort_records(ProposalRecord* rec, int64_t n, cudaStream_t s);
cudaError_t launch_masses(const MassArgs& a, cudaStream_t s);
cudaError_t launch_drift(const DriftArgs& a, cudaStream_t s);
cudaError_t launch_moments(const MomentArgs& a, cudaStream_t s);
// per (x cell, slot): int N f / E, its S_ex^0 part and the T_total term (Eq. (current conservation))
cudaError_t launch_energy_source(const MomentArgs& a, cudaStream_t s);
cudaError_t launch_convert(const long long* state, void* freal, int as_double, int64_t nxc,
                           int64_t npc, int nslots, const double* deg, cudaStream_t s);

}  // namespace bz
