/*
 * bz.h -- C ABI of libbz: the Monte Carlo 2->2 collision term of the
 * relativistic Boltzmann equation for g, u, d, s, ubar, dbar, sbar with
 * symmetrical sampling, the upwind drift and the moments, on one GB300
 * (sm_103a).  Method: Zhang, Wu, Pu, Qin, Wang, "Towards a full solution of
 * relativistic Boltzmann equation for quark-gluon matter on GPUs",
 * arXiv:1912.04457.
 *
 * Conventions
 * -----------
 * Units: momenta and masses in GeV, x in fm, t in fm/c (hbar c =
 *   0.1973269804 GeV fm converts dt into GeV^-1).
 * Species: 0 g, 1 u, 2 d, 3 s, 4 ubar, 5 dbar, 6 sbar.  Degeneracies
 *   N_g = 16, N_q = 6 (Sec. II).  Only the species of the mask are stored.
 * State: int64 n[slot][x][p] = N_s f_s(x, p) 2^40, round-half-even; slots
 *   are the active species in increasing index order; x = (ix, iy, iz) and
 *   p = (jx, jy, jz) row-major, last index fastest.  Momentum cells are
 *   centred: p_j = -L + (j + 1/2) 2L/n_p.  Spatial cells are periodic.
 * Memory: every pointer named "device" is CUDA device memory owned by the
 *   caller (e.g. a torch tensor's data_ptr); pointers named "host" are host
 *   memory.  The handle owns only its descriptors and device scratch.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  All
 *   work is enqueued on it; calls return without synchronising unless
 *   stated.  A handle's device scratch (masses, f, the FP32 deferral queue
 *   and work counter) serves one call at a time: calls on one handle must
 *   be ordered (one stream, or events between streams); separate handles
 *   run concurrently.
 * Errors: 0 on success; negative BZ_E* on error (nothing was enqueued
 *   after the failing check; bz_last_error gives the message).  No C++
 *   exception crosses this boundary.
 * Environment: BZ_F32_SCHEDULE (read at every FP32 collision call of a
 *   handle) = "counter" or "static" forces how the warps of the FP32 kernel
 *   share the work units -- taking them from a global counter, or one unit
 *   per warp -- which is otherwise chosen by size; both give the same bits
 *   (a test checks it).  Unset or any other value: chosen by size.
 *   BZ_STEP_GRAPH=0 (read by bz_step) launches every step of an FP32 run
 *   eagerly instead of replaying captured step graphs (same bits).
 */
#ifndef BZ_H
#define BZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BZ_OK 0
#define BZ_EINVAL (-1)    /* bad argument                                    */
#define BZ_ENOMEM (-2)    /* device allocation failed                        */
#define BZ_ECUDA (-3)     /* a CUDA call or launch failed                    */
#define BZ_EOVERFLOW (-4) /* fixed-point range exceeded (see bz_get_flags)   */
#define BZ_ENODEV (-5)    /* no CUDA device / wrong architecture             */

#define BZ_PREC_F64 0     /* integrand in FP64 (bit-exact with the CPU oracle) */
#define BZ_PREC_F32 1     /* integrand in FP32, uniforms with 23-bit resolution */

#define BZ_SAMPLER_SYMMETRIC 0 /* each root deposits +w/4 to p and k3, -w/4 to k1, k2 (Eq. small c relation) */
#define BZ_SAMPLER_PLAIN 1     /* usual MC: full weight to the anchor cell only (Fig. 3, 4 "without") */
#define BZ_SAMPLER_LEARNED 2   /* symmetric deposition, samples from the learned per-anchor proposal (bz_proposal_*) */

#define BZ_MASS_THERMAL 0   /* Eqs. (mg), (mq) every call; E = sqrt(p^2 + m^2) everywhere        */
#define BZ_MASS_MASSLESS 1  /* thermal m_g^2 as |M|^2 regulator only; E = |p| in kinematics     */
#define BZ_MASS_FIXED 2     /* masses set by bz_set_masses, never recomputed (Fig. 5)            */

typedef struct bz_handle_s* bz_handle;

typedef struct bz_grid {
    int32_t nx[3];   /* spatial cells per axis (1 = homogeneous along that axis)          */
    double dx;       /* spatial cell size, fm                                              */
    int32_t np[3];   /* momentum cells per axis; not odd along all three (a cell at p = 0) */
    double L;        /* momentum box [-L, L)^3, GeV; also the integration box of (k1_perp, k3) */
    uint64_t seed;   /* Philox4x32-10 key (low word xor box id, high word)                  */
    uint32_t box;    /* box id, xored into the key's low word                               */
    uint32_t reserved;
} bz_grid;

/* Creates a handle on the current CUDA device for the grid *g (host
 * pointer, copied).  Allocates the handle's device scratch (masses, flags,
 * one f-sized work array).  Defaults: gluons only, alpha_s = 0.3, mass mode
 * BZ_MASS_THERMAL, all anchors sampled, no equilibrium override.
 * Grid and seed follow the statement of the problem in Sec. II / III.
 * Errors: BZ_EINVAL (sizes <= 0, np > BZ max, all np odd, L <= 0, dx <= 0), BZ_ENODEV,
 * BZ_ENOMEM. */
int bz_init_grid(bz_handle* out, const bz_grid* g);

/* Releases the handle and its scratch (synchronises the device first). */
int bz_destroy(bz_handle h);

/* Message of the last error on h (or of the last failed bz_init_grid when h
 * is NULL).  Valid until the next call on h. */
const char* bz_last_error(bz_handle h);

/* Selects the species (bit s of species_mask = species s, Sec. II), the
 * coupling (g^2 = 4 pi alpha_s) and the mass mode (BZ_MASS_*).  A term of
 * Eqs. (C_quark)/(C_gluon) is evaluated only if all four of its species are
 * active.  Reallocates scratch if the slot count changes and forgets the
 * previous masses.  Errors: BZ_EINVAL (empty mask, alpha_s <= 0, mode). */
int bz_set_species(bz_handle h, uint32_t species_mask, double alpha_s, int mass_mode);

/* Number of active species (state slots), x cells, p cells; any out pointer
 * may be NULL. */
int bz_query_sizes(bz_handle h, int32_t* nslots, int64_t* nxcells, int64_t* npcells);

/* Collision increment, Eqs. (C_a_b), (work out delta E), (MC C_gg), (ca),
 * (small c relation):
 *   1. thermal masses from `state` (Eqs. mg, mq) unless mass mode FIXED,
 *      with E from the previous masses of this handle (E = |p| on the first
 *      call after init / bz_reset_masses); they become the handle's masses;
 *   2. for every anchor (species d, x cell, p cell) nsamples Philox samples
 *      of (p jitter, k1x, k1y, k3) in [-L, L)^5; for every term of species
 *      d's equation and every valid k1z root inside the box, the weight
 *      w = c~ (2L)^5/(4 nsamples) dt/hbar_c 2^40 is rounded to an integer q
 *      and deposited +q to (d, p), +q to (c, k3), -q to (a, k1), -q to (b, k2)
 *      (BZ_SAMPLER_PLAIN: +4w rounded to (d, p) only).
 * state (device, int64 [nslots][nx][np]) is read only.  A (device, int64,
 * same shape) is zeroed and filled with the increment of N f 2^40 over dt.
 * Sum of A is exactly 0 with the symmetric sampler.  step enters the
 * Philox counter (counter = (2 sample + block, p, x, step << 3 | d)).
 * prec: BZ_PREC_F64 (bit-exact with the FP64 CPU oracle) or BZ_PREC_F32.
 * Errors: BZ_EINVAL (nsamples <= 0, step outside [0, 2^29), prec/sampler),
 * BZ_ECUDA.  Overflows of the fixed point are counted (bz_get_flags). */
int bz_collision_term(bz_handle h, const int64_t* state, int64_t* A, int32_t nsamples,
                      int32_t step, double dt, int32_t prec, int32_t sampler, void* stream);

/* FP64 collision term (as bz_collision_term with BZ_PREC_F64 and the given
 * sampler) plus the audit of Sec. III.B's conservation laws, computed on
 * the GPU: audit_host (host double [8]) receives
 *   [0] sum_roots w (E_p + E_3 - E_1 - E_2)   energy balance of the continuous legs,
 *   [1..3] sum_roots w (p + k3 - k1 - k2)     momentum balance (x, y, z),
 *   [4] sum_roots |w| (E_p + E_3 + E_1 + E_2)  the scale of [0..3],
 *   [5] accepted roots, [6] sum_roots |w|,
 *   [7] sum of A over all cells (exactly 0 with the symmetric sampler),
 * w = c~ (2L)^5/(4N) dt/hbar_c 2^40 unquantised (the learned sampler
 * includes 1/(32 q)).  [0..3] vanish to rounding (energy and momentum are
 * conserved at the continuous leg momenta; the binned deposits are not,
 * Sec. III.B).  The FP64 sums are accumulated with atomics, so their last
 * bits depend on the order.  Synchronises.  Errors as bz_collision_term. */
int bz_collision_audit(bz_handle h, const int64_t* state, int64_t* A, int32_t nsamples, int32_t step, double dt,
                       int32_t sampler, double* audit_host, void* stream);

/* Free streaming, Eq. (left handside): first-order upwind in flux form,
 * periodic in x, v = p/E_p(x) with the handle's current masses (E = |p| in
 * mass mode MASSLESS), plus the force term when bz_set_force_term enabled
 * it.  Courant numbers in IEEE FP32 held in 2^-30 fixed point; each face
 * flux is an exact rounded integer product applied with opposite signs to
 * its two cells, so the sum of the state is invariant.  in, out: device
 * int64 [nslots][nx][np], must not overlap. */
int bz_drift(bz_handle h, const int64_t* in, int64_t* out, double dt, void* stream);

/* nsteps forward-Euler steps of Eq. (left handside) with all terms from
 * f^n (unsplit): per step, masses from n^n, then
 *   n^{n+1} = drift(n^n) + collision increment(n^n)
 * with Philox step index step0 + k.  state (device int64) is updated in
 * place.  moments_out (device, may be NULL): per step, the moments of
 * n^{n+1} as bz_moments, [nsteps][nx][nslots][5] doubles.
 * With BZ_PREC_F32 and nsteps >= 3 the first step is launched directly and
 * the following pairs of steps replay a CUDA graph of two captured steps
 * (the step index and moments slot live in device memory), kept on the
 * handle for the next call with the same state, moments buffer, dt and
 * nsamples and no setter call in between; the results are those of direct
 * launches, bit for bit.  While bz_profile is on every step is direct. */
int bz_step(bz_handle h, int64_t* state, double dt, int32_t nsteps, int32_t nsamples,
            int32_t prec, int32_t step0, double* moments_out, void* stream);

/* Moments, Eqs. (particle numbers), (energy momentum tensor), per x cell
 * and active species: out[x][slot][0..4] = (n, eps, T^01, T^02, T^03) as
 * densities (GeV^3, GeV^4), E at the bin centres with the handle's current
 * masses.  state: device int64; out: device double [nx][nslots][5]. */
int bz_moments(bz_handle h, const int64_t* state, double* out, void* stream);

/* Energy source of the kinetic energy-momentum tensor, Eq. (current
 * conservation): d_mu T_kin^{mu nu} = S_ex^nu = (1/2) sum_a d^nu m_a^2 I_a
 * with I_a = int d^3p/(2pi)^3 N_a f_a / E_a.  Per x cell and active species,
 * out[x][slot][0..2] = (I_a in GeV^2, (1/2)((m_a^2 - m_prev^2)/dt) I_a in
 * GeV^4 per fm/c -- the species' part of S_ex^0 --, -(1/4) m_a^2 I_a in
 * GeV^4 -- the term that turns T_kin^00 into the modified total energy
 * T_total^00 of a single flavour).  E and m_a^2 are the handle's current
 * masses (computed from state first if the handle has none); m2_prev_host
 * (host double [nx][4], as bz_get_masses) are the masses of the previous
 * evaluation, or NULL for no mass change (zero source).  I_a is an exact
 * integer sum of n round(2^24 / E), 1/E in IEEE FP32 at the bin centres;
 * with the massless dispersion both m^2 terms are zero.  state: device
 * int64; out: device double [nx][nslots][3].  Errors: BZ_EINVAL for null
 * pointers or dt <= 0, or mass mode FIXED without bz_set_masses. */
int bz_energy_source(bz_handle h, const int64_t* state, const double* m2_prev_host, double dt, double* out,
                     void* stream);

/* Current masses, host double [nx][4] = (m_g^2, m_u^2, m_d^2, m_s^2) in
 * GeV^2.  bz_get_masses synchronises the stream of the last call.
 * bz_set_masses also serves as the "previous" masses of the next call. */
int bz_get_masses(bz_handle h, double* m2_host);
int bz_set_masses(bz_handle h, const double* m2_host);
/* Forgets the previous masses: the next mass evaluation uses E = |p|. */
int bz_reset_masses(bz_handle h);

/* Counters (host int64 [4], synchronising): [0] roots dropped because a
 * regulated denominator t - m_g^2 or u - m_g^2 was >= 0 or s <= 0, [1]
 * deposits whose fixed-point weight exceeded 2^62, [2] mass fixed-point
 * overflows, [3] FP32-path terms that found the re-evaluation queue
 * full (kept in FP32).  bz_clear_flags zeroes them and the state warnings. */
int bz_get_flags(bz_handle h, int64_t* flags_host);
/* State warnings (host int64 [2], synchronising), added up by every moments
 * evaluation (bz_moments, and bz_step when it writes moments): [0] cells
 * with f < 0 (n < 0; the scheme does not clip, so a too large dt shows
 * here), [1] (anti)quark cells with f > 1 (Pauli blocking violated). */
int bz_get_state_flags(bz_handle h, int64_t* flags_host);
int bz_clear_flags(bz_handle h);

/* Resolution of the uniforms of the FP64 path: 32 (default, u = (x + 1/2)
 * 2^-32 from each Philox word x) or 23 (u = ((x >> 9) + 1/2) 2^-23, the
 * uniforms of the FP32 path, so both paths evaluate the same sample points).
 * Errors: BZ_EINVAL for other values. */
int bz_set_uniform_bits(bz_handle h, int32_t bits);

/* User-defined matrix elements (Sec. II: the API for the user's own |M|^2;
 * the Appendix table is the default).  Replaces row `row` of the |M|^2
 * table (0 q_a q_b -> q_a q_b, 1 q q -> q q, 2 q qb -> q qb, 3 q_a qb_a ->
 * q_b qb_b, 4 q qb -> g g (and g g -> q qb), 5 q g -> q g, 6 g g -> g g) for
 * every term that uses it, on the FP64 and FP32 paths, by
 *   |M|^2 = sum_k coef[k] s^a t^b u^c / (s^d (t - m_g^2)^e (u - m_g^2)^f),
 * (a, b, c, d, e, f) = exps[6k .. 6k+5], each in [0, 4]; 1 <= nterms <= 8
 * (host arrays, copied).  nterms = 0 restores the default row.  The FP32
 * path uses the FP32 rounding of each coefficient.  The batched ensemble
 * always uses the default table.  Errors: BZ_EINVAL for a bad row, count,
 * exponent or a non-finite coefficient. */
int bz_set_matrix_element(bz_handle h, int32_t row, int32_t nterms, const double* coef, const int32_t* exps);

/* Which momentum the delta function of Eq. (delta function) eliminates
 * (Sec. III.A): which = 0 (default, the paper's choice) k2 = k3 + p - k1,
 * with (k1x, k1y, k3) sampled and k1z from E1 + E2 = E3 + Ep; which = 1
 * k3 = k1 + k2 - p, with (k1x, k1y, k2) sampled and k1z from E1 - E3 =
 * Ep - E2 (the paper's "less stable" choice, for its stability comparison):
 * same box, volume (2L)^5, deposits and weights, the Jacobian of the
 * solved equation.  which = 1 is for the FP64 path with uniform samples;
 * collision calls with the FP32 path or the learned sampler then fail with
 * BZ_EINVAL.  Errors: BZ_EINVAL for other values. */
int bz_set_parameterisation(bz_handle h, int32_t which);

/* Force term -div_p[(grad_x E) f] of Eq. (left handside) (dp/dt = -grad_x E,
 * Eq. (boltzmann equation general form)), added to the drift of bz_drift and
 * bz_step when enable = 1 (default 0).  Along p_i the p cells of an x cell
 * move with -g_i / E, g_i = (m^2(x + e_i) - m^2(x - e_i)) / (4 dx) (the
 * central difference of the species' m^2, halved: dE/dx = (dm^2/dx)/(2E));
 * upwind in p with the Courant number ((-g_i) (1/E)) dt/dp_i held in 2^-30
 * fixed point like the x fluxes; no flux through the faces of the momentum
 * box, so the sum of the state stays exact.  It has no effect with one x
 * cell or the massless dispersion (no gradient).  Errors: BZ_EINVAL for
 * enable other than 0 or 1. */
int bz_set_force_term(bz_handle h, int32_t enable);

/* Restricts the anchors to those with linear index a = (slot nx + x) np + p
 * satisfying a % stride == offset (stride 1 = all).  Used to check full
 * size workloads against the CPU oracle on a sample of anchors. */
int bz_set_anchor_subset(bz_handle h, int64_t stride, int64_t offset);

/* Equilibrium check mode: when enable != 0, f at each leg is the Bose-
 * Einstein / Fermi-Dirac value at the leg's continuous momentum, Eqs. (fg),
 * (fq), with temperature T and chemical potentials mu (host double [7]),
 * instead of the bin value of the state. */
int bz_set_equilibrium(bz_handle h, int enable, double T, const double* mu_host);

/* Per-kernel timing of this handle's own launches (CUDA events recorded on
 * the caller's stream around each launch while enabled).  Kernel ids:
 * BZ_K_MASSES, BZ_K_DRIFT, BZ_K_COLLIDE, BZ_K_FIXUP, BZ_K_MOMENTS,
 * BZ_K_CONVERT.  bz_profile(h, 1) clears and starts, bz_profile(h, 0) stops;
 * bz_profile_read synchronises the device and returns, for the first n ids,
 * the summed milliseconds (host double [n]) and launch counts (host int64
 * [n]); either pointer may be NULL. */
#define BZ_K_MASSES 0
#define BZ_K_DRIFT 1
#define BZ_K_COLLIDE 2
#define BZ_K_FIXUP 3
#define BZ_K_MOMENTS 4
#define BZ_K_CONVERT 5
#define BZ_NKERNELS 6
int bz_profile(bz_handle h, int enable);
int bz_profile_read(bz_handle h, double* ms_host, int64_t* launches_host, int32_t n);

/* ------------------------------------------------------------------------
 * Batched ensemble: many independent, spatially homogeneous boxes (one x
 * cell each) with their own momentum grid, species set, coupling, mass mode
 * (THERMAL or MASSLESS) and sample count, advanced together with the FP32
 * integrand.  Each step runs the whole hot path of every box -- masses
 * (Eqs. mg, mq), collision sampling with symmetrical deposition (Eqs. ca,
 * small c relation) into the state in place, moments -- as one persistent
 * collision launch (warps take chunks of (box, anchor, 32 samples) units
 * from a global counter, so ragged boxes share the GPU evenly) inside one
 * captured CUDA graph that is replayed every step.
 * ------------------------------------------------------------------------ */
typedef struct bz_box {
    int32_t np[3];          /* momentum cells per axis                               */
    double L;               /* momentum box [-L, L)^3, GeV                           */
    uint32_t species_mask;  /* as bz_set_species                                     */
    int32_t nsamples;       /* samples per anchor, 1..2^20                           */
    double alpha_s;         /* coupling                                              */
    int32_t mass_mode;      /* BZ_MASS_THERMAL or BZ_MASS_MASSLESS                   */
    uint32_t box_id;        /* xored into the Philox key's low word                  */
    uint64_t seed;          /* Philox key                                            */
} bz_box;
typedef struct bz_batch_s* bz_batch;

/* Creates a batch of nboxes boxes (host array, copied) on the current
 * device and allocates its buffers.  Errors: BZ_EINVAL (sizes, masks,
 * nsamples, mass mode FIXED), BZ_ENODEV, BZ_ENOMEM. */
int bz_batch_create(bz_batch* out, int32_t nboxes, const bz_box* boxes);
int bz_batch_destroy(bz_batch b);
const char* bz_batch_last_error(bz_batch b);
/* Layout of the concatenated state and moments (host int64 / int32
 * [nboxes + 1]; either may be NULL): box i owns cells [cell_offsets[i],
 * cell_offsets[i+1]) of the state, laid out [slot][p] as for a handle, and
 * moment rows [slot_offsets[i], slot_offsets[i+1]) of 5 doubles each. */
int bz_batch_layout(bz_batch b, int64_t* cell_offsets, int32_t* slot_offsets);
/* nsteps Euler steps of every box; state (device int64, concatenated) is
 * updated in place; Philox step index step0 + k.  moments_out (device, may
 * be NULL): [nsteps][total slots][5] doubles as bz_moments.  The first call
 * runs the autotuner (on a copy of the state) and every call whose state,
 * moments_out or dt differs from the previous one re-captures the step
 * graph.  The previous masses persist across calls, as with a handle. */
int bz_batch_step(bz_batch b, int64_t* state, double dt, int32_t nsteps, int32_t step0, double* moments_out,
                  void* stream);
/* Tuned work-chunk size (units per grab), blocks per SM and the collision
 * time (ms per step) the autotuner measured; BZ_EINVAL before the first step. */
int bz_batch_tuning(bz_batch b, int32_t* chunk, int32_t* blocks_per_sm, double* ms_collide);
/* Current masses (host double [nboxes][4]) and counters (host int64 [4], as
 * bz_get_flags); both synchronise the device. */
int bz_batch_get_masses(bz_batch b, double* m2_host);
int bz_batch_get_flags(bz_batch b, int64_t* flags_host);

/* No-allocation variant of bz_collision_term (FP64 integrand, symmetric
 * sampler, all anchors).  The paper has no counterpart; this entry point
 * exists for callers that cannot allocate device memory themselves or let
 * a library do it -- code that runs inside another framework's memory pool,
 * under an allocator that forbids cudaMalloc, or in a plug-in that may only
 * touch the buffers it is handed.  It needs no handle and calls no
 * cudaMalloc, cudaFree or other allocating routine: its scratch (f of the
 * state, the mass accumulators, the counters) is a fixed set of file-scope
 * device arrays, about 2.2 MB, which every GPU that loads the library
 * holds until the process exits.
 *   Limits: nslots x nx x np <= BZ_STATIC_MAX_CELLS and nx <= BZ_STATIC_MAX_XCELLS
 *   (BZ_EINVAL with a message otherwise).
 *   Arguments: g (host), the species mask, alpha_s and mass mode as for
 *   bz_set_species; state (device int64 [nslots][nx][np], read only);
 *   m2_in (device double [nx][4]): BZ_MASS_THERMAL -- the masses of the
 *   previous call, which give the energies E = sqrt(p^2 + m^2) inside the
 *   thermal-mass sums, or NULL for E = |p|; BZ_MASS_MASSLESS -- ignored;
 *   BZ_MASS_FIXED -- the masses to use (required); m2_out (device double
 *   [nx][4], may be the same buffer as m2_in) receives the masses used; A
 *   (device int64, same shape as state) is zeroed and filled exactly as
 *   bz_collision_term fills it with BZ_PREC_F64 and BZ_SAMPLER_SYMMETRIC;
 *   nsamples, step, dt as there.  errbuf (host, may be NULL) receives a
 *   message of at most errbuf_len bytes when the return value is not BZ_OK.
 *   Set-up: the first call on a device looks up the device addresses of the
 *   scratch arrays (with that device current) and caches them for the life
 *   of the process; make that first call before any stream capture.  The
 *   cached addresses belong to the device's context: do not call this entry
 *   point again after cudaDeviceReset in the same process.
 *   Sharing: every call on a device uses the same scratch, which keeps the
 *   last call's contents; what must start at zero is cleared on the stream
 *   at the start of each call.  Calls that overlap on the GPU (different
 *   streams, or different threads) race and give wrong results. */
#define BZ_STATIC_MAX_CELLS (1 << 18)
#define BZ_STATIC_MAX_XCELLS 4096
int bz_collision_term_static(const bz_grid* g, uint32_t species_mask, double alpha_s, int32_t mass_mode,
                             const int64_t* state, const double* m2_in, double* m2_out, int64_t* A,
                             int32_t nsamples, int32_t step, double dt, void* stream, char* errbuf,
                             int32_t errbuf_len);

/* ------------------------------------------------------------------------
 * Learned importance-sampling proposal (not in the paper; it changes only
 * where the samples of Eq. (MC C_gg) fall).  For every anchor a small
 * network (9 -> 128 -> 128 -> 6, SiLU, BF16 tensor cores with FP32
 * accumulation) gives the parameters of a density over the normalised box
 * y = (k1x, k1y, k3)/L in [-1, 1)^5:
 *   q(y) = alpha/32 + (1 - alpha) prod_i g_i(y_i),  alpha >= 0.1,
 * g_i Student-t densities with two degrees of freedom truncated to [-1, 1)
 * (k1 components centred at 0 with scale sigma1, k3 components centred at
 * mu3 with scale sigma3; their CDF inverts with square roots only).  A
 * sample drawn from q carries the weight c~ L^5 / q(y) instead of c~ (2L)^5,
 * and its four legs still receive +-w/4, so the estimator stays unbiased
 * for any q > 0 and Sum A = 0 exactly.  Training maximises the |c~|-weighted
 * log-likelihood of samples recorded with the uniform sampler
 * (optimum q ~ |c~|).  Records: struct { int64 anchor; float w; float y[5]; }
 * (32 bytes), w = sum over the sample's terms and roots of |c~|.
 * ------------------------------------------------------------------------ */
/* Number of FP32 parameters of the network (flat: W1[16][128], b1[128],
 * W2[128][128], b2[128], W3[128][8], b3[8]; W[in][out], unused input rows
 * 9..15 and output columns 6, 7 are zero). */
int bz_proposal_nparams(void);
/* Allocates the network on h and draws Glorot-uniform weights from seed. */
int bz_proposal_init(bz_handle h, uint64_t seed);
int bz_proposal_get_params(bz_handle h, float* host);
int bz_proposal_set_params(bz_handle h, const float* host);
/* Uniform FP32 sampling of state in record mode: no deposits, no FP64
 * re-evaluation; for every unit (anchor, 32 samples) whose index is a
 * multiple of unit_stride one record is appended to records (device,
 * max_records) for each sample with w > 0 (samples whose roots were all
 * rejected or fell outside the box carry no information and are skipped).
 * Record order is not deterministic.  *n_written (host) receives the count,
 * at most max_records; synchronises.  Errors: BZ_EINVAL for a NULL pointer,
 * max_records <= 0, unit_stride <= 0 or 2^31 cells or more. */
int bz_record(bz_handle h, const int64_t* state, int32_t nsamples, int32_t step, double dt, int32_t unit_stride,
              void* records, int64_t max_records, int64_t* n_written, void* stream);
/* Loss L = -sum w log q / sum w over records [0, n) and its gradient (device
 * float [nparams], device float loss), forward and backward on the tensor
 * cores.  Synchronises (to read sum w). */
int bz_proposal_grad(bz_handle h, const void* records, int64_t n, float* grad, float* loss, void* stream);
/* steps Adam steps (lr, beta 0.9/0.999), each on a minibatch of `batch`
 * records drawn independently and uniformly from records [0, n) (index
 * SplitMix64(key_step + i) mod n, key_step from the handle's Adam step
 * count), so the minibatches do not follow the arrival order of the
 * records; losses_host (may be NULL) receives each step's loss. */
int bz_proposal_train(bz_handle h, const void* records, int64_t n, int32_t steps, int32_t batch, double lr,
                      float* losses_host, void* stream);
/* Runs the network for every anchor of h (8 floats each: mu3 x3, sigma3,
 * sigma1, alpha, 0, 0) on the tensor cores (tcgen05, 128 anchors per tile);
 * required before BZ_SAMPLER_LEARNED.  Synchronises; BZ_ECUDA if a
 * tensor-core wait timed out. */
int bz_proposal_infer(bz_handle h, void* stream);
/* Reads (out_host) and/or replaces (in_host) the per-anchor parameters,
 * host float [nslots nx np][8]; synchronises. */
int bz_proposal_anchor_params(bz_handle h, float* out_host, const float* in_host);
/* Sampler used by bz_step: BZ_SAMPLER_SYMMETRIC (default) or BZ_SAMPLER_LEARNED. */
int bz_set_step_sampler(bz_handle h, int32_t sampler);

/* ------------------------------------------------------------------------
 * Checkpoint (not in the paper).  The state, the step index (part of every
 * Philox counter) and the current thermal masses (the next mass evaluation's
 * dispersion) determine the rest of a run, so a run restarted from a
 * checkpoint continues bit for bit.
 * bz_save writes a little-endian file: a header (grid, seed, box, species
 * mask, alpha_s, mass mode, step), the masses if set, the state (device
 * int64 [ncell], copied; synchronises).
 * bz_load reads it into h, which must have the same grid, seed, box,
 * species, alpha_s and mass mode (else BZ_EINVAL): the state (device int64
 * [ncell]) and *step (host) receive the saved values, and the saved masses
 * become the handle's current masses.  Errors: BZ_EINVAL for a missing,
 * unreadable, truncated or mismatched file.
 * ------------------------------------------------------------------------ */
int bz_save(bz_handle h, const int64_t* state, int64_t step, const char* path);
int bz_load(bz_handle h, int64_t* state, int64_t* step, const char* path);

/* Bounds-checked builds (compiled with -DBZ_CHECK=1, a stand-in for a
 * memory sanitizer): the collision (FP64, FP32 and its re-evaluation) and the
 * drift kernels (streaming and row forms) test every index they compute into f, A, the
 * state and the mass table before the access, skip an access outside its
 * buffer and count it.  count: indices outside their buffers since the
 * last reset (host, may be NULL); first_bad: one of them, -1 if none (host,
 * may be NULL); reset = 1 clears the counters after reading.  The counters
 * are read with a synchronous copy: synchronize the streams that ran the
 * kernels first.  Errors: BZ_EINVAL in a build without BZ_CHECK (the
 * default), BZ_ECUDA if the copy fails. */
int bz_check_counts(int64_t* count, int64_t* first_bad, int32_t reset);

/* Library version string. */
const char* bz_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BZ_H */
