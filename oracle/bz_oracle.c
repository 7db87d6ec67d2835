/*
 * bz_oracle.c -- plain, slow, FP64 CPU oracle for the Monte Carlo 2->2
 * collision term with symmetrical sampling, the upwind drift and the
 * moment reductions of the relativistic Boltzmann equation for g, u, d, s
 * and their antiquarks (arXiv:1912.04457).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this
 * file; only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code with the CUDA library: everything
 * here (Philox, kinematics, |M|^2, deposition, drift, moments) is written
 * out independently from the paper's equations.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA
 * contraction, so each FP64 operation is one IEEE-rounded step in the
 * written order).
 *
 * Citations are to the paper's sections / equations / table:
 *   Eq. (C_quark), Eq. (C_gluon)  -- the collision terms of each species (Sec. II)
 *   Eq. (C_a_b)                   -- the 2->2 collision integral (Sec. II)
 *   Eqs. (mg), (mq)               -- thermal masses (Sec. II)
 *   Eq. (particle numbers), Eq. (energy momentum tensor) -- moments (Sec. II)
 *   Eqs. (delta function), (work out delta E), (delta replace) -- k2
 *                                    elimination and the k1z root (Sec. III.A)
 *   Eqs. (MC C_gg), (ca), (small c relation) -- MC estimator and symmetrical
 *                                    sampling (Sec. III.B)
 *   Eq. (left handside)           -- conservative (flux) form of the drift and the force term (Sec. III)
 *   Eq. (current conservation)    -- the energy source S_ex of a varying mass (Sec. II)
 *   Table (Matrix elements squared) -- |M|^2 (Appendix)
 *
 * Readings of the paper where it is silent (all listed in the design notes):
 *   - each of the four legs of a sample receives 1/4 of the sample weight;
 *   - each k1z root deposits to its own legs;
 *   - the anchor momentum p is jittered uniformly inside its cell;
 *   - the integration box is (k1x,k1y,k3) in [-L,L)^5; a root whose k1z or
 *     k2 leaves the box is rejected (run param 1: k3 eliminated instead,
 *     (k1x,k1y,k2) sampled, the paper's second choice of Sec. III.A);
 *   - user-defined |M|^2 rows are sums of terms c s^a t^b u^c /
 *     (s^d (t - m_g^2)^e (u - m_g^2)^f) replacing rows of the table;
 *   - the drift is first-order upwind in flux form, periodic in x;
 *   - the optional force term is upwind in p with dE/dx = (dm^2/dx)/(2E),
 *     dm^2/dx a central difference, and no flux through the momentum-box
 *     faces;
 *   - time is in fm/c, momenta in GeV, so dt enters as dt/hbar_c;
 *   - the mass integrals are summed exactly in 2^-30 fixed point, so their
 *     value does not depend on summation order.
 * Parity of the physical evolution curves (the paper's figures) is
 * unpinned: the figures are not available.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NSPEC 7
#define HBARC 0.1973269804 /* GeV fm */
#define PI 3.14159265358979323846
#define TWO_POW_40 1099511627776.0
#define TWO_POW_M40 (1.0 / 1099511627776.0)
#define MASS_SHIFT 30 /* fixed-point scale of the mass integrals: 2^30 */
#define MASS_FX (1.0 / 1024.0) /* state units (2^-40 of N f) to 2^-30 of f: 2^(MASS_SHIFT - 40) */

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random   */
/* numbers: as easy as 1, 2, 3"): ten rounds of the 4x32 S-box with the */
/* published multipliers and Weyl key increments.                      */
/* ------------------------------------------------------------------ */
void bzo_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------ */
/* Configuration                                                       */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t nx[3];          /* spatial cells per axis                          */
    double dx;              /* spatial cell size, fm                           */
    int32_t np[3];          /* momentum cells per axis                         */
    double L;               /* momentum box [-L, L)^3, GeV                     */
    uint64_t seed;          /* Philox key                                      */
    uint32_t box;           /* box id (xored into the key)                     */
    uint32_t species_mask;  /* bit s set: species s active (0 g,1 u,2 d,3 s,4 ub,5 db,6 sb) */
    double alpha_s;         /* strong coupling                                 */
    int32_t mass_mode;      /* 0 thermal dispersion+regulator, 1 massless dispersion, 2 fixed */
    int32_t analytic;       /* 1: f at each leg from the equilibrium formula (Eqs. fg, fq) */
    double T;               /* temperature for analytic f, GeV                 */
    double mu[NSPEC];       /* chemical potentials for analytic f, GeV         */
    int32_t force;          /* 1: the drift includes the force term -div_p[(grad_x E) f] */
    const struct bzo_urow_s* user;  /* user-defined |M|^2 rows (see msq_user), or NULL */
    uint32_t umask;         /* bit r set: row r of the |M|^2 table is user-defined */
} bzo_config;

static int is_quark(int s) { return s != 0; }
static double degeneracy(int s) { return s == 0 ? 16.0 : 6.0; } /* N_g, N_q (Sec. II) */
static int mass_slot(int s) { return s == 0 ? 0 : 1 + (s - 1) % 3; }

static int nslots(const bzo_config* c)
{
    int n = 0;
    for (int s = 0; s < NSPEC; ++s)
        if (c->species_mask & (1u << s)) ++n;
    return n;
}

static int slot_of(const bzo_config* c, int s)
{
    if (!(c->species_mask & (1u << s))) return -1;
    int n = 0;
    for (int q = 0; q < s; ++q)
        if (c->species_mask & (1u << q)) ++n;
    return n;
}

static int64_t n_xcells(const bzo_config* c) { return (int64_t)c->nx[0] * c->nx[1] * c->nx[2]; }
static int64_t n_pcells(const bzo_config* c) { return (int64_t)c->np[0] * c->np[1] * c->np[2]; }

/* ------------------------------------------------------------------ */
/* Terms of each species' equation, Eqs. (C_gluon) and (C_quark); the  */
/* antiquark equation is the charge conjugate of the quark one.  Legs  */
/* are (k1, k2, k3, p) = (a, b, c, d), labelled so that (k1, k3) is    */
/* the like-species / same-flavour line; then the table's t=(k1-k3)^2  */
/* and u=(k1-p)^2 apply to every row as printed.                       */
/* ------------------------------------------------------------------ */
enum { M_QQP = 0, M_QQ, M_QQB, M_QQB2, M_QQBGG, M_QG, M_GG };

typedef struct {
    int leg[4];   /* species of k1, k2, k3, p */
    double sym;   /* 1/2 for identical initial particles */
    int cls;      /* matrix element row */
} bzo_term;

static int quark_of(int f) { return 1 + f; }
static int anti_of(int f) { return 4 + f; }

/* Fills terms[] for anchor species d; returns the count (10 when all
 * species are active).  A term is kept only if all four of its species
 * are active. */
static int terms_for(const bzo_config* c, int d, bzo_term* out)
{
    bzo_term t[16];
    int n = 0;
#define ADD(A, B, C, D, SYM, CLS)                                                    \
    do {                                                                             \
        t[n].leg[0] = (A); t[n].leg[1] = (B); t[n].leg[2] = (C); t[n].leg[3] = (D);  \
        t[n].sym = (SYM); t[n].cls = (CLS); ++n;                                      \
    } while (0)
    if (d == 0) {
        ADD(0, 0, 0, 0, 0.5, M_GG);                      /* 1/2 gg <-> gg          */
        for (int f = 0; f < 3; ++f) {
            int q = quark_of(f), qb = anti_of(f);
            ADD(q, 0, q, 0, 1.0, M_QG);                  /* g q_f <-> g q_f        */
            ADD(qb, 0, qb, 0, 1.0, M_QG);                /* g qb_f <-> g qb_f      */
            ADD(q, qb, 0, 0, 1.0, M_QQBGG);              /* q_f qb_f <-> g g       */
        }
    } else {
        int anti = d >= 4;
        int fa = (d - 1) % 3;
        /* quark-equation legs written for a quark anchor, then charge-conjugated */
        int Q = quark_of(fa), QB = anti_of(fa);
        int me = anti ? QB : Q, bar = anti ? Q : QB;
        ADD(me, me, me, me, 0.5, M_QQ);                  /* 1/2 q_a q_a <-> q_a q_a */
        ADD(bar, me, bar, me, 1.0, M_QQB);               /* q_a qb_a <-> q_a qb_a   */
        ADD(0, 0, bar, me, 0.5, M_QQBGG);                /* 1/2 g g <-> q_a qb_a    */
        ADD(0, me, 0, me, 1.0, M_QG);                    /* q_a g <-> q_a g         */
        for (int fb = 0; fb < 3; ++fb) {
            if (fb == fa) continue;
            int Qb = anti ? anti_of(fb) : quark_of(fb);
            int QBb = anti ? quark_of(fb) : anti_of(fb);
            ADD(Qb, me, Qb, me, 1.0, M_QQP);             /* q_a q_b <-> q_a q_b     */
            ADD(QBb, me, QBb, me, 1.0, M_QQP);           /* q_a qb_b <-> q_a qb_b   */
            ADD(Qb, QBb, bar, me, 1.0, M_QQB2);          /* q_b qb_b <-> q_a qb_a   */
        }
    }
#undef ADD
    int m = 0;
    for (int i = 0; i < n; ++i) {
        int ok = 1;
        for (int l = 0; l < 4; ++l)
            if (!(c->species_mask & (1u << t[i].leg[l]))) ok = 0;
        if (ok) out[m++] = t[i];
    }
    return m;
}

/* ------------------------------------------------------------------ */
/* |M|^2 of the Appendix table, with t and u denominators regulated by */
/* m_g^2, written literally.  SU(3): d_F = C_A = 3, C_F = 4/3, d_A = 8. */
/* ------------------------------------------------------------------ */
/* A user-defined |M|^2 row (the API of Sec. II for the user's own matrix    */
/* elements): sum over its n <= 8 terms of coef s^a t^b u^c / (s^d          */
/* (t - m_g^2)^e (u - m_g^2)^f), e = (a, b, c, d, e, f), each power a       */
/* product of its factors from 1, left to right.                            */
typedef struct { double coef; uint8_t e[6]; uint8_t pad[2]; } bzo_uterm;
typedef struct bzo_urow_s { int32_t n; int32_t pad; bzo_uterm t[8]; } bzo_urow;

typedef struct { double A1, A2, A3, A4, A5; const bzo_urow* user; uint32_t umask; } bzo_mconst;

static double upow(double x, int n)
{
    double r = 1.0;
    for (int i = 0; i < n; ++i) r = r * x;
    return r;
}

static double msq_user(const bzo_urow* row, double s, double t, double u, double mg2)
{
    double tm = t - mg2, um = u - mg2;
    double acc = 0.0;
    for (int k = 0; k < row->n; ++k) {
        const bzo_uterm* T = &row->t[k];
        double num = (upow(s, T->e[0]) * upow(t, T->e[1])) * upow(u, T->e[2]);
        double den = (upow(s, T->e[3]) * upow(tm, T->e[4])) * upow(um, T->e[5]);
        acc = acc + T->coef * (num / den);
    }
    return acc;
}

static bzo_mconst mconst(double alpha_s)
{
    const double dF = 3.0, CA = 3.0, CF = 4.0 / 3.0, dA = 8.0;
    double g2 = 4.0 * PI * alpha_s;
    double g4 = g2 * g2;
    bzo_mconst k;
    k.A1 = 8.0 * g4 * dF * dF * CF * CF / dA;
    k.A2 = 16.0 * g4 * dF * CF * (CF - CA / 2.0);
    k.A3 = 8.0 * g4 * dF * CF * CF;
    k.A4 = 8.0 * g4 * dF * CF * CA;
    k.A5 = 16.0 * g4 * dA * CA * CA;
    k.user = NULL;
    k.umask = 0;
    return k;
}

static double msq(int cls, const bzo_mconst* k, double s, double t, double u, double mg2)
{
    if (k->user && (k->umask >> cls & 1u)) return msq_user(&k->user[cls], s, t, u, mg2);
    double tm = t - mg2, um = u - mg2;
    switch (cls) {
    case M_QQP:
        return k->A1 * ((s * s + u * u) / (tm * tm));
    case M_QQ:
        return k->A1 * ((s * s + u * u) / (tm * tm) + (s * s + t * t) / (um * um))
               + k->A2 * ((s * s) / (tm * um));
    case M_QQB:
        return k->A1 * ((s * s + u * u) / (tm * tm) + (u * u + t * t) / (s * s))
               + k->A2 * ((u * u) / (tm * s));
    case M_QQB2:
        return k->A1 * ((t * t + u * u) / (s * s));
    case M_QQBGG:
        return k->A3 * (u / tm + t / um) - k->A4 * ((t * t + u * u) / (s * s));
    case M_QG:
        return k->A4 * ((s * s + u * u) / (tm * tm)) - k->A3 * (u / s + s / um);
    case M_GG:
        return k->A5 * (3.0 - (s * u) / (tm * tm) - (s * t) / (um * um) - (t * u) / (s * s));
    }
    return 0.0;
}

/* Exported for the crossing-identity pins. */
double bzo_msq(int cls, double alpha_s, double s, double t, double u, double mg2)
{
    bzo_mconst k = mconst(alpha_s);
    return msq(cls, &k, s, t, u, mg2);
}

/* Exported for the user-row pins: one user-defined row at (s, t, u). */
double bzo_msq_user(const bzo_urow* row, double s, double t, double u, double mg2)
{
    return msq_user(row, s, t, u, mg2);
}

/* ------------------------------------------------------------------ */
/* k1z roots, Eqs. (work out delta E), (delta replace).  Given p, k3   */
/* and k1_perp, with k2 = p + k3 - k1, E1 + E2 = E3 + Ep has at most   */
/* two solutions in k1z; J = k1z/E1 - (k3z + pz - k1z)/E2.             */
/* ------------------------------------------------------------------ */
typedef struct { double z, E1, E2, J; } bzo_root;

static int solve_roots(const double p[3], double Ep, const double k3[3], double E3,
                       double k1x, double k1y, double ma2, double mb2, bzo_root r[2])
{
    double Px = p[0] + k3[0], Py = p[1] + k3[1], Pz = p[2] + k3[2];
    double E = Ep + E3;
    double a2 = (k1x * k1x + k1y * k1y) + ma2;
    double bx = Px - k1x, by = Py - k1y;
    double b2 = (bx * bx + by * by) + mb2;
    double D = E * E - Pz * Pz;
    double kap = (E * E + a2 - b2 - Pz * Pz) * 0.5;
    double H = kap * kap - a2 * D;
    if (H < 0.0 || D <= 0.0) return 0;
    double kp = kap * Pz;
    double sq = E * sqrt(H);
    double Q = kp >= 0.0 ? kp + sq : kp - sq;
    if (Q == 0.0) return 0;
    double zc[2];
    zc[0] = Q / D;
    zc[1] = (E * E * a2 - kap * kap) / Q;
    int n = 0;
    for (int i = 0; i < 2; ++i) {
        double z = zc[i];
        double e1 = (kap + Pz * z) / E;
        if (!(e1 > 0.0 && e1 < E)) continue;
        double E1 = sqrt(a2 + z * z);
        double dz = Pz - z;
        double E2 = sqrt(b2 + dz * dz);
        double J = z / E1 - dz / E2;
        if (J == 0.0) continue;
        r[n].z = z; r[n].E1 = E1; r[n].E2 = E2; r[n].J = J;
        ++n;
    }
    return n;
}

/* ------------------------------------------------------------------ */
/* The second choice of Sec. III.A: k3 = k1 + k2 - p eliminated.  Given */
/* p, k2 and k1_perp, E1 - E3 = Ep - E2 = dl with E3^2 = c2 + (k1z +    */
/* K)^2, c2 = (k1x + k2x - px)^2 + (k1y + k2y - py)^2 + mc^2, K = k2z - */
/* pz.  Squaring twice gives (K^2 - dl^2) z^2 - K (A0 + 2 dl^2) z +     */
/* A0^2/4 - dl^2 (c2 + K^2) = 0 with A0 = a2 - c2 - K^2 - dl^2; a root  */
/* of it solves the original equation iff A0 - 2 K z (= 2 dl E3) has   */
/* the sign of dl and E3 + dl > 0.  J = d(E1 - E3)/dk1z = k1z/E1 -      */
/* (k1z + K)/E3.  Returns the roots with (k1z, E1, E3, J) in r[].       */
/* ------------------------------------------------------------------ */
static int solve_roots_k3(const double p[3], double Ep, const double k2[3], double E2, double k1x, double k1y,
                          double ma2, double mc2, bzo_root r[2])
{
    double cx = (k1x + k2[0]) - p[0], cy = (k1y + k2[1]) - p[1], K = k2[2] - p[2];
    double a2 = (k1x * k1x + k1y * k1y) + ma2;
    double c2 = (cx * cx + cy * cy) + mc2;
    double dl = Ep - E2;
    double A0 = ((a2 - c2) - K * K) - dl * dl;
    double qa = K * K - dl * dl;
    double qb = -K * (A0 + 2.0 * dl * dl);
    double qc = 0.25 * A0 * A0 - dl * dl * (c2 + K * K);
    if (qa == 0.0 || dl == 0.0) return 0;
    double disc = qb * qb - 4.0 * qa * qc;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double Q = -0.5 * (qb >= 0.0 ? qb + sq : qb - sq);
    if (Q == 0.0) return 0;
    double zc[2] = {Q / qa, qc / Q};
    int n = 0;
    for (int i = 0; i < 2; ++i) {
        double z = zc[i];
        double w = A0 - 2.0 * K * z;
        if (!(dl > 0.0 ? w > 0.0 : w < 0.0)) continue;
        double zk = z + K;
        double E3 = sqrt(c2 + zk * zk);
        if (!(E3 + dl > 0.0)) continue;
        double E1 = sqrt(a2 + z * z);
        double J = z / E1 - zk / E3;
        if (J == 0.0) continue;
        r[n].z = z; r[n].E1 = E1; r[n].E2 = E3; r[n].J = J;  /* E2 slot carries E3 here */
        ++n;
    }
    return n;
}

/* Exported for the two-body phase-space pin: returns the number of valid
 * roots and, per root, (k1z, E1, E2, J) in out[4*i..4*i+3]. */
int bzo_roots(const double p[3], double md2, const double k3[3], double mc2,
              double k1x, double k1y, double ma2, double mb2, double out[8])
{
    double Ep = sqrt((p[0] * p[0] + p[1] * p[1]) + p[2] * p[2] + md2);
    double E3 = sqrt((k3[0] * k3[0] + k3[1] * k3[1]) + k3[2] * k3[2] + mc2);
    bzo_root r[2];
    int n = solve_roots(p, Ep, k3, E3, k1x, k1y, ma2, mb2, r);
    for (int i = 0; i < n; ++i) {
        out[4 * i + 0] = r[i].z; out[4 * i + 1] = r[i].E1;
        out[4 * i + 2] = r[i].E2; out[4 * i + 3] = r[i].J;
    }
    return n;
}

/* Two-body phase-space hook: midpoint sum over an m x m grid of
 * k1_perp in [-R, R)^2 of sum_roots 1/(|J| 2E1 2E2), i.e. the integral
 * over d^3k1/(2E1 2E2) delta(E1 + E2 - E3 - Ep) with k2 = p + k3 - k1
 * (no box cut), optionally weighted by J^2 (which keeps the integrand
 * bounded at the edge of the solution set, where J -> 0).  Unweighted it
 * equals (pi/2) lambda^{1/2}(s, ma2, mb2)/s when R covers the solution set. */
double bzo_two_body_sum(const double p[3], double md2, const double k3[3], double mc2,
                        double ma2, double mb2, double R, int m, int weight_j2)
{
    double Ep = sqrt((p[0] * p[0] + p[1] * p[1]) + p[2] * p[2] + md2);
    double E3 = sqrt((k3[0] * k3[0] + k3[1] * k3[1]) + k3[2] * k3[2] + mc2);
    double h = 2.0 * R / m;
    double total = 0.0;
#pragma omp parallel for reduction(+ : total)
    for (int i = 0; i < m; ++i) {
        double row = 0.0;
        for (int k = 0; k < m; ++k) {
            bzo_root r[2];
            int n = solve_roots(p, Ep, k3, E3, -R + (i + 0.5) * h, -R + (k + 0.5) * h, ma2, mb2, r);
            for (int q = 0; q < n; ++q) {
                double wgt = weight_j2 ? r[q].J * r[q].J : 1.0;
                row += wgt / (fabs(r[q].J) * 4.0 * r[q].E1 * r[q].E2);
            }
        }
        total += row;
    }
    return total * h * h;
}

/* ------------------------------------------------------------------ */
/* Grid helpers (cell-centred, Dp = 2L/n, centres -L + (j+1/2) Dp)     */
/* ------------------------------------------------------------------ */
static int bin_of(double k, double L, double dp, int n)
{
    int j = (int)floor((k + L) / dp);
    if (j < 0) j = 0;
    if (j >= n) j = n - 1;
    return j;
}

static int in_box(double k, double L) { return k >= -L && k < L; }

static double f_of_state(int64_t n, int s) { return (double)n * TWO_POW_M40 / degeneracy(s); }

/* equilibrium distribution, Eqs. (fg), (fq) */
static double f_equilibrium(const bzo_config* c, int s, double E)
{
    double x = (E - c->mu[s]) / c->T;
    return is_quark(s) ? 1.0 / (exp(x) + 1.0) : 1.0 / (exp(x) - 1.0);
}

/* ------------------------------------------------------------------ */
/* Thermal masses, Eqs. (mg), (mq).  Each species integral uses its    */
/* own dispersion E^a = sqrt(p^2 + m_a^2) with the previous masses      */
/* (E = |p| when m2_prev is NULL, the first step, and always in mass    */
/* mode 1, the massless dispersion).  The bin sums (3x the Eq. (mg)    */
/* integrand, 24x the Eq. (mq) one) are taken exactly in 2^-30 fixed    */
/* point of f; out[x][0] = m_g^2, out[x][1+i] =                         */
/* m_{q_i}^2.  Returns 0, or 1 if a fixed-point sum would overflow.     */
/* ------------------------------------------------------------------ */
int bzo_masses(const bzo_config* c, const int64_t* state, const double* m2_prev, double* out)
{
    const double CF = 4.0 / 3.0, dA = 8.0;  /* C_A = 3 and C_F enter the integrand coefficients */
    double g2 = 4.0 * PI * c->alpha_s;
    double dpx = 2.0 * c->L / c->np[0], dpy = 2.0 * c->L / c->np[1], dpz = 2.0 * c->L / c->np[2];
    double twopi = 2.0 * PI;
    double meas = dpx * dpy * dpz / (twopi * twopi * twopi);
    int64_t nxc = n_xcells(c), npc = n_pcells(c);
    int64_t limit = INT64_MAX / (npc > 0 ? npc : 1) / 2;
    int ovf = 0;
    for (int64_t x = 0; x < nxc; ++x) {
        int64_t sum_g = 0, sum_q[3] = {0, 0, 0};
        double m2p[4] = {0, 0, 0, 0};
        if (m2_prev && c->mass_mode != 1)
            for (int i = 0; i < 4; ++i) m2p[i] = m2_prev[x * 4 + i];
        for (int64_t j = 0; j < npc; ++j) {
            int jx = (int)(j / ((int64_t)c->np[1] * c->np[2]));
            int jy = (int)((j / c->np[2]) % c->np[1]);
            int jz = (int)(j % c->np[2]);
            double px = -c->L + ((double)jx + 0.5) * dpx;
            double py = -c->L + ((double)jy + 0.5) * dpy;
            double pz = -c->L + ((double)jz + 0.5) * dpz;
            double pp = (px * px + py * py) + pz * pz;
            /* N_s f_s = n_s 2^-40, so with r_a = 1/(2 E_a) the bin integrands are
             *   Eq. (mg): N_g C_A f_g r_g + sum_i N_q C_F (f_qi + f_qbi) r_qi
             *             = 2^-40 (3 n_g r_g + (4/3) sum_i q_i r_qi),
             *   Eq. (mq): 2 f_g r_g + (f_qi + f_qbi) r_qi = 2^-40 (n_g r_g / 8 + q_i r_qi / 6),
             * q_i = n_qi + n_qbi.  They are summed as 3x and 24x these (integer
             * coefficients), rounded to 2^-30 of f. */
            int64_t nsp[NSPEC];
            for (int s = 0; s < NSPEC; ++s) {
                int sl = slot_of(c, s);
                nsp[s] = sl < 0 ? 0 : state[((int64_t)sl * nxc + x) * npc + j];
            }
            double ng = (double)nsp[0];
            double rg = 0.5 / sqrt(pp + m2p[0]);
            double q[3], rq[3];
            for (int i = 0; i < 3; ++i) {
                q[i] = (double)(nsp[1 + i] + nsp[4 + i]);
                rq[i] = 0.5 / sqrt(pp + m2p[1 + i]);
            }
            double g3 = 9.0 * ng * rg + 4.0 * ((q[0] * rq[0] + q[1] * rq[1]) + q[2] * rq[2]);
            int64_t qg = llrint(g3 * MASS_FX);
            if (qg > limit || qg < -limit) ovf = 1;
            sum_g += qg;
            for (int i = 0; i < 3; ++i) {
                double q24 = 3.0 * ng * rg + 4.0 * q[i] * rq[i];
                int64_t qq = llrint(q24 * MASS_FX);
                if (qq > limit || qq < -limit) ovf = 1;
                sum_q[i] += qq;
            }
        }
        double inv = 1.0 / (double)(1LL << MASS_SHIFT);
        out[x * 4 + 0] = (2.0 * g2 / dA) * meas * ((double)sum_g * inv) / 3.0;
        for (int i = 0; i < 3; ++i)
            out[x * 4 + 1 + i] = (2.0 * CF * g2) * meas * ((double)sum_q[i] * inv) / 24.0;
    }
    return ovf;
}

/* ------------------------------------------------------------------ */
/* Collision term, Eqs. (C_a_b), (MC C_gg), (ca), (small c relation).  */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t nsamples;        /* N samples per anchor (x-cell, species d, p-cell)     */
    int32_t step;            /* time-step index, part of the Philox counter          */
    double dt;               /* fm/c                                                 */
    int32_t sampler;         /* 0 symmetrical (4 legs, 1/4 each), 1 plain (own cell), 2 symmetrical
                                with samples from a per-anchor proposal density              */
    int32_t ubits;           /* 32: u=(x+1/2)2^-32; 23: u=((x>>9)+1/2)2^-23          */
    int32_t p_center;        /* 1: p at the cell centre (no jitter)                  */
    int64_t anchor_stride;   /* anchors with index % stride == offset are sampled    */
    int64_t anchor_offset;
    const double* u_explicit;/* optional [anchor][sample][8] uniforms replacing Philox */
    const double* prop;      /* sampler 2: per-anchor proposal (mu3 x3, sigma3, sigma1, alpha, -, -) */
    int32_t param;           /* 0: k2 = k3 + p - k1 eliminated (the paper's choice); 1: k3 = k1 + k2 - p
                                eliminated, (k1_perp, k2) sampled (Sec. III.A, "less stable") */
    int32_t u_shared;        /* 1: u_explicit is one [sample][8] set used by every anchor */
} bzo_run;

/* Learned-proposal sample: defensive mixture q(y) = alpha/32 + (1 - alpha)
 * prod_i g_i(y_i) on y = (k1x, k1y, k3)/L in [-1, 1)^5, g_i the Student-t
 * density with two degrees of freedom, f(z) = (2 + z^2)^(-3/2), truncated to
 * [-1, 1) (centre 0 and scale sigma1 for the k1 components, centre mu3 and
 * scale sigma3 for k3); pr = (mu3 x3, sigma3, sigma1, alpha).  Its CDF is
 * F(z) = 1/2 + z / (2 sqrt(2 + z^2)), so with v = Fa + u (Fb - Fa) and
 * cv = 1 - v the inverse is z = (v - cv) / sqrt(2 v cv) and the density
 * there is f(z) = (2 v cv)^(3/2): square roots only.  usel < alpha picks the
 * uniform component (y = 2u - 1).  Returns 1/(32 q(y)), the factor that
 * turns the uniform weight V/N into 1/(N q_x). */
static double t2_tail(double z) /* F(-|z|) without cancellation */
{
    double s = sqrt(2.0 + z * z);
    return 1.0 / (s * (s + fabs(z)));
}

double bzo_proposal_sample(const double* pr, double usel, const double* u5, double* y)
{
    int uni = usel < pr[5];
    double G = 1.0;
    for (int i = 0; i < 5; ++i) {
        double mu = i < 2 ? 0.0 : pr[i - 2];
        double sg = i < 2 ? pr[4] : pr[3];
        double Fa = t2_tail((-1.0 - mu) / sg);  /* F(za), za < 0 */
        double cFb = t2_tail((1.0 - mu) / sg);  /* 1 - F(zb), zb > 0 */
        double D = (1.0 - cFb) - Fa;
        if (uni) {
            y[i] = 2.0 * u5[i] - 1.0;
            double z = (y[i] - mu) / sg;
            double s = sqrt(2.0 + z * z);
            G *= 1.0 / (s * s * s * sg * D);
        } else {
            double v = Fa + u5[i] * D, cv = cFb + (1.0 - u5[i]) * D;
            double t = 2.0 * v * cv;
            y[i] = mu + sg * ((v - cv) / sqrt(t));
            if (y[i] < -1.0) y[i] = -1.0;
            if (y[i] >= 1.0) y[i] = 0.99999994;
            G *= t * sqrt(t) / (sg * D);
        }
    }
    return 1.0 / (32.0 * (pr[5] / 32.0 + (1.0 - pr[5]) * G));
}

static double uniform_of(uint32_t x, int ubits)
{
    if (ubits == 23) return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
    return ((double)x + 0.5) * (1.0 / 4294967296.0);
}

/* One sample of the k3-eliminating parameterisation (run param 1):     */
/* (k1x, k1y, k2) uniform in the box, k1z from solve_roots_k3, k3 =      */
/* k1 + k2 - p; a root is kept if k1z and k3 lie in the box.  Weights,   */
/* |M|^2, W and the four deposits as in the k2 form, with the Jacobian   */
/* of this root.                                                         */
static void collide_sample_k3(const bzo_config* c, const bzo_run* r, const int64_t* state, const double* mdisp,
                              double mg2reg, int64_t x, const int jv[3], const double p[3], double k1x,
                              double k1y, const double k2[3], const bzo_term* terms, int nterms, const bzo_mconst* mk,
                              double Kq, double Kown, double twopi5, int64_t* A, double* c64, double* g64,
                              double* audit, int64_t* flags)
{
    int64_t nxc = n_xcells(c), npc = n_pcells(c);
    double L = c->L, twoL = 2.0 * c->L;
    double dp[3] = {twoL / c->np[0], twoL / c->np[1], twoL / c->np[2]};
    double pp = (p[0] * p[0] + p[1] * p[1]) + p[2] * p[2];
    double kk2 = (k2[0] * k2[0] + k2[1] * k2[1]) + k2[2] * k2[2];
    int64_t linp = ((int64_t)jv[0] * c->np[1] + jv[1]) * c->np[2] + jv[2];
    int64_t lin2 = ((int64_t)bin_of(k2[0], L, dp[0], c->np[0]) * c->np[1] + bin_of(k2[1], L, dp[1], c->np[1]))
                       * c->np[2] + bin_of(k2[2], L, dp[2], c->np[2]);
    for (int ti = 0; ti < nterms; ++ti) {
        const bzo_term* T = &terms[ti];
        int sa = T->leg[0], sb = T->leg[1], sc = T->leg[2], sd = T->leg[3];
        double ma2 = mdisp[mass_slot(sa)], mb2 = mdisp[mass_slot(sb)];
        double mc2 = mdisp[mass_slot(sc)], md2 = mdisp[mass_slot(sd)];
        double Ep = sqrt(pp + md2);
        double E2 = sqrt(kk2 + mb2);
        bzo_root rt[2];
        int nr = solve_roots_k3(p, Ep, k2, E2, k1x, k1y, ma2, mc2, rt);
        for (int ri = 0; ri < nr; ++ri) {
            double z = rt[ri].z, E1 = rt[ri].E1, E3 = rt[ri].E2, J = rt[ri].J;
            double k1[3] = {k1x, k1y, z};
            double k3[3] = {(k1x + k2[0]) - p[0], (k1y + k2[1]) - p[1], z + (k2[2] - p[2])};
            if (!in_box(z, L) || !in_box(k3[0], L) || !in_box(k3[1], L) || !in_box(k3[2], L)) continue;
            double E = Ep + E3;
            double PP = ((p[0] + k3[0]) * (p[0] + k3[0]) + (p[1] + k3[1]) * (p[1] + k3[1]))
                        + (p[2] + k3[2]) * (p[2] + k3[2]);
            double s = E * E - PP;
            double k1k3 = (k1[0] * k3[0] + k1[1] * k3[1]) + k1[2] * k3[2];
            double k1p = (k1[0] * p[0] + k1[1] * p[1]) + k1[2] * p[2];
            double t = (ma2 + mc2) - 2.0 * (E1 * E3 - k1k3);
            double uu = (ma2 + md2) - 2.0 * (E1 * Ep - k1p);
            if (s <= 0.0 || t - mg2reg >= 0.0 || uu - mg2reg >= 0.0) {
#pragma omp atomic
                flags[0] += 1;
                continue;
            }
            double M2 = msq(T->cls, mk, s, t, uu, mg2reg);
            int64_t lin1 = ((int64_t)bin_of(k1[0], L, dp[0], c->np[0]) * c->np[1] + bin_of(k1[1], L, dp[1], c->np[1]))
                               * c->np[2] + bin_of(k1[2], L, dp[2], c->np[2]);
            int64_t lin3 = ((int64_t)bin_of(k3[0], L, dp[0], c->np[0]) * c->np[1] + bin_of(k3[1], L, dp[1], c->np[1]))
                               * c->np[2] + bin_of(k3[2], L, dp[2], c->np[2]);
            double f1, f2, f3, fp;
            if (c->analytic) {
                f1 = f_equilibrium(c, sa, E1);
                f2 = f_equilibrium(c, sb, E2);
                f3 = f_equilibrium(c, sc, E3);
                fp = f_equilibrium(c, sd, Ep);
            } else {
                f1 = f_of_state(state[((int64_t)slot_of(c, sa) * nxc + x) * npc + lin1], sa);
                f2 = f_of_state(state[((int64_t)slot_of(c, sb) * nxc + x) * npc + lin2], sb);
                f3 = f_of_state(state[((int64_t)slot_of(c, sc) * nxc + x) * npc + lin3], sc);
                fp = f_of_state(state[((int64_t)slot_of(c, sd) * nxc + x) * npc + linp], sd);
            }
            double F1 = is_quark(sa) ? 1.0 - f1 : 1.0 + f1;
            double F2 = is_quark(sb) ? 1.0 - f2 : 1.0 + f2;
            double F3 = is_quark(sc) ? 1.0 - f3 : 1.0 + f3;
            double Fp = is_quark(sd) ? 1.0 - fp : 1.0 + fp;
            double gain = f1 * f2 * F3 * Fp;
            double W = gain - F1 * F2 * f3 * fp;
            double den = fabs(J) * twopi5 * 16.0 * E1 * E2 * E3 * Ep;
            double ct = T->sym * W * M2 / den;
            double wq = ct * Kown;
            if (!(fabs(wq) < 4611686018427387904.0)) {
#pragma omp atomic
                flags[1] += 1;
                continue;
            }
            int64_t q = llrint(wq);
            *c64 += ct * (Kq * 4.0) * (1.0 / TWO_POW_40);
            *g64 += (T->sym * gain * M2 / den) * (Kq * 4.0) * (1.0 / TWO_POW_40);
            {
                int64_t idx = ((int64_t)slot_of(c, sd) * nxc + x) * npc + linp;
#pragma omp atomic
                A[idx] += q;
            }
            if (r->sampler != 1) {
                int64_t i3 = ((int64_t)slot_of(c, sc) * nxc + x) * npc + lin3;
                int64_t i1 = ((int64_t)slot_of(c, sa) * nxc + x) * npc + lin1;
                int64_t i2 = ((int64_t)slot_of(c, sb) * nxc + x) * npc + lin2;
#pragma omp atomic
                A[i3] += q;
#pragma omp atomic
                A[i1] -= q;
#pragma omp atomic
                A[i2] -= q;
            }
            if (audit) {
                double w = ct * Kq;
                audit[0] += w * ((Ep + E3) - (E1 + E2));
                audit[1] += w * ((p[0] + k3[0]) - (k1[0] + k2[0]));
                audit[2] += w * ((p[1] + k3[1]) - (k1[1] + k2[1]));
                audit[3] += w * ((p[2] + k3[2]) - (k1[2] + k2[2]));
                audit[4] += fabs(w) * (Ep + E3 + E1 + E2);
                audit[5] += 1.0;
                audit[6] += fabs(w);
            }
        }
    }
}

/* Samples the anchor (slot sl / species d, x-cell x, p-cell j).  Deposits
 * into A (int64), adds the own-cell unquantised estimate into C64[anchor]
 * and its gain part into G64[anchor], and accumulates audit sums. */
static void collide_anchor(const bzo_config* c, const bzo_run* r, const int64_t* state,
                           const double* m2, int d, int64_t x, int64_t j, int64_t aidx,
                           const bzo_term* terms, int nterms, const bzo_mconst* mk,
                           double Kq, int64_t* A, double* C64, double* G64, double* audit,
                           int64_t* flags)
{
    int64_t nxc = n_xcells(c), npc = n_pcells(c);
    double L = c->L, twoL = 2.0 * c->L;
    double dp[3] = {twoL / c->np[0], twoL / c->np[1], twoL / c->np[2]};
    int jv[3] = {(int)(j / ((int64_t)c->np[1] * c->np[2])), (int)((j / c->np[2]) % c->np[1]),
                 (int)(j % c->np[2])};
    double mdisp[4], mg2reg = m2[x * 4 + 0];
    for (int i = 0; i < 4; ++i) mdisp[i] = c->mass_mode == 1 ? 0.0 : m2[x * 4 + i];
    const double twopi = 2.0 * PI;
    const double twopi5 = twopi * twopi * twopi * twopi * twopi;
    double Kown = r->sampler == 1 ? Kq * 4.0 : Kq;
    double c64 = 0.0, g64 = 0.0;
    uint32_t key[2] = {(uint32_t)(c->seed & 0xffffffffu) ^ c->box, (uint32_t)(c->seed >> 32)};

    for (int32_t smp = 0; smp < r->nsamples; ++smp) {
        double u[8];
        if (r->u_explicit) {
            int64_t ua = r->u_shared ? 0 : aidx;
            for (int i = 0; i < 8; ++i) u[i] = r->u_explicit[(ua * r->nsamples + smp) * 8 + i];
        } else {
            for (int blk = 0; blk < 2; ++blk) {
                uint32_t ctr[4] = {(uint32_t)(2 * smp + blk), (uint32_t)j, (uint32_t)x,
                                   ((uint32_t)r->step << 3) | (uint32_t)d};
                uint32_t o[4];
                bzo_philox4x32_10(ctr, key, o);
                for (int i = 0; i < 4; ++i) u[4 * blk + i] = uniform_of(o[i], r->ubits);
            }
        }
        double p[3], k3[3];
        for (int i = 0; i < 3; ++i) {
            double pc = -L + ((double)jv[i] + 0.5) * dp[i];
            p[i] = r->p_center ? pc : pc + dp[i] * (u[i] - 0.5);
        }
        double k1x, k1y, wfac = 1.0;
        if (r->sampler == 2) {
            const double* pr = r->prop + aidx * 8;
            uint32_t ctr[4] = {0x80000000u | (uint32_t)smp, (uint32_t)j, (uint32_t)x,
                               ((uint32_t)r->step << 3) | (uint32_t)d};
            uint32_t o[4];
            bzo_philox4x32_10(ctr, key, o);
            double y[5];
            wfac = bzo_proposal_sample(pr, uniform_of(o[0], r->ubits), u + 3, y);
            k1x = L * y[0];
            k1y = L * y[1];
            for (int i = 0; i < 3; ++i) k3[i] = L * y[2 + i];
        } else {
            k1x = -L + twoL * u[3];
            k1y = -L + twoL * u[4];
            for (int i = 0; i < 3; ++i) k3[i] = -L + twoL * u[5 + i];  /* k2 when param == 1 */
        }
        if (r->param == 1) {
            collide_sample_k3(c, r, state, mdisp, mg2reg, x, jv, p, k1x, k1y, k3, terms, nterms, mk, Kq, Kown,
                              twopi5, A, &c64, &g64, audit, flags);
            continue;
        }
        double pp = (p[0] * p[0] + p[1] * p[1]) + p[2] * p[2];
        double kk3 = (k3[0] * k3[0] + k3[1] * k3[1]) + k3[2] * k3[2];
        int bp[3] = {jv[0], jv[1], jv[2]};
        int b3[3] = {bin_of(k3[0], L, dp[0], c->np[0]), bin_of(k3[1], L, dp[1], c->np[1]),
                     bin_of(k3[2], L, dp[2], c->np[2])};
        int64_t lin3 = ((int64_t)b3[0] * c->np[1] + b3[1]) * c->np[2] + b3[2];
        int64_t linp = ((int64_t)bp[0] * c->np[1] + bp[1]) * c->np[2] + bp[2];

        for (int ti = 0; ti < nterms; ++ti) {
            const bzo_term* T = &terms[ti];
            int sa = T->leg[0], sb = T->leg[1], sc = T->leg[2], sd = T->leg[3];
            double ma2 = mdisp[mass_slot(sa)], mb2 = mdisp[mass_slot(sb)];
            double mc2 = mdisp[mass_slot(sc)], md2 = mdisp[mass_slot(sd)];
            double Ep = sqrt(pp + md2);
            double E3 = sqrt(kk3 + mc2);
            bzo_root rt[2];
            int nr = solve_roots(p, Ep, k3, E3, k1x, k1y, ma2, mb2, rt);
            for (int ri = 0; ri < nr; ++ri) {
                double z = rt[ri].z, E1 = rt[ri].E1, E2 = rt[ri].E2, J = rt[ri].J;
                double k1[3] = {k1x, k1y, z};
                double k2[3] = {(p[0] + k3[0]) - k1x, (p[1] + k3[1]) - k1y, (p[2] + k3[2]) - z};
                if (!in_box(z, L) || !in_box(k2[0], L) || !in_box(k2[1], L) || !in_box(k2[2], L))
                    continue;
                double E = Ep + E3;
                double PP = ((p[0] + k3[0]) * (p[0] + k3[0]) + (p[1] + k3[1]) * (p[1] + k3[1]))
                            + (p[2] + k3[2]) * (p[2] + k3[2]);
                double s = E * E - PP;
                double k1k3 = (k1[0] * k3[0] + k1[1] * k3[1]) + k1[2] * k3[2];
                double k1p = (k1[0] * p[0] + k1[1] * p[1]) + k1[2] * p[2];
                double t = (ma2 + mc2) - 2.0 * (E1 * E3 - k1k3);
                double uu = (ma2 + md2) - 2.0 * (E1 * Ep - k1p);
                if (s <= 0.0 || t - mg2reg >= 0.0 || uu - mg2reg >= 0.0) {
#pragma omp atomic
                    flags[0] += 1;
                    continue;
                }
                double M2 = msq(T->cls, mk, s, t, uu, mg2reg);
                int b1[3] = {bin_of(k1[0], L, dp[0], c->np[0]), bin_of(k1[1], L, dp[1], c->np[1]),
                             bin_of(k1[2], L, dp[2], c->np[2])};
                int b2[3] = {bin_of(k2[0], L, dp[0], c->np[0]), bin_of(k2[1], L, dp[1], c->np[1]),
                             bin_of(k2[2], L, dp[2], c->np[2])};
                int64_t lin1 = ((int64_t)b1[0] * c->np[1] + b1[1]) * c->np[2] + b1[2];
                int64_t lin2 = ((int64_t)b2[0] * c->np[1] + b2[1]) * c->np[2] + b2[2];
                double f1, f2, f3, fp;
                if (c->analytic) {
                    f1 = f_equilibrium(c, sa, E1);
                    f2 = f_equilibrium(c, sb, E2);
                    f3 = f_equilibrium(c, sc, E3);
                    fp = f_equilibrium(c, sd, Ep);
                } else {
                    f1 = f_of_state(state[((int64_t)slot_of(c, sa) * nxc + x) * npc + lin1], sa);
                    f2 = f_of_state(state[((int64_t)slot_of(c, sb) * nxc + x) * npc + lin2], sb);
                    f3 = f_of_state(state[((int64_t)slot_of(c, sc) * nxc + x) * npc + lin3], sc);
                    fp = f_of_state(state[((int64_t)slot_of(c, sd) * nxc + x) * npc + linp], sd);
                }
                /* F = 1 + f for gluons, 1 - f for (anti)quarks (Eq. C_a_b) */
                double F1 = is_quark(sa) ? 1.0 - f1 : 1.0 + f1;
                double F2 = is_quark(sb) ? 1.0 - f2 : 1.0 + f2;
                double F3 = is_quark(sc) ? 1.0 - f3 : 1.0 + f3;
                double Fp = is_quark(sd) ? 1.0 - fp : 1.0 + fp;
                double gain = f1 * f2 * F3 * Fp;
                double W = gain - F1 * F2 * f3 * fp;
                double den = fabs(J) * twopi5 * 16.0 * E1 * E2 * E3 * Ep;
                double ct = T->sym * W * M2 / den;        /* c~ of Eq. (ca), one root */
                double wq = ct * Kown * wfac;             /* weight in units 2^-40 of N f */
                if (!(fabs(wq) < 4611686018427387904.0)) {
#pragma omp atomic
                    flags[1] += 1;
                    continue;
                }
                int64_t q = llrint(wq);
                c64 += ct * (Kq * 4.0) * wfac * (1.0 / TWO_POW_40);
                g64 += (T->sym * gain * M2 / den) * (Kq * 4.0) * wfac * (1.0 / TWO_POW_40);
                /* own cell: +q to (d, p) */
                {
                    int64_t idx = ((int64_t)slot_of(c, sd) * nxc + x) * npc + linp;
#pragma omp atomic
                    A[idx] += q;
                }
                if (r->sampler != 1) {
                    int64_t i3 = ((int64_t)slot_of(c, sc) * nxc + x) * npc + lin3;
                    int64_t i1 = ((int64_t)slot_of(c, sa) * nxc + x) * npc + lin1;
                    int64_t i2 = ((int64_t)slot_of(c, sb) * nxc + x) * npc + lin2;
#pragma omp atomic
                    A[i3] += q;
#pragma omp atomic
                    A[i1] -= q;
#pragma omp atomic
                    A[i2] -= q;
                }
                if (audit) {
                    /* continuous-leg E / P balance of each deposit set */
                    double w = ct * Kq * wfac;
                    audit[0] += w * ((Ep + E3) - (E1 + E2));
                    audit[1] += w * ((p[0] + k3[0]) - (k1[0] + k2[0]));
                    audit[2] += w * ((p[1] + k3[1]) - (k1[1] + k2[1]));
                    audit[3] += w * ((p[2] + k3[2]) - (k1[2] + k2[2]));
                    audit[4] += fabs(w) * (Ep + E3 + E1 + E2);
                    audit[5] += 1.0;
                    audit[6] += fabs(w);
                }
            }
        }
    }
    if (C64) C64[aidx] += c64;
    if (G64) G64[aidx] += g64;
}

/* Collision deposit for every sampled anchor.  A[slot][x][p] is zeroed and
 * filled with the int64 fixed-point increments of N_s f (scale 2^40),
 * already multiplied by dt (dt/hbar_c in GeV^-1).  C64 / G64 (optional)
 * receive, per anchor, the plain (own-cell, full-weight) FP64 estimate of
 * the increment of N f and of its gain part.  audit (optional, 8 doubles)
 * receives the continuous-leg E/P balance.  flags[0] counts roots dropped
 * for a non-negative regulated denominator, flags[1] quantisation
 * overflows.  Returns 0. */
int bzo_collision(const bzo_config* c, const bzo_run* r, const int64_t* state, const double* m2,
                  int64_t* A, double* C64, double* G64, double* audit, int64_t* flags)
{
    int ns = nslots(c);
    int64_t nxc = n_xcells(c), npc = n_pcells(c);
    int64_t ncell = (int64_t)ns * nxc * npc;
    memset(A, 0, sizeof(int64_t) * (size_t)ncell);
    if (C64) memset(C64, 0, sizeof(double) * (size_t)ncell);
    if (G64) memset(G64, 0, sizeof(double) * (size_t)ncell);
    if (audit) memset(audit, 0, 8 * sizeof(double));
    flags[0] = flags[1] = 0;
    bzo_mconst mk = mconst(c->alpha_s);
    mk.user = c->user;
    mk.umask = c->umask;
    double twoL = 2.0 * c->L;
    double V = twoL * twoL * twoL * twoL * twoL;
    /* weight of one root per leg, in units of 2^-40 of N f:
     * c~ * V/(4N) * dt/hbar_c * 2^40 */
    double Kq = ((V * r->dt) / (4.0 * (double)r->nsamples)) / HBARC * TWO_POW_40;
    bzo_term terms[NSPEC][16];
    int nterms[NSPEC];
    int slot_species[NSPEC];
    for (int s = 0; s < NSPEC; ++s) {
        nterms[s] = terms_for(c, s, terms[s]);
        int sl = slot_of(c, s);
        if (sl >= 0) slot_species[sl] = s;
    }
    int64_t stride = r->anchor_stride > 0 ? r->anchor_stride : 1;
    double audit_acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma omp parallel
    {
        double aud[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t aidx = 0; aidx < ncell; ++aidx) {
            if (aidx % stride != r->anchor_offset) continue;
            int sl = (int)(aidx / (nxc * npc));
            int64_t x = (aidx / npc) % nxc;
            int64_t j = aidx % npc;
            int d = slot_species[sl];
            collide_anchor(c, r, state, m2, d, x, j, aidx, terms[d], nterms[d], &mk, Kq, A, C64,
                           G64, audit ? aud : NULL, flags);
        }
#pragma omp critical
        for (int i = 0; i < 8; ++i) audit_acc[i] += aud[i];
    }
    if (audit)
        for (int i = 0; i < 8; ++i) audit[i] = audit_acc[i];
    return 0;
}

/* ------------------------------------------------------------------ */
/* Drift, Eq. (left handside), flux form, first-order upwind, periodic */
/* in x.  Face flux F_{i+1/2} = c_d n_i if p_d > 0 else c_d n_{i+1},    */
/* with the Courant number c_d = (p_d / E_p(x_up)) dt/dx taken at the   */
/* upwind cell.  On the int64 state the Courant number is evaluated in  */
/* IEEE single precision as (p_d (1/sqrt(p^2 + m^2))) dt/dx (correctly  */
/* rounded sqrt and divide) and held                                    */
/* in 2^-30 fixed point; each face flux round((n c) 2^-30) is an exact  */
/* integer product, computed once and applied with opposite signs to    */
/* the two cells, so the sum of the state is invariant.                 */
/* ------------------------------------------------------------------ */
static double courant(const bzo_config* c, const double* m2, int64_t x, int s, double pd, double pp,
                      double dtdx)
{
    double m = 0.0;
    if (c->mass_mode != 1) m = m2[x * 4 + mass_slot(s)];
    double E = sqrt(pp + m);
    return (pd / E) * dtdx;
}

static int64_t courant_fx(const bzo_config* c, const double* m2, int64_t x, int s, float pdf,
                          float ppf, float dtdxf)
{
    float m = 0.0f;
    if (c->mass_mode != 1) m = (float)m2[x * 4 + mass_slot(s)];
    float inv = 1.0f / sqrtf(ppf + m);
    float cf = (pdf * inv) * dtdxf;
    return llrintf(cf * 1073741824.0f);
}

static int64_t flux_fx(int64_t n, int64_t C)
{
    __int128 prod = (__int128)n * (__int128)C + ((__int128)1 << 29);
    return (int64_t)(prod >> 30);
}

static int64_t xlin(const bzo_config* c, int ix, int iy, int iz)
{
    return ((int64_t)ix * c->nx[1] + iy) * c->nx[2] + iz;
}

/* Force term of Eq. (left handside), -div_p[(grad_x E) f] (Eq. (boltzmann  */
/* equation general form): dp/dt = -grad_x E).  Along p_i a cell moves     */
/* with -dE/dx_i = -(dm^2/dx_i) / (2E); dm^2/dx_i is the central           */
/* difference (m^2(x + e_i) - m^2(x - e_i)) / (2 dx) of the species' mass,  */
/* so with g_i = (m^2(x + e_i) - m^2(x - e_i)) / (4 dx) (FP64, then FP32)   */
/* the Courant number is ((-g_i) (1/E)) dt/dp_i in IEEE single precision,   */
/* held in 2^-30 fixed point like the x fluxes.  Upwind in p (every p cell  */
/* of an x cell moves the same way), and no flux crosses a face of the      */
/* momentum box, so the sum of the state stays exact.                       */
static float force_g(const bzo_config* c, const double* m2, int64_t xl, int64_t xh, int s, double inv4dx)
{
    if (c->mass_mode == 1) return 0.0f;
    return (float)((m2[xh * 4 + mass_slot(s)] - m2[xl * 4 + mass_slot(s)]) * inv4dx);
}

static int64_t force_courant(float g, float inv, float dtdpf)
{
    float cf = ((-g) * inv) * dtdpf;
    return llrintf(cf * 1073741824.0f);
}

int bzo_drift(const bzo_config* c, const int64_t* in, const double* m2, double dt, int64_t* out)
{
    int ns = nslots(c);
    int64_t nxc = n_xcells(c), npc = n_pcells(c);
    float dtdxf = (float)(dt / c->dx);
    double dp[3] = {2.0 * c->L / c->np[0], 2.0 * c->L / c->np[1], 2.0 * c->L / c->np[2]};
    float dtdpf[3] = {(float)(dt / dp[0]), (float)(dt / dp[1]), (float)(dt / dp[2])};
    double inv4dx = 1.0 / (4.0 * c->dx);
    int species[NSPEC];
    for (int s = 0; s < NSPEC; ++s)
        if (slot_of(c, s) >= 0) species[slot_of(c, s)] = s;
#pragma omp parallel for collapse(2)
    for (int sl = 0; sl < ns; ++sl) {
        for (int64_t x = 0; x < nxc; ++x) {
            int s = species[sl];
            int ix = (int)(x / ((int64_t)c->nx[1] * c->nx[2]));
            int iy = (int)((x / c->nx[2]) % c->nx[1]);
            int iz = (int)(x % c->nx[2]);
            int xi[3] = {ix, iy, iz};
            for (int64_t j = 0; j < npc; ++j) {
                int jv[3] = {(int)(j / ((int64_t)c->np[1] * c->np[2])),
                             (int)((j / c->np[2]) % c->np[1]), (int)(j % c->np[2])};
                float pf[3];
                for (int d = 0; d < 3; ++d) pf[d] = (float)(-c->L + ((double)jv[d] + 0.5) * dp[d]);
                float ppf = (pf[0] * pf[0] + pf[1] * pf[1]) + pf[2] * pf[2];
                int64_t nc = in[((int64_t)sl * nxc + x) * npc + j];
                int64_t acc = 0;
                for (int d = 0; d < 3; ++d) {
                    if (c->nx[d] == 1) continue;
                    int lo[3] = {xi[0], xi[1], xi[2]}, hi[3] = {xi[0], xi[1], xi[2]};
                    lo[d] = (xi[d] - 1 + c->nx[d]) % c->nx[d];
                    hi[d] = (xi[d] + 1) % c->nx[d];
                    int64_t xl = xlin(c, lo[0], lo[1], lo[2]), xh = xlin(c, hi[0], hi[1], hi[2]);
                    int64_t fplus, fminus;
                    if (pf[d] > 0.0f) {
                        fplus = flux_fx(nc, courant_fx(c, m2, x, s, pf[d], ppf, dtdxf));
                        fminus = flux_fx(in[((int64_t)sl * nxc + xl) * npc + j],
                                         courant_fx(c, m2, xl, s, pf[d], ppf, dtdxf));
                    } else {
                        fplus = flux_fx(in[((int64_t)sl * nxc + xh) * npc + j],
                                        courant_fx(c, m2, xh, s, pf[d], ppf, dtdxf));
                        fminus = flux_fx(nc, courant_fx(c, m2, x, s, pf[d], ppf, dtdxf));
                    }
                    acc += fplus - fminus;
                }
                if (c->force) {
                    float m = c->mass_mode == 1 ? 0.0f : (float)m2[x * 4 + mass_slot(s)];
                    float inv = 1.0f / sqrtf(ppf + m);
                    for (int i = 0; i < 3; ++i) {
                        if (c->nx[i] == 1) continue;
                        int lo[3] = {xi[0], xi[1], xi[2]}, hi[3] = {xi[0], xi[1], xi[2]};
                        lo[i] = (xi[i] - 1 + c->nx[i]) % c->nx[i];
                        hi[i] = (xi[i] + 1) % c->nx[i];
                        float g = force_g(c, m2, xlin(c, lo[0], lo[1], lo[2]), xlin(c, hi[0], hi[1], hi[2]), s,
                                          inv4dx);
                        int up = (-g) > 0.0f;  /* this x cell's p cells move towards larger p_i */
                        int64_t own = 0, behind = 0;
                        int jo = jv[i] + (up ? 1 : -1), jb = jv[i] + (up ? -1 : 1);
                        if (jo >= 0 && jo < c->np[i]) own = flux_fx(nc, force_courant(g, inv, dtdpf[i]));
                        if (jb >= 0 && jb < c->np[i]) {
                            int jw[3] = {jv[0], jv[1], jv[2]};
                            float pw[3] = {pf[0], pf[1], pf[2]};
                            jw[i] = jb;
                            pw[i] = (float)(-c->L + ((double)jb + 0.5) * dp[i]);
                            float ppw = (pw[0] * pw[0] + pw[1] * pw[1]) + pw[2] * pw[2];
                            float invb = 1.0f / sqrtf(ppw + m);
                            int64_t jbl = ((int64_t)jw[0] * c->np[1] + jw[1]) * c->np[2] + jw[2];
                            behind = flux_fx(in[((int64_t)sl * nxc + x) * npc + jbl], force_courant(g, invb, dtdpf[i]));
                        }
                        acc += up ? own - behind : behind - own;
                    }
                }
                out[((int64_t)sl * nxc + x) * npc + j] = nc - acc;
            }
        }
    }
    return 0;
}

/* Same scheme on an FP64 f state (no rounding of the fluxes); used for the
 * Fourier-mode pin of the scheme itself. */
int bzo_drift_f64(const bzo_config* c, const double* in, const double* m2, double dt, double* out)
{
    int ns = nslots(c);
    int64_t nxc = n_xcells(c), npc = n_pcells(c);
    double dtdx = dt / c->dx;
    double dp[3] = {2.0 * c->L / c->np[0], 2.0 * c->L / c->np[1], 2.0 * c->L / c->np[2]};
    int species[NSPEC];
    for (int s = 0; s < NSPEC; ++s)
        if (slot_of(c, s) >= 0) species[slot_of(c, s)] = s;
    for (int sl = 0; sl < ns; ++sl) {
        for (int64_t x = 0; x < nxc; ++x) {
            int s = species[sl];
            int xi[3] = {(int)(x / ((int64_t)c->nx[1] * c->nx[2])), (int)((x / c->nx[2]) % c->nx[1]),
                         (int)(x % c->nx[2])};
            for (int64_t j = 0; j < npc; ++j) {
                int jv[3] = {(int)(j / ((int64_t)c->np[1] * c->np[2])),
                             (int)((j / c->np[2]) % c->np[1]), (int)(j % c->np[2])};
                double pv[3];
                for (int d = 0; d < 3; ++d) pv[d] = -c->L + ((double)jv[d] + 0.5) * dp[d];
                double pp = (pv[0] * pv[0] + pv[1] * pv[1]) + pv[2] * pv[2];
                double fc = in[((int64_t)sl * nxc + x) * npc + j];
                double acc = 0.0;
                for (int d = 0; d < 3; ++d) {
                    if (c->nx[d] == 1) continue;
                    int lo[3] = {xi[0], xi[1], xi[2]}, hi[3] = {xi[0], xi[1], xi[2]};
                    lo[d] = (xi[d] - 1 + c->nx[d]) % c->nx[d];
                    hi[d] = (xi[d] + 1) % c->nx[d];
                    int64_t xl = xlin(c, lo[0], lo[1], lo[2]), xh = xlin(c, hi[0], hi[1], hi[2]);
                    double fplus, fminus;
                    if (pv[d] > 0.0) {
                        fplus = courant(c, m2, x, s, pv[d], pp, dtdx) * fc;
                        fminus = courant(c, m2, xl, s, pv[d], pp, dtdx)
                                 * in[((int64_t)sl * nxc + xl) * npc + j];
                    } else {
                        fplus = courant(c, m2, xh, s, pv[d], pp, dtdx)
                                * in[((int64_t)sl * nxc + xh) * npc + j];
                        fminus = courant(c, m2, x, s, pv[d], pp, dtdx) * fc;
                    }
                    acc = acc + (fplus - fminus);
                }
                out[((int64_t)sl * nxc + x) * npc + j] = fc - acc;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Moments, Eqs. (particle numbers), (energy momentum tensor): per      */
/* x-cell and active species, out[x][slot][0..4] = (n, eps, T01, T02,   */
/* T03) as densities in GeV^3 / GeV^4.  The sums are exact integer sums */
/* (order independent): the number is sum n; the energy uses E at the   */
/* bin centre in IEEE single precision, sqrt(p^2 + m^2) (|p| in mass     */
/* mode 1), held in 2^-24 fixed point; the momentum uses p_d =          */
/* (2 j_d + 1 - n_d) dp_d / 2.  nsum[slot] = exact sum of the state.    */
/* ------------------------------------------------------------------ */
static double i128_to_double(__int128 v)
{
    return (double)(int64_t)(v >> 64) * 18446744073709551616.0 + (double)(uint64_t)v;
}

int bzo_moments(const bzo_config* c, const int64_t* state, const double* m2, double* out,
                int64_t* nsum)
{
    int ns = nslots(c);
    int64_t nxc = n_xcells(c), npc = n_pcells(c);
    double dp[3] = {2.0 * c->L / c->np[0], 2.0 * c->L / c->np[1], 2.0 * c->L / c->np[2]};
    double twopi = 2.0 * PI;
    double pref = dp[0] * dp[1] * dp[2] / (twopi * twopi * twopi) * TWO_POW_M40;
    int species[NSPEC];
    for (int s = 0; s < NSPEC; ++s)
        if (slot_of(c, s) >= 0) species[slot_of(c, s)] = s;
    for (int sl = 0; sl < ns; ++sl) nsum[sl] = 0;
    for (int64_t x = 0; x < nxc; ++x) {
        for (int sl = 0; sl < ns; ++sl) {
            int s = species[sl];
            float m = c->mass_mode == 1 ? 0.0f : (float)m2[x * 4 + mass_slot(s)];
            __int128 ntot = 0, e = 0, t[3] = {0, 0, 0};
            for (int64_t j = 0; j < npc; ++j) {
                int jv[3] = {(int)(j / ((int64_t)c->np[1] * c->np[2])),
                             (int)((j / c->np[2]) % c->np[1]), (int)(j % c->np[2])};
                float pf[3];
                for (int d = 0; d < 3; ++d) pf[d] = (float)(-c->L + ((double)jv[d] + 0.5) * dp[d]);
                float ppf = (pf[0] * pf[0] + pf[1] * pf[1]) + pf[2] * pf[2];
                int64_t Efx = llrintf(sqrtf(ppf + m) * 16777216.0f);
                int64_t n = state[((int64_t)sl * nxc + x) * npc + j];
                ntot += n;
                e += (__int128)Efx * n;
                for (int d = 0; d < 3; ++d) t[d] += (__int128)(2 * jv[d] + 1 - c->np[d]) * n;
            }
            nsum[sl] += (int64_t)ntot;
            double* o = out + (x * ns + sl) * 5;
            o[0] = i128_to_double(ntot) * pref;
            o[1] = i128_to_double(e) * pref * (1.0 / 16777216.0);
            for (int d = 0; d < 3; ++d) o[2 + d] = i128_to_double(t[d]) * pref * (0.5 * dp[d]);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Source of the kinetic energy-momentum tensor, Eq. (current            */
/* conservation): S_ex^0 = (1/2) sum_a (dm_a^2/dt) I_a with              */
/* I_a = int d^3p/(2pi)^3 N_a f_a / E_a, and the term -(1/4) m_a^2 I_a   */
/* of the modified total energy T_total^00 (single flavour).  Per        */
/* (x cell, slot), out[3] = {I_a, S_ex^0 part (1/2)((m^2 - m^2_prev)/dt) */
/* I_a, -(1/4) m^2 I_a}.  I_a is an exact integer sum of n R with        */
/* R = round(2^24 / E), 1/E = 1/sqrt(p^2 + m^2) in IEEE FP32 at the bin  */
/* centre with the masses m2 (as the drift); with the massless           */
/* dispersion E does not depend on m^2 and both m^2 terms are zero.      */
/* ------------------------------------------------------------------ */
int bzo_energy_source(const bzo_config* c, const int64_t* state, const double* m2, const double* m2_prev, double dt,
                      double* out)
{
    int ns = nslots(c);
    int64_t nxc = n_xcells(c), npc = n_pcells(c);
    double dp[3] = {2.0 * c->L / c->np[0], 2.0 * c->L / c->np[1], 2.0 * c->L / c->np[2]};
    double twopi = 2.0 * PI;
    double pref = dp[0] * dp[1] * dp[2] / (twopi * twopi * twopi) * TWO_POW_M40;
    int species[NSPEC];
    for (int s = 0; s < NSPEC; ++s)
        if (slot_of(c, s) >= 0) species[slot_of(c, s)] = s;
    for (int64_t x = 0; x < nxc; ++x) {
        for (int sl = 0; sl < ns; ++sl) {
            int ms = mass_slot(species[sl]);
            float m = c->mass_mode == 1 ? 0.0f : (float)m2[x * 4 + ms];
            __int128 acc = 0;
            for (int64_t j = 0; j < npc; ++j) {
                int jv[3] = {(int)(j / ((int64_t)c->np[1] * c->np[2])),
                             (int)((j / c->np[2]) % c->np[1]), (int)(j % c->np[2])};
                float pf[3];
                for (int d = 0; d < 3; ++d) pf[d] = (float)(-c->L + ((double)jv[d] + 0.5) * dp[d]);
                float ppf = (pf[0] * pf[0] + pf[1] * pf[1]) + pf[2] * pf[2];
                float inv = 1.0f / sqrtf(ppf + m);
                int64_t R = llrintf(inv * 16777216.0f);
                acc += (__int128)R * state[((int64_t)sl * nxc + x) * npc + j];
            }
            double I = i128_to_double(acc) * pref * (1.0 / 16777216.0);
            double mc = c->mass_mode == 1 ? 0.0 : m2[x * 4 + ms];
            double mp = c->mass_mode == 1 ? 0.0 : m2_prev[x * 4 + ms];
            double* o = out + (x * ns + sl) * 3;
            o[0] = I;
            o[1] = 0.5 * ((mc - mp) / dt) * I;
            o[2] = -0.25 * mc * I;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* One forward-Euler step, all terms from f^n (unsplit):                */
/*   m^2 <- masses(n^n, E from m2_prev);  n^{n+1} = drift(n^n) + A(n^n) */
/* m2 (in/out): previous masses on entry (ignored when first != 0),     */
/* this step's masses on exit (mass mode 2: left as given).             */
/* ------------------------------------------------------------------ */
int bzo_step(const bzo_config* c, const bzo_run* r, const int64_t* in, double* m2, int first,
             int64_t* out, int64_t* flags)
{
    int64_t nxc = n_xcells(c), npc = n_pcells(c);
    int ns = nslots(c);
    int64_t ncell = (int64_t)ns * nxc * npc;
    int rc = 0;
    if (c->mass_mode != 2) {
        double* mnew = (double*)malloc(sizeof(double) * 4 * (size_t)nxc);
        rc = bzo_masses(c, in, first ? NULL : m2, mnew);
        memcpy(m2, mnew, sizeof(double) * 4 * (size_t)nxc);
        free(mnew);
    }
    int64_t* A = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    bzo_collision(c, r, in, m2, A, NULL, NULL, NULL, flags);
    bzo_drift(c, in, m2, r->dt, out);
    for (int64_t i = 0; i < ncell; ++i) out[i] += A[i];
    free(A);
    return rc;
}

int bzo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int bzo_sizeof_config(void) { return (int)sizeof(bzo_config); }
int bzo_sizeof_run(void) { return (int)sizeof(bzo_run); }
