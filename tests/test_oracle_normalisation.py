"""Pin of the absolute normalisation of the oracle's Monte Carlo estimator,
Eqs. (C_a_b), (MC C_gg), (ca), against a closed form.

Setup: gluons, u and ubar on the massless dispersion (E = |k|), f at every leg
the equilibrium value at the leg's continuous momentum (Eqs. (fg), (fq)) with
T = 0.15 GeV, one species set at chemical potential -8 T ("hot") and the other
at -20 T ("cold"), and a user |M|^2 table whose q_a qbar_a <-> g g row is the
constant M0 and whose other rows are 0.  In the Boltzmann limit of the hot
legs (f = e^{(mu - E)/T}, F = 1 +- f -> 1), the statistical factor of that
term depends on k3 only, through energy conservation E1 + E2 = E3 + Ep, and
Eq. (C_a_b) factorises:

  the two-body phase space of (k1, k2) at fixed P = k3 + p,
    int d^3k1/((2pi)^3 2E1) d^3k2/((2pi)^3 2E2) (2pi)^4 delta^4(k1 + k2 - P) = 1/(8 pi)
  for massless legs, and
    int d^3k3/((2pi)^3 2E3) e^{-E3/T} = T^2/(4 pi^2),

so per unit time (dt/hbar_c) the anchor's increment of N f is
    C(p) = sym M0 e^{(2 mu_hot - Ep)/T} T^2 / (64 pi^3 Ep)
with the sign of gain (+) or loss (-).  Quarks hot: the gluon equation's
q qbar -> g g term is a gain (sym 1).  Gluons hot: it is a loss for the gluon
anchor (sym 1) and the quark equations' 1/2 g g -> q qbar term is a gain
(sym 1/2); quarks hot, that term is a loss of the quark anchors.  Corrections: Fermi-Dirac/Bose-Einstein beyond the Boltzmann limit
<= 2 e^{-8} relative, the cold legs e^{-12} relative.

The integrand is concentrated at |k3| <~ a few T, while the estimator draws
(k1_perp, k3) uniformly from the whole box, so the test feeds the oracle
explicit points: uniform in shells r0 <= |k3| < r1 with |k1_perp| <= Ep +
|k3| (every root has |k1_perp| <= |k1| <= E1 <= Ep + E3 for massless legs, so
these regions hold every root of their k3), their sizes chosen by the weight
of each shell.  For points uniform in a region B of volume |B|, the
estimator V/N sum c~ has the expectation (V/|B|) int_B c~, so the integral is
recovered as sum over shells of C64 |B|/V, and the k3 integral is cut at
|k3| = 10 T: the factor 1 - e^{-10} 11 is applied.  The anchors are the eight
centre cells of a 16^3 grid on [-2, 2) GeV (|p| = sqrt(3) dp/2, p at the
cell centre), whose shells lie inside the momentum box, so no root is
rejected by the box.  A mistake of (2 pi)^6 for (2 pi)^5, a dropped
1/(2 Ep), V/(2N) for V/N or dt hbar_c for dt/hbar_c changes the ratio by a
factor of 2 or more; the measured spread of the ratio over point sets is
0.3%.
"""
import numpy as np
import pytest

import oracle as O

HBARC = 0.1973269804
N_GRID, L = 16, 2.0


def _shell_points(rng, n, Ep, r0, r1):
    """n points uniform in {r0 <= |k3| < r1, |k1_perp| <= Ep + |k3|} as the
    oracle's explicit uniforms (p jitter unused: p at the cell centre)."""
    h1 = Ep + r1
    pts = np.zeros((0, 5))
    while pts.shape[0] < n:
        k3 = rng.uniform(-r1, r1, size=(4 * n, 3))
        k1 = rng.uniform(-h1, h1, size=(4 * n, 2))
        r3 = np.sqrt((k3 ** 2).sum(1))
        ok = (r3 >= r0) & (r3 < r1) & (np.sqrt((k1 ** 2).sum(1)) <= Ep + r3)
        pts = np.concatenate([pts, np.concatenate([k1[ok], k3[ok]], 1)])
    u = np.full((n, 8), 0.5)
    u[:, 3:8] = (pts[:n] + L) / (2 * L)
    return u


def _shell_volume(Ep, r0, r1):
    """|B| = int_{r0 <= |k3| < r1} pi (Ep + |k3|)^2 d^3k3."""
    F = lambda R: Ep ** 2 * R ** 3 / 3 + Ep * R ** 4 / 2 + R ** 5 / 5
    return 4 * np.pi ** 2 * (F(r1) - F(r0))


def _integral(T, hot, seed, N=1 << 19, M0=1e9):
    """Per slot (g, u, ubar): the oracle's plain estimate summed over the 8
    centre anchors and the k3 shells, in units of dt/hbar_c, with the
    closed form of each and the deposits of the int64 plain estimator."""
    mu = [0.0] * 7
    hot_mu, cold_mu = -8 * T, -20 * T
    mu[0] = hot_mu if hot == "g" else cold_mu
    mu[1] = mu[4] = hot_mu if hot == "q" else cold_mu
    zero = [(0.0, (0, 0, 0, 0, 0, 0))]
    rows = {r: zero for r in range(7)}
    rows[O.M_QQBGG] = [(M0, (0, 0, 0, 0, 0, 0))]
    n = N_GRID
    cfg = O.make_config(np_=(n, n, n), L=L, seed=seed, species_mask=0x13, alpha_s=0.3, mass_mode=2,
                        analytic=True, T=T, mu=mu, user_rows=rows)
    npc = n ** 3
    st = np.zeros(3 * npc, dtype=np.int64)
    m2 = np.zeros((1, 4))          # fixed masses 0: E = |k|, regulator 0
    dt = 0.01
    dp = 2 * L / n
    Ep = np.sqrt(3.0) * dp / 2
    c = n // 2
    anchors = [((c - 1 + a) * n + (c - 1 + b)) * n + (c - 1 + e) for a in (0, 1) for b in (0, 1) for e in (0, 1)]
    edges = np.array([0, .5, 1, 1.5, 2, 2.5, 3, 4, 5, 6, 8, 10]) * T
    G = lambda R: -np.exp(-R / T) * T * (R + T)                  # int k e^{-k/T} dk
    w = np.array([G(b) - G(a) for a, b in zip(edges[:-1], edges[1:])])
    counts = np.maximum(4096, (N * w / w.sum()).astype(int))
    V = (2 * L) ** 5
    rng = np.random.default_rng(seed)
    est = np.zeros(3)
    dev_A = 0.0
    for (r0, r1), k in zip(zip(edges[:-1], edges[1:]), counts):
        u = _shell_points(rng, int(k), Ep, r0, r1)
        vol = _shell_volume(Ep, r0, r1)
        for j in anchors:
            r = O.collision(cfg, st, m2, int(k), step=0, dt=dt, sampler=O.PLAIN, p_center=True, want_c64=True,
                            anchor_stride=npc, anchor_offset=j, u_explicit=u, u_shared=True)
            for sl in range(3):
                est[sl] += r["C64"][sl, 0, j] / (dt / HBARC) * vol / V
                # the int64 plain deposit is the same weight, quantised per root
                dev_A = max(dev_A, abs(r["A"][sl, 0, j] / 2.0 ** 40 - r["C64"][sl, 0, j]) /
                            max(abs(r["C64"][sl, 0, j]), 1e-300))
    cut = 1 - np.exp(-10.0) * 11.0
    base = M0 * np.exp((2 * hot_mu - Ep) / T) * T ** 2 / (64 * np.pi ** 3 * Ep) * cut * len(anchors)
    if hot == "q":   # gain of the gluon anchor; loss of the quark anchors' 1/2 g g <-> q qbar
        expect = np.array([base, -0.5 * base, -0.5 * base])
    else:            # loss of the gluon anchor; gain of the quark anchors
        expect = np.array([-base, 0.5 * base, 0.5 * base])
    return est, expect, dev_A


@pytest.mark.parametrize("T", [0.15, 0.1])
def test_gain_of_q_qbar_to_g_g_equals_the_closed_form(T):
    est, expect, dev_A = _integral(T, "q", seed=11)
    assert est[0] > 0
    assert est[0] / expect[0] == pytest.approx(1.0, abs=0.02)       # gain of the gluon anchor, sym 1
    assert est[1] / expect[1] == pytest.approx(1.0, abs=0.02)       # loss of u: 1/2 g g <-> u ubar
    assert est[2] / expect[2] == pytest.approx(1.0, abs=0.02)
    assert dev_A < 1e-4


def test_loss_term_and_the_half_of_g_g_to_q_qbar():
    est, expect, dev_A = _integral(0.15, "g", seed=12)
    assert est[0] < 0
    assert est[0] / expect[0] == pytest.approx(1.0, abs=0.02)       # loss of the gluon anchor, sym 1
    assert est[1] / expect[1] == pytest.approx(1.0, abs=0.02)       # gain of u: 1/2 g g -> u ubar
    assert est[2] / expect[2] == pytest.approx(1.0, abs=0.02)       # gain of ubar
    assert dev_A < 1e-4
