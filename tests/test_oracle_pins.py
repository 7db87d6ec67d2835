"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms, crossing identities of the |M|^2 table,
exact invariants, an independent CM-frame quadrature, and expectation
identities between estimators.  All run on the CPU in seconds.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1912_04457_gb300 import inputs as I

HBARC = 0.1973269804


# ---------------------------------------------------------------------------
# Philox4x32-10 (counter-based stream of the sampler)
# ---------------------------------------------------------------------------
def _kat_rows():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert list(O.philox(ctr, key)) == expect


def test_philox_uniformity_chi2():
    # 64-bin chi^2 of 2^17 words drawn along the sample counter.
    key = [12345, 678]
    words = []
    for i in range(1 << 15):
        words.extend(O.philox([i, 7, 3, 9], key))
    words = np.array(words, dtype=np.uint64)
    counts = np.bincount((words >> np.uint64(26)).astype(np.int64), minlength=64)
    expect = len(words) / 64.0
    chi2 = ((counts - expect) ** 2 / expect).sum()
    # 63 dof: mean 63, sd ~11.2; 5 sd bounds
    assert 63 - 56 < chi2 < 63 + 56


# ---------------------------------------------------------------------------
# |M|^2 table (Appendix): crossing identities of the massless rows
# ---------------------------------------------------------------------------
def _stu(rng, n=50):
    out = []
    for _ in range(n):
        s = rng.uniform(0.1, 10.0)
        c = rng.uniform(-0.99, 0.99)
        t = -0.5 * s * (1 - c)
        out.append((s, t, -s - t))
    return out


def test_msq_crossing_identities():
    rng = np.random.default_rng(0)
    a = 0.3
    for s, t, u in _stu(rng):
        m = lambda cls, S, T, U: O.msq(cls, a, S, T, U, 0.0)
        # q g -> q g  =  - (q qbar -> g g) crossed s <-> t (one fermion crossed)
        assert m(O.M_QG, s, t, u) == pytest.approx(-m(O.M_QQBGG, t, s, u), rel=1e-12)
        # q1 qbar1 -> q1 qbar1 = q1 q1 -> q1 q1 with s <-> u
        assert m(O.M_QQB, s, t, u) == pytest.approx(m(O.M_QQ, u, t, s), rel=1e-12)
        # q1 qbar1 -> q2 qbar2 = q1 q2 -> q1 q2 with s <-> t
        assert m(O.M_QQB2, s, t, u) == pytest.approx(m(O.M_QQP, t, s, u), rel=1e-12)
        # gg -> gg symmetric under all permutations of (s, t, u)
        ref = m(O.M_GG, s, t, u)
        for perm in [(s, u, t), (t, s, u), (t, u, s), (u, s, t), (u, t, s)]:
            assert m(O.M_GG, *perm) == pytest.approx(ref, rel=1e-12)
        # identical-particle rows are t <-> u symmetric
        assert m(O.M_QQ, s, t, u) == pytest.approx(m(O.M_QQ, s, u, t), rel=1e-12)
        assert m(O.M_QQBGG, s, t, u) == pytest.approx(m(O.M_QQBGG, s, u, t), rel=1e-12)
        # all rows are positive in the physical region
        for cls in range(7):
            assert m(cls, s, t, u) > 0


def test_msq_known_values():
    # massless gg -> gg at 90 degrees in the CM frame: s = 1, t = u = -1/2:
    # 16 g^4 dA CA^2 (3 - 2 * (-1/2)/(1/4) - 1/4) = 16 g^4 * 72 * (27/4)
    a = 0.3
    g4 = (4 * math.pi * a) ** 2
    assert O.msq(O.M_GG, a, 1.0, -0.5, -0.5, 0.0) == pytest.approx(16 * g4 * 72 * 6.75, rel=1e-14)
    # q1 q2 -> q1 q2: 8 g^4 (9 * 16/9 / 8) (s^2 + u^2)/t^2 = 16 g^4 (1 + 1/4)/(1/4)
    assert O.msq(O.M_QQP, a, 1.0, -0.5, -0.5, 0.0) == pytest.approx(16 * g4 * 5.0, rel=1e-14)


# ---------------------------------------------------------------------------
# k1z roots and Jacobian, Eqs. (work out delta E), (delta replace)
# ---------------------------------------------------------------------------
def _cm_frame_j2(p, md2, k3, mc2, ma2, mb2, nc=96, nphi=192):
    """Integral of J^2 over the two-body phase space d^3k1/(2E1) d^3k2/(2E2)
    delta^4(k1 + k2 - p - k3), done in the CM frame (|k*| / (4 sqrt s) dOmega*)
    with the lab momenta obtained by a boost; independent of the oracle."""
    Ep = math.sqrt(p @ p + md2)
    E3 = math.sqrt(k3 @ k3 + mc2)
    E = Ep + E3
    P = p + k3
    s = E * E - P @ P
    rs = math.sqrt(s)
    k = math.sqrt((s - ma2 - mb2) ** 2 - 4 * ma2 * mb2) / (2 * rs)
    E1s = math.sqrt(k * k + ma2)
    x, wx = np.polynomial.legendre.leggauss(nc)
    phi = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    n = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1)
    ks = k * n
    beta = P / E
    b = np.linalg.norm(beta)
    bh = beta / b
    g = E / rs
    kb = ks @ bh
    k1 = ks + ((g - 1) * kb + g * E1s * b)[..., None] * bh
    E1 = g * (E1s + b * kb)
    k2 = P - k1
    E2 = E - E1
    J = k1[..., 2] / E1 - k2[..., 2] / E2
    return k / (4 * rs) * (J ** 2 * wx[:, None]).sum() * (2 * math.pi / nphi)


@pytest.mark.parametrize("case", [
    (np.array([0.3, -0.2, 0.5]), 0.15, np.array([-0.4, 0.1, 0.2]), 0.05, 0.1, 0.2),
    (np.array([1.1, 0.4, -0.7]), 0.0, np.array([0.2, -0.9, 0.3]), 0.0, 0.0, 0.0),
    (np.array([-0.2, 0.05, 0.1]), 0.3, np.array([0.6, 0.6, -1.2]), 0.3, 0.13, 0.3),
])
def test_two_body_phase_space_vs_cm_frame(case):
    p, md2, k3, mc2, ma2, mb2 = case
    E = math.sqrt(p @ p + md2) + math.sqrt(k3 @ k3 + mc2)
    lab = O.two_body_sum(p, md2, k3, mc2, ma2, mb2, E + 0.1, 2000, weight_j2=True)
    cm = _cm_frame_j2(p, md2, k3, mc2, ma2, mb2)
    assert lab == pytest.approx(cm, rel=2e-5)


def test_roots_energy_balance_jacobian_and_scan():
    rng = np.random.default_rng(1)
    checked = 0
    for _ in range(300):
        p = rng.uniform(-2, 2, 3)
        k3 = rng.uniform(-2, 2, 3)
        k1x, k1y = rng.uniform(-2, 2, 2)
        ma2, mb2, mc2, md2 = rng.uniform(0, 0.4, 4)
        r = O.roots(p, md2, k3, mc2, k1x, k1y, ma2, mb2)
        Ep = math.sqrt(p @ p + md2)
        E3 = math.sqrt(k3 @ k3 + mc2)
        E = Ep + E3
        P = p + k3
        a2 = k1x ** 2 + k1y ** 2 + ma2
        b2 = (P[0] - k1x) ** 2 + (P[1] - k1y) ** 2 + mb2
        g = lambda z: math.sqrt(a2 + z * z) + math.sqrt(b2 + (P[2] - z) ** 2) - E
        for z, E1, E2, J in r:
            assert abs(E1 + E2 - E) <= 1e-13 * E
            h = 1e-6
            fd = (g(z + h) - g(z - h)) / (2 * h)
            assert J == pytest.approx(fd, rel=1e-6, abs=1e-9)
        # brute-force scan of g(z) over a wide window finds the same number of roots
        zs = np.linspace(-8 * E, 8 * E, 40001)
        gv = np.sqrt(a2 + zs ** 2) + np.sqrt(b2 + (P[2] - zs) ** 2) - E
        changes = int(np.sum(np.sign(gv[1:]) != np.sign(gv[:-1])))
        assert changes == len(r)
        checked += len(r)
    assert checked > 100


# ---------------------------------------------------------------------------
# Thermal masses, Eqs. (mg), (mq): closed forms with E = |p| at mu = 0
#   gluons only:         m_g^2 = g^2 T^2 / 2
#   g + 3 flavours:      m_g^2 = 3/4 g^2 T^2, m_q^2 = g^2 T^2 / 3
#   u, ubar only:        m_g^2 = g^2 T^2 / 12, m_u^2 = g^2 T^2 / 9
# With gluons the cell-centred sum has an O(dp) error from the 1/p^2
# region of f_BE/p; one Richardson step removes it (Fermi-Dirac alone
# converges faster).
# ---------------------------------------------------------------------------
def _mass_state(n, L, mask, T):
    fs = [I.equilibrium_f((n, n, n), L, s, T) for s in I.slots(mask)]
    return I.encode(np.stack(fs).reshape(len(fs), 1, -1), mask)


@pytest.mark.parametrize("mask,expect", [
    (0x01, {0: 0.5}),
    (0x7F, {0: 0.75, 1: 1.0 / 3.0, 2: 1.0 / 3.0, 3: 1.0 / 3.0}),
    (0x12, {0: 1.0 / 12.0, 1: 1.0 / 9.0}),
])
def test_thermal_mass_closed_form(mask, expect):
    T, a, L = 0.5, 0.3, 4.0
    g2 = 4 * math.pi * a
    res = {}
    for n in (32, 64):
        cfg = O.make_config(np_=(n, n, n), L=L, species_mask=mask, alpha_s=a)
        res[n] = O.masses(cfg, _mass_state(n, L, mask, T))[0]
    for slot, coef in expect.items():
        exact = coef * g2 * T * T
        e32 = res[32][slot] / exact - 1
        e64 = res[64][slot] / exact - 1
        assert abs(e64) < abs(e32)
        if mask & 1:
            assert 1.7 < e32 / e64 < 2.3       # Bose-Einstein 1/p^2 region: first order in dp
        rich = 2 * res[64][slot] - res[32][slot]
        assert rich / exact - 1 == pytest.approx(0.0, abs=0.01)


def test_mass_uses_previous_dispersion():
    # With E = sqrt(p^2 + m^2) the integrals shrink; zero previous masses
    # reproduce the first-step (E = |p|) result bit for bit.
    n, L = 16, 2.0
    w = I.gluon_step_box(n=n, L=L)
    cfg = O.make_config(np_=w.np_, L=L, species_mask=w.species_mask)
    m0 = O.masses(cfg, w.state())
    mz = O.masses(cfg, w.state(), np.zeros((1, 4)))
    assert np.array_equal(m0, mz)
    m1 = O.masses(cfg, w.state(), m0)
    assert m1[0, 0] < m0[0, 0]


# ---------------------------------------------------------------------------
# Equilibrium: C vanishes for Bose-Einstein / Fermi-Dirac f (detailed
# balance) when f is taken at the continuous leg momenta.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mask,mass_mode", [(0x01, 0), (0x7F, 0), (0x7F, 1), (0x09, 0)])
def test_equilibrium_collision_vanishes(mask, mass_mode):
    n, L, T = 8, 2.0, 0.5
    fs = [I.equilibrium_f((n, n, n), L, s, T) for s in I.slots(mask)]
    st = I.encode(np.stack(fs).reshape(len(fs), 1, -1), mask)
    cfg = O.make_config(np_=(n, n, n), L=L, species_mask=mask, alpha_s=0.3,
                        mass_mode=mass_mode, analytic=True, T=T)
    m2 = O.masses(cfg, st)
    r = O.collision(cfg, st, m2, 64, want_c64=True)
    C, G = r["C64"], r["G64"]
    assert (G > 0).sum() > 0.5 * G.size
    ratio = np.abs(C[G > 0]) / G[G > 0]
    assert ratio.max() < 1e-12
    # the quantised increments vanish up to the rounding of cancelled terms
    assert np.abs(r["A"]).max() <= 4 * 10 * 64 * 2


def test_nonequilibrium_collision_does_not_vanish():
    # same grid, f on the grid (CGC step): |C|/gain is O(1)
    w = I.gluon_step_box(n=8)
    cfg = O.make_config(np_=w.np_, L=w.L, species_mask=1)
    m2 = O.masses(cfg, w.state())
    r = O.collision(cfg, w.state(), m2, 64, want_c64=True)
    G = r["G64"]
    assert (np.abs(r["C64"][G > 0]) / G[G > 0]).max() > 0.1


# ---------------------------------------------------------------------------
# Number conservation (Sec. III.B): sum of A is exactly zero with symmetrical
# sampling and not without it.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mask", [0x01, 0x7F])
def test_number_conservation_exact(mask):
    n, L = 10, 2.0
    rng = np.random.default_rng(5)
    f = rng.uniform(0, 0.5, size=(bin(mask).count("1"), 1, n ** 3))
    st = I.encode(f, mask)
    cfg = O.make_config(np_=(n, n, n), L=L, species_mask=mask)
    m2 = O.masses(cfg, st)
    sym = O.collision(cfg, st, m2, 16)["A"]
    assert int(sym.sum()) == 0
    assert np.abs(sym).sum() > 0
    plain = O.collision(cfg, st, m2, 16, sampler=O.PLAIN)["A"]
    assert int(plain.sum()) != 0


def test_number_conserved_over_steps_with_drift():
    # inhomogeneous 4^3 x 6^3 gluon box, 5 steps of drift + collisions
    w = I.gluon_bump_xp(nxs=4, dx=0.2, n=6, L=2.0)
    cfg = O.make_config(nx=w.nx, dx=w.dx, np_=w.np_, L=w.L, species_mask=1)
    st = w.state()
    total = int(st.sum())
    m2 = None
    for k in range(5):
        st, m2, flags = O.step(cfg, st, m2, k == 0, 8, k, 0.02)
        assert int(st.sum()) == total


# ---------------------------------------------------------------------------
# Energy / momentum: each deposit set balances at the continuous leg
# momenta to rounding; on the bin centres the imbalance obeys
# |dE| <= 4 (sqrt(3)/2) dp sum|w| since |grad E| <= 1.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mask", [0x01, 0x7F])
def test_energy_momentum_audit(mask):
    n, L = 10, 2.0
    rng = np.random.default_rng(9)
    f = rng.uniform(0, 0.5, size=(bin(mask).count("1"), 1, n ** 3))
    st = I.encode(f, mask)
    cfg = O.make_config(np_=(n, n, n), L=L, species_mask=mask, mass_mode=2)
    m2 = np.array([[0.3, 0.1, 0.1, 0.1]])
    r = O.collision(cfg, st, m2, 16, want_audit=True)
    a = r["audit"]
    assert a[5] > 1000
    for i in range(4):
        assert abs(a[i]) <= 1e-12 * a[4]
    # bin-centre audit
    A = r["A"][:, 0, :].astype(np.float64)
    pc = I.momentum_centres((n, n, n), L)
    dE = 0.0
    for sl, s in enumerate(I.slots(mask)):
        msq = m2[0, 0] if s == 0 else m2[0, 1 + (s - 1) % 3]
        dE += (np.sqrt((pc * pc).sum(1) + msq) * A[sl]).sum()
    dp = 2 * L / n
    bound = 4 * (math.sqrt(3) / 2) * dp * a[6] + 4 * 0.5 * a[5] * 2 * math.sqrt(3) * L
    assert abs(dE) <= bound
    assert abs(dE) > 0  # binning does break it (Sec. IV.C)


def test_energy_binning_error_shrinks_with_grid():
    # Fig. 5 trend: the bin-centre energy change relative to the gross
    # energy throughput falls as the grid is refined.
    rel = []
    for n in (8, 16):
        L = 2.0
        st = I.encode(I.step_f((n, n, n), L, 0.5, 1.5).reshape(1, 1, -1), 1)
        cfg = O.make_config(np_=(n, n, n), L=L, species_mask=1, mass_mode=2)
        m2 = np.array([[0.5, 0, 0, 0]])
        A = O.collision(cfg, st, m2, 64)["A"][0, 0].astype(np.float64)
        pc = I.momentum_centres((n, n, n), L)
        E = np.sqrt((pc * pc).sum(1) + 0.5)
        rel.append(abs((E * A).sum()) / (E * np.abs(A)).sum())
    assert rel[1] < rel[0]


# ---------------------------------------------------------------------------
# Symmetrical sampling is unbiased: E[A_symmetric] = E[A_plain] (plain = the
# usual MC, own cell only with the full weight), over independent seeds.
# A wrong leg weight (e.g. 1/2 instead of 1/4) or a wrong sign fails this.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mask", [0x01, 0x7F])
def test_symmetric_equals_plain_in_expectation(mask):
    n, L, N = 6, 2.0, 256
    ns = bin(mask).count("1")
    f = np.stack([I.step_f((n, n, n), L, 0.5, 1.2) if s == 0 else I.exp_f((n, n, n), L, 0.2, 0.4)
                  for s in I.slots(mask)]).reshape(ns, 1, -1)
    st = I.encode(f, mask)
    seeds = range(1, 61)
    pc = I.momentum_centres((n, n, n), L)
    shell = np.minimum((np.sqrt((pc * pc).sum(1)) / (L * math.sqrt(3)) * 4).astype(int), 3)
    def agg(A):
        return np.array([[A[sl, 0, shell == k].sum() for k in range(4)] for sl in range(ns)])
    sy, pl = [], []
    for sd in seeds:
        cfg = O.make_config(np_=(n, n, n), L=L, species_mask=mask, seed=sd)
        m2 = O.masses(cfg, st)
        sy.append(agg(O.collision(cfg, st, m2, N)["A"].astype(np.float64)))
        pl.append(agg(O.collision(cfg, st, m2, N, sampler=O.PLAIN)["A"].astype(np.float64)))
    sy, pl = np.array(sy), np.array(pl)
    diff = sy.mean(0) - pl.mean(0)
    err = np.sqrt(sy.var(0, ddof=1) / len(seeds) + pl.var(0, ddof=1) / len(seeds))
    live = err > 0
    assert np.array_equal(diff[~live], np.zeros_like(diff[~live]))
    z = diff[live] / err[live]
    assert np.abs(z).max() < 5.0
    # the signal is far above the noise, so a wrong leg weight (which scales
    # the symmetric mean) would fail the z test above
    assert (np.abs(pl.mean(0))[live] / err[live]).max() > 8


# ---------------------------------------------------------------------------
# Drift, Eq. (left handside) in flux form, first-order upwind, periodic
# ---------------------------------------------------------------------------
def test_drift_fourier_amplification():
    nxs, n, L, dx, dt = 16, 4, 2.0, 0.1, 0.03
    cfg = O.make_config(nx=(nxs, nxs, 1), dx=dx, np_=(n, n, n), L=L, species_mask=1, mass_mode=2)
    m2 = np.full((nxs * nxs, 4), 0.2)
    xc = I.space_centres((nxs, nxs, 1), dx)
    kx, ky = 2 * math.pi * 3 / (nxs * dx), 2 * math.pi * 5 / (nxs * dx)
    phase = kx * xc[:, 0] + ky * xc[:, 1]
    f0 = (1.0 + 0.1 * np.cos(phase))[:, None] * np.ones((1, n ** 3))
    f1 = O.drift_f64(cfg, f0.reshape(1, nxs * nxs, -1), m2, dt)[0]
    pc = I.momentum_centres((n, n, n), L)
    for j in range(n ** 3):
        p = pc[j]
        E = math.sqrt(p @ p + 0.2)
        g = 1.0 + 0j
        for d, k in ((0, kx), (1, ky)):
            c = p[d] / E * dt / dx
            g -= abs(c) * (1 - np.exp(-1j * np.sign(p[d]) * k * dx))
        expect = 1.0 + 0.1 * np.real(g * np.exp(1j * phase))
        assert np.abs(f1[:, j] - expect).max() < 1e-13


def test_drift_exact_shift_at_unit_courant():
    # massless, p along x (n_py = n_pz = 1 puts p_y = p_z = 0), dt = dx: shift by one cell
    nxs, dx = 8, 0.25
    cfg = O.make_config(nx=(nxs, 1, 1), dx=dx, np_=(2, 1, 1), L=1.0, species_mask=1, mass_mode=1)
    rng = np.random.default_rng(3)
    st = rng.integers(0, 1 << 44, size=(1, nxs, 2)).astype(np.int64)
    out = O.drift(cfg, st, np.zeros((nxs, 4)), dx)
    assert np.array_equal(out[0, :, 1], np.roll(st[0, :, 1], 1))   # p_x > 0 moves +x
    assert np.array_equal(out[0, :, 0], np.roll(st[0, :, 0], -1))  # p_x < 0 moves -x


def test_drift_conserves_exactly_with_x_dependent_mass():
    nxs, n = 6, 6
    cfg = O.make_config(nx=(nxs, nxs, nxs), dx=0.2, np_=(n, n, n), L=2.0, species_mask=0x03,
                        mass_mode=2)
    rng = np.random.default_rng(4)
    st = rng.integers(0, 1 << 43, size=(2, nxs ** 3, n ** 3)).astype(np.int64)
    m2 = rng.uniform(0.0, 0.5, size=(nxs ** 3, 4))
    out = O.drift(cfg, st, m2, 0.05)
    assert out[0].sum() == st[0].sum() and out[1].sum() == st[1].sum()
    assert not np.array_equal(out, st)


def test_drift_first_order_convergence():
    # smooth 1-D profile advected at v = p/E; error vs f(x - vt) halves with dx
    errs = []
    for nxs in (32, 64):
        dx = 3.2 / nxs
        cfg = O.make_config(nx=(nxs, 1, 1), dx=dx, np_=(2, 1, 1), L=1.0, species_mask=1,
                            mass_mode=2)
        m2 = np.full((nxs, 4), 0.3)
        xc = I.space_centres((nxs, 1, 1), dx)[:, 0]
        f = np.stack([np.exp(np.sin(2 * math.pi * xc / 3.2))] * 2, 1).reshape(1, nxs, 2)
        dt = 0.4 * dx
        steps = int(round(0.8 / dt))
        for _ in range(steps):
            f = O.drift_f64(cfg, f, m2, dt)
        v = 0.5 / math.sqrt(0.25 + 0.3)
        exact = np.exp(np.sin(2 * math.pi * (xc - v * steps * dt) / 3.2))
        errs.append(np.abs(f[0, :, 1] - exact).max())
    assert 1.6 < errs[0] / errs[1] < 2.4


# ---------------------------------------------------------------------------
# Moments, Eqs. (particle numbers), (energy momentum tensor)
#   Bose-Einstein, mu = 0, massless: n = N_g zeta(3) T^3 / pi^2, eps = N_g pi^2 T^4 / 30
# ---------------------------------------------------------------------------
def test_moments_closed_form():
    T, L = 0.5, 8.0
    zeta3 = 1.2020569031595942
    n_exact = 16 * zeta3 * T ** 3 / math.pi ** 2
    e_exact = 16 * math.pi ** 2 * T ** 4 / 30
    num, en = [], []
    for n in (32, 64):
        st = I.encode(I.equilibrium_f((n, n, n), L, 0, T).reshape(1, 1, -1), 1)
        cfg = O.make_config(np_=(n, n, n), L=L, species_mask=1, mass_mode=1)
        mom, nsum = O.moments(cfg, st, np.zeros((1, 4)))
        num.append(mom[0, 0, 0])
        en.append(mom[0, 0, 1])
        assert np.abs(mom[0, 0, 2:]).max() < 1e-12 * mom[0, 0, 1]
        assert nsum[0] == st.sum()
    # the number sum converges at second order in dp; Richardson removes it
    e32, e64 = num[0] / n_exact - 1, num[1] / n_exact - 1
    assert 3.0 < e32 / e64 < 5.0
    assert (4 * num[1] - num[0]) / 3 / n_exact - 1 == pytest.approx(0.0, abs=1e-3)
    assert en[1] / e_exact - 1 == pytest.approx(0.0, abs=2e-4)
