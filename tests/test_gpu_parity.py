"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: int64 deposits, masses, drifted states and moments of the FP64 path
are bit-identical to the oracle's; the FP32 integrand path is within 2e-5
relative L2 of the oracle evaluated on the same (23-bit) uniforms; the sum
of every symmetric deposit is exactly zero.
"""
import numpy as np
import pytest

import oracle as O
from paper_1912_04457_gb300 import inputs as I

pytestmark = pytest.mark.gpu

F32_TOL = 2e-5


def torch_mod():
    import torch
    return torch


def make_pair(nx=(1, 1, 1), dx=1.0, np_=(8, 8, 8), L=2.0, seed=1, mask=1, alpha=0.3, mass_mode=0):
    from paper_1912_04457_gb300 import bz
    h = bz.Handle(nx=nx, dx=dx, np_=np_, L=L, seed=seed, species_mask=mask, alpha_s=alpha,
                  mass_mode=mass_mode)
    cfg = O.make_config(nx=nx, dx=dx, np_=np_, L=L, seed=seed, species_mask=mask, alpha_s=alpha,
                        mass_mode=mass_mode)
    return h, cfg


def random_state(mask, nxc, np_, seed, lo=0.0, hi=0.6):
    ns = bin(mask).count("1")
    f = I.random_f(np_, ns, nxc, seed, lo, hi)
    return I.encode(f, mask)


def to_dev(a):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_l2(a, b):
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


COLLISION_CASES = [
    # name, np, mask, N, mass_mode, sampler
    ("gluon_8cube_N64", (8, 8, 8), 0x01, 64, 0, 0),
    ("gluon_ragged_N48", (6, 10, 8), 0x01, 48, 0, 0),
    ("qgp7_6cube_N32", (6, 6, 6), 0x7F, 32, 0, 0),
    ("g_u_ubar_N1", (8, 8, 8), 0x13, 1, 0, 0),
    ("qgp7_massless_N32", (6, 6, 6), 0x7F, 32, 1, 0),
    ("gluon_plain_N64", (8, 8, 8), 0x01, 64, 0, 1),
    ("qgp7_plain_N33", (6, 6, 6), 0x7F, 33, 0, 1),
]


@pytest.mark.parametrize("name,np_,mask,N,mass_mode,sampler", COLLISION_CASES)
def test_collision_f64_bit_exact(name, np_, mask, N, mass_mode, sampler):
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    h, cfg = make_pair(np_=np_, mask=mask, mass_mode=mass_mode, seed=7)
    st = random_state(mask, 1, np_, 11)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    dt, step = 0.01, 3
    h.collision_term(to_dev(st), A, N, step, dt, bz.PREC_F64, sampler)
    m_gpu = h.get_masses()
    m2 = O.masses(cfg, st)
    assert np.array_equal(m_gpu, m2)
    ref = O.collision(cfg, st, m2, N, step=step, dt=dt, sampler=sampler)
    got = A.cpu().numpy().reshape(ref["A"].shape)
    assert np.array_equal(got, ref["A"])
    assert np.abs(got).sum() > 0
    if sampler == 0:
        assert int(got.sum()) == 0
    assert np.array_equal(h.flags()[:2], ref["flags"])


@pytest.mark.parametrize("mask,mass_mode,sampler", [(0x01, 0, 0), (0x7F, 0, 0), (0x7F, 1, 1)])
def test_collision_audit_matches_oracle(mask, mass_mode, sampler):
    """bz_collision_audit: the same int64 deposits as the oracle, its continuous-leg
    energy / momentum balance (zero to rounding against the |w| E scale), the root
    count exactly, the other sums to FP64 summation-order rounding, and sum A = 0
    for the symmetric sampler."""
    torch = torch_mod()
    np_ = (8, 8, 8)
    h, cfg = make_pair(np_=np_, mask=mask, mass_mode=mass_mode, seed=5)
    st = random_state(mask, 1, np_, 21)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    N, step, dt = 48, 2, 0.01
    aud = h.collision_audit(to_dev(st), A, N, step, dt, sampler)
    ref = O.collision(cfg, st, O.masses(cfg, st), N, step=step, dt=dt, sampler=sampler, want_audit=True)
    assert np.array_equal(A.cpu().numpy().reshape(ref["A"].shape), ref["A"])
    ra = ref["audit"]
    assert aud[5] == ra[5] and aud[5] > 0
    for k in (4, 6):
        assert aud[k] == pytest.approx(ra[k], rel=1e-12)
    for k in range(4):
        assert abs(aud[k]) <= 1e-12 * aud[4] and abs(aud[k] - ra[k]) <= 1e-12 * aud[4]
    if sampler == 0:
        assert aud[7] == 0.0
    else:
        assert aud[7] == float(ref["A"].sum()) and aud[7] != 0.0


def test_f64_path_on_23_bit_uniforms():
    """With bz_set_uniform_bits(23) the FP64 path evaluates the FP32 path's sample
    points: bit-identical to the oracle at ubits = 23, and the FP32 path within
    the FP32 tolerance of it."""
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    np_, mask, N = (8, 8, 8), 0x7F, 48
    h, cfg = make_pair(np_=np_, mask=mask, seed=13)
    st = random_state(mask, 1, np_, 17)
    A64 = torch.empty(st.size, dtype=torch.int64, device="cuda")
    A32 = torch.empty_like(A64)
    h.set_uniform_bits(23)
    h.collision_term(to_dev(st), A64, N, 4, 0.01, bz.PREC_F64)
    h.reset_masses()
    h.collision_term(to_dev(st), A32, N, 4, 0.01, bz.PREC_F32)
    ref = O.collision(cfg, st, O.masses(cfg, st), N, step=4, dt=0.01, ubits=23)["A"]
    assert np.array_equal(A64.cpu().numpy().reshape(ref.shape), ref)
    assert rel_l2(A32.cpu().numpy(), A64.cpu().numpy()) <= F32_TOL
    with pytest.raises(bz.BzError):
        h.set_uniform_bits(24)


def test_second_call_uses_previous_dispersion():
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    h, cfg = make_pair(np_=(6, 6, 6), mask=0x7F)
    st = random_state(0x7F, 1, (6, 6, 6), 5)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    h.collision_term(to_dev(st), A, 32, 0, 0.01, bz.PREC_F64)
    m_first = O.masses(cfg, st)
    h.collision_term(to_dev(st), A, 32, 1, 0.01, bz.PREC_F64)
    m_second = O.masses(cfg, st, m_first)
    assert np.array_equal(h.get_masses(), m_second)
    ref = O.collision(cfg, st, m_second, 32, step=1, dt=0.01)
    assert np.array_equal(A.cpu().numpy().reshape(ref["A"].shape), ref["A"])


def test_fixed_masses_and_anchor_subset():
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    h, cfg = make_pair(np_=(8, 8, 8), mask=0x0F, mass_mode=2)
    m2 = np.array([[0.31, 0.12, 0.14, 0.16]])
    h.set_masses(m2)
    h.set_anchor_subset(7, 3)
    st = random_state(0x0F, 1, (8, 8, 8), 6)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    h.collision_term(to_dev(st), A, 64, 2, 0.02, bz.PREC_F64)
    ref = O.collision(cfg, st, m2, 64, step=2, dt=0.02, anchor_stride=7, anchor_offset=3)
    assert np.array_equal(A.cpu().numpy().reshape(ref["A"].shape), ref["A"])
    assert np.array_equal(h.get_masses(), m2)


@pytest.mark.parametrize("np_,mask,N", [((12, 12, 12), 0x01, 64), ((8, 8, 8), 0x7F, 64),
                                        ((10, 6, 8), 0x13, 40)])
def test_collision_f32_within_tolerance(np_, mask, N):
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    h, cfg = make_pair(np_=np_, mask=mask, seed=3)
    st = random_state(mask, 1, np_, 12, 0.05, 0.5)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    h.collision_term(to_dev(st), A, N, 1, 0.01, bz.PREC_F32)
    m2 = O.masses(cfg, st)
    ref = O.collision(cfg, st, m2, N, step=1, dt=0.01, ubits=23)["A"]
    got = A.cpu().numpy().reshape(ref.shape)
    assert int(got.sum()) == 0
    assert rel_l2(got, ref) <= F32_TOL


@pytest.mark.parametrize("mask,N", [(0x7F, 48), (0x13, 40)])
def test_collision_f32_massless_one_group(mask, N):
    """With the massless dispersion every term of an equation has the same
    kinematics, so all of them (up to ten) form one group and ride on each
    root that phase B evaluates."""
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    np_ = (8, 8, 8)
    h, cfg = make_pair(np_=np_, mask=mask, seed=4, mass_mode=1)
    st = random_state(mask, 1, np_, 13, 0.05, 0.5)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    h.collision_term(to_dev(st), A, N, 2, 0.01, bz.PREC_F32)
    m2 = O.masses(cfg, st)
    ref = O.collision(cfg, st, m2, N, step=2, dt=0.01, ubits=23)["A"]
    got = A.cpu().numpy().reshape(ref.shape)
    assert int(got.sum()) == 0
    assert rel_l2(got, ref) <= F32_TOL
    assert np.count_nonzero(ref) > 0


def test_equilibrium_vanishes_on_gpu():
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    np_ = (8, 8, 8)
    h, cfg = make_pair(np_=np_, mask=0x7F)
    fs = [I.equilibrium_f(np_, 2.0, s, 0.5) for s in I.slots(0x7F)]
    st = I.encode(np.stack(fs).reshape(7, 1, -1), 0x7F)
    h.set_equilibrium(True, 0.5)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    h.collision_term(to_dev(st), A, 64, 0, 0.01, bz.PREC_F64)
    h.set_equilibrium(False)
    B = torch.empty_like(A)
    h.reset_masses()
    h.collision_term(to_dev(st), B, 64, 0, 0.01, bz.PREC_F64)
    eq = np.abs(A.cpu().numpy()).max()
    off = np.abs(B.cpu().numpy()).max()   # on the grid the residual is O(dp), not zero
    assert eq <= 4 * 64 * 10
    assert off > 1000 * max(eq, 1)


DRIFT_CASES = [
    # nx, np, mask, dt (dx = 0.2), f range
    ((4, 3, 5), (6, 6, 6), 0x03, 0.05, (0.0, 0.6)),
    ((1, 4, 1), (5, 6, 4), 0x01, 0.3, (-0.2, 0.6)),     # y only, odd np_x (p_x = 0 cells)
    ((3, 1, 1), (4, 4, 4), 0x01, 0.1, (0.0, 0.6)),      # x only
    ((1, 1, 5), (6, 5, 4), 0x01, 0.2, (-0.2, 0.6)),     # z only, |c| up to 1
    ((2, 5, 3), (4, 6, 4), 0x11, 0.39, (-0.2, 0.6)),    # dt/dx = 1.95, narrow integer form
    ((2, 3, 2), (4, 4, 4), 0x01, 0.45, (0.0, 0.6)),     # dt/dx = 2.25, wide (128-bit) form
    ((1, 2, 41), (4, 4, 4), 0x01, 0.05, (0.0, 0.6)),    # n_z above the plane kernel's buffer
    ((2, 2, 40), (4, 4, 4), 0x01, 0.1, (-0.2, 0.6)),    # n_z at the plane kernel's largest buffer
    ((10, 16, 2), (16, 16, 16), 0x01, 0.1, (0.0, 0.6)),  # y segments of several rows (1.3 M cells)
    ((7, 6, 5), (6, 8, 10), 0x7F, 0.1, (-0.1, 0.6)),    # 7 species, ragged
    ((2, 3, 4), (4, 6, 4), 0x01, 0.3, (-1e4, 1e4)),     # |n| near 2^57: large high words in every flux
    ((2, 2, 3), (4, 4, 4), 0x01, 0.45, (-1e4, 1e4)),    # the same through the 128-bit (wide) form
]


@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("nx,np_,mask,dt,frange", DRIFT_CASES)
def test_drift_bit_exact_with_x_dependent_masses(nx, np_, mask, dt, frange, force):
    """x drift (and with force=True the force term -div_p[(grad_x E) f]) on
    random masses per x cell, bit for bit."""
    torch = torch_mod()
    nxc = nx[0] * nx[1] * nx[2]
    h, cfg = make_pair(nx=nx, dx=0.2, np_=np_, mask=mask, mass_mode=2)
    cfg.force = 1 if force else 0
    h.set_force_term(force)
    rng = np.random.default_rng(2)
    m2 = rng.uniform(0.0, 0.5, size=(nxc, 4))
    h.set_masses(m2)
    st = random_state(mask, nxc, np_, 8, *frange)
    out = torch.empty(st.size, dtype=torch.int64, device="cuda")
    h.drift(to_dev(st), out, dt)
    ref = O.drift(cfg, st, m2, dt)
    got = out.cpu().numpy().reshape(ref.shape)
    assert np.array_equal(got, ref)
    assert got.sum() == st.sum()


@pytest.mark.parametrize("mask", [0x01, 0x06, 0x31])
def test_masses_bit_exact_species_subsets(mask):
    """Masses with some species absent (their 1/(2E) is not evaluated) equal
    the oracle's, which evaluates every species; the second call uses the
    first call's dispersion."""
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    np_ = (6, 8, 6)
    h, cfg = make_pair(np_=np_, mask=mask)
    st = random_state(mask, 1, np_, 12)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    h.collision_term(to_dev(st), A, 1, 0, 0.01, bz.PREC_F32)
    m_first = O.masses(cfg, st)
    assert np.array_equal(h.get_masses(), m_first)
    h.collision_term(to_dev(st), A, 1, 1, 0.01, bz.PREC_F32)
    assert np.array_equal(h.get_masses(), O.masses(cfg, st, m_first))


@pytest.mark.parametrize("frange", [(0.0, 0.6), (-0.3, 0.6), (-1e5, 1e5)])
def test_moments_bit_exact(frange):
    """Exact sums, including negative cells and values near 2^61 (the high
    words of every split product)."""
    torch = torch_mod()
    nx, np_, mask = (2, 1, 3), (6, 8, 10), 0x7F
    h, cfg = make_pair(nx=nx, dx=0.2, np_=np_, mask=mask, mass_mode=2)
    m2 = np.random.default_rng(3).uniform(0.0, 0.4, size=(6, 4))
    h.set_masses(m2)
    st = random_state(mask, 6, np_, 9, *frange)
    out = torch.empty(6 * 7 * 5, dtype=torch.float64, device="cuda")
    h.moments(to_dev(st), out)
    ref, _ = O.moments(cfg, st, m2)
    assert np.array_equal(out.cpu().numpy().reshape(ref.shape), ref)


@pytest.mark.parametrize("mask,mass_mode,force", [(0x01, 0, False), (0x13, 0, False), (0x01, 1, False),
                                                   (0x13, 0, True), (0x01, 1, True)])
def test_step_bit_exact_inhomogeneous(mask, mass_mode, force):
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    nx, np_, N, dt = (4, 4, 2), (6, 6, 6), 32, 0.02
    h, cfg = make_pair(nx=nx, dx=0.2, np_=np_, mask=mask, mass_mode=mass_mode)
    cfg.force = 1 if force else 0
    h.set_force_term(force)
    nxc = 32
    st = random_state(mask, nxc, np_, 10, 0.0, 0.4)
    dev = to_dev(st)
    nsteps = 3
    mom = torch.empty(nsteps * nxc * bin(mask).count("1") * 5, dtype=torch.float64, device="cuda")
    h.step(dev, dt, nsteps, N, bz.PREC_F64, step0=5, moments_out=mom)
    ref, m2 = st, None
    moms = []
    for k in range(nsteps):
        ref, m2, _ = O.step(cfg, ref, m2, k == 0, N, 5 + k, dt)
        moms.append(O.moments(cfg, ref, m2)[0])
    assert np.array_equal(dev.cpu().numpy().reshape(ref.shape), ref)
    assert int(ref.sum()) == int(st.sum())
    assert np.array_equal(h.get_masses(), m2)
    assert np.array_equal(mom.cpu().numpy().reshape(np.array(moms).shape), np.array(moms))


# ---------------------------------------------------------------------------
# Full-size workloads (the benchmark configurations), checked on sampled
# anchors the oracle computes one by one, and by invariants that hold at any
# size.
# ---------------------------------------------------------------------------
def test_gluon_step_box_full_run_bit_exact():
    """Pure gluons, 20^3, N = 64, 10 Euler steps of dt = 0.01, FP64: whole run."""
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    w = I.gluon_step_box()
    h, cfg = make_pair(np_=w.np_, L=w.L, seed=w.seed, mask=w.species_mask, alpha=w.alpha_s)
    st = w.state()
    dev = to_dev(st)
    h.step(dev, w.dt, w.nsteps, w.nsamples, bz.PREC_F64)
    ref, m2 = st, None
    for k in range(w.nsteps):
        ref, m2, _ = O.step(cfg, ref, m2, k == 0, w.nsamples, k, w.dt)
    got = dev.cpu().numpy().reshape(ref.shape)
    assert np.array_equal(got, ref)
    assert int(got.sum()) == int(st.sum())


def test_qgp_box_full_size_sampled_anchors():
    """7 species, 32^3 over [-3, 3), N = 1024: FP64 bit-exact and FP32 within
    tolerance on every 997th anchor; FP32 over all anchors conserves exactly."""
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    w = I.qgp_box()
    h, cfg = make_pair(np_=w.np_, L=w.L, seed=w.seed, mask=w.species_mask, alpha=w.alpha_s)
    st = w.state()
    dev = to_dev(st)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    m2 = O.masses(cfg, st)
    h.set_anchor_subset(997, 5)
    h.collision_term(dev, A, w.nsamples, 0, w.dt, bz.PREC_F64)
    assert np.array_equal(h.get_masses(), m2)
    ref = O.collision(cfg, st, m2, w.nsamples, step=0, dt=w.dt, anchor_stride=997, anchor_offset=5)
    assert np.array_equal(A.cpu().numpy().reshape(ref["A"].shape), ref["A"])
    h.reset_masses()
    h.collision_term(dev, A, w.nsamples, 0, w.dt, bz.PREC_F32)
    ref32 = O.collision(cfg, st, m2, w.nsamples, step=0, dt=w.dt, ubits=23, anchor_stride=997,
                        anchor_offset=5)["A"]
    assert rel_l2(A.cpu().numpy().reshape(ref32.shape), ref32) <= F32_TOL
    h.set_anchor_subset(1, 0)
    h.reset_masses()
    h.collision_term(dev, A, w.nsamples, 0, w.dt, bz.PREC_F32)
    assert int(A.sum().item()) == 0
    assert int(A.abs().sum().item()) > 0


def test_gluon_bump_full_size(monkeypatch):
    """16^3 x 20^3 gluons, N = 256: masses and drift over all 33M cells are
    bit-exact; collisions on sampled anchors (FP64 bit-exact, the FP32 kernel of
    the timed step within tolerance under both work schedules, the same bits
    from each); one full FP32 step conserves."""
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    w = I.gluon_bump_xp()
    h, cfg = make_pair(nx=w.nx, dx=w.dx, np_=w.np_, L=w.L, seed=w.seed, mask=w.species_mask,
                       alpha=w.alpha_s)
    st = w.state()
    dev = to_dev(st)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    h.set_anchor_subset(65537, 11)
    h.collision_term(dev, A, w.nsamples, 0, w.dt, bz.PREC_F64)
    m2 = O.masses(cfg, st)
    assert np.array_equal(h.get_masses(), m2)
    ref = O.collision(cfg, st, m2, w.nsamples, step=0, dt=w.dt, anchor_stride=65537, anchor_offset=11)
    assert np.array_equal(A.cpu().numpy().reshape(ref["A"].shape), ref["A"])
    out = torch.empty_like(dev)
    h.drift(dev, out, w.dt)
    assert np.array_equal(out.cpu().numpy().reshape(st.shape), O.drift(cfg, st, m2, w.dt))
    ref32 = O.collision(cfg, st, m2, w.nsamples, step=0, dt=w.dt, ubits=23, anchor_stride=65537,
                        anchor_offset=11)["A"]
    got = {}
    for sched in ("counter", "static"):
        monkeypatch.setenv("BZ_F32_SCHEDULE", sched)
        h.reset_masses()
        h.collision_term(dev, A, w.nsamples, 0, w.dt, bz.PREC_F32)
        got[sched] = A.cpu().numpy().reshape(ref32.shape)
        assert int(got[sched].sum()) == 0
        assert rel_l2(got[sched], ref32) <= F32_TOL
    monkeypatch.delenv("BZ_F32_SCHEDULE")
    assert np.array_equal(got["counter"], got["static"])
    h.set_anchor_subset(1, 0)
    h.reset_masses()
    total = int(dev.sum().item())
    h.step(dev, w.dt, 1, w.nsamples, bz.PREC_F32)
    assert int(dev.sum().item()) == total


def test_argument_errors():
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    h, _ = make_pair(np_=(4, 4, 4))
    st = torch.zeros(64, dtype=torch.int64, device="cuda")
    A = torch.zeros(64, dtype=torch.int64, device="cuda")
    with pytest.raises(bz.BzError) as e:
        h.collision_term(st, A, 0)
    assert e.value.code == bz.BZ_EINVAL
    with pytest.raises(bz.BzError):
        h.collision_term(st, A, 4, step=1 << 29)
    with pytest.raises(TypeError):
        h.collision_term(st.double(), A, 4)
    with pytest.raises(ValueError):
        h.collision_term(st[:32], A[:32], 4)
    with pytest.raises(bz.BzError):
        h.drift(st, st, 0.01)
    h2, _ = make_pair(np_=(4, 4, 4), mass_mode=2)
    with pytest.raises(bz.BzError):
        h2.collision_term(st, A, 4)   # fixed masses not set


K3_CASES = [
    # np, mask, N, mass_mode, sampler
    ((8, 8, 8), 0x01, 64, 0, 0),
    ((6, 6, 6), 0x7F, 32, 0, 0),
    ((6, 10, 8), 0x13, 33, 1, 1),
]


@pytest.mark.parametrize("np_,mask,N,mass_mode,sampler", K3_CASES)
def test_collision_k3_parameterisation_bit_exact(np_, mask, N, mass_mode, sampler):
    """The k3-eliminating form (bz_set_parameterisation(1)) of the FP64 path
    equals the oracle's (run param 1) bit for bit; symmetric deposits sum to 0."""
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    h, cfg = make_pair(np_=np_, mask=mask, mass_mode=mass_mode)
    h.set_parameterisation(1)
    st = random_state(mask, 1, np_, 21)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    h.collision_term(to_dev(st), A, N, 3, 0.01, bz.PREC_F64, sampler)
    m2 = O.masses(cfg, st)
    ref = O.collision(cfg, st, m2, N, step=3, dt=0.01, sampler=sampler, param=1)["A"]
    got = A.cpu().numpy().reshape(ref.shape)
    assert np.array_equal(got, ref)
    if sampler == 0:
        assert int(got.sum()) == 0
    with pytest.raises(bz.BzError):
        h.collision_term(to_dev(st), A, N, 3, 0.01, bz.PREC_F32, sampler)   # FP64 only


def test_option_argument_errors():
    """Option setters refuse values outside their domain."""
    from paper_1912_04457_gb300 import bz
    h, _ = make_pair(np_=(4, 4, 4))
    for bad in (2, -1):
        with pytest.raises(bz.BzError):
            h._check(h.lib.bz_set_force_term(h.h, bad))   # the binding passes 0 or 1 only
        with pytest.raises(bz.BzError):
            h.set_parameterisation(bad)
    with pytest.raises(bz.BzError):
        h.set_uniform_bits(16)


def test_f32_step_with_force_conserves_number():
    """An FP32 step of an inhomogeneous box with the force term and thermal
    masses: drift, force, collisions and the fixup together keep sum n exact."""
    from paper_1912_04457_gb300 import bz
    nx, np_, mask = (4, 3, 2), (8, 8, 8), 0x13
    h, _ = make_pair(nx=nx, dx=0.2, np_=np_, mask=mask, mass_mode=0)
    h.set_force_term(True)
    st = random_state(mask, 24, np_, 31, 0.0, 0.5)
    dev = to_dev(st)
    h.step(dev, 0.01, 3, 64, bz.PREC_F32)
    got = dev.cpu().numpy()
    assert int(got.sum()) == int(st.sum())
    assert not np.array_equal(got.reshape(st.shape), st)


@pytest.mark.parametrize("mask", [0x01, 0x13])
def test_masses_table_path_extreme_states(mask):
    """The thermal masses through the p^2 table (one 1/(2E) per distinct p^2
    and x cell) and, for gluon-only states, the integer evaluation of the bin
    products: bit-identical to the oracle on an inhomogeneous grid with
    negative cells and cells beyond 2^49 (which take the FP64 instructions),
    for the first evaluation (E = |p|) and the second (E from the first)."""
    from paper_1912_04457_gb300 import bz
    torch = torch_mod()
    nx, np_ = (4, 2, 3), (20, 20, 20)
    nxc = 24
    h, cfg = make_pair(nx=nx, dx=0.2, np_=np_, mask=mask)
    st = random_state(mask, nxc, np_, 14, -0.2, 0.8)
    rng = np.random.default_rng(15)
    flat = st.reshape(-1)
    big = rng.choice(flat.size, size=200, replace=False)
    flat[big] = rng.integers(1 << 49, 1 << 52, size=200) * rng.choice([-1, 1], size=200)
    dev = to_dev(st)
    A = torch.empty(st.size, dtype=torch.int64, device="cuda")
    h.collision_term(dev, A, 1, 0, 0.01, bz.PREC_F32)
    m1 = O.masses(cfg, st)
    assert np.array_equal(h.get_masses(), m1)
    h.collision_term(dev, A, 1, 1, 0.01, bz.PREC_F32)
    assert np.array_equal(h.get_masses(), O.masses(cfg, st, m1))
