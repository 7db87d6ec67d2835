"""Parity of the FP32 time step that the benchmark times (bz_step with
BZ_PREC_F32, Sec. III: masses, drift with the FP32 f of n^n, collision
deposits straight into n^{n+1}, float-float re-evaluation of ill-conditioned
terms) with the FP64 oracle's Euler step on the same 23-bit sample points.

Each step starts from the GPU's state and masses; the oracle's step from
the same state gives the masses (bit-identical), the drift (bit-identical:
the collision part is isolated by subtracting the oracle's drift) and the
collision increment, which the FP32 path matches within 2e-5 relative L2.
Sum n is exact every step.  The same holds for the learned step sampler on
given per-anchor proposal parameters and for boxes of a batched ensemble."""
import numpy as np
import pytest

import oracle as O
from paper_1912_04457_gb300 import inputs as I

pytestmark = pytest.mark.gpu

F32_TOL = 2e-5


def _rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


STEP_CASES = [
    # name, nx, np, mask, mass_mode, force, N, dt
    ("qgp7_homogeneous", (1, 1, 1), (8, 8, 8), 0x7F, 0, False, 48, 0.01),
    ("g_u_ubar_inhomogeneous_force", (4, 3, 2), (6, 6, 6), 0x13, 0, True, 32, 0.01),
    ("gluon_inhomogeneous_massless", (3, 2, 4), (8, 6, 6), 0x01, 1, False, 40, 0.02),
]


@pytest.mark.parametrize("name,nx,np_,mask,mass_mode,force,N,dt", STEP_CASES)
def test_f32_step_increments_match_the_oracle(name, nx, np_, mask, mass_mode, force, N, dt):
    import torch
    from paper_1912_04457_gb300 import bz
    nxc = int(np.prod(nx))
    h = bz.Handle(nx=nx, dx=0.2, np_=np_, L=2.0, seed=9, species_mask=mask, alpha_s=0.3, mass_mode=mass_mode)
    h.set_force_term(force)
    cfg = O.make_config(nx=nx, dx=0.2, np_=np_, L=2.0, seed=9, species_mask=mask, alpha_s=0.3,
                        mass_mode=mass_mode, force=force)
    st = I.encode(I.random_f(np_, bin(mask).count("1"), nxc, 41, 0.02, 0.5), mask)
    dev = torch.from_numpy(st.reshape(-1)).cuda()
    cur = st.copy()
    m_prev = None
    for k in range(3):
        h.step(dev, dt, 1, N, bz.PREC_F32, step0=7 + k)
        got = dev.cpu().numpy().reshape(st.shape)
        ref, m_used, _ = O.step(cfg, cur, m_prev, k == 0, N, 7 + k, dt, ubits=23)
        assert np.array_equal(h.get_masses(), m_used), "step %d masses" % k
        drift = O.drift(cfg, cur, m_used, dt)
        err = _rel_l2(got - drift, ref - drift)
        assert err <= F32_TOL, "step %d: collision increment off by %.2e" % (k, err)
        assert int(got.sum()) == int(cur.sum())
        assert np.count_nonzero(ref - drift) > 0
        cur, m_prev = got, m_used
    h.close()


def test_f32_step_with_the_learned_sampler_matches_the_oracle():
    """bz_set_step_sampler(BZ_SAMPLER_LEARNED) on fixed per-anchor proposal
    parameters: each step's collision increment against the oracle's learned
    estimator on the same parameters and 23-bit uniforms."""
    import torch
    from paper_1912_04457_gb300 import bz
    np_, mask, N, dt = (6, 6, 6), 0x7F, 48, 0.01
    h = bz.Handle(np_=np_, L=2.0, seed=5, species_mask=mask, alpha_s=0.3)
    cfg = O.make_config(np_=np_, L=2.0, seed=5, species_mask=mask, alpha_s=0.3)
    ncell = bin(mask).count("1") * int(np.prod(np_))
    rng = np.random.default_rng(8)
    prm = np.zeros((ncell, 8), dtype=np.float32)
    prm[:, 0:3] = rng.uniform(-0.3, 0.3, size=(ncell, 3))     # mu3
    prm[:, 3] = rng.uniform(0.3, 0.8, size=ncell)             # sigma3
    prm[:, 4] = rng.uniform(0.3, 0.8, size=ncell)             # sigma1
    prm[:, 5] = rng.uniform(0.15, 0.5, size=ncell)            # alpha
    h.set_anchor_params(prm)
    h.set_step_sampler(bz.SAMPLER_LEARNED)
    st = I.encode(I.random_f(np_, 7, 1, 43, 0.02, 0.5), mask)
    dev = torch.from_numpy(st.reshape(-1)).cuda()
    cur, m_prev = st.copy(), None
    for k in range(2):
        h.step(dev, dt, 1, N, bz.PREC_F32, step0=3 + k)
        got = dev.cpu().numpy().reshape(st.shape)
        ref, m_used, _ = O.step(cfg, cur, m_prev, k == 0, N, 3 + k, dt, sampler=O.LEARNED, ubits=23,
                                prop=prm.astype(np.float64))
        assert np.array_equal(h.get_masses(), m_used)
        drift = O.drift(cfg, cur, m_used, dt)      # one x cell: the drift is the identity
        err = _rel_l2(got - drift, ref - drift)
        assert err <= F32_TOL, "step %d: learned increment off by %.2e" % (k, err)
        assert int(got.sum()) == int(cur.sum())
        cur, m_prev = got, m_used
    h.close()


def test_batch_boxes_match_the_oracle():
    """Boxes of a batched ensemble (one persistent launch per step, graph
    replay) against the oracle's step of each box: masses bit-identical,
    collision increments within 2e-5, number exact."""
    import torch
    from paper_1912_04457_gb300 import bz
    specs = [((6, 6, 6), 0x01, 40, 0.30, 0), ((6, 8, 6), 0x7F, 48, 0.25, 0), ((8, 8, 8), 0x01, 33, 0.35, 1),
             ((4, 6, 8), 0x13, 50, 0.30, 0)]
    boxes, states = [], []
    for i, (np_, mask, N, a, mm) in enumerate(specs):
        boxes.append({"np_": np_, "L": 2.0, "species_mask": mask, "nsamples": N, "alpha_s": a,
                      "mass_mode": mm, "box_id": 3 + i, "seed": 13})
        states.append(I.encode(I.random_f(np_, bin(mask).count("1"), 1, 50 + i, 0.02, 0.5), mask))
    dt = 0.01
    B = bz.Batch(boxes)
    flat = torch.from_numpy(np.concatenate([s.reshape(-1) for s in states])).cuda()
    cur = [s.copy() for s in states]
    m_prev = [None] * len(boxes)
    for k in range(2):
        B.step(flat, dt, 1, step0=2 + k)
        torch.cuda.synchronize()
        got_all = flat.cpu().numpy()
        m_batch = B.get_masses()
        for i, bx in enumerate(boxes):
            cfg = O.make_config(np_=bx["np_"], L=2.0, seed=13, box=bx["box_id"], species_mask=bx["species_mask"],
                                alpha_s=bx["alpha_s"], mass_mode=bx["mass_mode"])
            ref, m_used, _ = O.step(cfg, cur[i], m_prev[i], k == 0, bx["nsamples"], 2 + k, dt, ubits=23)
            lo, hi = B.cell_offsets[i], B.cell_offsets[i + 1]
            got = got_all[lo:hi].reshape(ref.shape)
            assert np.array_equal(m_batch[i], m_used[0]), "box %d step %d masses" % (i, k)
            err = _rel_l2(got - cur[i], ref - cur[i])   # one x cell: the whole increment is the collision
            assert err <= F32_TOL, "box %d step %d: increment off by %.2e" % (i, k, err)
            assert int(got.sum()) == int(cur[i].sum())
            cur[i], m_prev[i] = got, m_used
    B.close()


@pytest.mark.parametrize("np_,mask,N", [((8, 8, 8), 0x7F, 48), ((20, 20, 20), 0x01, 256)])
def test_counter_and_static_schedules_give_the_same_bits(np_, mask, N, monkeypatch):
    """The FP32 kernel's two ways of sharing work units among warps (a global
    counter, the default for large problems, or one unit per warp, the
    default for small ones) give bit-identical deposits, and both are within
    the FP32 tolerance of the oracle (first case) or conserve exactly."""
    import torch
    from paper_1912_04457_gb300 import bz
    h = bz.Handle(np_=np_, L=2.0, seed=3, species_mask=mask, alpha_s=0.3)
    st = I.encode(I.random_f(np_, bin(mask).count("1"), 1, 12, 0.05, 0.5), mask)
    dev = torch.from_numpy(st.reshape(-1)).cuda()
    out = {}
    for sched in ("counter", "static"):
        monkeypatch.setenv("BZ_F32_SCHEDULE", sched)
        A = torch.empty_like(dev)
        h.reset_masses()
        h.collision_term(dev, A, N, 1, 0.01, bz.PREC_F32)
        out[sched] = A.cpu().numpy()
    monkeypatch.delenv("BZ_F32_SCHEDULE")
    assert np.array_equal(out["counter"], out["static"])
    assert int(out["counter"].sum()) == 0 and np.count_nonzero(out["counter"]) > 0
    if np.prod(np_) <= 512:
        cfg = O.make_config(np_=np_, L=2.0, seed=3, species_mask=mask, alpha_s=0.3)
        ref = O.collision(cfg, st, O.masses(cfg, st), N, step=1, dt=0.01, ubits=23)["A"]
        assert _rel_l2(out["counter"].reshape(ref.shape), ref) <= F32_TOL
    h.close()


@pytest.mark.parametrize("nx,np_,mask,force,nsteps", [((1, 1, 1), (12, 12, 12), 0x01, False, 7),
                                                      ((4, 3, 2), (6, 6, 6), 0x13, True, 6)])
def test_replayed_step_graph_gives_the_eager_bits(nx, np_, mask, force, nsteps, monkeypatch):
    """FP32 runs of several steps replay a captured pair of steps (device-side
    step index and moments slot): state, masses and per-step moments equal
    those of the same run with every step launched eagerly (BZ_STEP_GRAPH=0),
    over two calls (the second reuses the graph)."""
    import torch
    from paper_1912_04457_gb300 import bz
    nxc = int(np.prod(nx))
    ns = bin(mask).count("1")
    st = I.encode(I.random_f(np_, ns, nxc, 61, 0.02, 0.5), mask)
    out = {}
    for mode in ("graph", "eager"):
        if mode == "eager":
            monkeypatch.setenv("BZ_STEP_GRAPH", "0")
        h = bz.Handle(nx=nx, dx=0.2, np_=np_, L=2.0, seed=4, species_mask=mask, alpha_s=0.3)
        h.set_force_term(force)
        dev = torch.from_numpy(st.reshape(-1)).cuda()
        mom = torch.zeros(nsteps * nxc * ns * 5, dtype=torch.float64, device="cuda")
        h.step(dev, 0.01, nsteps, 32, bz.PREC_F32, step0=3, moments_out=mom)
        a = (dev.cpu().numpy().copy(), mom.cpu().numpy().copy(), h.get_masses())
        h.step(dev, 0.01, nsteps, 32, bz.PREC_F32, step0=3 + nsteps, moments_out=mom)
        out[mode] = (a, (dev.cpu().numpy().copy(), mom.cpu().numpy().copy(), h.get_masses()))
        h.close()
    monkeypatch.delenv("BZ_STEP_GRAPH")
    for call in range(2):
        for g, e in zip(out["graph"][call], out["eager"][call]):
            assert np.array_equal(g, e)
    assert int(out["graph"][1][0].sum()) == int(st.sum())
