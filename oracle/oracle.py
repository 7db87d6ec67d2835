"""ctypes wrapper of the C oracle (test infrastructure only).

Arrays are numpy; the state is int64 n[slot][x][p] = N_s f 2^40 with the
active species in increasing index order (0 g, 1 u, 2 d, 3 s, 4 ubar,
5 dbar, 6 sbar), x and p row-major with the last axis fastest.
"""
import ctypes as C
import os

import numpy as np

from .build import build_oracle

NSPEC = 7
SYMMETRIC, PLAIN, LEARNED = 0, 1, 2
M_QQP, M_QQ, M_QQB, M_QQB2, M_QQBGG, M_QG, M_GG = range(7)


class Config(C.Structure):
    _fields_ = [
        ("nx", C.c_int32 * 3), ("dx", C.c_double),
        ("np", C.c_int32 * 3), ("L", C.c_double),
        ("seed", C.c_uint64), ("box", C.c_uint32),
        ("species_mask", C.c_uint32), ("alpha_s", C.c_double),
        ("mass_mode", C.c_int32), ("analytic", C.c_int32),
        ("T", C.c_double), ("mu", C.c_double * NSPEC),
        ("force", C.c_int32),
        ("user", C.c_void_p), ("umask", C.c_uint32),
    ]


class Run(C.Structure):
    _fields_ = [
        ("nsamples", C.c_int32), ("step", C.c_int32), ("dt", C.c_double),
        ("sampler", C.c_int32), ("ubits", C.c_int32), ("p_center", C.c_int32),
        ("anchor_stride", C.c_int64), ("anchor_offset", C.c_int64),
        ("u_explicit", C.POINTER(C.c_double)),
        ("prop", C.POINTER(C.c_double)),
        ("param", C.c_int32),
        ("u_shared", C.c_int32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        _lib = C.CDLL(path)
        P = C.c_void_p
        _lib.bzo_philox4x32_10.argtypes = [P, P, P]
        _lib.bzo_msq.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]
        _lib.bzo_msq.restype = C.c_double
        _lib.bzo_msq_user.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double]
        _lib.bzo_msq_user.restype = C.c_double
        _lib.bzo_roots.argtypes = [P, C.c_double, P, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_double, P]
        _lib.bzo_two_body_sum.argtypes = [P, C.c_double, P, C.c_double, C.c_double, C.c_double,
                                          C.c_double, C.c_int, C.c_int]
        _lib.bzo_two_body_sum.restype = C.c_double
        _lib.bzo_masses.argtypes = [P, P, P, P]
        _lib.bzo_collision.argtypes = [P, P, P, P, P, P, P, P, P]
        _lib.bzo_drift.argtypes = [P, P, P, C.c_double, P]
        _lib.bzo_drift_f64.argtypes = [P, P, P, C.c_double, P]
        _lib.bzo_moments.argtypes = [P, P, P, P, P]
        _lib.bzo_energy_source.argtypes = [P, P, P, P, C.c_double, P]
        _lib.bzo_step.argtypes = [P, P, P, P, C.c_int, P, P]
        _lib.bzo_num_threads.restype = C.c_int
        _lib.bzo_proposal_sample.argtypes = [P, C.c_double, P, P]
        _lib.bzo_proposal_sample.restype = C.c_double
        assert _lib.bzo_sizeof_config() == C.sizeof(Config)
        assert _lib.bzo_sizeof_run() == C.sizeof(Run)
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# user-defined |M|^2 rows: 7 rows of (n, pad, 8 x (coef, a, b, c, d, e, f, pad, pad))
UTERM = np.dtype([("coef", "<f8"), ("e", "u1", (6,)), ("pad", "u1", (2,))])
UROW = np.dtype([("n", "<i4"), ("pad", "<i4"), ("t", UTERM, (8,))])


def user_table(rows):
    """rows: {row index: [(coef, (a, b, c, d, e, f)), ...]} -> (structured array of 7 rows, mask)."""
    tab = np.zeros(7, dtype=UROW)
    mask = 0
    for r, terms in rows.items():
        assert 0 <= r < 7 and 0 < len(terms) <= 8
        tab[r]["n"] = len(terms)
        for k, (c, e) in enumerate(terms):
            tab[r]["t"][k]["coef"] = c
            tab[r]["t"][k]["e"] = e
        mask |= 1 << r
    return tab, mask


def msq_user(terms, s, t, u, mg2):
    tab, _ = user_table({0: terms})
    return lib().bzo_msq_user(tab.ctypes.data_as(C.c_void_p), s, t, u, mg2)


def make_config(nx=(1, 1, 1), dx=1.0, np_=(20, 20, 20), L=2.0, seed=1, box=0,
                species_mask=1, alpha_s=0.3, mass_mode=0, analytic=False, T=0.5, mu=None, force=False,
                user_rows=None):
    c = Config()
    c.nx[:] = list(nx)
    c.dx = dx
    c.np[:] = list(np_)
    c.L = L
    c.seed = seed
    c.box = box
    c.species_mask = species_mask
    c.alpha_s = alpha_s
    c.mass_mode = mass_mode
    c.analytic = 1 if analytic else 0
    c.T = T
    c.mu[:] = list(mu) if mu is not None else [0.0] * NSPEC
    c.force = 1 if force else 0
    if user_rows:
        c._user_keep, c.umask = user_table(user_rows)
        c.user = c._user_keep.ctypes.data
    return c


def nslots(cfg):
    return bin(cfg.species_mask).count("1")


def ncells(cfg):
    nxc = cfg.nx[0] * cfg.nx[1] * cfg.nx[2]
    npc = cfg.np[0] * cfg.np[1] * cfg.np[2]
    return nslots(cfg), nxc, npc


def philox(ctr, key):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().bzo_philox4x32_10(_ptr(ctr), _ptr(key), _ptr(out))
    return out


def msq(cls, alpha_s, s, t, u, mg2):
    return lib().bzo_msq(cls, alpha_s, s, t, u, mg2)


def roots(p, md2, k3, mc2, k1x, k1y, ma2, mb2):
    p = np.ascontiguousarray(p, dtype=np.float64)
    k3 = np.ascontiguousarray(k3, dtype=np.float64)
    out = np.zeros(8)
    n = lib().bzo_roots(_ptr(p), md2, _ptr(k3), mc2, k1x, k1y, ma2, mb2, _ptr(out))
    return out[: 4 * n].reshape(n, 4)


def two_body_sum(p, md2, k3, mc2, ma2, mb2, R, m, weight_j2=False):
    p = np.ascontiguousarray(p, dtype=np.float64)
    k3 = np.ascontiguousarray(k3, dtype=np.float64)
    return lib().bzo_two_body_sum(_ptr(p), md2, _ptr(k3), mc2, ma2, mb2, R, m,
                                  1 if weight_j2 else 0)


def masses(cfg, state, m2_prev=None):
    ns, nxc, npc = ncells(cfg)
    state = np.ascontiguousarray(state, dtype=np.int64).reshape(-1)
    assert state.size == ns * nxc * npc
    out = np.zeros((nxc, 4))
    mp = None if m2_prev is None else np.ascontiguousarray(m2_prev, dtype=np.float64)
    rc = lib().bzo_masses(C.byref(cfg), _ptr(state), _ptr(mp), _ptr(out))
    if rc:
        raise OverflowError("mass fixed-point sum overflow")
    return out


def make_run(nsamples, step=0, dt=0.01, sampler=SYMMETRIC, ubits=32, p_center=False,
             anchor_stride=1, anchor_offset=0, u_explicit=None, prop=None, param=0, u_shared=False):
    r = Run()
    r.param = param
    r.u_shared = 1 if u_shared else 0
    r.nsamples = nsamples
    r.step = step
    r.dt = dt
    r.sampler = sampler
    r.ubits = ubits
    r.p_center = 1 if p_center else 0
    r.anchor_stride = anchor_stride
    r.anchor_offset = anchor_offset
    if u_explicit is not None:
        r._u_keep = np.ascontiguousarray(u_explicit, dtype=np.float64)
        r.u_explicit = r._u_keep.ctypes.data_as(C.POINTER(C.c_double))
    else:
        r.u_explicit = None
    if prop is not None:
        r._prop_keep = np.ascontiguousarray(prop, dtype=np.float64)
        r.prop = r._prop_keep.ctypes.data_as(C.POINTER(C.c_double))
    else:
        r.prop = None
    return r


def collision(cfg, state, m2, nsamples, step=0, dt=0.01, sampler=SYMMETRIC, ubits=32,
              p_center=False, anchor_stride=1, anchor_offset=0, u_explicit=None,
              want_c64=False, want_audit=False, prop=None, param=0, u_shared=False):
    """Returns dict with A (int64 [slot][x][p]), flags, and optionally C64/G64/audit.
    param 0: k2 eliminated (the paper's choice), 1: k3 eliminated.  u_explicit:
    [anchor][sample][8] uniforms replacing Philox, or with u_shared one
    [sample][8] set used by every anchor."""
    ns, nxc, npc = ncells(cfg)
    state = np.ascontiguousarray(state, dtype=np.int64).reshape(-1)
    m2 = np.ascontiguousarray(m2, dtype=np.float64).reshape(nxc, 4)
    if sampler == LEARNED:
        assert prop is not None and np.asarray(prop).size == ns * nxc * npc * 8
        assert param == 0, "the learned sampler draws (k1_perp, k3)"
    run = make_run(nsamples, step, dt, sampler, ubits, p_center, anchor_stride, anchor_offset,
                   u_explicit, prop, param, u_shared)
    A = np.zeros(ns * nxc * npc, dtype=np.int64)
    C64 = np.zeros(ns * nxc * npc) if want_c64 else None
    G64 = np.zeros(ns * nxc * npc) if want_c64 else None
    audit = np.zeros(8) if want_audit else None
    flags = np.zeros(2, dtype=np.int64)
    lib().bzo_collision(C.byref(cfg), C.byref(run), _ptr(state), _ptr(m2), _ptr(A), _ptr(C64),
                        _ptr(G64), _ptr(audit), _ptr(flags))
    out = {"A": A.reshape(ns, nxc, npc), "flags": flags}
    if want_c64:
        out["C64"] = C64.reshape(ns, nxc, npc)
        out["G64"] = G64.reshape(ns, nxc, npc)
    if want_audit:
        out["audit"] = audit
    return out


def drift(cfg, state, m2, dt):
    ns, nxc, npc = ncells(cfg)
    state = np.ascontiguousarray(state, dtype=np.int64).reshape(-1)
    m2 = np.ascontiguousarray(m2, dtype=np.float64).reshape(nxc, 4)
    out = np.zeros_like(state)
    lib().bzo_drift(C.byref(cfg), _ptr(state), _ptr(m2), dt, _ptr(out))
    return out.reshape(ns, nxc, npc)


def drift_f64(cfg, f, m2, dt):
    ns, nxc, npc = ncells(cfg)
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    m2 = np.ascontiguousarray(m2, dtype=np.float64).reshape(nxc, 4)
    out = np.zeros_like(f)
    lib().bzo_drift_f64(C.byref(cfg), _ptr(f), _ptr(m2), dt, _ptr(out))
    return out.reshape(ns, nxc, npc)


def moments(cfg, state, m2):
    ns, nxc, npc = ncells(cfg)
    state = np.ascontiguousarray(state, dtype=np.int64).reshape(-1)
    m2 = np.ascontiguousarray(m2, dtype=np.float64).reshape(nxc, 4)
    out = np.zeros((nxc, ns, 5))
    nsum = np.zeros(ns, dtype=np.int64)
    lib().bzo_moments(C.byref(cfg), _ptr(state), _ptr(m2), _ptr(out), _ptr(nsum))
    return out, nsum


def energy_source(cfg, state, m2, m2_prev, dt):
    """Per (x cell, slot): [I = int d^3p/(2pi)^3 N f / E, S_ex^0 part
    (1/2)((m^2 - m^2_prev)/dt) I, -(1/4) m^2 I] (Eq. (current conservation))."""
    ns, nxc, npc = ncells(cfg)
    state = np.ascontiguousarray(state, dtype=np.int64).reshape(-1)
    m2 = np.ascontiguousarray(m2, dtype=np.float64).reshape(nxc, 4)
    m2_prev = np.ascontiguousarray(m2_prev, dtype=np.float64).reshape(nxc, 4)
    out = np.zeros((nxc, ns, 3))
    lib().bzo_energy_source(C.byref(cfg), _ptr(state), _ptr(m2), _ptr(m2_prev), C.c_double(dt), _ptr(out))
    return out


def step(cfg, state, m2, first, nsamples, step_index, dt, sampler=SYMMETRIC, ubits=32, prop=None):
    """One Euler step; returns (new state, masses used, flags).  prop: the
    per-anchor proposal parameters [anchor][8] of the learned sampler."""
    ns, nxc, npc = ncells(cfg)
    state = np.ascontiguousarray(state, dtype=np.int64).reshape(-1)
    m2 = np.array(m2 if m2 is not None else np.zeros((nxc, 4)), dtype=np.float64).reshape(nxc, 4)
    if sampler == LEARNED:
        assert prop is not None and np.asarray(prop).size == ns * nxc * npc * 8
    run = make_run(nsamples, step_index, dt, sampler, ubits, prop=prop)
    out = np.zeros_like(state)
    flags = np.zeros(2, dtype=np.int64)
    rc = lib().bzo_step(C.byref(cfg), C.byref(run), _ptr(state), _ptr(m2), 1 if first else 0,
                        _ptr(out), _ptr(flags))
    if rc:
        raise OverflowError("mass fixed-point sum overflow")
    return out.reshape(ns, nxc, npc), m2, flags


def num_threads():
    return lib().bzo_num_threads()


def proposal_sample(prm, usel, u5):
    """One learned-proposal sample: (y [5], 1/(32 q(y)))."""
    prm = np.ascontiguousarray(prm, dtype=np.float64)
    u5 = np.ascontiguousarray(u5, dtype=np.float64)
    y = np.zeros(5)
    wf = lib().bzo_proposal_sample(_ptr(prm), float(usel), _ptr(u5), _ptr(y))
    return y, wf
