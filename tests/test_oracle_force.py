"""Pins of the oracle's force term, -div_p[(grad_x E) f] of Eq. (left
handside): upwind in p with dE/dx_i = (dm^2/dx_i)/(2E) (central difference of
m^2), no flux through the faces of the momentum box.  Checked against what
does not depend on that discretisation: exact number conservation, no force
without a mass gradient, the momentum change against the paper's own
central difference of E in Eq. (descrete left hand), and the cancellation of
drift and force for any f = F(E(x, p)) (a stationary solution of the
collisionless equation: E is conserved along dx/dt = p/E, dp/dt = -grad_x E),
whose residual is of first order in the cell sizes."""
import numpy as np
import pytest

import oracle as O
from paper_1912_04457_gb300 import inputs as I

L = 2.0


def _centres(np_):
    pc = [-L + (np.arange(n) + 0.5) * 2 * L / n for n in np_]
    return np.stack(np.meshgrid(*pc, indexing="ij"), 0).reshape(3, -1)   # [3, npc]


def _energies(np_, m2x):
    P = _centres(np_)
    return P, np.sqrt((P ** 2).sum(0)[None, :] + m2x[:, None])          # [nxc, npc]


def _zero_edges(f, np_, nxc, w=1):
    f = f.reshape(-1, nxc, *np_).copy()
    f[..., :w, :, :] = 0
    f[..., -w:, :, :] = 0
    f[..., :, :w, :] = 0
    f[..., :, -w:, :] = 0
    f[..., :, :, :w] = 0
    f[..., :, :, -w:] = 0
    return f.reshape(-1, nxc, int(np.prod(np_)))


def _pair(nx, np_, dx, mask=0x01, mass_mode=2):
    on = O.make_config(nx=nx, dx=dx, np_=np_, species_mask=mask, mass_mode=mass_mode, force=True)
    off = O.make_config(nx=nx, dx=dx, np_=np_, species_mask=mask, mass_mode=mass_mode, force=False)
    return on, off


def test_force_conserves_number_exactly():
    nx, np_, mask = (4, 3, 5), (8, 6, 8), 0x13
    nxc = 60
    on, off = _pair(nx, np_, 0.2, mask)
    st = I.encode(I.random_f(np_, 3, nxc, 8, -0.1, 0.6), mask)     # f up to the box faces
    m2 = np.random.default_rng(2).uniform(0.0, 0.5, size=(nxc, 4))
    a, b = O.drift(on, st, m2, 0.05), O.drift(off, st, m2, 0.05)
    assert int(a.sum()) == int(st.sum())
    assert not np.array_equal(a, b)


@pytest.mark.parametrize("mass_mode", [1, 2])
def test_no_force_without_a_mass_gradient(mass_mode):
    """Equal masses in every x cell (or the massless dispersion): the force
    term adds nothing, bit for bit."""
    nx, np_ = (3, 4, 2), (6, 6, 6)
    on, off = _pair(nx, np_, 0.2, 0x01, mass_mode)
    st = I.encode(I.random_f(np_, 1, 24, 4, 0.0, 0.6), 0x01)
    m2 = np.tile([0.3, 0.2, 0.2, 0.25], (24, 1))
    assert np.array_equal(O.drift(on, st, m2, 0.05), O.drift(off, st, m2, 0.05))


def test_momentum_change_matches_the_central_difference_of_E():
    """With f zero in the outer p cells no flux meets a box face, and the x
    drift moves nothing between p cells, so the change of sum_p p_i n is the
    force alone: dt sum F_i n with F_i = -(E(x + e_i, p) - E(x - e_i, p))/(2 dx)
    (the paper's difference form), per axis (different gradient per axis)."""
    nx, np_, dx, dt = (12, 10, 8), (12, 12, 12), 0.2, 0.002
    on, off = _pair(nx, np_, dx)
    ix, iy, iz = np.meshgrid(*[np.arange(n) for n in nx], indexing="ij")
    m2x = (0.3 + 0.05 * np.sin(2 * np.pi * ix / nx[0]) - 0.03 * np.cos(2 * np.pi * iy / nx[1])
           + 0.015 * np.sin(2 * np.pi * iz / nx[2] + 0.3)).reshape(-1)
    m2 = np.repeat(m2x[:, None], 4, axis=1)
    nxc = m2x.size
    st = I.encode(_zero_edges(I.random_f(np_, 1, nxc, 3, 0.1, 0.6), np_, nxc), 0x01)
    n0 = st.reshape(nxc, -1).astype(np.float64)
    n_on = O.drift(on, st, m2, dt).reshape(n0.shape).astype(np.float64)
    n_off = O.drift(off, st, m2, dt).reshape(n0.shape).astype(np.float64)
    P, E = _energies(np_, m2x)
    Eg = E.reshape(nx + (-1,))
    for i in range(3):
        F = -(np.roll(Eg, -1, axis=i) - np.roll(Eg, 1, axis=i)) / (2 * dx)
        want = dt * (F.reshape(n0.shape) * n0).sum()
        got = ((n_on - n0) * P[i][None, :]).sum()
        assert abs(((n_off - n0) * P[i][None, :]).sum()) < 1e-9 * abs(want)
        assert got == pytest.approx(want, rel=0.02), i


def test_drift_and_force_cancel_for_a_function_of_the_energy():
    """f = exp(-E(x, p)/T) with m^2 varying along x: the residual of drift
    plus force is a small fraction of the drift alone and shrinks as the
    cells shrink (a wrong sign doubles the change, a wrong factor leaves a
    residual of the drift's own size)."""
    ratios = []
    for nxx, npp in [(16, 16), (64, 32)]:
        nx, np_, dx, dt = (nxx, 1, 1), (npp, 4, 4), 3.2 / nxx, 0.001
        m2x = 0.4 + 0.1 * np.sin(2 * np.pi * np.arange(nxx) / nxx)
        m2 = np.repeat(m2x[:, None], 4, axis=1)
        _, E = _energies(np_, m2x)
        f = np.exp(-E / 0.3).reshape(1, nxx, *np_)
        f[..., :1, :, :] = 0
        f[..., -1:, :, :] = 0
        st = I.encode(f.reshape(1, nxx, -1), 0x01)
        on, off = _pair(nx, np_, dx)
        n0 = st.reshape(nxx, -1).astype(np.float64)
        d_on = O.drift(on, st, m2, dt).reshape(n0.shape) - n0
        d_off = O.drift(off, st, m2, dt).reshape(n0.shape) - n0
        inner = np.ones(np_, bool)
        inner[:2] = False
        inner[-2:] = False
        inner = inner.reshape(-1)
        ratios.append(np.abs(d_on[:, inner]).sum() / np.abs(d_off[:, inner]).sum())
    assert ratios[0] < 0.45
    assert ratios[1] < 0.6 * ratios[0]
