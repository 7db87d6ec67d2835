"""Pins of the oracle's energy source (Eq. (current conservation)):
I = int d^3p/(2pi)^3 N f / E, S_ex^0 = (1/2)(dm^2/dt) I and the T_total term
-(1/4) m^2 I.  I is checked against the closed form N T^2/12 of massless
Bose-Einstein gluons (Richardson extrapolation of the O(dp) grid error), and
S_ex^0 against the change of the kinetic energy T^00 (Eq. (energy momentum
tensor), the moments) when only the masses change: for a fixed f,
T^00(m_b) - T^00(m_a) = sum N f (E_b - E_a) = (1/2) (m_b^2 - m_a^2) I up to
second order in the mass change.  The -(1/4) m^2 I term of T_total is the
product of the pinned I and the masses; beyond that it is unpinned."""
import numpy as np
import pytest

import oracle as O
from paper_1912_04457_gb300 import inputs as I


def test_closed_form_massless_bose_einstein():
    T, L = 0.3, 3.0
    vals = []
    for n in (16, 32, 64):
        cfg = O.make_config(np_=(n, n, n), L=L, species_mask=1, mass_mode=1)
        st = I.encode(I.equilibrium_f((n, n, n), L, 0, T).reshape(1, 1, -1), 1)
        r = O.energy_source(cfg, st, np.zeros((1, 4)), np.zeros((1, 4)), 1.0)
        vals.append(r[0, 0, 0])
        assert r[0, 0, 1] == 0.0 and r[0, 0, 2] == 0.0   # massless dispersion: no m^2 terms
    exact = 16 * T * T / 12
    r1a, r1b = 2 * vals[1] - vals[0], 2 * vals[2] - vals[1]      # first-order error removed
    r2 = (4 * r1b - r1a) / 3                                     # and the second-order one
    assert abs(vals[2] / exact - 1) > 0.05                       # the raw grid value is off ...
    assert abs(r2 / exact - 1) < 2e-3                            # ... the extrapolation is not


@pytest.mark.parametrize("mask", [0x01, 0x02])
def test_source_matches_the_energy_change_from_the_masses(mask):
    """First (E = |p|) and second mass evaluation of one state, and 1/10 of
    that change: the relative mismatch is second order (shrinks ~10x)."""
    n, L, dt = 24, 2.0, 0.01
    cfg = O.make_config(np_=(n, n, n), L=L, species_mask=mask, mass_mode=2)
    f = I.step_f((n, n, n), L, 0.5, 1.5).reshape(1, 1, -1)
    st = I.encode(f, mask)
    cth = O.make_config(np_=(n, n, n), L=L, species_mask=mask, mass_mode=0)
    ma = O.masses(cth, st)
    mb_full = O.masses(cth, st, ma)
    rels = []
    for eps in (1.0, 0.1):
        mb = ma + eps * (mb_full - ma)
        dT = O.moments(cfg, st, mb)[0][0, 0, 1] - O.moments(cfg, st, ma)[0][0, 0, 1]
        r = O.energy_source(cfg, st, mb, ma, dt)[0, 0]
        assert r[1] * dt == pytest.approx(0.5 * (mb - ma)[0, 0 if mask == 1 else 1] * r[0], rel=1e-12)
        rels.append(abs(dT / (r[1] * dt) - 1))
    assert rels[0] < 0.05
    assert rels[1] < 0.15 * rels[0]


def test_source_sign_and_time_step():
    n, L = 12, 2.0
    cfg = O.make_config(np_=(n, n, n), L=L, species_mask=1, mass_mode=2)
    st = I.encode(I.step_f((n, n, n), L, 0.5, 1.0).reshape(1, 1, -1), 1)
    ma = np.tile([0.40, 0.1, 0.1, 0.1], (1, 1))
    mb = np.tile([0.45, 0.1, 0.1, 0.1], (1, 1))
    up = O.energy_source(cfg, st, mb, ma, 0.01)[0, 0]
    down = O.energy_source(cfg, st, ma, mb, 0.01)[0, 0]
    half = O.energy_source(cfg, st, mb, ma, 0.02)[0, 0]
    assert up[1] > 0 > down[1]
    assert half[1] == pytest.approx(up[1] / 2, rel=1e-12)
    assert up[2] == pytest.approx(-0.25 * 0.45 * up[0], rel=1e-12)
