"""Pins of the oracle's energy source (Eq. (current conservation)):
I = int d^3p/(2pi)^3 N f / E, S_ex^0 = (1/2)(dm^2/dt) I and the T_total term
-(1/4) m^2 I.  I is checked against the closed form N T^2/12 of massless
Bose-Einstein gluons (Richardson extrapolation of the O(dp) grid error), and
S_ex^0 against the change of the kinetic energy T^00 (Eq. (energy momentum
tensor), the moments) when only the masses change: for a fixed f,
T^00(m_b) - T^00(m_a) = sum N f (E_b - E_a) = (1/2) (m_b^2 - m_a^2) I up to
second order in the mass change.  The -(1/4) m^2 I term of T_total is
checked against a quadrature of its definition, and against the property
the paper derives it from: for one flavour with self-consistent masses its
change cancels S_ex^0 dt."""
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


def test_T_total_term_against_a_quadrature_of_its_definition():
    """-(1/4) m^2 int d^3p/(2pi)^3 N f/E for Bose-Einstein gluons at T = 0.3 GeV
    with a fixed m^2 = 0.2 GeV^2 (E = sqrt(p^2 + m^2) in f and in 1/E): the
    grid values, with the O(dp^2) error of the cell-centred sums removed by
    Richardson extrapolation over 16^3, 32^3, 64^3, against a radial
    quadrature of the same definition over the momentum box [-L, L)^3 (scipy;
    the part of the sphere of radius p inside the cube is 1 - 3 (p - L)/p for
    L <= p <= sqrt(2) L; beyond, the integrand is below e^{-14} of its peak)."""
    quad = pytest.importorskip("scipy.integrate").quad
    T, L, m2 = 0.3, 3.0, 0.2
    vals = []
    for n in (16, 32, 64):
        cfg = O.make_config(np_=(n, n, n), L=L, species_mask=1, mass_mode=2)
        st = I.encode(I.equilibrium_f((n, n, n), L, 0, T, m2=m2).reshape(1, 1, -1), 1)
        m = np.array([[m2, 0.0, 0.0, 0.0]])
        r = O.energy_source(cfg, st, m, m, 1.0)
        vals.append(r[0, 0, 2])
    E = lambda p: np.sqrt(p * p + m2)
    g = lambda p: p * p / (E(p) * np.expm1(E(p) / T))
    I_exact = 16.0 / (2 * np.pi ** 2) * (quad(g, 0, L)[0] +
                                        quad(lambda p: (1 - 3 * (p - L) / p) * g(p), L, np.sqrt(2) * L)[0])
    exact = -0.25 * m2 * I_exact
    r1a, r1b = (4 * vals[1] - vals[0]) / 3, (4 * vals[2] - vals[1]) / 3
    assert abs(r1b / exact - 1) < 2e-5
    assert abs(r1b / exact - 1) < 0.2 * abs(vals[0] / exact - 1)


def test_T_total_term_cancels_the_source_for_one_flavour():
    """For pure gluons with self-consistent masses (Eq. (mg) evaluated with E
    from the same m^2), m_g^2 = (g^2 C_A / d_A) I, so -(1/4) m^2 I =
    -(1/4)(d_A/(g^2 C_A)) m^4 and its change over a step is minus S_ex^0 dt:
    the modified T_total of the paper is conserved up to second order in the
    mass change.  Checked for a 1% and a 0.1% change of the state."""
    n, L, alpha = 24, 2.0, 0.3
    cfg_th = O.make_config(np_=(n, n, n), L=L, species_mask=1, alpha_s=alpha, mass_mode=0)
    cfg_fx = O.make_config(np_=(n, n, n), L=L, species_mask=1, alpha_s=alpha, mass_mode=2)
    f = I.step_f((n, n, n), L, 0.5, 1.5).reshape(1, 1, -1)

    def self_consistent(st):
        m = O.masses(cfg_th, st)
        for _ in range(60):
            m_new = O.masses(cfg_th, st, m)
            if np.array_equal(m_new, m):
                break
            m = m_new
        return m

    g2 = 4 * np.pi * alpha
    st_a = I.encode(f, 1)
    ma = self_consistent(st_a)
    ra = O.energy_source(cfg_fx, st_a, ma, ma, 1.0)[0, 0]
    assert ra[0] * g2 * 3.0 / 8.0 == pytest.approx(ma[0, 0], rel=1e-5)   # m_g^2 = (g^2 C_A/d_A) I
    rels = []
    for eps in (1e-2, 1e-3):
        st_b = I.encode(f * (1 + eps), 1)
        mb = self_consistent(st_b)
        dt = 0.01
        rb = O.energy_source(cfg_fx, st_b, mb, ma, dt)[0, 0]
        d_term = rb[2] - ra[2]                 # change of -(1/4) m^2 I
        rels.append(abs(d_term / (-rb[1] * dt) - 1))
    assert rels[0] < 0.02
    assert rels[1] < 0.2 * rels[0]
