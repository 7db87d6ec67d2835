"""Pins of user-defined |M|^2 rows (the API for the user's own matrix
elements, Sec. II): a row is sum_k c_k s^a t^b u^c / (s^d (t - m_g^2)^e
(u - m_g^2)^f).  Every row of the Appendix table written in this form equals
the built-in row (pinned by its crossing identities) to rounding; the
collision estimate is linear in the row (same samples); detailed balance
holds for a user row too (equilibrium f)."""
import numpy as np
import pytest

import oracle as O
from paper_1912_04457_gb300 import inputs as I


def _consts(alpha):
    g2 = 4 * np.pi * alpha
    g4, dF, CA, CF, dA = g2 * g2, 3.0, 3.0, 4.0 / 3.0, 8.0
    return (8 * g4 * dF * dF * CF * CF / dA, 16 * g4 * dF * CF * (CF - CA / 2), 8 * g4 * dF * CF * CF,
            8 * g4 * dF * CF * CA, 16 * g4 * dA * CA * CA)


def table_rows(alpha):
    """The Appendix table in user form: (coef, (a, b, c, d, e, f)) with t~ = t - m_g^2, u~ = u - m_g^2."""
    A1, A2, A3, A4, A5 = _consts(alpha)
    return {
        0: [(A1, (2, 0, 0, 0, 2, 0)), (A1, (0, 0, 2, 0, 2, 0))],                                  # q q' -> q q'
        1: [(A1, (2, 0, 0, 0, 2, 0)), (A1, (0, 0, 2, 0, 2, 0)), (A1, (2, 0, 0, 0, 0, 2)),
            (A1, (0, 2, 0, 0, 0, 2)), (A2, (2, 0, 0, 0, 1, 1))],                                  # q q -> q q
        2: [(A1, (2, 0, 0, 0, 2, 0)), (A1, (0, 0, 2, 0, 2, 0)), (A1, (0, 0, 2, 2, 0, 0)),
            (A1, (0, 2, 0, 2, 0, 0)), (A2, (0, 0, 2, 1, 1, 0))],                                  # q qb -> q qb
        3: [(A1, (0, 2, 0, 2, 0, 0)), (A1, (0, 0, 2, 2, 0, 0))],                                  # q qb -> q' qb'
        4: [(A3, (0, 0, 1, 0, 1, 0)), (A3, (0, 1, 0, 0, 0, 1)), (-A4, (0, 2, 0, 2, 0, 0)),
            (-A4, (0, 0, 2, 2, 0, 0))],                                                           # q qb -> g g
        5: [(A4, (2, 0, 0, 0, 2, 0)), (A4, (0, 0, 2, 0, 2, 0)), (-A3, (0, 0, 1, 1, 0, 0)),
            (-A3, (1, 0, 0, 0, 0, 1))],                                                           # q g -> q g
        6: [(3 * A5, (0, 0, 0, 0, 0, 0)), (-A5, (1, 0, 1, 0, 2, 0)), (-A5, (1, 1, 0, 0, 0, 2)),
            (-A5, (0, 1, 1, 2, 0, 0))],                                                           # g g -> g g
    }


def test_table_rows_in_user_form_equal_the_builtin_rows():
    rng = np.random.default_rng(3)
    rows = table_rows(0.3)
    for r, terms in rows.items():
        for _ in range(200):
            s = rng.uniform(0.1, 20.0)
            t, u = -rng.uniform(0.05, 10.0), -rng.uniform(0.05, 10.0)
            mg2 = rng.uniform(0.0, 0.6)
            want = O.msq(r, 0.3, s, t, u, mg2)
            got = O.msq_user(terms, s, t, u, mg2)
            assert got == pytest.approx(want, rel=1e-12, abs=1e-12 * abs(want)), (r, s, t, u)


def _box(user=None, mask=0x13, analytic=False):
    return O.make_config(np_=(6, 6, 6), L=2.0, seed=5, species_mask=mask, alpha_s=0.3, mass_mode=0,
                         analytic=analytic, T=0.4, user_rows=user)


def test_estimate_is_linear_in_a_user_row():
    st = I.encode(I.random_f((6, 6, 6), 3, 1, 9, 0.0, 0.5), 0x13)
    base = _box()
    m2 = O.masses(base, st)
    ref = O.collision(base, st, m2, 64, want_c64=True)["C64"]
    same = O.collision(_box(table_rows(0.3)), st, m2, 64, want_c64=True)["C64"]
    assert np.allclose(same, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    doubled = {r: [(2 * c, e) for c, e in terms] for r, terms in table_rows(0.3).items()}
    twice = O.collision(_box(doubled), st, m2, 64, want_c64=True)["C64"]
    assert np.allclose(twice, 2 * ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    # a single row replaced changes the estimate
    only_gg = O.collision(_box({6: [(100.0, (0, 0, 0, 0, 0, 0))]}), st, m2, 64, want_c64=True)["C64"]
    assert not np.allclose(only_gg, ref)


def test_detailed_balance_with_a_user_row():
    """Equilibrium f (Bose-Einstein / Fermi-Dirac at the continuous leg
    energies): W = 0 at every root whatever |M|^2 is, so a constant and an
    s-channel-like user row both give |C| << gain."""
    st = I.encode(I.random_f((6, 6, 6), 3, 1, 9, 0.0, 0.5), 0x13)
    user = {6: [(50.0, (0, 0, 0, 0, 0, 0))], 5: [(10.0, (2, 0, 0, 0, 1, 1))], 4: [(3.0, (0, 2, 0, 2, 0, 0))]}
    cfg = _box(user, analytic=True)
    m2 = O.masses(_box(), st)
    r = O.collision(cfg, st, m2, 64, want_c64=True)
    assert np.abs(r["C64"]).max() < 1e-12 * np.abs(r["G64"]).max()
    assert np.abs(r["G64"]).max() > 0
