"""User-defined |M|^2 rows (bz_set_matrix_element) against the oracle's:
FP64 bit for bit, FP32 within the FP32 tolerance on the same uniforms, the
default restored bit for bit, and argument errors."""
import numpy as np
import pytest

import oracle as O
from paper_1912_04457_gb300 import inputs as I
from test_oracle_user_msq import table_rows

pytestmark = pytest.mark.gpu

USER = {6: [(50.0, (0, 0, 0, 0, 0, 0)), (-3.0, (1, 0, 1, 0, 2, 0))],      # constant + a t-channel piece
        5: [(12.0, (2, 0, 0, 0, 1, 1))],
        2: table_rows(0.3)[2]}


def _pair(mask, user):
    from paper_1912_04457_gb300 import bz
    h = bz.Handle(np_=(6, 8, 6), L=2.0, seed=3, species_mask=mask, alpha_s=0.3)
    for r, terms in user.items():
        h.set_matrix_element(r, terms)
    cfg = O.make_config(np_=(6, 8, 6), L=2.0, seed=3, species_mask=mask, alpha_s=0.3, user_rows=user)
    return h, cfg


@pytest.mark.parametrize("mask", [0x01, 0x7F])
def test_user_rows_f64_bit_exact_and_f32_within_tolerance(mask):
    import torch
    from paper_1912_04457_gb300 import bz
    h, cfg = _pair(mask, USER)
    st = I.encode(I.random_f((6, 8, 6), bin(mask).count("1"), 1, 14, 0.0, 0.5), mask)
    dev = torch.from_numpy(st.reshape(-1)).cuda()
    A = torch.empty_like(dev)
    h.collision_term(dev, A, 48, 2, 0.01, bz.PREC_F64)
    m2 = O.masses(cfg, st)
    ref = O.collision(cfg, st, m2, 48, step=2, dt=0.01)["A"]
    assert np.array_equal(A.cpu().numpy().reshape(ref.shape), ref)
    h.reset_masses()
    h.collision_term(dev, A, 48, 2, 0.01, bz.PREC_F32)
    ref23 = O.collision(cfg, st, m2, 48, step=2, dt=0.01, ubits=23)["A"].astype(float)
    got = A.cpu().numpy().reshape(ref23.shape).astype(float)
    assert int(got.sum()) == 0
    assert np.linalg.norm(got - ref23) / np.linalg.norm(ref23) <= 2e-5
    # the default rows come back with nterms = 0
    for r in USER:
        h.set_matrix_element(r, [])
    h.reset_masses()
    h.collision_term(dev, A, 48, 2, 0.01, bz.PREC_F64)
    base = O.make_config(np_=(6, 8, 6), L=2.0, seed=3, species_mask=mask, alpha_s=0.3)
    assert np.array_equal(A.cpu().numpy().reshape(ref.shape), O.collision(base, st, m2, 48, step=2, dt=0.01)["A"])


def test_user_row_argument_errors():
    from paper_1912_04457_gb300 import bz
    h = bz.Handle(np_=(6, 6, 6), species_mask=1)
    for row, terms in [(7, [(1.0, (0,) * 6)]), (-1, [(1.0, (0,) * 6)]), (0, [(1.0, (5, 0, 0, 0, 0, 0))]),
                       (0, [(float("nan"), (0,) * 6)]), (0, [(1.0, (0,) * 6)] * 9)]:
        with pytest.raises(bz.BzError):
            h.set_matrix_element(row, terms)
