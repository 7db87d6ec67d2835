"""The paper's stability comparison of the two ways to use the delta
function (Sec. III.A, Fig. 2): gluons, random f in [0, 1], the plain
(own-cell) estimator, independent evaluations of one step; the spread of the
total gluon number is larger when k3 is eliminated than when k2 is (the
paper's "less stable" choice), while both have the same mean within errors."""
import numpy as np
import pytest

from paper_1912_04457_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_k3_elimination_spreads_more():
    import torch
    from paper_1912_04457_gb300 import bz
    n, L, N, dt, seeds = 20, 2.0, 100, 0.01, 24
    st = I.encode(I.random_f((n, n, n), 1, 1, 7, 0.0, 1.0), 0x01)
    dev = torch.from_numpy(st.reshape(-1)).cuda()
    totals = {0: [], 1: []}
    for param in (0, 1):
        for sd in range(seeds):
            h = bz.Handle(np_=(n, n, n), L=L, seed=1000 + sd, species_mask=0x01, alpha_s=0.3)
            h.set_parameterisation(param)
            A = torch.empty_like(dev)
            h.collision_term(dev, A, N, 0, dt, bz.PREC_F64, bz.SAMPLER_PLAIN)
            totals[param].append(float(A.sum().item()))
            h.close()
    t0, t1 = np.array(totals[0]), np.array(totals[1])
    err = np.sqrt(t0.var(ddof=1) / seeds + t1.var(ddof=1) / seeds)
    assert abs(t0.mean() - t1.mean()) < 5 * err
    assert t1.std(ddof=1) > 1.2 * t0.std(ddof=1)
