"""Pins of the learned-proposal parts of the oracle.

* the proposal density is normalised on [-1, 1)^5 and the oracle's sampler
  (C, inverse CDF) draws from exactly the density the loss uses (numpy);
* the loss gradient of the FP64 network equals central finite differences;
* importance sampling keeps the collision estimator unbiased: the mean of the
  learned-proposal deposits over seeds equals the mean of the uniform ones.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp
from paper_1912_04457_gb300 import inputs as I


def _prm(mu=(0.2, -0.3, 0.1), s3=0.25, s1=0.4, alpha=0.3):
    return np.array([mu[0], mu[1], mu[2], s3, s1, alpha, 0.0, 0.0])


def test_proposal_density_is_normalised():
    rng = np.random.default_rng(0)
    for prm in (_prm(), _prm((0.8, 0.0, -0.6), 0.05, 0.1, 0.1), _prm((0, 0, 0), 0.5, 0.5, 0.9)):
        y = rng.uniform(-1, 1, (400000, 5))
        q = mlp.proposal_density(np.tile(prm, (len(y), 1)), y)
        est = 32.0 * q.mean()                      # E_uniform[q] * volume
        err = 32.0 * q.std() / np.sqrt(len(y))
        assert abs(est - 1.0) < 5 * err + 1e-12


def test_oracle_sampler_draws_from_the_density():
    rng = np.random.default_rng(1)
    prm = _prm()
    n = 60000
    ys, wf = np.zeros((n, 5)), np.zeros(n)
    for i in range(n):
        ys[i], wf[i] = O.proposal_sample(prm, rng.uniform(), rng.uniform(size=5))
    q = mlp.proposal_density(np.tile(prm, (n, 1)), ys)
    assert np.allclose(wf, 1.0 / (32.0 * q), rtol=1e-10)
    # marginal histograms vs the density's marginals (mixture of uniform and truncated Student-t with
    # two degrees of freedom, whose CDF is 1/2 + z / (2 sqrt(2 + z^2)))
    edges = np.linspace(-1, 1, 21)
    for i in range(5):
        mu = 0.0 if i < 2 else prm[i - 2]
        s = prm[4] if i < 2 else prm[3]
        cdf2 = lambda z: 0.5 + z / (2.0 * np.sqrt(2.0 + z * z))
        Fa, Fb = cdf2((-1 - mu) / s), cdf2((1 - mu) / s)
        cdf = (cdf2((edges - mu) / s) - Fa) / (Fb - Fa)
        p = prm[5] * np.diff(edges) / 2.0 + (1 - prm[5]) * np.diff(cdf)
        counts, _ = np.histogram(ys[:, i], edges)
        chi2 = ((counts - n * p) ** 2 / (n * p)).sum()
        assert chi2 < 19 + 6 * np.sqrt(2 * 19)
    # the importance weight has unit mean under the proposal: E_q[1/(32 q)] = 1
    assert abs(wf.mean() - 1.0) < 5 * wf.std() / np.sqrt(n)


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = mlp.init_params(3).astype(np.float64)
    n = 64
    a = rng.integers(0, 7 * 6 ** 3, n)
    X = mlp.features(a, (6, 6, 6), 2.0, 1, list(range(7)))
    y = rng.uniform(-1, 1, (n, 5))
    w = rng.uniform(0.1, 2.0, n)
    loss, g = mlp.loss_grad(params, X, y, w, bf=False)
    W1, b1, W2, b2, W3, b3 = mlp.split(np.arange(mlp.NPARAM))
    picks = [int(W1[0, 5]), int(W1[8, 100]), int(b1[17]), int(W2[3, 4]), int(W2[120, 7]), int(b2[60]),
             int(W3[10, 0]), int(W3[99, 5]), int(b3[3]), int(b3[5])]
    for k in picks:
        h = 1e-6 * max(1.0, abs(params[k]))
        pp, pm = params.copy(), params.copy()
        pp[k] += h
        pm[k] -= h
        fd = (mlp.loss_grad(pp, X, y, w, bf=False)[0] - mlp.loss_grad(pm, X, y, w, bf=False)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    # padded inputs / outputs carry no gradient
    idx = lambda v: np.asarray(v, dtype=np.int64).ravel()
    assert np.all(g[idx(W1[9:])] == 0) and np.all(g[idx(W3[:, 6:])] == 0) and np.all(g[idx(b3[6:])] == 0)


@pytest.mark.parametrize("mask", [0x01, 0x7F])
def test_learned_sampler_is_unbiased(mask):
    n, L, N = 6, 2.0, 64
    ns = bin(mask).count("1")
    f = np.stack([I.step_f((n, n, n), L, 0.5, 1.2) if s == 0 else I.exp_f((n, n, n), L, 0.2, 0.4)
                  for s in I.slots(mask)]).reshape(ns, 1, -1)
    st = I.encode(f, mask)
    rng = np.random.default_rng(4)
    prop = np.zeros((ns * n ** 3, 8))
    prop[:, 0:3] = rng.uniform(-0.3, 0.3, (len(prop), 3))
    prop[:, 3] = rng.uniform(0.1, 0.4, len(prop))
    prop[:, 4] = rng.uniform(0.1, 0.4, len(prop))
    prop[:, 5] = 0.2
    pc = I.momentum_centres((n, n, n), L)
    shell = np.minimum((np.sqrt((pc * pc).sum(1)) / (L * np.sqrt(3)) * 4).astype(int), 3)

    def agg(A):
        return np.array([[A[sl, 0, shell == k].sum() for k in range(4)] for sl in range(ns)])
    un, le = [], []
    for sd in range(1, 41):
        cfg = O.make_config(np_=(n, n, n), L=L, species_mask=mask, seed=sd)
        m2 = O.masses(cfg, st)
        un.append(agg(O.collision(cfg, st, m2, N)["A"].astype(float)))
        r = O.collision(cfg, st, m2, N, sampler=O.LEARNED, prop=prop)
        assert int(r["A"].sum()) == 0
        le.append(agg(r["A"].astype(float)))
    un, le = np.array(un), np.array(le)
    err = np.sqrt(un.var(0, ddof=1) / len(un) + le.var(0, ddof=1) / len(le))
    live = err > 0
    z = (un.mean(0) - le.mean(0))[live] / err[live]
    assert np.abs(z).max() < 5.0
    assert (np.abs(un.mean(0))[live] / err[live]).max() > 8
