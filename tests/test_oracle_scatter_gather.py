"""Brute force on a 4^3 grid: the oracle's symmetrical deposition (a
scatter: each root adds +q to the bins of p and k3 and -q to those of k1 and
k2, Sec. III.B) against an independently coded gather on the same explicit
sample points — for every bin, the sum over all (anchor, sample, root) whose
legs land in it.  The kinematics here are written from the paper's equations
(Eqs. (delta function), (work out delta E), (delta replace)) with numpy, not
taken from the oracle; only |M|^2 (pinned by its own identities) is shared.
The int64 quanta must agree bin by bin (up to a unit where a quantum's
rounding sits on a half-integer)."""
import numpy as np

import oracle as O
from paper_1912_04457_gb300 import inputs as I

HBARC = 0.1973269804
L, NP, ALPHA = 2.0, 4, 0.3


def _gather(f, m2, u, dt, N):
    """Returns the int64 deposit array [NP^3] of the symmetrical estimator (gluons)."""
    dp = 2 * L / NP
    mg2 = m2
    V = (2 * L) ** 5
    Kq = V * dt / (4.0 * N) / HBARC * 2.0 ** 40            # one root's quantum per leg, 2^-40 N f units
    binof = lambda k: np.clip(np.floor((k + L) / dp).astype(np.int64), 0, NP - 1)
    lin = lambda b: (b[..., 0] * NP + b[..., 1]) * NP + b[..., 2]
    A = np.zeros(NP ** 3, dtype=np.int64)
    fl = f.reshape(-1)
    na = NP ** 3
    jv = np.stack(np.meshgrid(*[np.arange(NP)] * 3, indexing="ij"), -1).reshape(na, 3)
    for a in range(na):
        uu = u[a]                                           # [N, 8]
        p = -L + (jv[a] + 0.5) * dp + dp * (uu[:, 0:3] - 0.5)
        k1p = -L + 2 * L * uu[:, 3:5]
        k3 = -L + 2 * L * uu[:, 5:8]
        Ep = np.sqrt((p ** 2).sum(1) + mg2)
        E3 = np.sqrt((k3 ** 2).sum(1) + mg2)
        P = p + k3
        E = Ep + E3
        # k2 = P - k1: E1 + E2 = E with E1^2 = a2 + z^2, E2^2 = b2 + (Pz - z)^2
        a2 = (k1p ** 2).sum(1) + mg2
        b2 = ((P[:, :2] - k1p) ** 2).sum(1) + mg2
        # squaring: E^2 + a2 - b2 - Pz^2 + 2 Pz z = 2 E E1 -> (E^2 - Pz^2) z^2 - 2 c Pz z + (a2 E^2 - c^2) = 0
        c = 0.5 * (E * E + a2 - b2 - P[:, 2] ** 2)
        qa, qb, qc = E * E - P[:, 2] ** 2, -2 * c * P[:, 2], a2 * E * E - c * c
        disc = qb * qb - 4 * qa * qc
        ok = (disc >= 0) & (qa > 0) & (np.abs(P[:, 0] - k1p[:, 0]) <= 1e9)
        sq = np.sqrt(np.where(ok, disc, 0.0))
        for sgn in (1.0, -1.0):
            z = (-qb + sgn * sq) / np.where(ok, 2 * qa, 1.0)
            E1 = np.sqrt(a2 + z * z)
            k2 = np.stack([P[:, 0] - k1p[:, 0], P[:, 1] - k1p[:, 1], P[:, 2] - z], 1)
            E2 = np.sqrt((k2 ** 2).sum(1) + mg2)
            good = ok & (np.abs(E1 + E2 - E) <= 1e-10 * E)
            good &= (z >= -L) & (z < L) & np.all((k2 >= -L) & (k2 < L), 1)
            J = z / E1 - k2[:, 2] / E2
            good &= J != 0
            k1 = np.stack([k1p[:, 0], k1p[:, 1], z], 1)
            s = E * E - (P ** 2).sum(1)
            t = (E1 - E3) ** 2 - ((k1 - k3) ** 2).sum(1)
            uu_ = (E1 - Ep) ** 2 - ((k1 - p) ** 2).sum(1)
            good &= (s > 0) & (t - mg2 < 0) & (uu_ - mg2 < 0)
            for i in np.nonzero(good)[0]:
                M2 = O.msq(6, ALPHA, s[i], t[i], uu_[i], mg2)
                b1, b2_, b3 = lin(binof(k1[i])), lin(binof(k2[i])), lin(binof(k3[i]))
                f1, f2, f3, fp = fl[b1], fl[b2_], fl[b3], fl[a]
                W = f1 * f2 * (1 + f3) * (1 + fp) - (1 + f1) * (1 + f2) * f3 * fp
                ct = 0.5 * W * M2 / (abs(J[i]) * (2 * np.pi) ** 5 * 16 * E1[i] * E2[i] * E3[i] * Ep[i])
                q = int(np.rint(ct * Kq))
                # gather: each bin collects the quanta of the legs that land in it
                A[a] += q
                A[b3] += q
                A[b1] -= q
                A[b2_] -= q
    return A


def test_symmetric_scatter_equals_gather_on_explicit_samples():
    N, dt, m2 = 24, 0.01, 0.3
    cfg = O.make_config(np_=(NP,) * 3, L=L, seed=2, species_mask=0x01, alpha_s=ALPHA, mass_mode=2)
    st = I.encode(I.random_f((NP,) * 3, 1, 1, 41, 0.05, 0.7), 0x01)
    f = I.decode(st, 0x01)[0, 0]
    u = np.random.default_rng(9).random((NP ** 3, N, 8))
    ref = O.collision(cfg, st, np.full((1, 4), m2), N, dt=dt, u_explicit=u)["A"].reshape(-1)
    got = _gather(f, m2, u, dt, N)
    assert int(ref.sum()) == 0 and int(got.sum()) == 0
    assert np.abs(ref).sum() > 1000 * NP ** 3                 # the comparison has substance
    diff = np.abs(ref - got)
    assert diff.max() <= 1 and (diff > 0).sum() <= 2, (diff.max(), (diff > 0).sum())   # measured: identical
