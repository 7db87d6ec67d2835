"""FP64 reference of the learned proposal network and its loss (test
infrastructure only).

The network maps anchor features (9) to the 6 parameters of a proposal
density over the normalised sample box y = (k1x, k1y, k3)/L in [-1, 1)^5:
a 9 -> 128 -> 128 -> 6 MLP with SiLU.  The GPU evaluates every GEMM on BF16
operands with FP32 accumulation; this reference rounds to BF16 at the same
points (features, weights, pre-activations, activations, output gradients,
pre-activation gradients) and accumulates in FP64.  With `bf16=False` every
rounding is skipped, which gives a smooth loss for finite-difference checks.

Proposal (defensive mixture):
  mu3 = tanh(o0..2), sigma3 = 0.02 + 0.5 sigmoid(o3), sigma1 = 0.02 + 0.5 sigmoid(o4),
  alpha = 0.1 + 0.9 sigmoid(o5),
  q(y) = alpha / 32 + (1 - alpha) prod_i g_i(y_i),
g_i the Student-t density with two degrees of freedom, f(z) = (2 + z^2)^(-3/2)
(z = (y - centre)/scale), with centre 0 (k1 components) or mu3 (k3
components), truncated to [-1, 1): its CDF, inverse CDF and density need
only square roots, F(z) = 1/2 + z / (2 sqrt(2 + z^2)).  Loss over records
(anchor a, weight w, sample y): L = -sum_i w_i log q(y_i | a_i) / sum_i w_i.
"""
import numpy as np

H, NIN, NOUT = 128, 16, 8
NPARAM = NIN * H + H + H * H + H + H * NOUT + NOUT


def split(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + NIN * H].reshape(NIN, H); o += NIN * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H * NOUT].reshape(H, NOUT); o += H * NOUT
    b3 = p[o:o + NOUT]
    return W1, b1, W2, b2, W3, b3


def join(W1, b1, W2, b2, W3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])


def bf16(x):
    """Round to BF16 the way the GPU does (to FP32 first, then nearest-even on the top 16 bits)."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def features(a, np_, L, nxc, slot_species):
    """Features of anchors a (global index [slot][x][p]) at their cell centres, FP32."""
    a = np.asarray(a, dtype=np.int64)
    npc = int(np.prod(np_))
    sl = a // (nxc * npc)
    j = a % npc
    jv = [j // (np_[1] * np_[2]), (j // np_[2]) % np_[1], j % np_[2]]
    L32 = np.float32(L)
    p = []
    for i in range(3):
        dp = np.float32(np.float32(2.0) * L32 / np.float32(np_[i]))
        c = (-L32 + (jv[i].astype(np.float32) + np.float32(0.5)) * dp) / L32
        p.append(c.astype(np.float32))
    pp = (p[0] * p[0] + p[1] * p[1] + p[2] * p[2]).astype(np.float32)
    d = np.asarray(slot_species)[sl]
    F = np.zeros((a.size, NIN))
    F[:, 0], F[:, 1], F[:, 2] = p[0], p[1], p[2]
    F[:, 3] = np.sqrt(pp)
    F[:, 4] = pp
    F[:, 5] = d == 0
    F[:, 6] = (d >= 1) & (d <= 3)
    F[:, 7] = d >= 4
    F[:, 8] = 1.0
    return F


def _sig(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(params, X, bf=True):
    """Returns outputs o [n, 8] and the cached intermediates."""
    r = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    c = _f32 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = split(params)
    Xb = r(X)
    W1b, W2b, W3b = r(W1), r(W2), r(W3)
    Z1 = r(c(Xb @ W1b + b1))
    H1 = r(c(Z1 * _sig(Z1)))
    Z2 = r(c(H1 @ W2b + b2))
    H2 = r(c(Z2 * _sig(Z2)))
    O = H2 @ W3b + b3
    return O, (Xb, W1b, W2b, W3b, Z1, H1, Z2, H2)


def head(O):
    o = np.asarray(O, dtype=np.float64)
    prm = np.zeros((o.shape[0], 8))
    prm[:, 0:3] = np.tanh(o[:, 0:3])
    prm[:, 3] = 0.02 + 0.5 * _sig(o[:, 3])
    prm[:, 4] = 0.02 + 0.5 * _sig(o[:, 4])
    prm[:, 5] = 0.1 + 0.9 * _sig(o[:, 5])
    return prm


def t2_pdf(z):
    """Student-t density with two degrees of freedom."""
    return (2.0 + z * z) ** -1.5


def t2_cdf(z):
    """Its CDF, 1/2 + z / (2 sqrt(2 + z^2)), written without cancellation in the tails."""
    s = np.sqrt(2.0 + z * z)
    tail = 1.0 / (s * (s + np.abs(z)))         # F(-|z|)
    return np.where(z < 0, tail, 1.0 - tail)


def proposal_density(prm, y):
    """q(y) for rows of per-sample parameters prm [n, 8] and samples y [n, 5]."""
    G = np.ones(len(y))
    for i in range(5):
        mu = np.zeros(len(y)) if i < 2 else prm[:, i - 2]
        s = prm[:, 4] if i < 2 else prm[:, 3]
        Z = t2_cdf((1.0 - mu) / s) - t2_cdf((-1.0 - mu) / s)
        G = G * t2_pdf((y[:, i] - mu) / s) / (s * Z)
    al = prm[:, 5]
    return al / 32.0 + (1.0 - al) * G


def logq_grad(O, y):
    """log q and d log q / d o (n x 6), analytic."""
    prm = head(O)
    n = len(y)
    G = np.ones(n)
    dmu = np.zeros((n, 3))
    ds3 = np.zeros(n)
    ds1 = np.zeros(n)
    for i in range(5):
        k3 = i >= 2
        mu = prm[:, i - 2] if k3 else np.zeros(n)
        s = prm[:, 3] if k3 else prm[:, 4]
        z, za, zb = (y[:, i] - mu) / s, (-1.0 - mu) / s, (1.0 - mu) / s
        Z = t2_cdf(zb) - t2_cdf(za)
        pa, pb = t2_pdf(za), t2_pdf(zb)
        G = G * t2_pdf(z) / (s * Z)
        dlf = -3.0 * z / (2.0 + z * z)            # d log f / dz
        dm = -dlf / s + (pb - pa) / (s * Z)
        dsg = -dlf * z / s - 1.0 / s + (pb * zb - pa * za) / (s * Z)
        if k3:
            dmu[:, i - 2] = dm
            ds3 += dsg
        else:
            ds1 += dsg
    al = prm[:, 5]
    q = al / 32.0 + (1 - al) * G
    r = (1 - al) * G / q
    g = np.zeros((n, 6))
    g[:, 0:3] = r[:, None] * dmu * (1 - prm[:, 0:3] ** 2)
    s3 = (prm[:, 3] - 0.02) / 0.5
    s1 = (prm[:, 4] - 0.02) / 0.5
    g[:, 3] = r * ds3 * 0.5 * s3 * (1 - s3)
    g[:, 4] = r * ds1 * 0.5 * s1 * (1 - s1)
    sa = (al - 0.1) / 0.9
    g[:, 5] = (1.0 / 32.0 - G) / q * 0.9 * sa * (1 - sa)
    return np.log(q), g


def loss_grad(params, X, y, w, bf=True):
    """Loss -sum w log q / sum w and its gradient with respect to the flat parameters."""
    r = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = split(params)
    O, (Xb, W1b, W2b, W3b, Z1, H1, Z2, H2) = forward(params, X, bf)
    wn = np.asarray(w, dtype=np.float64) / np.sum(w)
    if bf:
        wn = _f32(wn)
    lq, gq = logq_grad(O[:, :6], y)
    loss = -np.sum(wn * lq)
    dO = np.zeros((len(y), 16))
    dO[:, :6] = r(-wn[:, None] * gq)
    dO8 = dO[:, :NOUT]
    dW3 = H2.T @ dO8
    db3 = dO8.sum(0)
    dsil = lambda Z: _sig(Z) * (1 + Z * (1 - _sig(Z)))
    dZ2 = r(c32(bf)(dO8 @ W3b.T * dsil(Z2)))
    dW2 = H1.T @ dZ2
    db2 = dZ2.sum(0)
    dZ1 = r(c32(bf)(dZ2 @ W2b.T * dsil(Z1)))
    dW1 = Xb.T @ dZ1
    db1 = dZ1.sum(0)
    return loss, join(dW1, db1, dW2, db2, dW3, db3)


def c32(bf):
    return _f32 if bf else (lambda v: np.asarray(v, dtype=np.float64))


def init_params(seed):
    """Glorot-uniform weights from numpy's seeded generator (zero biases, zero padding)."""
    rng = np.random.default_rng(seed)
    W1 = np.zeros((NIN, H))
    W1[:9] = rng.uniform(-1, 1, (9, H)) * np.sqrt(6.0 / (9 + H))
    W2 = rng.uniform(-1, 1, (H, H)) * np.sqrt(6.0 / (2 * H))
    W3 = np.zeros((H, NOUT))
    W3[:, :6] = rng.uniform(-1, 1, (H, 6)) * np.sqrt(6.0 / (H + 6))
    b1 = rng.uniform(-0.1, 0.1, H)
    b2 = rng.uniform(-0.1, 0.1, H)
    b3 = np.zeros(NOUT)
    b3[:6] = rng.uniform(-0.5, 0.5, 6)
    return join(W1, b1, W2, b2, W3, b3).astype(np.float32)
