"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no step of the method: it only builds initial
distributions f_s(x, p) of the closed forms the paper uses (CGC-like step,
Eq. (CGC); exponential quark tail; Bose-Einstein / Fermi-Dirac, Eqs. (fg),
(fq); a Gaussian spatial bump) and encodes them as the library's int64
state n = round(N_s f 2^40) (N_g = 16, N_q = 6).

State layout: n[slot][x][p], slots = active species in increasing index
order (0 g, 1 u, 2 d, 3 s, 4 ubar, 5 dbar, 6 sbar), x = (ix, iy, iz) and
p = (jx, jy, jz) row-major with the last index fastest.  Momentum cells
are centred: p_j = -L + (j + 1/2) 2L/n.
"""
from dataclasses import dataclass, field
from typing import Tuple

import numpy as np

NSPEC = 7
SPECIES = ("g", "u", "d", "s", "ubar", "dbar", "sbar")
DEGENERACY = (16.0, 6.0, 6.0, 6.0, 6.0, 6.0, 6.0)
ALL_SPECIES = 0x7F
GLUON_ONLY = 0x01
SCALE = 2.0 ** 40


@dataclass
class Workload:
    name: str
    nx: Tuple[int, int, int]
    dx: float
    np_: Tuple[int, int, int]
    L: float
    species_mask: int
    alpha_s: float
    nsamples: int
    nsteps: int
    dt: float
    seed: int
    f: np.ndarray = field(repr=False)  # float64 [slot][x][p]

    @property
    def nslots(self):
        return bin(self.species_mask).count("1")

    @property
    def nxc(self):
        return int(np.prod(self.nx))

    @property
    def npc(self):
        return int(np.prod(self.np_))

    def state(self):
        return encode(self.f, self.species_mask)


def slots(species_mask):
    return [s for s in range(NSPEC) if species_mask & (1 << s)]


def momentum_centres(np_, L):
    """Cell-centre momenta, shape [npc, 3]."""
    axes = [-L + (np.arange(n) + 0.5) * (2.0 * L / n) for n in np_]
    px, py, pz = np.meshgrid(*axes, indexing="ij")
    return np.stack([px.ravel(), py.ravel(), pz.ravel()], axis=1)


def space_centres(nx, dx):
    """Cell-centre positions of a grid centred on 0, shape [nxc, 3]."""
    axes = [(np.arange(n) + 0.5 - n / 2.0) * dx for n in nx]
    x, y, z = np.meshgrid(*axes, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def encode(f, species_mask):
    """f[slot][x][p] (float64) -> int64 state N_s f 2^40 (round half even)."""
    f = np.asarray(f, dtype=np.float64)
    deg = np.array([DEGENERACY[s] for s in slots(species_mask)]).reshape(-1, 1, 1)
    return np.rint(f * deg * SCALE).astype(np.int64)


def decode(n, species_mask):
    deg = np.array([DEGENERACY[s] for s in slots(species_mask)]).reshape(-1, 1, 1)
    return np.asarray(n, dtype=np.float64) / SCALE / deg


def step_f(np_, L, f0=0.5, Qs=1.0):
    """CGC-like step f0 theta(1 - |p|/Qs) at the cell centres, Eq. (CGC)."""
    p = momentum_centres(np_, L)
    return np.where(np.sqrt((p * p).sum(1)) < Qs, f0, 0.0)


def exp_f(np_, L, a=0.05, T0=0.4):
    p = momentum_centres(np_, L)
    return a * np.exp(-np.sqrt((p * p).sum(1)) / T0)


def equilibrium_f(np_, L, species, T, mu=0.0, m2=0.0):
    """Bose-Einstein (gluons) / Fermi-Dirac (quarks) at the cell centres, Eqs. (fg), (fq)."""
    p = momentum_centres(np_, L)
    E = np.sqrt((p * p).sum(1) + m2)
    x = (E - mu) / T
    return 1.0 / (np.exp(x) + 1.0) if species != 0 else 1.0 / np.expm1(x)


def random_f(np_, nslots, nxc, seed, lo=0.0, hi=1.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(nslots, nxc, int(np.prod(np_))))


# ---------------------------------------------------------------------------
# The workloads of the benchmark configurations.
# ---------------------------------------------------------------------------
def gluon_step_box(n=20, L=2.0, nsamples=64, nsteps=10, dt=0.01, seed=1, f0=0.5, Qs=1.0):
    """Pure gluons, one spatial cell, n^3 momentum grid on [-L, L)^3, step IC."""
    f = step_f((n, n, n), L, f0, Qs).reshape(1, 1, -1)
    return Workload("gluon_step_%d^3_N%d" % (n, nsamples), (1, 1, 1), 1.0, (n, n, n), L,
                    GLUON_ONLY, 0.3, nsamples, nsteps, dt, seed, f)


def qgp_box(n=32, L=3.0, nsamples=1024, nsteps=200, dt=0.005, seed=2):
    """Seven species, one spatial cell: gluons 0.5 theta(1 - |p|), (anti)quarks
    0.05 exp(-|p|/0.4 GeV), each times (1 + 0.01 (2u - 1)), u uniform per cell."""
    np_ = (n, n, n)
    rng = np.random.default_rng(seed)
    f = np.zeros((7, 1, n ** 3))
    f[0, 0] = step_f(np_, L, 0.5, 1.0)
    for s in range(1, 7):
        f[s, 0] = exp_f(np_, L, 0.05, 0.4)
    f *= 1.0 + 0.01 * (2.0 * rng.uniform(size=f.shape) - 1.0)
    return Workload("qgp_7species_%d^3_N%d" % (n, nsamples), (1, 1, 1), 1.0, np_, L,
                    ALL_SPECIES, 0.3, nsamples, nsteps, dt, seed, f)


def gluon_bump_xp(nxs=16, dx=0.2, n=20, L=2.0, nsamples=256, nsteps=100, dt=0.005, seed=3):
    """Pure gluons on an nxs^3 periodic spatial grid: 0.5 theta(1 - |p|) (1 + 0.3 exp(-|x|^2/(2 0.8^2)))."""
    np_ = (n, n, n)
    x = space_centres((nxs,) * 3, dx)
    bump = 1.0 + 0.3 * np.exp(-(x * x).sum(1) / (2.0 * 0.8 ** 2))
    f = (bump[:, None] * step_f(np_, L, 0.5, 1.0)[None, :]).reshape(1, nxs ** 3, n ** 3)
    return Workload("gluon_bump_x%d^3_p%d^3_N%d" % (nxs, n, nsamples), (nxs,) * 3, dx, np_, L,
                    GLUON_ONLY, 0.3, nsamples, nsteps, dt, seed, f)


def batched_boxes(nboxes=64, seed=5, dt=0.01, nsteps=50):
    """Ensemble of independent homogeneous boxes: grids drawn from {12, 16, 20,
    24, 32}^3 on [-2, 2) GeV, species sets from {gluons only, 7 species},
    alpha_s ~ U[0.2, 0.4], Q_s ~ U[0.8, 1.5] GeV, f0 ~ U[0.1, 1.0], samples per
    cell ~ U{256..1024}.  Gluons start as f0 theta(Q_s - |p|), (anti)quarks
    empty.  Returns (list of box dicts, list of int64 states, dt, nsteps)."""
    rng = np.random.default_rng(seed)
    boxes, states = [], []
    for i in range(nboxes):
        n = int(rng.choice([12, 16, 20, 24, 32]))
        mask = ALL_SPECIES if rng.uniform() < 0.5 else GLUON_ONLY
        alpha = float(rng.uniform(0.2, 0.4))
        qs = float(rng.uniform(0.8, 1.5))
        f0 = float(rng.uniform(0.1, 1.0))
        N = int(rng.integers(256, 1025))
        L = 2.0
        f = np.zeros((bin(mask).count("1"), 1, n ** 3))
        f[0, 0] = step_f((n, n, n), L, f0, qs)
        boxes.append({"np_": (n, n, n), "L": L, "species_mask": mask, "nsamples": N, "alpha_s": alpha,
                      "mass_mode": 0, "box_id": i, "seed": seed, "Qs": qs, "f0": f0})
        states.append(encode(f, mask))
    return boxes, states, dt, nsteps
