"""Seeded synthetic workloads shaped like the paper's experiments.

This module only draws inputs: design X, responses Y, reference locations
Xref, per-location sizes, and the noise-free truth at Xref.  It holds none of
the method's arithmetic, so both the CUDA path and the FP64 oracle may use it.

Draw order for every workload (numpy.random.default_rng(seed)): design X,
then response noise, then reference locations, then per-location sizes.

Workloads (the paper's own data is not available; these stand in for it):
  toy2d      2-d toy surface of Sec. 4 (data of Gramacy & Apley):
             y = x1 exp(-x1^2 - x2^2) + N(0, 0.001^2) on [-2,2]^2.
  borehole   8-d borehole function of Sec. 5.2 on U[0,1]^8 inputs mapped to
             the physical ranges; y standardised by the design mean/sd.
             (The paper used Latin hypercube samples; i.i.d. uniform here.)
  clustered2d  the 2-d toy surface on a design of tight clusters, nugget
             1e-7 (local matrices with cond ~2e8).
  slab3d     3-d nonstationary surface, 70% of the design in the slab
             0.4 < x1 < 0.6, predicted on a 60 x 60 x 56 grid (a synthetic
             stand-in for the LGBB experiment of Sec. 5.1, whose data is not
             available).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    X: np.ndarray          # N x p design (float64 or float32)
    Y: np.ndarray          # N responses (same dtype as X)
    Xref: np.ndarray       # M x p reference locations (same dtype as X)
    truth: np.ndarray      # M noise-free responses at Xref (float64)
    n0: int
    n: np.ndarray          # M final local design sizes (int32)
    Np: np.ndarray         # M candidate-set sizes N' (int32)
    d: float               # lengthscale (starting value when mle is set)
    g: float               # nugget
    mle: tuple | None = None  # (dmin, dmax, max_iter) when the MLE step runs
    meta: dict = field(default_factory=dict)

    @property
    def N(self):
        return self.X.shape[0]

    @property
    def M(self):
        return self.Xref.shape[0]

    @property
    def p(self):
        return self.X.shape[1]


def toy2d_f(X):
    X = np.asarray(X, dtype=np.float64)
    return X[:, 0] * np.exp(-X[:, 0] ** 2 - X[:, 1] ** 2)


def borehole_f(U):
    """Borehole flow rate on unit-cube inputs mapped to the physical ranges."""
    U = np.asarray(U, dtype=np.float64)
    rw = 0.05 + 0.10 * U[:, 0]
    r = 100.0 + (50000.0 - 100.0) * U[:, 1]
    Tu = 63070.0 + (115600.0 - 63070.0) * U[:, 2]
    Hu = 990.0 + (1110.0 - 990.0) * U[:, 3]
    Tl = 63.1 + (116.0 - 63.1) * U[:, 4]
    Hl = 700.0 + (820.0 - 700.0) * U[:, 5]
    L = 1120.0 + (1680.0 - 1120.0) * U[:, 6]
    Kw = 9855.0 + (12045.0 - 9855.0) * U[:, 7]
    lr = np.log(r / rw)
    return 2.0 * np.pi * Tu * (Hu - Hl) / (lr * (1.0 + 2.0 * L * Tu / (lr * rw ** 2 * Kw) + Tu / Tl))


def slab3d_f(X):
    X = np.asarray(X, dtype=np.float64)
    return (np.sin(6.0 * X[:, 1]) + X[:, 2] ** 2
            + 2.0 * (X[:, 0] > 0.5) * np.exp(-5.0 * (X[:, 1] - 0.5) ** 2))


def toy2d(seed=0, N=10_000, M=100, n0=6, n=50, Np=1000, d=0.5, g=1e-4, dtype=np.float64):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-2.0, 2.0, size=(N, 2))
    noise = rng.normal(0.0, 0.001, size=N)
    Xref = rng.uniform(-2.0, 2.0, size=(M, 2))
    Y = toy2d_f(X) + noise
    return Workload("toy2d", X.astype(dtype), Y.astype(dtype), Xref.astype(dtype), toy2d_f(Xref),
                    n0, np.full(M, n, np.int32), np.full(M, Np, np.int32), d, g)


def clustered2d(seed=5, N=20_000, M=40, clusters=1000, spread=0.02, n0=6, n=30, Np=300, d=0.05, g=1e-7,
                dtype=np.float64):
    """The 2-d toy surface on a design of tight clusters (each point within
    `spread` of one of `clusters` uniform centres) with a tiny nugget: local
    matrices with cond ~2e8, the hard case for a reduced-precision screen.
    (At g = 1e-8 the FP64 method itself breaks down on this design: m_j^{-1}
    of Eq. (piedef) evaluates <= 0 in FP64 at almost every location.)"""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-2.0, 2.0, size=(clusters, 2))
    X = centres[rng.integers(0, clusters, N)] + rng.uniform(-spread, spread, size=(N, 2))
    noise = rng.normal(0.0, 0.001, size=N)
    Xref = rng.uniform(-2.0, 2.0, size=(M, 2))
    Y = toy2d_f(X) + noise
    return Workload("clustered2d", X.astype(dtype), Y.astype(dtype), Xref.astype(dtype), toy2d_f(Xref),
                    n0, np.full(M, n, np.int32), np.full(M, Np, np.int32), d, g)


def borehole(seed=1, N=100_000, M=10_000, n0=6, n=50, Np=1000, d=2.0, g=1e-6,
             dtype=np.float64, n_range=None, Np_range=None, mle=None):
    """Borehole workload.  n_range / Np_range = (lo, hi) draw per-location
    sizes uniformly from {lo..hi} (the batched uneven configuration)."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, size=(N, 8))
    # the borehole function is deterministic; no noise draw is consumed
    Xref = rng.uniform(0.0, 1.0, size=(M, 8))
    f = borehole_f(X)
    mu, sd = f.mean(), f.std()
    Y = (f - mu) / sd
    truth = (borehole_f(Xref) - mu) / sd
    n_arr = (rng.integers(n_range[0], n_range[1] + 1, size=M).astype(np.int32)
             if n_range else np.full(M, n, np.int32))
    Np_arr = (rng.integers(Np_range[0], Np_range[1] + 1, size=M).astype(np.int32)
              if Np_range else np.full(M, Np, np.int32))
    return Workload("borehole", X.astype(dtype), Y.astype(dtype), Xref.astype(dtype), truth, n0,
                    n_arr, Np_arr, d, g, mle, meta=dict(y_mean=mu, y_sd=sd))


def slab3d(seed=3, N=500_000, grid=(60, 60, 56), n0=6, n=60, Np=1500, d=0.05, g=1e-4,
           dtype=np.float32, mle=(1e-3, 20.0, 10)):
    rng = np.random.default_rng(seed)
    n_slab = int(round(0.7 * N))
    slab = rng.uniform(0.0, 1.0, size=(n_slab, 3))
    slab[:, 0] = 0.4 + 0.2 * slab[:, 0]
    rest = rng.uniform(0.0, 1.0, size=(N - n_slab, 3))
    # x1 uniform on [0, 0.4) U (0.6, 1]: map a U[0,0.8) draw around the slab
    u = rest[:, 0] * 0.8
    rest[:, 0] = np.where(u < 0.4, u, u + 0.2)
    X = np.concatenate([slab, rest])
    noise = rng.normal(0.0, 0.01, size=N)
    g1, g2, g3 = (np.linspace(0.0, 1.0, k) for k in grid)
    Xref = np.stack(np.meshgrid(g1, g2, g3, indexing="ij"), -1).reshape(-1, 3)
    Y = slab3d_f(X) + noise
    M = Xref.shape[0]
    return Workload("slab3d", X.astype(dtype), Y.astype(dtype), Xref.astype(dtype),
                    slab3d_f(Xref), n0, np.full(M, n, np.int32), np.full(M, Np, np.int32), d, g,
                    mle)


# The five configurations of the benchmark specification, by name.
def c1_toy2d_fp64(**kw):
    """2-d toy, N=10,000, M=100, (n0, n, N') = (6, 50, 1000), d=0.5, g=1e-4."""
    return toy2d(seed=0, **kw)


def c2_borehole_100k(**kw):
    """Borehole, N=100,000, M=10,000, (6, 50, 1000), d=2.0, g=1e-6."""
    return borehole(seed=1, **kw)


def c3_borehole_1m_uneven(**kw):
    """Borehole, N=1,000,000 FP32, M=20,000, n~U{30..100}, N'~U{500..2000},
    Newton MLE of d from 2.0 within [1e-3, 20], <= 10 iterations."""
    args = dict(seed=2, N=1_000_000, M=20_000, dtype=np.float32, n_range=(30, 100),
                Np_range=(500, 2000), mle=(1e-3, 20.0, 10))
    args.update(kw)
    return borehole(**args)


def c4_slab3d(**kw):
    """Nonstationary 3-d, N=500,000 FP32, 60x60x56 grid, (6, 60, 1500), MLE."""
    return slab3d(seed=3, **kw)


def c5_borehole_4m(**kw):
    """Borehole, N=4,000,000 FP32, M=100,000, (6, 50, 2000), MLE."""
    args = dict(seed=4, N=4_000_000, M=100_000, Np=2000, dtype=np.float32,
                mle=(1e-3, 20.0, 10))
    args.update(kw)
    return borehole(**args)


CONFIGS = {
    "c1_toy2d_fp64": c1_toy2d_fp64,
    "c2_borehole_100k": c2_borehole_100k,
    "c3_borehole_1m_uneven": c3_borehole_1m_uneven,
    "c4_slab3d": c4_slab3d,
    "c5_borehole_4m": c5_borehole_4m,
}
