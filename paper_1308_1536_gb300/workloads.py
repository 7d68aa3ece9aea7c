"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds generators only: it draws random numbers with numpy's PCG64
and does none of the method's arithmetic (no lifting, no rounding, no
elimination).  Both the CUDA path and the CPU oracle consume its output.

The paper's matrices (eq. det and eq. betaNew) need high-accuracy zeta zeros
that are not available here; nearly singular seeded matrices with the same
shape stand in for them:

* Cauchy matrices A_ij = 1/(x_i + y_j) with x, y in (0, 1] sorted and
  distinct: their determinant has a closed form and they are extremely
  ill-conditioned, like the interpolating matrices of Sec. 2.
* Integer matrices with entries uniform in [-1000, 1000]: exact determinants
  and cofactors are known by modular arithmetic.
* Gaussian f64 matrices with an exact near rank deficiency (det = 1e-30 times
  a cofactor) for the adjoint.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1308

# The five workloads (seed = SEED_BASE + workload number).
C1 = dict(name="cauchy_N64_p512", N=64, p=512, seed=SEED_BASE + 1)
C2 = dict(name="cauchy_and_int_N1024_p2048_lastcol", N=1024, p=2048, seed=SEED_BASE + 2)
C3 = dict(name="batch_4096_N8-256_p1024", count=4096, Nmin=8, Nmax=256, p=1024, seed=SEED_BASE + 3)
C4 = dict(name="adjoint_N512_p4096", N=512, p=4096, seed=SEED_BASE + 4)
C5 = dict(name="cauchy_N4096_p32768", N=4096, p=32768, seed=SEED_BASE + 5)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def cauchy_xy(N: int, seed: int, g: np.random.Generator | None = None):
    """x, y: N doubles each, 1 - U[0,1) (so in (0, 1]), sorted ascending,
    all distinct within each vector (redrawn until they are)."""
    g = rng(seed) if g is None else g
    out = []
    for _ in range(2):
        while True:
            v = np.sort(1.0 - g.random(N))
            if N < 2 or np.all(np.diff(v) > 0):
                break
        out.append(v)
    return out[0], out[1]


def int_matrix(N: int, seed: int, lo: int = -1000, hi: int = 1000, g: np.random.Generator | None = None):
    """N x N int64 matrix, entries uniform in [lo, hi]."""
    g = rng(seed) if g is None else g
    return g.integers(lo, hi + 1, size=(N, N), dtype=np.int64)


def nearly_singular_f64(N: int, seed: int, eps: float = 1e-30):
    """N(0,1) matrix with an exact near rank deficiency: G[0, N-2] = 0,
    column N-1 := column N-2, then G[0, N-1] = eps, so that
    det = eps * C_{1N} (cofactor of entry (1, N))."""
    g = rng(seed)
    G = g.standard_normal((N, N))
    if N >= 2:
        G[0, N - 2] = 0.0
        G[:, N - 1] = G[:, N - 2]
        G[0, N - 1] = eps
    return G


def batch_sizes(count: int, Nmin: int, Nmax: int, seed: int):
    """Sizes N uniform in [Nmin, Nmax] and, per matrix, its kind: even index
    Cauchy, odd index integer; plus one derived seed per matrix."""
    g = rng(seed)
    Ns = g.integers(Nmin, Nmax + 1, size=count, dtype=np.int64)
    seeds = g.integers(0, 2**62, size=count, dtype=np.int64)
    kinds = np.array(["cauchy" if i % 2 == 0 else "int" for i in range(count)])
    return Ns, kinds, seeds


def batch_inputs(count: int, Nmin: int, Nmax: int, seed: int, which=None):
    """Per-matrix raw inputs for the batch workload: list of
    ("cauchy", (x, y)) or ("int", A) for the selected indices."""
    Ns, kinds, seeds = batch_sizes(count, Nmin, Nmax, seed)
    idx = range(count) if which is None else which
    out = []
    for i in idx:
        N = int(Ns[i])
        if kinds[i] == "cauchy":
            out.append(("cauchy", cauchy_xy(N, int(seeds[i]))))
        else:
            out.append(("int", int_matrix(N, int(seeds[i]))))
    return out
