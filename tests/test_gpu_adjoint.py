"""GPU parity of the adjoint: the inverse X = U^-1 L at p bits and the
binary64 gradient G = A^-T equal the oracle's bit for bit; at the workload
size (N = 512, p = 4096, nearly singular) sampled entries of X A equal the
identity to the rounding bound and the last row of X equals the last-column
minors over the determinant; the torch autograd wrapper returns the same
gradient."""
from fractions import Fraction

import numpy as np
import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def same(a, b):
    return all(np.array_equal(np.asarray(x), np.asarray(y)) for x, y in zip(a, b))


@pytest.mark.parametrize("N,p", [(1, 512), (2, 512), (9, 512), (33, 1024), (20, 4096), (5, 32768)])
def test_adjoint_vs_oracle(mpdet, oracle_lib, N, p):
    A = W.rng(40 + N).standard_normal((N, N))
    h = mpdet.Mpdet(N, p, lastcol=True)
    s, la, G = h.logabsdet_grad(A)
    Xi = h.get_inverse()
    h.close()
    st, zk, D, Xm = oracle_lib.ge(oracle_lib.from_f64(A.reshape(-1), p), N, p, lastcol=True, nthreads=8)
    assert st == 0
    OX = oracle_lib.usolve(Xm, N, p, nthreads=8)
    assert same(Xi, OX), "A^-1 differs from the oracle"
    OG = oracle_lib.to_f64(OX, p).reshape(N, N).T
    assert np.array_equal(G, OG), "binary64 gradient differs from the oracle"
    osg, ola = oracle_lib.logabsdet(D, N, p)
    assert s == osg and la == pytest.approx(ola, rel=0, abs=1e-12)


def test_adjoint_workload_C4(mpdet, oracle_lib):
    """N = 512, p = 4096, the nearly singular Gaussian matrix (det = 1e-30 *
    C_1N): log|det| against numpy's slogdet (binary64, conditioning-limited),
    sampled entries of X A - I at p bits, and the last row of X against the
    last-column minors over the determinant."""
    cfg = W.C4
    N, p = cfg["N"], cfg["p"]
    A = W.nearly_singular_f64(N, cfg["seed"])
    h = mpdet.Mpdet(N, p, lastcol=True)
    s, la, G = h.logabsdet_grad(A)
    Xi = h.get_inverse()
    C = h.lastcol_minors()
    D = h.get_minors()
    h.close()
    assert np.isfinite(la) and np.all(np.isfinite(G))
    det = X.to_fraction(D[0][N - 1], D[1][N - 1], D[2][N - 1], p)
    g = W.rng(1)
    for _ in range(6):  # entries of X A - I
        r, c = int(g.integers(N)), int(g.integers(N))
        acc = sum(X.to_fraction(Xi[0][r * N + j], Xi[1][r * N + j], Xi[2][r * N + j], p) * Fraction(float(A[j, c]))
                  for j in range(N))
        assert abs(acc - (1 if r == c else 0)) < Fraction(1, 2 ** 2000)
    for j in list(range(5)) + [N - 2, N - 1]:  # (A^-1)_Nj = C_jN / det
        xnj = X.to_fraction(Xi[0][(N - 1) * N + j], Xi[1][(N - 1) * N + j], Xi[2][(N - 1) * N + j], p)
        cj = X.to_fraction(C[0][j], C[1][j], C[2][j], p)
        assert abs(xnj - cj / det) <= abs(cj / det) * Fraction(1, 2 ** 2000) + Fraction(1, 2 ** 3000)


def test_torch_autograd_wrapper(mpdet):
    import torch

    N, p = 24, 1024
    A = torch.tensor(W.rng(7).standard_normal((N, N)), dtype=torch.float64, device="cuda", requires_grad=True)
    y = mpdet.mp_logabsdet(A, p)
    (3.0 * y).backward()
    h = mpdet.Mpdet(N, p, lastcol=True)
    s, la, G = h.logabsdet_grad(A.detach().cpu().numpy(), scale=3.0)
    h.close()
    assert float(y.detach()) == la
    assert np.array_equal(A.grad.cpu().numpy(), G)
    ref = torch.linalg.slogdet(A.detach())[1].item()
    assert abs(ref - la) < 1e-9
    assert np.allclose(G, 3.0 * np.linalg.inv(A.detach().cpu().numpy()).T, rtol=1e-8, atol=1e-10)
