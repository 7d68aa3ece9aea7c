"""The method on the paper's own interpolating matrix (eq. det), at small N,
on CPU: Delta_N has entries beta_i(gamma_j) built from the first nontrivial
zeta zeros gamma_j (computed here with mpmath, not taken from any table).
The oracle's leading minors are compared with high-precision determinants of
the same p-bit matrix; Sec. 4.3 reports a loss of about 1.4 bits per row
operation for this matrix (0.42 decimal digits per row, fitted over large N
at 8192 bits).  At N = 24 the measured loss per row stays within that figure,
and the leading minors decay as the paper describes (the matrices are nearly
singular).  Needs mpmath; no GPU."""
from fractions import Fraction

import pytest

import exactref as X

pytestmark = pytest.mark.usefixtures("oracle_lib")


def beta(mp, n, t):
    """beta_n(t) of Sec. 2: minus twice the real part of
    pi^(-1/4 + it/2) (t^2 + 1/4) Gamma(1/4 - it/2) / (4 n^(1/2 - it))."""
    z = (mp.power(mp.pi, -mp.mpf(1) / 4 + 1j * t / 2) * (t * t + mp.mpf(1) / 4) * mp.gamma(mp.mpf(1) / 4 - 1j * t / 2)
         / (4 * mp.power(n, mp.mpf(1) / 2 - 1j * t)))
    return -2 * z.real


def test_bit_loss_on_the_interpolating_matrix(oracle_lib):
    mp = pytest.importorskip("mpmath").mp
    N, p = 24, 512
    mp.dps = p // 3 + 40
    g = [mp.zetazero(j).imag for j in range(1, N + 1)]
    vals = []
    for i in range(1, N + 1):
        for j in range(N):
            m, e = mp.frexp(beta(mp, i, g[j]))
            vals.append(Fraction(int(mp.floor(m * mp.mpf(2) ** (p + 8)))) * Fraction(2) ** (int(e) - p - 8))
    A = X.pack(vals, p)
    Av = X.unpack(A, p)
    st, zk, D, _ = oracle_lib.ge(A, N, p, nthreads=4)
    assert st == 0
    Dv = X.unpack(D, p)
    mp.dps = p + 60
    ks, losses, mags = [], [], []
    for k in range(1, N + 1):
        B = mp.matrix([[mp.mpf(Av[i * N + j].numerator) / Av[i * N + j].denominator for j in range(k)]
                       for i in range(k)])
        d = mp.det(B)
        got = mp.mpf(Dv[k - 1].numerator) / Dv[k - 1].denominator
        rel = abs(got - d) / abs(d)
        bits = float(-mp.log(rel, 2)) if rel else p + 1.0
        ks.append(k)
        losses.append(p - bits)
        mags.append(float(mp.log10(abs(d))))
    kb, lb = sum(ks) / N, sum(losses) / N
    slope = sum((a - kb) * (b - lb) for a, b in zip(ks, losses)) / sum((a - kb) ** 2 for a in ks)
    assert 0.0 < slope <= 1.4, slope
    assert max(losses) < 0.1 * p
    # nearly singular: the leading minors fall by ever larger factors per row
    steps = [mags[k] - mags[k + 1] for k in range(N - 1)]
    assert mags[-1] < -250 and steps[-1] > steps[0] > 0
