"""Pins of the oracle's adjoint: X = U^-1 L must be A^-1 (exact inverses of
small integer matrices), its last row must be C_jN / det (the last-column
minors over the determinant, eq. minorsdef), it must match p-bit central
finite differences of log|det|, and the binary64 rounding must agree with
Python's correctly rounded float(Fraction)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.usefixtures("oracle_lib")


def exact_inverse(M):
    N = len(M)
    A = [[Fraction(v) for v in row] + [Fraction(int(i == j)) for j in range(N)] for i, row in enumerate(M)]
    for c in range(N):
        piv = next(r for r in range(c, N) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        f = A[c][c]
        A[c] = [v / f for v in A[c]]
        for r in range(N):
            if r != c and A[r][c] != 0:
                g = A[r][c]
                A[r] = [a - g * b for a, b in zip(A[r], A[c])]
    return [row[N:] for row in A]


def factor_lastcol(oracle, M, p):
    N = len(M)
    A = oracle.from_f64(np.asarray(M, np.float64).reshape(-1), p)
    st, zk, D, Xm = oracle.ge(A, N, p, lastcol=True)
    if st != 0 or zk != 0:
        return None, None
    return D, Xm


@pytest.mark.parametrize("N", [1, 2, 3, 6])
def test_usolve_is_the_inverse(oracle_lib, N):
    p = 256
    g = W.rng(300 + N)
    for _ in range(3):
        M = g.integers(-9, 10, (N, N))
        try:
            inv = exact_inverse(M.tolist())
        except StopIteration:
            continue
        D, Xm = factor_lastcol(oracle_lib, M, p)
        if D is None:
            continue  # a zero leading minor: no elimination without pivoting
        Xi = X.unpack(oracle_lib.usolve(Xm, N, p), p)
        scale = max(abs(v) for row in inv for v in row)
        for i in range(N):
            for j in range(N):
                assert abs(Xi[i * N + j] - inv[i][j]) <= scale * Fraction(1, 2 ** (p - 32))


def test_last_row_is_lastcol_minors_over_det(oracle_lib):
    N, p = 10, 512
    M = W.int_matrix(N, 11)
    D, Xm = factor_lastcol(oracle_lib, M, p)
    Xi = X.unpack(oracle_lib.usolve(Xm, N, p), p)
    C = X.unpack(oracle_lib.lastcol_minors(Xm, D, N, p), p)
    det = X.to_fraction(D[0][N - 1], D[1][N - 1], D[2][N - 1], p)
    for j in range(N):
        want = C[j] / det  # d log|det| / dA_jN = C_jN / det = (A^-1)_Nj
        assert abs(Xi[(N - 1) * N + j] - want) <= abs(want) * Fraction(1, 2 ** (p - 48)) + Fraction(1, 2 ** (p // 2))


def test_finite_differences_of_logabsdet(oracle_lib):
    """Central differences of log|det| at p bits, h = 2^-40 relative:
    (log|det(A + h E_ij)| - log|det(A - h E_ij)|) / 2h = (A^-T)_ij + O(h^2)."""
    N, p = 6, 512
    A = W.rng(12).standard_normal((N, N))
    D, Xm = factor_lastcol(oracle_lib, A, p)
    Xi = X.unpack(oracle_lib.usolve(Xm, N, p), p)
    h = 2.0 ** -40

    def logdet(M):
        st, zk, Dd, _ = oracle_lib.ge(oracle_lib.from_f64(M.reshape(-1), p), N, p)
        d = X.to_fraction(Dd[0][N - 1], Dd[1][N - 1], Dd[2][N - 1], p)
        # log of a rational to ~1e-30 relative: use the exact ratio of the two determinants
        return d

    for (i, j) in ((0, 0), (2, 5), (5, 3), (4, 4)):
        Ap, Am = A.copy(), A.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        dp, dm = logdet(Ap), logdet(Am)
        hp = Fraction(float(Ap[i, j])) - Fraction(float(A[i, j]))
        hm = Fraction(float(A[i, j])) - Fraction(float(Am[i, j]))
        assert hp == hm == Fraction(h)
        # log(dp/dm) / 2h with log(1+u) = u - u^2/2 + ..., u = dp/dm - 1 = O(h)
        u = dp / dm - 1
        fd = (u - u * u / 2 + u ** 3 / 3) / (2 * Fraction(h))
        grad = Xi[j * N + i]  # (A^-T)_ij = (A^-1)_ji
        assert abs(fd - grad) <= abs(grad) * Fraction(1, 2 ** 60) + Fraction(1, 2 ** 60)


def test_to_f64_is_correctly_rounded(oracle_lib):
    p = 128
    g = W.rng(99)
    vals = []
    for _ in range(300):
        m = (1 << (p - 1)) | int.from_bytes(g.bytes(p // 8), "little") & ((1 << (p - 1)) - 1)
        e = int(g.integers(-1200, 1200))
        vals.append(Fraction(m) * Fraction(2) ** (e - p) * (-1 if g.integers(0, 2) else 1))
    # ties at the binary64 boundary, the smallest subnormal, the largest finite
    vals += [Fraction(1) + Fraction(1, 2 ** 53), Fraction(1) + Fraction(3, 2 ** 53), Fraction(1, 2 ** 1075),
             Fraction(3, 2 ** 1076), Fraction(2 ** 1024 - 2 ** 970), Fraction(1, 2 ** 1022) * (1 - Fraction(1, 2 ** 60))]
    # just above half the smallest subnormal: one rounding gives 2^-1074; rounding to 53 bits first and
    # then to the subnormal grid gives a tie and 0 (the subnormal quantum must be applied directly)
    vals += [Fraction(1, 2 ** 1075) * (1 + Fraction(1, 2 ** 59)), Fraction(5, 2 ** 1060) * (1 + Fraction(1, 2 ** 70))]
    packed = X.pack(vals, p)
    got = oracle_lib.to_f64(packed, p)
    for v, gv in zip(X.unpack(packed, p), got):
        try:
            want = float(v)
        except OverflowError:
            want = math.inf if v > 0 else -math.inf
        assert gv == want or (gv == 0 and want == 0), (v, gv, want)
        if want == 0:
            assert math.copysign(1, gv) == math.copysign(1, want) or v == 0


def test_logabsdet_helper(oracle_lib):
    p = 256
    for M, want in (([[2, 0], [0, 3]], math.log(6)), ([[0.5, 1], [1, 0.5]], math.log(0.75))):
        D, Xm = factor_lastcol(oracle_lib, M, p)
        s, la = oracle_lib.logabsdet(D, len(M), p)
        assert abs(la - want) < 1e-15
        assert s == (1.0 if np.linalg.det(np.array(M, float)) > 0 else -1.0)


def brute_force_usolve(Aw, p):
    """Op-by-op exact emulation of the back substitution X = U^-1 L with
    Fractions and RN, in reading G12's order (right-looking, bottom row
    first): S = L (unit diagonal, zero above); for k = N..1 the row
    X_k. = RN(S_k. * RN(1/u_kk)), then S_ic = RN(S_ic - RN(u_ik * X_kc)) for
    every i < k and every column c.  Aw is the eliminated array of
    brute_force_ge in last-column mode (U on and above the diagonal, L
    below)."""
    N = len(Aw)
    r = lambda q: X.to_fraction(*X.rn_tuple(q, p), p)
    S = [[Aw[i][j] if j < i else Fraction(int(i == j)) for j in range(N)] for i in range(N)]
    for k in reversed(range(N)):
        rk = r(1 / Aw[k][k])
        S[k] = [r(v * rk) for v in S[k]]
        for i in range(k):
            S[i] = [r(S[i][c] - r(Aw[i][k] * S[k][c])) for c in range(N)]
    return S


@pytest.mark.parametrize("p", [64, 96, 128])
def test_usolve_brute_force_op_sequence(oracle_lib, p):
    """The oracle's back substitution performs exactly the rounded operations
    of reading G12 in that order: every entry of X equals the brute-force
    emulation bit for bit (the inverse and finite-difference pins above only
    bound the error, which a different order or rounding would also meet)."""
    from test_oracle_ge import brute_force_ge

    g = W.rng(500 + p)
    done = 0
    for trial in range(40):
        N = int(g.integers(1, 6))
        M = (g.standard_normal((N, N)) * 10.0).tolist() if trial % 2 else g.integers(-9, 10, (N, N)).tolist()
        D, Xm = factor_lastcol(oracle_lib, M, p)
        if D is None:
            continue
        Dw, Aw = brute_force_ge(M, p, lastcol=True)
        assert X.unpack(Xm, p) == [v for row in Aw for v in row]
        want = brute_force_usolve(Aw, p)
        got = X.unpack(oracle_lib.usolve(Xm, N, p), p)
        for i in range(N):
            for c in range(N):
                assert got[i * N + c] == want[i][c], (trial, N, i, c)
        done += 1
    assert done >= 25
