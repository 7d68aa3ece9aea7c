"""Pins of the oracle's elimination against mathematics it must reproduce.

* det and leading minors of small integer matrices against exact rational
  determinants computed by the paper's condensation identity (Sec. 3, eq.
  condensation), an independent route to the same numbers;
* the whole rounded operation sequence of Gaussian elimination without
  pivoting re-derived op by op with exact rationals and RNE (brute force on
  tiny inputs);
* Cauchy determinants against their closed form at every k;
* last-column signed minors (eq. minorsdef) against exact cofactors, the
  2x2 hand case, C_NN = D_{N-1} and the Laplace identity det = sum a_jN C_jN;
* structural invariants: the leading K x K block of a run equals a K x K run,
  thread count and step windows do not change any bit, zero pivots stop with
  the documented status.
"""
from fractions import Fraction

import numpy as np
import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.usefixtures("oracle_lib")


def lg2(q: Fraction) -> int:
    """floor-ish log2 of a positive rational (exact enough for bit counts)."""
    return q.numerator.bit_length() - q.denominator.bit_length()


def det_condensation(M):
    """Exact determinant by repeated condensation (Sec. 3, eq. condensation):
    b_ij = a_1l * a_{i+1,j+1} - a_{i+1,l} * a_{1,j+1} with l the first
    non-zero column of row 1 (columns before l give b_ij = -a_{i+1,j} a_1l),
    det A = det B / a_1l^(N-2).  Exact rationals; independent of GE."""
    A = [[Fraction(v) for v in row] for row in M]
    N = len(A)
    scale = Fraction(1)
    sign = 1
    while N > 1:
        l = next((j for j in range(N) if A[0][j] != 0), None)
        if l is None:
            return Fraction(0)
        p = A[0][l]
        # Moving column l to the front changes the sign by (-1)^l.
        if l:
            for row in A:
                row.insert(0, row.pop(l))
            sign *= (-1) ** l
        B = [[p * A[i + 1][j + 1] - A[i + 1][0] * A[0][j + 1] for j in range(N - 1)] for i in range(N - 1)]
        if N > 2:
            scale *= p ** (N - 2)
        A, N = B, N - 1
    return sign * A[0][0] / scale


def exact_leading_minors(M):
    N = len(M)
    return [det_condensation([row[:k] for row in M[:k]]) for k in range(1, N + 1)]


def exact_lastcol_cofactors(M):
    N = len(M)
    out = []
    for j in range(N):
        minor = [row[: N - 1] for i, row in enumerate(M) if i != j]
        out.append((-1) ** (j + N - 1) * (det_condensation(minor) if N > 1 else Fraction(1)))
    return out


def lift_int(oracle, A, p):
    return oracle.from_int(np.asarray(A, np.int64).reshape(-1), p)


def test_condensation_reference_is_a_determinant():
    # sanity of the exact reference itself: a permutation matrix, a triangular
    # matrix and a matrix with a leading zero in row 1
    assert det_condensation([[0, 1], [1, 0]]) == -1
    assert det_condensation([[2, 5, 7], [0, 3, 1], [0, 0, 4]]) == 24
    assert det_condensation([[0, 0, 1], [0, 1, 0], [1, 0, 0]]) == -1
    assert det_condensation([[1, 2, 3], [4, 5, 6], [7, 8, 10]]) == -3


def test_2x2_by_hand(oracle_lib):
    # [[a, b], [c, d]] = [[2, 5], [6, 7]]: D = (2, 2*7 - 5*6 = -16); every op
    # is exact here (z = 3).  Cofactors of the last column: C_12 = -c = -6,
    # C_22 = a = 2.
    p = 128
    A = lift_int(oracle_lib, [[2, 5], [6, 7]], p)
    st, zk, D, Xm = oracle_lib.ge(A, 2, p, lastcol=True)
    assert st == 0 and zk == 0
    assert X.unpack(D, p) == [2, -16]
    assert X.unpack(oracle_lib.lastcol_minors(Xm, D, 2, p), p) == [-6, 2]
    # normalised minors delta = C_j2 / C_12 = (1, -1/3)
    dl = X.unpack(oracle_lib.lastcol_minors(Xm, D, 2, p, normalised=True), p)
    assert dl[0] == 1 and dl[1] == X.unpack(X.pack([Fraction(-1, 3)], p), p)[0]


def brute_force_ge(M, p, lastcol):
    """Op-by-op exact emulation of the elimination with Fractions and RN."""
    N = len(M)
    r = lambda q: X.to_fraction(*X.rn_tuple(q, p), p)
    A = [[r(Fraction(v)) for v in row] for row in M]
    D = []
    prev = Fraction(1)
    for k in range(N):
        prev = r(prev * A[k][k])
        D.append(prev)
        if A[k][k] == 0:
            return D + [Fraction(0)] * (N - k - 1), A
        if k == N - 1:
            break
        rk = r(1 / A[k][k])
        z = {i: r(A[i][k] * rk) for i in range(k + 1, N)}
        for i in range(k + 1, N):
            for j in range(N):
                if j == k or (not lastcol and j < k):
                    continue
                A[i][j] = r(A[i][j] - r(z[i] * A[k][j]))
            if lastcol:
                A[i][k] = -z[i]
    return D, A


@pytest.mark.parametrize("p", [64, 96, 128])
@pytest.mark.parametrize("lastcol", [False, True])
def test_brute_force_op_sequence(oracle_lib, p, lastcol):
    g = W.rng(20 + p)
    for trial in range(12):
        N = int(g.integers(1, 6))
        if trial % 2:
            M = (g.standard_normal((N, N)) * 10.0).tolist()
            A = oracle_lib.from_f64(np.asarray(M).reshape(-1), p)
        else:
            M = g.integers(-9, 10, (N, N)).tolist()
            A = lift_int(oracle_lib, M, p)
        st, zk, D, Xm = oracle_lib.ge(A, N, p, lastcol=lastcol)
        Dw, Aw = brute_force_ge(M, p, lastcol)
        assert X.unpack(D, p) == Dw
        got = X.unpack(Xm, p)
        if st == 0:
            for i in range(N):
                for j in range(N):
                    if j >= i or lastcol:  # the strict lower part is L only in lastcol mode
                        assert got[i * N + j] == Aw[i][j], (trial, i, j)


@pytest.mark.parametrize("N", [3, 5, 8])
def test_integer_minors_vs_exact(oracle_lib, N):
    p = 256
    g = W.rng(100 + N)
    for _ in range(3):
        M = g.integers(-9, 10, (N, N)).tolist()
        st, zk, D, Xm = oracle_lib.ge(lift_int(oracle_lib, M, p), N, p, lastcol=True)
        exact = exact_leading_minors(M)
        if any(v == 0 for v in exact[:-1]):
            continue  # a zero leading minor stops GE without pivoting
        got = X.unpack(D, p)
        for k in range(N):
            if exact[k] == 0:
                assert got[k] == 0 or abs(got[k]) < Fraction(1, 2 ** (p // 2))
            else:
                assert abs(got[k] - exact[k]) <= abs(exact[k]) * Fraction(1, 2 ** (p - 24))
        C = X.unpack(oracle_lib.lastcol_minors(Xm, D, N, p), p)
        Cx = exact_lastcol_cofactors(M)
        scale = max(abs(c) for c in Cx)
        for c, cx in zip(C, Cx):
            assert abs(c - cx) <= scale * Fraction(1, 2 ** (p - 24))
        assert C[-1] == (got[N - 2] if N > 1 else 1)  # C_NN = D_{N-1}, bitwise


def test_cauchy_closed_form_every_k(oracle_lib):
    """Config-1 shape: N = 64, p = 512.  det of the leading k x k Cauchy block
    is prod_{i<j<=k}(x_j-x_i)(y_j-y_i) / prod_{i,j<=k}(x_i+y_j).  The oracle
    works on RN(1/RN(x_i+y_j)), so the agreement decays with k as the matrix
    conditioning amplifies the 2^-p input perturbation: the test requires
    more than p-16 correct bits for k <= 2, a loss of at most 12 bits per
    row, and that the loss grows (monotone within 8 bits)."""
    N, p = W.C1["N"], W.C1["p"]
    x, y = W.cauchy_xy(N, W.C1["seed"])
    st, zk, D, _ = oracle_lib.ge(oracle_lib.cauchy(x, y, p), N, p)
    assert st == 0
    fx = [Fraction(float(v)) for v in x]
    fy = [Fraction(float(v)) for v in y]
    num = den = Fraction(1)
    Dv = X.unpack(D, p)
    bits = []
    for k in range(1, N + 1):
        i = k - 1
        for j in range(i):
            num *= (fx[i] - fx[j]) * (fy[i] - fy[j])
        for j in range(k):
            den *= (fx[i] + fy[j]) * ((fx[j] + fy[i]) if j != i else 1)
        ex = num / den
        assert (Dv[k - 1] > 0) == (ex > 0)
        rel = abs(Dv[k - 1] - ex) / abs(ex)
        b = -lg2(rel) if rel else p + 1
        bits.append(b)
        assert b >= p - 16 - 12 * (k - 1), (k, b)
    assert bits[0] >= p - 2 and bits[1] >= p - 16
    assert all(bits[k] <= bits[k - 8] + 8 for k in range(8, N))


def test_lastcol_integer_cofactors_and_laplace(oracle_lib):
    N, p = 12, 512
    M = W.int_matrix(N, 7)
    Ml = M.tolist()
    st, zk, D, Xm = oracle_lib.ge(lift_int(oracle_lib, Ml, p), N, p, lastcol=True)
    assert st == 0
    C = X.unpack(oracle_lib.lastcol_minors(Xm, D, N, p), p)
    Cx = exact_lastcol_cofactors(Ml)
    for c, cx in zip(C, Cx):
        assert abs(c - cx) <= abs(cx) * Fraction(1, 2 ** (p - 64))
    det = X.unpack(D, p)[-1]
    lap = sum(Fraction(int(M[j, N - 1])) * C[j] for j in range(N))
    assert abs(lap - det) <= sum(abs(Fraction(int(M[j, N - 1])) * C[j]) for j in range(N)) * Fraction(1, 2 ** (p - 64))
    # delta_{N,j} = C_jN / C_1N
    dl = X.unpack(oracle_lib.lastcol_minors(Xm, D, N, p, normalised=True), p)
    for j in range(N):
        assert abs(dl[j] - Cx[j] / Cx[0]) <= abs(Cx[j] / Cx[0]) * Fraction(1, 2 ** (p - 64))


def test_leading_block_equals_standalone(oracle_lib):
    N, K, p = 20, 9, 256
    x, y = W.cauchy_xy(N, 3)
    A = oracle_lib.cauchy(x, y, p)
    _, _, D, _ = oracle_lib.ge(A, N, p)
    _, _, Dk, _ = oracle_lib.ge(oracle_lib.cauchy(x[:K], y[:K], p), K, p)
    assert X.same(tuple(t[:K] for t in D), Dk)


def test_threads_and_windows_do_not_change_bits(oracle_lib):
    N, p = 24, 512
    A = lift_int(oracle_lib, W.int_matrix(N, 5), p)
    ref = oracle_lib.ge(A, N, p, lastcol=True, nthreads=1)
    par = oracle_lib.ge(A, N, p, lastcol=True, nthreads=5)
    assert X.same(ref[2], par[2]) and X.same(ref[3], par[3])
    # run steps [0, 7), then [7, N) from the saved state
    st1, _, D1, X1 = oracle_lib.ge(A, N, p, lastcol=True, k_end=7)
    st2, _, D2, X2 = oracle_lib.ge(X1, N, p, lastcol=True, k0=7, D=D1)
    assert X.same(D2, ref[2]) and X.same(X2, ref[3])


def test_zero_pivots(oracle_lib):
    p = 128
    st, zk, D, _ = oracle_lib.ge(lift_int(oracle_lib, [[0, 1], [1, 0]], p), 2, p)
    assert (st, zk) == (oracle_lib.EZEROPIVOT, 1) and X.unpack(D, p) == [0, 0]
    # a_22 becomes exactly zero after step 1: D_1 valid, D_2 = D_3 = +0
    st, zk, D, _ = oracle_lib.ge(lift_int(oracle_lib, [[1, 2, 3], [2, 4, 5], [1, 1, 1]], p), 3, p)
    assert (st, zk) == (oracle_lib.EZEROPIVOT, 2) and X.unpack(D, p) == [1, 0, 0]
    assert D[1][1] == X.ZEXP and D[0][1] == 0  # canonical +0
    # zero at k = N is a singular matrix, not a failure: det = +0
    st, zk, D, Xm = oracle_lib.ge(lift_int(oracle_lib, [[1, 2], [2, 4]], p), 2, p, lastcol=True)
    assert (st, zk) == (0, 2) and X.unpack(D, p) == [1, 0]
    assert X.unpack(oracle_lib.lastcol_minors(Xm, D, 2, p), p) == [-2, 1]


def test_single_element(oracle_lib):
    p = 64
    st, zk, D, Xm = oracle_lib.ge(oracle_lib.from_f64([-3.5], p), 1, p, lastcol=True)
    assert st == 0 and X.unpack(D, p) == [Fraction(-7, 2)]
    assert X.unpack(oracle_lib.lastcol_minors(Xm, D, 1, p), p) == [1]  # C_11 = D_0 = 1


def test_minor_series_integer_exact(oracle_lib):
    """Series of last-column minors for every leading size (Sec. 3): series n
    against exact cofactors of the leading n x n block's last column, its
    normalised form against C_jn / C_1n, and the Laplace identity per n."""
    N, p = 10, 512
    M = W.int_matrix(N, 11)
    Ml = M.tolist()
    st, zk, D, Xm = oracle_lib.ge(lift_int(oracle_lib, Ml, p), N, p, lastcol=True)
    assert st == 0
    S = X.unpack(oracle_lib.minor_series(Xm, D, N, p), p)
    Sd = X.unpack(oracle_lib.minor_series(Xm, D, N, p, normalised=True), p)
    Dl = X.unpack(D, p)
    tol = Fraction(1, 2 ** (p - 64))
    for nn in range(1, N + 1):
        off = nn * (nn - 1) // 2
        blk = [row[:nn] for row in Ml[:nn]]
        Cx = exact_lastcol_cofactors(blk)
        C = S[off:off + nn]
        for c, cx in zip(C, Cx):
            assert abs(c - cx) <= abs(cx) * tol
        # Laplace along the last column of the n x n block: D_n = sum_j a_jn C_jn
        lap = sum(Fraction(blk[j][nn - 1]) * C[j] for j in range(nn))
        assert abs(lap - Dl[nn - 1]) <= sum(abs(Fraction(blk[j][nn - 1]) * C[j]) for j in range(nn)) * tol
        d = Sd[off:off + nn]
        assert d[0] == 1
        for j in range(nn):
            assert abs(d[j] - Cx[j] / Cx[0]) <= abs(Cx[j] / Cx[0]) * tol


def test_minor_series_equals_standalone_runs(oracle_lib):
    """Series n is bit-identical to the last-column minors of a standalone
    n x n elimination of the leading block (both modes), Cauchy input."""
    N, p = 14, 256
    x, y = W.cauchy_xy(N, 21)
    _, _, D, Xm = oracle_lib.ge(oracle_lib.cauchy(x, y, p), N, p, lastcol=True)
    for normalised in (False, True):
        S = oracle_lib.minor_series(Xm, D, N, p, normalised=normalised)
        for nn in (1, 2, 3, 7, N):
            _, _, Dn, Xn = oracle_lib.ge(oracle_lib.cauchy(x[:nn], y[:nn], p), nn, p, lastcol=True)
            Cn = oracle_lib.lastcol_minors(Xn, Dn, nn, p, normalised=normalised)
            off = nn * (nn - 1) // 2
            assert X.same(tuple(t[off:off + nn] for t in S), Cn)


def test_minor_series_2x2_by_hand(oracle_lib):
    """[[a, b], [c, d]]: series 1 is (1), series 2 the cofactors (-c, a)."""
    p = 128
    A = [[3, 5], [7, 2]]
    _, _, D, Xm = oracle_lib.ge(lift_int(oracle_lib, A, p), 2, p, lastcol=True)
    S = X.unpack(oracle_lib.minor_series(Xm, D, 2, p), p)
    # C^(2)_22 = D_1 = a exactly; C^(2)_12 = RN(a * l_21) = -c within three roundings
    assert S[0] == 1 and S[2] == 3 and abs(S[1] + 7) <= 7 * Fraction(1, 2 ** (p - 3))
    Sd = X.unpack(oracle_lib.minor_series(Xm, D, 2, p, normalised=True), p)
    # delta^(2) = (1, C_22 / C_12) = (1, RN(1/l_21)), l_21 = -RN(c RN(1/a))
    assert Sd[:2] == [1, 1] and abs(Sd[2] - Fraction(3, -7)) <= Fraction(3, 7) * Fraction(1, 2 ** (p - 3))


def test_minor_series_zero_l_n1(oracle_lib):
    """A leading block whose C_1n is zero: its normalised series is all +0,
    the unnormalised one holds the exact (zero) cofactor."""
    p = 128
    # leading 2x2 block [[1, 0], [0, 1]]: l_21 = 0, C^(2)_12 = 0
    A = [[1, 0, 2], [0, 1, 3], [4, 5, 6]]
    _, _, D, Xm = oracle_lib.ge(lift_int(oracle_lib, A, p), 3, p, lastcol=True)
    S = X.unpack(oracle_lib.minor_series(Xm, D, 3, p), p)
    Sd = X.unpack(oracle_lib.minor_series(Xm, D, 3, p, normalised=True), p)
    assert S[1:3] == [0, 1]
    assert Sd[1:3] == [0, 0]
    Cx = exact_lastcol_cofactors(A)
    assert S[3:6] == Cx


def test_oracle_reproduces_stored_values(oracle_lib):
    """The oracle's results for workload C1 (leading and last-column minors)
    equal the stored values written by tests/golden/make_golden.py, number for
    number: any change to the oracle's arithmetic shows here."""
    import os
    import sys

    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
    import make_golden

    want = open(make_golden.GOLDEN).read().splitlines()
    got = make_golden.lines(*make_golden.compute())
    assert got == want


def test_integer_minors_vs_multimodular_exact(oracle_lib):
    """Every leading minor of a 96 x 96 integer matrix (entries in [-1000,
    1000]) against its exact value from elimination modulo many primes and
    Chinese remaindering (an exact route independent of the oracle): at most
    40 bits lost at p = 512, i.e. relative error below 2^-(p-40)."""
    from fractions import Fraction as F

    import bench

    N, p = 96, 512
    A = W.int_matrix(N, 1396)
    exact = bench.exact_leading_minors_int(A, N)
    st, zk, D, _ = oracle_lib.ge(lift_int(oracle_lib, A, p), N, p, nthreads=4)
    assert st == 0
    got = X.unpack(D, p)
    for k in range(N):
        assert exact[k] != 0
        assert abs(got[k] - exact[k]) <= abs(F(exact[k])) / 2 ** (p - 40), k


def test_two_rounding_multiplier_costs_no_accuracy(oracle_lib):
    """Reading G3: the multipliers are RN(a_ik * RN(1/a_kk)), two roundings,
    instead of the correctly rounded RN(a_ik / a_kk).  Against the Cauchy
    closed form at every k the two choices lose the same number of bits per
    row (the matrix's conditioning, about 5 bits per row, dominates one extra
    rounding per multiplier)."""
    import bench

    N, p = W.C1["N"], W.C1["p"]
    x, y = W.cauchy_xy(N, W.C1["seed"])
    A = oracle_lib.cauchy(x, y, p)
    r = {}
    for divide in (False, True):
        st, zk, D, _ = oracle_lib.ge(A, N, p, divide=divide)
        assert st == 0
        r[divide] = bench.cauchy_bit_loss(x, y, D, p, every=8)
    assert abs(r[False]["bits_per_row"] - r[True]["bits_per_row"]) < 0.2
    for a, b in zip(r[False]["per_k"], r[True]["per_k"]):
        assert abs(a["bits"] - b["bits"]) < 12
