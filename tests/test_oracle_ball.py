"""Pins of the oracle's ball mode (values with rigorous radii, the bounds the
paper leaves to future work in Sec. 4.4):

* the radius arithmetic against exact rationals: every operation is the
  exact result rounded up (or down) to a 32-bit mantissa, checked against a
  rounding written here from that definition;
* the values of the ball elimination are the plain elimination's bit for bit;
* containment: exact leading minors (condensation, eq. condensation), exact
  last-column cofactors and normalised minors, the Cauchy closed form at every
  k, and every entry of the exactly eliminated array lie within value +-
  radius;
* brute force: the radius recurrences re-derived op by op with Fractions
  (RU32 after every operation, in the stated order) equal the oracle's radii
  bit for bit on tiny matrices.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W
from test_oracle_ge import brute_force_ge, det_condensation, exact_lastcol_cofactors, exact_leading_minors

pytestmark = pytest.mark.usefixtures("oracle_lib")

ZEXP = np.iinfo(np.int64).min
RAD_INF = np.iinfo(np.int64).max


def rad_value(m, e):
    if int(m) == 0:
        return Fraction(0)
    assert int(e) != RAD_INF
    return Fraction(int(m)) * Fraction(2) ** (int(e) - 32)


def r32(v: Fraction, up: bool):
    """v >= 0 rounded up (or down) to m * 2^(e-32), 2^31 <= m < 2^32."""
    if v == 0:
        return 0, ZEXP
    e = v.numerator.bit_length() - v.denominator.bit_length() + 1
    while v >= Fraction(2) ** e:
        e += 1
    while v < Fraction(2) ** (e - 1):
        e -= 1
    s = v * Fraction(2) ** (32 - e)
    m = math.ceil(s) if up else math.floor(s)
    if m == 1 << 32:
        m, e = 1 << 31, e + 1
    return m, e


def rand_rad(g):
    return int(g.integers(1 << 31, 1 << 32)), int(g.integers(-300, 300))


def test_radius_arithmetic_rounds_as_defined(oracle_lib):
    g = W.rng(91)
    cases = [(rand_rad(g), rand_rad(g)) for _ in range(400)]
    # equal exponents, gaps at and around 31/32/63/64 bits, all-ones mantissas
    for d in (0, 1, 30, 31, 32, 33, 62, 63, 64, 65, 200):
        cases.append(((0xFFFFFFFF, 10), (0xFFFFFFFF, 10 - d)))
        cases.append(((0x80000000, 10), (0x80000001, 10 - d)))
    cases.append(((0x80000000, 5), (0, ZEXP)))
    for a, b in cases:
        va, vb = rad_value(*a), rad_value(*b)
        got, _ = oracle_lib.rad_op(0, a, b)
        assert got == r32(va + vb, True), (a, b)
        got, _ = oracle_lib.rad_op(1, a, b)
        assert got == r32(va * vb, True), (a, b)
        got, _ = oracle_lib.rad_op(2, a, b)
        assert got == r32(va * vb, False), (a, b)
        if vb:
            got, _ = oracle_lib.rad_op(3, a, b)
            assert got == r32(va / vb, True), (a, b)
        got, pos = oracle_lib.rad_op(4, a, b)
        assert pos == (va > vb)
        if va > vb:
            assert got == r32(va - vb, False), (a, b)


@pytest.mark.parametrize("lastcol", [False, True])
def test_ball_values_are_the_plain_elimination(oracle_lib, lastcol):
    N, p = 20, 512
    x, y = W.cauchy_xy(N, 3)
    A, RA = oracle_lib.cauchy_ball(x, y, p)
    assert X.same(A, oracle_lib.cauchy(x, y, p))
    st, zk, D, Xm, RD, RX = oracle_lib.ge_ball(A, RA, N, p, lastcol=lastcol)
    st2, zk2, D2, X2 = oracle_lib.ge(A, N, p, lastcol=lastcol)
    assert (st, zk) == (st2, zk2) and X.same(D, D2) and X.same(Xm, X2)


def contained(v, exact, m, e):
    return abs(exact - v) <= rad_value(m, e)


@pytest.mark.parametrize("N", [2, 4, 7])
def test_ball_contains_exact_integer_minors_and_cofactors(oracle_lib, N):
    p = 128
    g = W.rng(400 + N)
    done = 0
    for _ in range(6):
        M = g.integers(-9, 10, (N, N)).tolist()
        ex = exact_leading_minors(M)
        if any(v == 0 for v in ex[:-1]):
            continue
        A = oracle_lib.from_int(np.asarray(M).reshape(-1), p)
        st, zk, D, Xm, RD, RX = oracle_lib.ge_ball(A, None, N, p, lastcol=True)
        got = X.unpack(D, p)
        for k in range(N):
            assert contained(got[k], ex[k], RD[0][k], RD[1][k]), k
        C, RC = oracle_lib.lastcol_ball(Xm, RX, D, RD, N, p)
        Cx = exact_lastcol_cofactors(M)
        for j, (c, cx) in enumerate(zip(X.unpack(C, p), Cx)):
            assert contained(c, cx, RC[0][j], RC[1][j]), j
        if Cx[0] != 0:
            Dl, RDl = oracle_lib.lastcol_ball(Xm, RX, D, RD, N, p, normalised=True)
            for j, dv in enumerate(X.unpack(Dl, p)):
                if int(RDl[1][j]) != RAD_INF:
                    assert contained(dv, Cx[j] / Cx[0], RDl[0][j], RDl[1][j]), j
        done += 1
    assert done >= 2


def test_ball_contains_exact_f64_determinants(oracle_lib):
    p = 96
    g = W.rng(77)
    for N in (3, 5, 6):
        Mf = g.standard_normal((N, N))
        A = oracle_lib.from_f64(Mf.reshape(-1), p)
        st, zk, D, Xm, RD, RX = oracle_lib.ge_ball(A, None, N, p)
        ex = exact_leading_minors([[Fraction(float(v)) for v in row] for row in Mf])
        for k, (d, dx) in enumerate(zip(X.unpack(D, p), ex)):
            assert contained(d, dx, RD[0][k], RD[1][k]), (N, k)


def test_ball_contains_every_entry_of_the_exact_elimination(oracle_lib):
    """The in-place array after elimination in last-column mode, exactly:
    U and L of exact Gaussian elimination without pivoting of the same input
    (Fractions), entry by entry within the oracle's value +- radius."""
    N, p = 6, 64
    x, y = W.cauchy_xy(N, 11)
    A, RA = oracle_lib.cauchy_ball(x, y, p)
    st, zk, D, Xm, RD, RX = oracle_lib.ge_ball(A, RA, N, p, lastcol=True)
    ex = [[1 / (Fraction(float(x[i])) + Fraction(float(y[j]))) for j in range(N)] for i in range(N)]
    for k in range(N - 1):
        for i in range(k + 1, N):
            z = ex[i][k] / ex[k][k]
            for j in range(N):
                if j != k:
                    ex[i][j] -= z * ex[k][j]
            ex[i][k] = -z
    got = X.unpack(Xm, p)
    for i in range(N):
        for j in range(N):
            assert contained(got[i * N + j], ex[i][j], RX[0][i * N + j], RX[1][i * N + j]), (i, j)


def test_ball_contains_the_cauchy_closed_form_at_every_k(oracle_lib):
    """Workload C1 (Cauchy N = 64, p = 512): det of every leading k x k block
    in closed form, prod_{i<j}(x_j-x_i)(y_j-y_i) / prod(x_i+y_j), lies within
    D_k +- radius while the radius is bounded; the radius certifies fewer
    bits than are actually correct (interval bounds are pessimistic, Sec.
    4.4): measured here, about 12.4 bits per row against the 4.9 actually
    lost, and unbounded from k = 41 on (a pivot's ball then holds zero)."""
    cfg = W.C1
    N, p = cfg["N"], cfg["p"]
    x, y = W.cauchy_xy(N, cfg["seed"])
    A, RA = oracle_lib.cauchy_ball(x, y, p)
    st, zk, D, Xm, RD, RX = oracle_lib.ge_ball(A, RA, N, p)
    got = X.unpack(D, p)
    xs = [Fraction(float(v)) for v in x]
    ys = [Fraction(float(v)) for v in y]
    num, den = Fraction(1), Fraction(1)
    for k in range(1, N + 1):
        i = k - 1
        for j in range(i):
            num *= (xs[i] - xs[j]) * (ys[i] - ys[j])
        for j in range(k):
            den *= xs[i] + ys[j]
            if j != i:
                den *= xs[j] + ys[i]
        det = num / den
        if int(RD[1][i]) == RAD_INF:
            assert k > 32
            continue
        r = rad_value(RD[0][i], RD[1][i])
        assert abs(got[i] - det) <= r, k
        certified = -math.log2(r / abs(det)) if r else p
        actual = -math.log2(abs(got[i] - det) / abs(det)) if got[i] != det else p
        assert certified <= actual + 1
        assert certified >= p - 13 * k  # no more than 13 bits per row lost in the bound here


# ---------------------------------------------------------------------------
# brute force of the radius recurrences
# ---------------------------------------------------------------------------
def rv(r):
    return rad_value(*r)


def ru(v):
    return r32(v, True)


def rd(v):
    return r32(v, False)


def mag(q: Fraction, p: int, up: bool):
    """|q| rounded to the 32-bit grid of its binade (from the top limb)."""
    return r32(abs(q), up)


def hu(u: Fraction, p: int):
    if u == 0:
        return 0, ZEXP
    e = abs(u).numerator.bit_length() - abs(u).denominator.bit_length() + 1
    while abs(u) >= Fraction(2) ** e:
        e += 1
    while abs(u) < Fraction(2) ** (e - 1):
        e -= 1
    return 1 << 31, e - p


INF = "inf"


def radd(a, b):
    if a == INF or b == INF:
        return INF
    return ru(rv(a) + rv(b))


def rmul(a, b, up=True):
    if (a != INF and a[0] == 0) or (b != INF and b[0] == 0):
        return 0, ZEXP
    if a == INF or b == INF:
        return INF
    return ru(rv(a) * rv(b)) if up else rd(rv(a) * rv(b))


def bmul(u, x, rx, y, ry, p):
    r = radd(hu(u, p), rmul(mag(x, p, True), ry))
    r = radd(r, rmul(mag(y, p, True), rx))
    return radd(r, rmul(rx, ry))


def bsub(u, rx, rt, p):
    return radd(radd(hu(u, p), rx), rt)


def brecip(u, a, ra, p):
    lo = mag(a, p, False)
    if ra == INF or rv(ra) >= rv(lo):
        return INF
    gap = rd(rv(lo) - rv(ra))
    den = rmul(lo, gap, up=False)
    return radd(hu(u, p), (0, ZEXP) if ra[0] == 0 else ru(rv(ra) / rv(den)))


def brute_force_ball(M, p, lastcol):
    """The elimination of brute_force_ge with the radius rules applied op by
    op (exact input: radius 0); returns the radii of D and of the array."""
    N = len(M)
    r = lambda q: X.to_fraction(*X.rn_tuple(q, p), p)
    A = [[r(Fraction(v)) for v in row] for row in M]
    R = [[(0, ZEXP)] * N for _ in range(N)]
    RDv = []
    prev, rprev = Fraction(1), (0, ZEXP)
    for k in range(N):
        d = r(prev * A[k][k])
        rprev = bmul(d, prev, rprev, A[k][k], R[k][k], p)
        prev = d
        RDv.append(rprev)
        if A[k][k] == 0 or k == N - 1:
            break
        rk = r(1 / A[k][k])
        rrk = brecip(rk, A[k][k], R[k][k], p)
        z = {i: r(A[i][k] * rk) for i in range(k + 1, N)}
        rz = {i: bmul(z[i], A[i][k], R[i][k], rk, rrk, p) for i in range(k + 1, N)}
        for i in range(k + 1, N):
            for j in range(N):
                if j == k or (not lastcol and j < k):
                    continue
                t = r(z[i] * A[k][j])
                rt = bmul(t, z[i], rz[i], A[k][j], R[k][j], p)
                u = r(A[i][j] - t)
                R[i][j] = bsub(u, R[i][j], rt, p)
                A[i][j] = u
            if lastcol:
                A[i][k] = -z[i]
                R[i][k] = rz[i]
    return RDv, R


@pytest.mark.parametrize("p", [64, 96, 128])
@pytest.mark.parametrize("lastcol", [False, True])
def test_ball_brute_force_radius_sequence(oracle_lib, p, lastcol):
    g = W.rng(600 + p + lastcol)
    for trial in range(8):
        N = int(g.integers(1, 6))
        M = (g.standard_normal((N, N)) * 10.0).tolist() if trial % 2 else g.integers(-9, 10, (N, N)).tolist()
        A = oracle_lib.from_f64(np.asarray(M, np.float64).reshape(-1), p)
        st, zk, D, Xm, RD, RX = oracle_lib.ge_ball(A, None, N, p, lastcol=lastcol)
        if st != 0:
            continue
        RDw, Rw = brute_force_ball(M, p, lastcol)
        for k in range(N):
            want = RDw[k]
            got = INF if int(RD[1][k]) == RAD_INF else (int(RD[0][k]), int(RD[1][k]))
            if want != INF and want[0] == 0:
                want = (0, ZEXP)
            assert got == want, (trial, k)
        for i in range(N):
            for j in range(N):
                if j >= i or lastcol:
                    want = Rw[i][j]
                    q = i * N + j
                    got = INF if int(RX[1][q]) == RAD_INF else (int(RX[0][q]), int(RX[1][q]))
                    if want != INF and want[0] == 0:
                        want = (0, ZEXP)
                    assert got == want, (trial, i, j)
