"""Pins of the oracle's element operations against exact rational arithmetic.

Each case is computed exactly with fractions.Fraction and rounded by the
independent integer RNE of tests/exactref.py; the oracle must agree bit for
bit.  The cases cover the corners where a multiprecision rounding goes wrong:
ties to even, carries through every limb, renormalisation after rounding up,
exponent gaps on both sides of p+2, total and partial cancellation, binade
drops at powers of two, and p from 64 to 32768 bits.
"""
from fractions import Fraction

import numpy as np
import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.usefixtures("oracle_lib")

PS = [64, 128, 512, 2048]


def rand_num(g, p, emin=-200, emax=200):
    m = 1 << (p - 1)
    m |= int.from_bytes(g.bytes(p // 8), "little") & ((1 << (p - 1)) - 1)
    s = int(g.integers(0, 2))
    e = int(g.integers(emin, emax))
    v = Fraction(m) * Fraction(2) ** (e - p)
    return -v if s else v


def special_mantissas(p):
    return [
        1 << (p - 1),                      # power of two
        (1 << p) - 1,                      # all ones
        (1 << (p - 1)) + 1,                # just above a power of two
        (1 << (p - 1)) | ((1 << (p - 1)) - 1) & 0x5555555555555555,
        (3 << (p - 2)),                    # 1.1b
        ((1 << p) - 1) ^ (1 << (p // 2)),  # a zero bit in the middle
    ]


def division_corner_mantissas(p):
    """Divisors that drive every branch of a base-2^32 long division of
    2^(2p): one and two decrements of the quotient-limb estimate by the
    two-limb test, the add-back (2^(p-1) + 1 and top limbs 2^31 over
    all-ones), the estimate clamped to 2^32 - 1 when the remainder's top limb
    equals the divisor's (every limb 2^31), and the power-of-two case."""
    top = 1 << (p - 1)
    return special_mantissas(p) + [
        top | ((1 << (p - 64)) - 1),          # v1 = 2^31, v0 = 0, lower limbs all ones
        top | (1 << (p - 64)),                # lowest bit of the second limb
        top | ((1 << (p - 32)) - 1),          # v1 = 2^31, everything below all ones
        (1 << p) - (1 << (p - 32)),           # top limb all ones, the rest zero
        ((1 << p) - 1) ^ ((1 << (p - 33)) | 1),
        sum(0x80000000 << (32 * i) for i in range(p // 32)) + 1,  # remainder top limb = v1: clamped estimate
        top | (0x7FFFFFFF << (p - 64)) | ((1 << (p - 64)) - (1 << 32)) | 0x80000000,
    ]


def values_with_specials(g, p, count):
    vals = [rand_num(g, p) for _ in range(count)]
    for m in special_mantissas(p):
        for e in (0, 1, -1, 37):
            vals.append(Fraction(m) * Fraction(2) ** (e - p))
            vals.append(-Fraction(m) * Fraction(2) ** (e - p))
    return vals


def check_binary(oracle, op, p, a_vals, b_vals, exact):
    A = X.pack(a_vals, p)
    B = X.pack(b_vals, p)
    got = op(A, B, p)
    # inputs are representable, so pack() did not round them
    ua, ub = X.unpack(A, p), X.unpack(B, p)
    want = X.pack([exact(x, y) for x, y in zip(ua, ub)], p)
    bad = [i for i in range(len(ua)) if not (got[0][i] == want[0][i] and got[1][i] == want[1][i]
                                               and np.array_equal(got[2][i], want[2][i]))]
    assert not bad, f"{len(bad)} mismatches, first at {bad[0]}: {ua[bad[0]]} op {ub[bad[0]]}"


@pytest.mark.parametrize("p", PS)
def test_mul_random_and_specials(oracle_lib, p):
    g = np.random.Generator(np.random.PCG64(11 + p))
    a = values_with_specials(g, p, 300)
    b = values_with_specials(g, p, 300)
    g.shuffle(b)
    a += [Fraction(0), a[0], Fraction(0)]
    b += [b[0], Fraction(0), Fraction(0)]
    check_binary(oracle_lib, oracle_lib.mul, p, a, b, lambda x, y: x * y)


@pytest.mark.parametrize("p", PS)
def test_mul_ties_to_even(oracle_lib, p):
    # m_b = 3*2^(p-2), m_a odd and < 2^(p+1)/3: the product has 2p-1 bits and
    # the p-1 dropped bits are exactly 100..0, a tie; RN keeps the even
    # neighbour.  Half the cases round up, half down.
    g = np.random.Generator(np.random.PCG64(7 + p))
    a, b = [], []
    lim = (1 << (p + 1)) // 3
    for _ in range(60):
        m = int.from_bytes(g.bytes(p // 8), "little") % (lim - (1 << (p - 1))) + (1 << (p - 1))
        m |= 1
        a.append(Fraction(m) * Fraction(2) ** (-p))
        b.append(Fraction(3 << (p - 2)) * Fraction(2) ** (-p))
    exact = [x * y for x, y in zip(a, b)]
    # confirm they really are ties
    for q in exact:
        s, e, m = X.rn(q, p)
        scaled = abs(q) * Fraction(2) ** (p - e)
        assert scaled.denominator == 2 or (m & 1) == 0
    check_binary(oracle_lib, oracle_lib.mul, p, a, b, lambda x, y: x * y)


@pytest.mark.parametrize("p", PS)
@pytest.mark.parametrize("kind", ["add", "sub"])
def test_addsub_exponent_gaps(oracle_lib, p, kind):
    g = np.random.Generator(np.random.PCG64(3 + p + (kind == "sub")))
    a, b = [], []
    gaps = list(range(0, 70)) + [p - 2, p - 1, p, p + 1, p + 2, p + 3, p + 40, 5 * p, 10**6]
    for d in gaps:
        for _ in range(4):
            x = rand_num(g, p, 0, 1)
            y = rand_num(g, p, 0, 1)
            y = y * Fraction(2) ** (-d)
            if g.integers(0, 2):
                x, y = y, x
            a.append(x)
            b.append(y)
    op = oracle_lib.add if kind == "add" else oracle_lib.sub
    exact = (lambda x, y: x + y) if kind == "add" else (lambda x, y: x - y)
    check_binary(oracle_lib, op, p, a, b, exact)


@pytest.mark.parametrize("p", PS)
def test_addsub_power_of_two_far_operand(oracle_lib, p):
    """A = +-1 (a power of two) minus or plus B at exponent gaps p-1 .. p+3.
    Below a power of two the spacing halves, so at gap p+1 a B above half
    that spacing moves A - B to the grid point under A: an exact-gap shortcut
    that returns A one bit too early fails here."""
    g = np.random.Generator(np.random.PCG64(77 + p))
    a, b = [], []
    ulp = Fraction(2) ** (-p + 1)  # ulp of A = 1 (mantissa 2^(p-1), value 1)
    for d in (p - 1, p, p + 1, p + 2, p + 3):
        for mb in ((1 << (p - 1)) + 1, 3 << (p - 2), (1 << p) - 1, int(g.integers(1 << 62, 1 << 63)) << (p - 63)):
            y = Fraction(mb) * Fraction(2) ** (-p) * 2 * ulp * Fraction(2) ** (p - 1 - d)
            a += [Fraction(1), Fraction(-1), Fraction(1)]
            b += [y, -y, -y]
    check_binary(oracle_lib, oracle_lib.sub, p, a, b, lambda x, y: x - y)
    check_binary(oracle_lib, oracle_lib.add, p, a, b, lambda x, y: x + y)


@pytest.mark.parametrize("p", PS)
def test_sub_cancellation_ties_and_binade_drop(oracle_lib, p):
    g = np.random.Generator(np.random.PCG64(5 + p))
    a, b = [], []
    ulp = Fraction(2) ** (-p)  # ulp of numbers in [1/2, 1)
    for _ in range(40):
        x = abs(rand_num(g, p, 0, 1))
        a.append(x); b.append(x)                        # exact zero -> +0
        a.append(x); b.append(x - ulp)                  # one-ulp difference
        a.append(x); b.append(x * (1 - Fraction(1, 1 << 20)))  # partial cancellation
        a.append(-x); b.append(-x)
    for m in special_mantissas(p):
        x = Fraction(m) * ulp
        for k in range(1, 6):  # ties and near-ties just below a power of two
            t = ulp / (1 << k)
            a += [x, x, Fraction(1, 2), Fraction(1, 2), Fraction(1)]
            b += [t, -t, t, -t, t * 3]
    check_binary(oracle_lib, oracle_lib.sub, p, a, b, lambda x, y: x - y)
    check_binary(oracle_lib, oracle_lib.add, p, a, b, lambda x, y: x + y)


@pytest.mark.parametrize("p", PS + [4096])
def test_recip(oracle_lib, p):
    g = np.random.Generator(np.random.PCG64(9 + p))
    vals = values_with_specials(g, p, 40 if p <= 2048 else 8)
    A = X.pack(vals, p)
    got = oracle_lib.recip(A, p)
    want = X.pack([1 / v for v in X.unpack(A, p)], p)
    assert X.same(got, want)


@pytest.mark.parametrize("p", [128, 256, 2048])
def test_recip_division_corners(oracle_lib, p):
    vals = [Fraction(m) * Fraction(2) ** (e - p) for m in division_corner_mantissas(p) for e in (0, -3)]
    A = X.pack(vals, p)
    assert X.same(oracle_lib.recip(A, p), X.pack([1 / v for v in vals], p))


def test_recip_of_zero_is_an_error(oracle_lib):
    with pytest.raises(RuntimeError):
        oracle_lib.recip(X.pack([Fraction(0)], 128), 128)


def test_large_precision_ops(oracle_lib):
    p = 32768
    g = np.random.Generator(np.random.PCG64(32768))
    a = [rand_num(g, p, -5, 5) for _ in range(3)]
    b = [rand_num(g, p, -5, 5) for _ in range(3)]
    check_binary(oracle_lib, oracle_lib.mul, p, a, b, lambda x, y: x * y)
    check_binary(oracle_lib, oracle_lib.sub, p, a, b, lambda x, y: x - y)
    A = X.pack(a[:1], p)
    assert X.same(oracle_lib.recip(A, p), X.pack([1 / X.unpack(A, p)[0]], p))


@pytest.mark.parametrize("p", [64, 512])
def test_lift_f64_and_int_exact(oracle_lib, p):
    g = np.random.Generator(np.random.PCG64(1))
    d = np.concatenate([g.standard_normal(50), [0.0, -0.0, 5e-324, -2.2250738585072014e-308, 1.7976931348623157e308,
                                                 1e-30, 1.0, -1.0]])
    got = oracle_lib.from_f64(d, p)
    want = X.pack([Fraction(float(v)) for v in d], p)
    assert X.same(got, want)
    assert got[0][d.tolist().index(-0.0)] == 0  # -0.0 lifts to +0
    iv = np.concatenate([g.integers(-1000, 1001, 50), [0, 1, -1, 2**62, -(2**63)]]).astype(np.int64)
    assert X.same(oracle_lib.from_int(iv, p), X.pack([Fraction(int(v)) for v in iv], p))


def test_mpmath_second_opinion(oracle_lib):
    mpmath = pytest.importorskip("mpmath")
    from mpmath import libmp

    p = 256
    g = np.random.Generator(np.random.PCG64(99))
    a = [rand_num(g, p, -50, 50) for _ in range(100)]
    b = [rand_num(g, p, -50, 50) for _ in range(100)]
    A, B = X.pack(a, p), X.pack(b, p)
    got_m, got_s = oracle_lib.mul(A, B, p), oracle_lib.sub(A, B, p)

    def to_mpf(q):
        return libmp.from_rational(q.numerator, q.denominator, p + 64, "n")

    for i in range(100):
        xa, xb = to_mpf(a[i]), to_mpf(b[i])  # exact: inputs have p bits
        m = libmp.mpf_mul(xa, xb, p, "n")
        s = libmp.mpf_sub(xa, xb, p, "n")
        for got, ref in ((got_m, m), (got_s, s)):
            q = X.to_fraction(got[0][i], got[1][i], got[2][i], p)
            sign, man, exp, _bc = ref  # value = (-1)^sign * man * 2^exp
            assert q == (-1) ** sign * Fraction(int(man)) * Fraction(2) ** exp


@pytest.mark.parametrize("p", [64, 512])
def test_cauchy_entries(oracle_lib, p):
    from paper_1308_1536_gb300 import workloads as W

    x, y = W.cauchy_xy(7, 42)
    got = oracle_lib.cauchy(x, y, p)
    r = lambda q: X.to_fraction(*X.rn_tuple(q, p), p)
    want = X.pack([1 / r(Fraction(float(a)) + Fraction(float(b))) for a in x for b in y], p)
    assert X.same(got, want)


@pytest.mark.parametrize("p", [64, 128, 512, 2048])
def test_div_is_correctly_rounded(oracle_lib, p):
    """The oracle's optional one-rounding division RN(a/b) (used only to
    measure what the method's two-rounding multiplier costs) against the
    exact rational quotient rounded by the independent reference."""
    g = W.rng(500 + p)
    va, vb = [], []
    for _ in range(150):
        for out in (va, vb):
            m = (1 << (p - 1)) | int.from_bytes(g.bytes(p // 8), "little") & ((1 << (p - 1)) - 1)
            out.append(Fraction(m) * Fraction(2) ** int(g.integers(-400, 400) - p) * (-1 if g.integers(0, 2) else 1))
    va += [Fraction(3), Fraction(1), Fraction(-7, 2), Fraction(0)]
    vb += [Fraction(3), Fraction(3), Fraction(5), Fraction(9)]
    A, B = X.pack(va, p), X.pack(vb, p)
    got = oracle_lib.div(A, B, p)
    want = X.pack([a / b for a, b in zip(X.unpack(A, p), X.unpack(B, p))], p)
    assert X.same(got, want)
    with pytest.raises(RuntimeError):
        oracle_lib.div(X.pack([Fraction(1)], p), X.pack([Fraction(0)], p), p)
