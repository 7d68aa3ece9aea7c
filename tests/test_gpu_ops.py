"""GPU element-wise arithmetic (the kernels' mul_round / sub_round /
recip_round through mpdet_ops) against the oracle, bit for bit, on the
corner cases of tests/test_oracle_ops.py: ties to even, carries through every
limb, exponent gaps on both sides of 64 and p+2 (the register and the
shared-memory alignment paths), cancellations of 0..p bits (the register and
the shared-memory normalisation paths), zeros, and p from 128 to 32768."""
from fractions import Fraction

import numpy as np
import pytest

import exactref as X
from test_oracle_ops import division_corner_mantissas, rand_num, values_with_specials

pytestmark = pytest.mark.gpu


def cases(p, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    a = values_with_specials(g, p, 200)
    b = values_with_specials(g, p, 200)
    g.shuffle(b)
    ulp = Fraction(2) ** (-p)
    gaps = list(range(0, 40)) + [60, 62, 63, 64, 65, 66, 95, 96, 97, p - 2, p - 1, p, p + 1, p + 2, p + 3, 3 * p, 10**6]
    for d in gaps:
        for _ in range(3):
            x = rand_num(g, p, 0, 1)
            y = rand_num(g, p, 0, 1) * Fraction(2) ** (-d)
            if g.integers(0, 2):
                x, y = y, x
            a.append(x)
            b.append(y)
    for _ in range(30):  # cancellations of 1..p bits
        x = abs(rand_num(g, p, 0, 1))
        k = int(g.integers(1, p))
        a.append(x)
        b.append(x - ulp * int(g.integers(1, 1 << min(k, 60))) * Fraction(2) ** max(0, k - 60))
        a.append(x)
        b.append(x)
    a += [Fraction(0), Fraction(0), a[0]]
    b += [Fraction(0), b[0], Fraction(0)]
    return X.pack(a, p), X.pack(b, p)


def first_bad(got, want):
    for i in range(len(got[0])):
        if got[0][i] != want[0][i] or got[1][i] != want[1][i] or not np.array_equal(got[2][i], want[2][i]):
            return i
    return None


@pytest.mark.parametrize("p", [64, 96, 128, 160, 256, 512, 1024, 2048, 3072, 4096, 32768])
def test_ops_vs_oracle(mpdet, oracle_lib, p):
    A, B = cases(p, 5000 + p)
    for op in ("mul", "sub", "add"):
        got = mpdet.ops(op, A, B, p)
        want = getattr(oracle_lib, op)(A, B, p)
        i = first_bad(got, want)
        assert i is None, f"{op} p={p}: first mismatch at {i}"
    nz = np.nonzero(A[1] != X.ZEXP)[0][:60 if p >= 4096 else 400]
    Anz = tuple(t[nz] for t in A)
    got = mpdet.ops("recip", Anz, Anz, p)
    assert first_bad(got, oracle_lib.recip(Anz, p)) is None


@pytest.mark.parametrize("p", [128, 256, 512, 1024, 2048, 4096, 8192, 32768])
def test_recip_division_corners(mpdet, oracle_lib, p):
    vals = []
    for m in division_corner_mantissas(p):
        for e in (0, 5, -3):
            vals.append(Fraction(m) * Fraction(2) ** (e - p))
            vals.append(-Fraction(m) * Fraction(2) ** (e - p))
    A = X.pack(vals, p)
    got = mpdet.ops("recip", A, A, p)
    i = first_bad(got, oracle_lib.recip(A, p))
    assert i is None, f"p={p}: first mismatch at {i}"
    want = X.pack([1 / v for v in vals], p)
    assert first_bad(got, want) is None


@pytest.mark.parametrize("p", [128, 256, 512, 1024, 2048, 4096, 8192])
def test_pivot_reciprocal_corners(mpdet, oracle_lib, p):
    """The pivot kernel's reciprocal (its own lane grouping) on the same
    divisors: a_00 is the corner mantissa, the multipliers of column 0 expose
    r_1 in lastcol mode and must equal the oracle's bit for bit."""
    g = np.random.Generator(np.random.PCG64(900 + p))
    for m in division_corner_mantissas(p):
        vals = [Fraction(m) * Fraction(2) ** (-p)] + [rand_num(g, p) for _ in range(8)]
        A = X.pack(vals, p)
        h = mpdet.Mpdet(3, p, lastcol=True)
        h.set_mp(A)
        rc, zk, D = h.factor()
        Xg = h.get_mp()
        h.close()
        st, ozk, OD, OX = oracle_lib.ge(A, 3, p, lastcol=True)
        assert rc == st and zk == ozk
        assert first_bad(D, OD) is None
        assert first_bad(Xg, OX) is None, f"p={p} m={hex(m)[:20]}"
