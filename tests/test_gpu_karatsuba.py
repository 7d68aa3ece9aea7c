"""One Karatsuba level against the schoolbook product on the IMAD engine's
lane layout (mpdet_mulbench): RN(a*b) at p = 8192, 16384 and 32768 by both
methods equals the oracle's product bit for bit, on random operands and on
mantissas that make every carry of the method appear: all-ones halves (the
sums z0 + z1 and b0 + b1 carry out), powers of two, a product that rounds up
through every limb, and zeros."""
from fractions import Fraction

import numpy as np
import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W
from test_oracle_ops import rand_num, special_mantissas

pytestmark = pytest.mark.gpu


def karatsuba_corners(p):
    h = p // 2
    ms = [(1 << p) - 1,                                   # both halves all ones
          (1 << (p - 1)) | ((1 << h) - 1),                # low half all ones
          ((1 << p) - 1) ^ ((1 << h) - 1),               # high half all ones, low half zero
          (1 << (p - 1)) | (1 << (h - 1)),
          (1 << (p - 1)) + 1,
          (3 << (p - 2)) | ((1 << (h + 5)) - 1)]
    return ms + list(special_mantissas(p))


@pytest.mark.parametrize("p", [8192, 16384, 32768])
def test_karatsuba_equals_schoolbook_and_oracle(mpdet, oracle_lib, p):
    g = np.random.Generator(np.random.PCG64(7000 + p))
    a = [rand_num(g, p) for _ in range(90)]
    b = [rand_num(g, p) for _ in range(90)]
    cm = karatsuba_corners(p)
    for i, ma in enumerate(cm):
        for mb in cm[i:i + 3]:
            a.append(Fraction(ma) * Fraction(2) ** (-p + int(g.integers(-5, 5))))
            b.append(-Fraction(mb) * Fraction(2) ** (-p))
    a += [Fraction(0), a[0]]
    b += [b[0], Fraction(0)]
    A, B = X.pack(a, p), X.pack(b, p)
    want = oracle_lib.mul(A, B, p)
    school, _ = mpdet.mulbench("school", A, B, p)
    kara, _ = mpdet.mulbench("kara", A, B, p, reps=2)
    for name, got in (("schoolbook", school), ("karatsuba", kara)):
        for i in range(len(a)):
            assert got[0][i] == want[0][i] and got[1][i] == want[1][i] and np.array_equal(got[2][i], want[2][i]), \
                f"{name} p={p}: product {i} differs from the oracle"


@pytest.mark.parametrize("p,N", [(8192, 11), (16384, 7), (32768, 5)])
def test_update_with_karatsuba_products_equals_oracle(mpdet, oracle_lib, p, N):
    """The elimination with the IMAD update's products formed by one
    Karatsuba level (MPDET_TUNE_KARATSUBA) equals the oracle bit for bit:
    leading minors, the whole in-place array and the last-column minors."""
    x, y = W.cauchy_xy(N, 4000 + N)
    h = mpdet.Mpdet(N, p, lastcol=True)
    h.tune(karatsuba=True, engine=0)
    h.set_cauchy(x, y)
    rc, zk, D = h.factor()
    Xm = h.get_mp()
    C = h.lastcol_minors()
    h.close()
    st, ozk, OD, OX = oracle_lib.ge(oracle_lib.cauchy(x, y, p), N, p, lastcol=True, nthreads=8)
    assert (rc, zk) == (st, ozk)
    assert X.same(D, OD) and X.same(Xm, OX)
    assert X.same(C, oracle_lib.lastcol_minors(OX, OD, N, p))
