"""The tensor-core engine (exact digit convolution on tcgen05, p = 512, 1024,
2048) and
the IMAD engine must give the same bits for the whole elimination, in both
modes, for the adjoint's back substitution, and match the oracle."""
import numpy as np
import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run(mpdet, N, p, kind, data, engine, lastcol=True, tc_min_rows=0):
    """tc_min_rows=0: the tensor engine takes every update launch, down to
    one row (the default hands short launches to the IMAD kernel)."""
    h = mpdet.Mpdet(N, p, lastcol=lastcol)
    h.tune(engine=engine, tc_min_rows=tc_min_rows)
    if kind == "cauchy":
        h.set_cauchy(*data)
    elif kind == "int":
        h.set_i32(data)
    else:
        h.set_f64(data)
    rc, zk, D = h.factor()
    Xm = h.get_mp()
    h.close()
    return rc, zk, D, Xm


@pytest.mark.parametrize("p", [512, 1024, 2048])
@pytest.mark.parametrize("N", [1, 2, 5, 130, 300])
@pytest.mark.parametrize("kind", ["cauchy", "int", "f64"])
def test_tensor_engine_equals_imad_engine(mpdet, p, N, kind):
    g = W.rng(N * 7 + len(kind) + p)
    data = W.cauchy_xy(N, N) if kind == "cauchy" else (W.int_matrix(N, N) if kind == "int" else g.standard_normal((N, N)))
    for lastcol in (False, True):
        b = run(mpdet, N, p, kind, data, 0, lastcol)
        for engine in ((1, 2) if p == 2048 else (1,)):
            a = run(mpdet, N, p, kind, data, engine, lastcol)
            assert a[:2] == b[:2]
            assert X.same(a[2], b[2]), f"leading minors differ between engines {engine} and 0"
            assert X.same(a[3], b[3]), f"in-place arrays differ between engines {engine} and 0"


@pytest.mark.parametrize("p", [512, 1024, 2048])
def test_tensor_engine_vs_oracle(mpdet, oracle_lib, p):
    N = 150
    A = W.int_matrix(N, 3)
    rc, zk, D, Xm = run(mpdet, N, p, "int", A, 1)
    st, ozk, OD, OX = oracle_lib.ge(oracle_lib.from_int(A.reshape(-1), p), N, p, lastcol=True, nthreads=16)
    assert (rc, zk) == (st, ozk)
    assert X.same(D, OD) and X.same(Xm, OX)


def test_tensor_engine_adjoint(mpdet):
    N, p = 140, 2048
    A = W.rng(9).standard_normal((N, N))
    out = []
    for engine in (1, 0):
        h = mpdet.Mpdet(N, p, lastcol=True)
        h.tune(engine=engine, tc_min_rows=0)
        s, la, G = h.logabsdet_grad(A)
        out.append((s, la, G, h.get_inverse()))
        h.close()
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2]) and X.same(out[0][3], out[1][3])


@pytest.mark.parametrize("tc_min_rows", [16, 64, 1 << 20])
def test_engine_switch_by_rows(mpdet, tc_min_rows):
    """Mixing the engines within one elimination (tensor cores for the long
    launches, IMAD for the short ones) changes no bit."""
    N, p = 200, 1024
    data = W.int_matrix(N, 17)
    ref = run(mpdet, N, p, "int", data, 0)
    got = run(mpdet, N, p, "int", data, 1, tc_min_rows=tc_min_rows)
    assert got[:2] == ref[:2] and X.same(got[2], ref[2]) and X.same(got[3], ref[3])


@pytest.mark.parametrize("p", [512, 1024, 2048])
def test_tensor_engine_rare_subtraction_paths(mpdet, oracle_lib, p):
    """Inputs that drive the subtraction's rare paths in the tensor engine's
    row subtraction: entries spread over 2^-300..2^300 (exponent gaps of 64
    and more between x_ij and the product), rank-deficient integer matrices
    (exact cancellation to zero), and near-duplicate rows (cancellation of
    more than 32 bits).  Bit-identical to the IMAD engine and the oracle."""
    g = W.rng(500 + p)
    N = 140
    spread = g.standard_normal((N, N)) * np.exp2(g.integers(-300, 300, (N, N)).astype(np.float64))
    B = g.integers(-5, 6, (N, 3))
    lowrank = (B @ g.integers(-5, 6, (3, N))).astype(np.int64)
    near = g.standard_normal((N, N))
    near[1::2] = near[0::2] + g.standard_normal((N // 2, N)) * 2.0 ** -40
    for kind, data in (("f64", spread), ("int", lowrank), ("f64", near)):
        a = run(mpdet, N, p, kind, data, 1)
        b = run(mpdet, N, p, kind, data, 0)
        assert a[:2] == b[:2]
        assert X.same(a[2], b[2]) and X.same(a[3], b[3])
    A = oracle_lib.from_f64(near.reshape(-1), p)
    st, zk, D, OX = oracle_lib.ge(A, N, p, lastcol=True, nthreads=16)
    a = run(mpdet, N, p, "f64", near, 1)
    assert a[:2] == (st, zk) and X.same(a[2], D) and X.same(a[3], OX)


@pytest.mark.parametrize("p", [512, 1024, 2048])
def test_tensor_engine_lazy_drain_fallback(mpdet, oracle_lib, p):
    """The epilogue reads the low half of a product only when limbs n-8..n-2
    of its upper part are all zeros or all ones above bit 14.  With a_00 = 1
    the first step's multipliers are column 0 exactly, so column 0 and row 0
    choose the products: (2^(p-1) + 1)(2^p - 1) has a low half of all ones,
    (2^p - 1)^2 and products with a power of two have (almost) all zeros, the
    random entries take the fast path.  Bit-identical to the IMAD engine and
    the oracle."""
    from fractions import Fraction

    from test_oracle_ops import rand_num

    g = np.random.Generator(np.random.PCG64(4242 + p))
    N = 40
    half, ones, top = (1 << (p - 1)) + 1, (1 << p) - 1, 1 << (p - 1)
    col0 = [half, ones, top, None]
    row0 = [ones, top, half, None]
    vals = []
    for i in range(N):
        for j in range(N):
            if i == 0 and j == 0:
                v = Fraction(1)
            elif j == 0:
                m = col0[i % 4]
                v = rand_num(g, p) if m is None else Fraction(m) * Fraction(2) ** (int(g.integers(-3, 4)) - p)
            elif i == 0:
                m = row0[j % 4]
                v = rand_num(g, p) if m is None else Fraction(m) * Fraction(2) ** (int(g.integers(-3, 4)) - p)
            else:
                v = rand_num(g, p)
            vals.append(v)
    A = X.pack(vals, p)
    out = []
    for engine in (1, 0):
        h = mpdet.Mpdet(N, p, lastcol=True)
        h.tune(engine=engine, tc_min_rows=0)
        h.set_mp(A)
        rc, zk, D = h.factor()
        out.append((rc, zk, D, h.get_mp()))
        h.close()
    assert out[0][:2] == out[1][:2]
    assert X.same(out[0][2], out[1][2]) and X.same(out[0][3], out[1][3])
    st, ozk, OD, OX = oracle_lib.ge(A, N, p, lastcol=True, nthreads=8)
    assert out[0][:2] == (st, ozk) and X.same(out[0][2], OD) and X.same(out[0][3], OX)


@pytest.mark.parametrize("p", [2048, 4096, 8192, 16384])
def test_imad_update_geometries_are_bit_identical(mpdet, oracle_lib, p):
    """The IMAD update with 32 limbs per lane (both register budgets) gives
    the bits of the precision's own geometry, in both modes and for the
    adjoint's back substitution, and the oracle's."""
    N = 37 if p <= 4096 else 21
    data = W.cauchy_xy(N, p + 1)

    def go(geom, lastcol):
        h = mpdet.Mpdet(N, p, lastcol=lastcol)
        h.tune(engine=0, update_geometry=geom)
        h.set_cauchy(*data)
        rc, zk, D = h.factor()
        Xm = h.get_mp()
        h.close()
        return rc, zk, D, Xm

    for lastcol in (False, True):
        base = go(0, lastcol)
        for geom in (1, 2, -1):
            a = go(geom, lastcol)
            assert a[:2] == base[:2] and X.same(a[2], base[2]) and X.same(a[3], base[3]), (geom, lastcol)
    st, ozk, OD, OX = oracle_lib.ge(oracle_lib.cauchy(*data, p), N, p, lastcol=True, nthreads=8)
    assert X.same(base[2], OD) and X.same(base[3], OX)
    A = W.rng(p).standard_normal((N, N))
    g = []
    for geom in (0, 1):
        h = mpdet.Mpdet(N, p, lastcol=True)
        h.tune(engine=0, update_geometry=geom)
        g.append(h.logabsdet_grad(A, grad=True))
        h.close()
    assert g[0][0] == g[1][0] and g[0][1] == g[1][1] and np.array_equal(g[0][2], g[1][2])
