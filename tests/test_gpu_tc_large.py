"""The large-precision tensor engine (p = 4096 .. 32768: 8-bit digits of the
multiplier against 4-bit digits of the pivot-row element on tcgen05, the
lower half of each product skipped when it cannot change the rounding) gives
the same bits as the IMAD engine and the oracle: whole eliminations in both
modes, every launch down to one row, the exact fallback (products with an
all-zero or all-one band below the rounding point), the adjoint's back
substitution, and a zero pivot."""
import numpy as np
import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run(mpdet, N, p, kind, data, engine, lastcol=True, tc_min_rows=0):
    h = mpdet.Mpdet(N, p, lastcol=lastcol)
    h.tune(engine=engine, tc_min_rows=tc_min_rows)
    if kind == "cauchy":
        h.set_cauchy(*data)
    elif kind == "int":
        h.set_i32(np.asarray(data, dtype=np.int32))
    else:
        h.set_f64(data)
    rc, zk, D = h.factor()
    Xm = h.get_mp()
    h.close()
    return rc, zk, D, Xm


def data_for(kind, N, seed):
    if kind == "cauchy":
        return W.cauchy_xy(N, seed)
    if kind == "int":
        return W.int_matrix(N, seed)
    return W.rng(seed).standard_normal((N, N))


def same_run(a, b, what):
    assert a[:2] == b[:2], what
    assert X.same(a[2], b[2]), f"{what}: leading minors differ"
    assert X.same(a[3], b[3]), f"{what}: in-place arrays differ"


@pytest.mark.parametrize("p,N", [(4096, 2), (4096, 70), (4096, 200), (8192, 140), (16384, 130), (32768, 131)])
@pytest.mark.parametrize("kind", ["cauchy", "int", "f64"])
def test_large_tensor_engine_equals_imad_engine(mpdet, p, N, kind):
    data = data_for(kind, N, N + p // 1024)
    for lastcol in (False, True):
        ref = run(mpdet, N, p, kind, data, 0, lastcol)
        got = run(mpdet, N, p, kind, data, 1, lastcol)
        same_run(got, ref, f"p={p} N={N} {kind} lastcol={lastcol}")


@pytest.mark.parametrize("p,N", [(4096, 96), (32768, 20)])
def test_large_tensor_engine_vs_oracle(mpdet, oracle_lib, p, N):
    x, y = W.cauchy_xy(N, 5)
    rc, zk, D, Xm = run(mpdet, N, p, "cauchy", (x, y), 1)
    st, ozk, OD, OX = oracle_lib.ge(oracle_lib.cauchy(x, y, p), N, p, lastcol=True, nthreads=16)
    assert (rc, zk) == (st, ozk)
    assert X.same(D, OD) and X.same(Xm, OX)


@pytest.mark.parametrize("p", [4096, 32768])
def test_large_tensor_engine_exact_fallback(mpdet, oracle_lib, p):
    """a_11 = 1 and powers of two in the first row: the first step's products
    are exact (their bits below the rounding point are all zero), which the
    lazy low half cannot decide; they take the exact path."""
    N = 40
    A = W.int_matrix(N, 23)
    A[0, 0] = 1
    A[0, 1:8] = [1, 2, -4, 8, 1024, -1, 0]
    A[1:6, 0] = [1, -2, 0, 64, 3]
    rc, zk, D, Xm = run(mpdet, N, p, "int", A, 1)
    ref = run(mpdet, N, p, "int", A, 0)
    same_run((rc, zk, D, Xm), ref, "exact products")
    st, ozk, OD, OX = oracle_lib.ge(oracle_lib.from_int(A.reshape(-1), p), N, p, lastcol=True, nthreads=16)
    assert (rc, zk) == (st, ozk)
    assert X.same(D, OD) and X.same(Xm, OX)


def test_large_tensor_engine_zero_pivot(mpdet):
    N, p = 100, 4096
    A = W.int_matrix(N, 31)
    A[1] = A[0] * 3  # D_2 = 0 exactly
    ref = run(mpdet, N, p, "int", A, 0)
    got = run(mpdet, N, p, "int", A, 1)
    assert got[1] == 2
    same_run(got, ref, "zero pivot")


def test_large_tensor_engine_adjoint(mpdet):
    N, p = 100, 4096
    A = W.nearly_singular_f64(N, 77)
    out = []
    for engine in (1, 0):
        h = mpdet.Mpdet(N, p, lastcol=True)
        h.tune(engine=engine, tc_min_rows=0)
        s, la, G = h.logabsdet_grad(A)
        out.append((s, la, G, h.get_inverse()))
        h.close()
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2]) and X.same(out[0][3], out[1][3])
