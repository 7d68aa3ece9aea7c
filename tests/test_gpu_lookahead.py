"""Look-ahead (column k+1 of step k updated first on a second stream, then
the pivot and multipliers of step k+1 while the rest of step k runs) changes
no bit: the same operations on the same operands.  Checked against the
one-stream order and the oracle, across windows, zero pivots (the update of
step k still completes when step k+1's pivot, running beside it, is zero) and
every engine."""
import numpy as np
import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run(mpdet, N, p, lastcol, kind, data, lookahead, windows=None, **tune):
    h = mpdet.Mpdet(N, p, lastcol=lastcol)
    h.tune(lookahead=lookahead, **tune)
    if kind == "cauchy":
        h.set_cauchy(*data)
    elif kind == "int":
        h.set_i32(data)
    else:
        h.set_f64(data)
    mids = []
    if windows:
        k = 0
        for w in windows:
            h.factor_range(k, min(k + w, N))
            k = min(k + w, N)
            mids.append((h.get_mp(), h.get_minors()))
    rc, zk, D = h.factor()
    Xm = h.get_mp()
    C = h.lastcol_minors() if (lastcol and rc == 0) else None
    h.close()
    return rc, zk, D, Xm, C, mids


def data_for(kind, N, seed):
    if kind == "cauchy":
        return W.cauchy_xy(N, seed)
    if kind == "int":
        return W.int_matrix(N, seed)
    return W.rng(seed).standard_normal((N, N))


def assert_runs_equal(a, b):
    assert a[:2] == b[:2]
    assert X.same(a[2], b[2]), "leading minors"
    assert X.same(a[3], b[3]), "in-place array"
    if a[4] is not None or b[4] is not None:
        assert X.same(a[4], b[4]), "last-column minors"


@pytest.mark.parametrize("p", [512, 1024, 2048, 4096])
@pytest.mark.parametrize("N", [2, 3, 37, 150])
@pytest.mark.parametrize("lastcol", [False, True])
def test_lookahead_equals_serial(mpdet, p, N, lastcol):
    kind = ("cauchy", "int", "f64")[(N + p // 512) % 3]
    data = data_for(kind, N, N + p)
    assert_runs_equal(run(mpdet, N, p, lastcol, kind, data, True), run(mpdet, N, p, lastcol, kind, data, False))


@pytest.mark.parametrize("p", [1024, 2048])
def test_lookahead_vs_oracle(mpdet, oracle_lib, p):
    N = 70
    A = W.int_matrix(N, 21)
    got = run(mpdet, N, p, True, "int", A, True)
    st, zk, D, OX = oracle_lib.ge(oracle_lib.from_int(A.reshape(-1), p), N, p, lastcol=True, nthreads=16)
    assert got[:2] == (st, zk)
    assert X.same(got[2], D) and X.same(got[3], OX)
    assert X.same(got[4], oracle_lib.lastcol_minors(OX, D, N, p))


def test_lookahead_windows_end_in_the_serial_state(mpdet):
    """Each window's last step updates all its columns, so the in-place array
    and the minors after every window equal those of the one-stream order."""
    N, p = 60, 2048
    data = data_for("cauchy", N, 4)
    windows = [1, 2, 5, 13, 1, 30, 8]
    a = run(mpdet, N, p, True, "cauchy", data, True, windows)
    b = run(mpdet, N, p, True, "cauchy", data, False, windows)
    assert_runs_equal(a, b)
    for (xa, da), (xb, db) in zip(a[5], b[5]):
        assert X.same(xa, xb) and X.same(da, db)


def exact_zero_pivot_matrix(N, kz, seed):
    """A = L U with small integer entries, unit lower L and an upper U whose
    diagonal holds powers of two except u_kk = 0 at k = kz (0-based): every
    operation of the elimination is exact at p >= 256, so step kz + 1 meets an
    exactly zero pivot."""
    g = W.rng(seed)
    L = np.tril(g.integers(-3, 4, (N, N)), -1) + np.eye(N, dtype=np.int64)
    U = np.triu(g.integers(-3, 4, (N, N)), 1)
    d = g.choice([1, 2, 4, -2], N)
    d[kz] = 0
    U = U + np.diag(d)
    return (L @ U).astype(np.int64)


@pytest.mark.parametrize("lastcol", [False, True])
@pytest.mark.parametrize("kz", [0, 1, 4, 10])
def test_lookahead_zero_pivot_state(mpdet, oracle_lib, lastcol, kz):
    N, p = 12, 512
    A = exact_zero_pivot_matrix(N, kz, 100 + kz)
    a = run(mpdet, N, p, lastcol, "int", A, True)
    b = run(mpdet, N, p, lastcol, "int", A, False)
    st, zk, D, OX = oracle_lib.ge(oracle_lib.from_int(A.reshape(-1), p), N, p, lastcol=lastcol)
    assert a[:2] == b[:2] == (st, zk) == (mpdet.EZEROPIVOT, kz + 1)
    assert X.same(a[2], b[2]) and X.same(a[2], D)
    # the array after the steps before the zero pivot, complete
    assert X.same(a[3], b[3])
    iu = np.array([i * N + j for i in range(N) for j in range(N) if lastcol or j >= i])
    sub = lambda t: tuple(np.asarray(v)[iu] for v in t)
    assert X.same(sub(a[3]), sub(OX))


@pytest.mark.parametrize("reserve", [0, 16])
@pytest.mark.parametrize("engine", [0, 1])
def test_lookahead_reserve_and_engines(mpdet, reserve, engine):
    N, p = 160, 2048
    data = data_for("int", N, 8)
    a = run(mpdet, N, p, True, "int", data, True, engine=engine, lookahead_reserve=reserve)
    b = run(mpdet, N, p, True, "int", data, False, engine=0)
    assert_runs_equal(a, b)
