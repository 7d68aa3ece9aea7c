"""GPU parity of the series of last-column minors for every leading size
(Sec. 3: the minor arrays for N = 2, 3, ... from one elimination), of
sampled reads of the in-place array, and a full-size sampled check of the
N = 4096, p = 32768 Cauchy workload over its first elimination steps.
Everything is compared bit for bit with the CPU oracle."""
import numpy as np
import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def assert_same(got, want, what):
    for i in range(len(want[0])):
        ok = got[0][i] == want[0][i] and got[1][i] == want[1][i] and np.array_equal(got[2][i], want[2][i])
        assert ok, f"{what}: first mismatch at {i}: got ({got[0][i]}, {got[1][i]}) want ({want[0][i]}, {want[1][i]})"


def _inputs(kind, N, seed):
    if kind == "cauchy":
        return W.cauchy_xy(N, seed)
    return W.int_matrix(N, seed)


@pytest.mark.parametrize("kind,N,p", [("cauchy", 150, 1024), ("int", 130, 2048), ("cauchy", 33, 512),
                                      ("int", 40, 4096), ("cauchy", 1, 512), ("int", 2, 256)])
def test_minor_series_vs_oracle(mpdet, oracle_lib, kind, N, p):
    data = _inputs(kind, N, 1308 + N)
    h = mpdet.Mpdet(N, p, lastcol=True)
    if kind == "cauchy":
        h.set_cauchy(*data)
        A = oracle_lib.cauchy(*data, p)
    else:
        h.set_i32(data.astype(np.int32))
        A = oracle_lib.from_int(data.reshape(-1), p)
    rc, zk, D = h.factor()
    S = h.minor_series()
    Sd = h.minor_series(normalised=True)
    h.close()
    st, ozk, OD, OX = oracle_lib.ge(A, N, p, lastcol=True, nthreads=8)
    assert rc == st == 0
    assert_same(S, oracle_lib.minor_series(OX, OD, N, p), "series")
    assert_same(Sd, oracle_lib.minor_series(OX, OD, N, p, normalised=True), "normalised series")
    # the largest series is the last-column minors of the whole matrix
    off = N * (N - 1) // 2
    assert_same(tuple(t[off:] for t in S), oracle_lib.lastcol_minors(OX, OD, N, p), "series N")


def test_minor_series_device_output_and_zero_pivot(mpdet, oracle_lib):
    """Device outputs; a zero pivot at step kz leaves series 1..kz valid and
    every later series +0."""
    import torch

    N, p, kz = 24, 512, 9
    # A = L U with unit lower L, integer U with unit diagonal except u_kz,kz = 0:
    # elimination without pivoting is exact and meets an exactly zero pivot at kz
    g = W.rng(77)
    L = np.tril(g.integers(-2, 3, (N, N)), -1) + np.eye(N, dtype=np.int64)
    U = np.triu(g.integers(-3, 4, (N, N)), 1) + np.diag(g.choice([-1, 1], N))
    U[kz - 1, kz - 1] = 0
    A = L @ U
    assert np.abs(A).max() < 2**31
    h = mpdet.Mpdet(N, p, lastcol=True)
    h.set_i32(A.astype(np.int32))
    rc, zk, D = h.factor()
    assert rc == mpdet.EZEROPIVOT and zk == kz
    n, tot = p // 32, N * (N + 1) // 2
    out = (torch.empty(tot, dtype=torch.int8, device="cuda"), torch.empty(tot, dtype=torch.int64, device="cuda"),
           torch.empty((tot, n), dtype=torch.int32, device="cuda"))
    h.minor_series(out=out)
    torch.cuda.synchronize()
    S = (out[0].cpu().numpy(), out[1].cpu().numpy(), out[2].cpu().numpy().view(np.uint32))
    h.close()
    st, ozk, OD, OX = oracle_lib.ge(oracle_lib.from_int(A.reshape(-1), p), N, p, lastcol=True)
    assert ozk == kz
    lim = kz * (kz + 1) // 2
    assert_same(tuple(t[:lim] for t in S), tuple(t[:lim] for t in oracle_lib.minor_series(OX, OD, N, p)),
                "series 1..kz")
    assert np.all(S[1][lim:] == X.ZEXP) and np.all(S[0][lim:] == 0) and not S[2][lim:].any()


def test_get_entries_equals_get_mp(mpdet):
    N, p = 50, 1024
    h = mpdet.Mpdet(N, p, lastcol=True)
    h.set_cauchy(*W.cauchy_xy(N, 5))
    h.factor_range(0, 20)
    Xm = h.get_mp()
    idx = np.array([0, 1, N - 1, N, 20 * N + 20, N * N - 1, 777], np.int64)
    E = h.get_entries(idx)
    h.close()
    assert_same(E, tuple(t[idx] for t in Xm), "entries")


def test_full_size_C5_first_steps_sampled(mpdet, oracle_lib):
    """Workload C5 at full size (Cauchy, N = 4096, p = 32768: 68.9 GB in HBM),
    first two elimination steps in last-column mode, in the launch
    configuration of a full factorisation.  After k steps entry (i, j) depends
    only on rows {0..k-1, i} and columns {0..k-1, j}, so each sampled entry
    (U part and L part) is checked against an oracle elimination of that
    (k+1) x (k+1) submatrix; D_1, D_2 against the leading 2 x 2 block."""
    cfg = W.C5
    N, p, k = cfg["N"], cfg["p"], 2
    x, y = W.cauchy_xy(N, cfg["seed"])
    g = W.rng(cfg["seed"] + 7)
    h = mpdet.Mpdet(N, p, lastcol=True)
    try:
        h.set_cauchy(x, y)
        h.factor_range(0, k)
        assert h.status()[0] == 0
        D = h.get_minors()
        rows = sorted({k, N - 1, *g.integers(k, N, 6).tolist()})
        cols = sorted({k, N - 1, *g.integers(k, N, 3).tolist()})
        idx, want = [], []
        for i in rows:
            for j in cols:
                ri, cj = np.array([0, 1, i]), np.array([0, 1, j])
                st, _, OD, OX = oracle_lib.ge(oracle_lib.cauchy(x[ri], y[cj], p), k + 1, p, lastcol=True, k_end=k)
                # (i, j): the Schur complement entry; (i, 0), (i, 1): row i of L
                for c, full in ((2, i * N + j), (0, i * N), (1, i * N + 1)):
                    idx.append(full)
                    want.append(tuple(t[2 * (k + 1) + c] for t in OX))
                if i == rows[0]:  # rows 0 and 1 (U and l_10) once per column
                    for r, c in ((0, 2), (1, 2), (1, 0)):
                        idx.append((r * N + j) if c == 2 else N)
                        want.append(tuple(t[r * (k + 1) + c] for t in OX))
        E = h.get_entries(np.array(idx, np.int64))
        for q, w in enumerate(want):
            got = (E[0][q], E[1][q], E[2][q])
            assert got[0] == w[0] and got[1] == w[1] and np.array_equal(got[2], w[2]), f"entry {idx[q]}"
        _, _, OD2, _ = oracle_lib.ge(oracle_lib.cauchy(x[:k], y[:k], p), k, p)
        assert_same(tuple(t[:k] for t in D), OD2, "D_1, D_2")
    finally:
        h.close()


def test_full_size_C2_series_sampled(mpdet, oracle_lib):
    """Workload C2 at full size (N = 1024, p = 2048, last-column mode, the
    benchmark's configuration): the series of last-column minors of the full
    run, at sampled sizes n, equals the oracle's last-column minors of the
    leading n x n block (bit for bit); this checks the L bookkeeping (a5) of
    rows below n in the full-size launches."""
    N, p = W.C2["N"], W.C2["p"]
    x, y = W.cauchy_xy(N, W.C2["seed"])
    A = W.int_matrix(N, W.C2["seed"] + 100)
    for kind in ("cauchy", "int"):
        h = mpdet.Mpdet(N, p, lastcol=True)
        if kind == "cauchy":
            h.set_cauchy(x, y)
        else:
            h.set_i32(A.astype(np.int32))
        rc, zk, D = h.factor()
        assert rc == 0
        S = h.minor_series()
        h.close()
        for nn in (1, 2, 17, 64):
            if kind == "cauchy":
                M = oracle_lib.cauchy(x[:nn], y[:nn], p)
            else:
                M = oracle_lib.from_int(A[:nn, :nn].reshape(-1), p)
            st, _, OD, OX = oracle_lib.ge(M, nn, p, lastcol=True, nthreads=8)
            assert st == 0
            off = nn * (nn - 1) // 2
            assert_same(tuple(t[off:off + nn] for t in S), oracle_lib.lastcol_minors(OX, OD, nn, p),
                        f"{kind}: series {nn}")
