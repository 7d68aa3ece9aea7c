"""The allocation-free entry point (mpdet_factor_noalloc) against the regular
one (mpdet_factor + mpdet_lastcol_minors).

mpdet_factor_noalloc serves callers that cannot allocate device memory (host
frameworks that own every buffer and forbid a plugin its own allocations,
latency-bound loops that cannot take an allocation mid-step): it keeps its
working memory in a static device array.  Its results must equal the regular path's bit for bit, also
on a second call in a row, which finds the array holding the first call's
contents.  This file is named to be collected last."""
import numpy as np
import pytest

from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(triple, torch):
    s, e, m = triple
    return (torch.from_numpy(np.ascontiguousarray(s)).cuda(), torch.from_numpy(np.ascontiguousarray(e)).cuda(),
            torch.from_numpy(np.ascontiguousarray(m).view(np.int32)).cuda())


def _host(triple):
    s, e, m = triple
    return (s.cpu().numpy(), e.cpu().numpy(), m.cpu().numpy().view(np.uint32))


def _empty(count, p, torch):
    n = p // 32
    return (torch.zeros(count, dtype=torch.int8, device="cuda"),
            torch.zeros(count, dtype=torch.int64, device="cuda"),
            torch.zeros((count, n), dtype=torch.int32, device="cuda"))


def _equal(a, b):
    return all(np.array_equal(np.asarray(x), np.asarray(y)) for x, y in zip(a, b))


@pytest.mark.parametrize("N,p,kind", [(64, 512, "cauchy"), (40, 2048, "int"), (7, 4096, "cauchy"), (1, 512, "int")])
def test_noalloc_matches_regular_entry_point_twice(mpdet, N, p, kind):
    import torch

    # input at p bits and the regular path's results
    h = mpdet.Mpdet(N, p, lastcol=True)
    if kind == "cauchy":
        h.set_cauchy(*W.cauchy_xy(N, 1308 + N))
    else:
        h.set_i32(W.int_matrix(N, 1308 + N))
    A = h.get_mp()
    rc, zk, D_ref = h.factor()
    C_ref = h.lastcol_minors()
    h.close()
    Ad = _dev(A, torch)
    for call in range(2):
        D, C = _empty(N, p, torch), _empty(N, p, torch)
        st, z = mpdet.factor_noalloc(Ad, N, p, D, C)
        torch.cuda.synchronize()
        assert (st, z) == (rc, zk), call
        assert _equal(_host(D), D_ref), f"minors differ on call {call + 1}"
        assert _equal(_host(C), C_ref), f"last-column minors differ on call {call + 1}"


def test_noalloc_zero_pivot_and_size_limit(mpdet):
    import torch

    p = 512
    h = mpdet.Mpdet(2, p)
    h.set_i32(np.array([[0, 1], [1, 0]]))
    A = h.get_mp()
    h.close()
    D = _empty(2, p, torch)
    assert mpdet.factor_noalloc(_dev(A, torch), 2, p, D) == (mpdet.EZEROPIVOT, 1)
    # beyond the static working memory: a clear status, nothing launched
    big = _empty(600 * 600, p, torch)
    with pytest.raises(mpdet.MpdetError) as ei:
        mpdet.factor_noalloc(big, 600, p, _empty(600, p, torch))
    assert ei.value.code == mpdet.ENOSCRATCH
