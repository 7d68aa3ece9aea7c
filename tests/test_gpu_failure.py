"""Failure detection on the GPU without a fault: a bounded mbarrier wait on a
barrier that nothing completes must give up and report MPDET_ETIMEOUT (the
control, a barrier its block completes, reports OK), and the context must
stay usable afterwards: a factorisation right after it still equals the
oracle bit for bit."""
import numpy as np
import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(mpdet, oracle_lib):
    assert mpdet.selftest_timeout(limit=4096, arrive=True) == mpdet.OK
    assert mpdet.selftest_timeout(limit=4096, arrive=False) == mpdet.ETIMEOUT
    assert mpdet.selftest_timeout(limit=1, arrive=False) == mpdet.ETIMEOUT
    N, p = 40, 2048
    x, y = W.cauchy_xy(N, 777)
    h = mpdet.Mpdet(N, p, lastcol=True)
    h.set_cauchy(x, y)
    rc, zk, D = h.factor()
    h.close()
    st, ozk, OD, OX = oracle_lib.ge(oracle_lib.cauchy(x, y, p), N, p, lastcol=True)
    assert rc == st == 0 and X.same(D, OD)
