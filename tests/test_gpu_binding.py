"""The binding refuses buffers the library would read or write past their end
or in the wrong memory, before any call reaches the library, and the handle
stays usable."""
import numpy as np
import pytest

from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_binding_refuses_short_mistyped_or_misplaced_buffers(mpdet):
    import torch

    N, p = 8, 512
    n = p // 32
    x, y = W.cauchy_xy(N, 3)
    h = mpdet.Mpdet(N, p, lastcol=True)
    h.set_cauchy(x, y)
    short = (torch.zeros(N - 1, dtype=torch.int8, device="cuda"), torch.zeros(N - 1, dtype=torch.int64, device="cuda"),
             torch.zeros((N - 1, n), dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        h.factor(out=short)
    host = (np.zeros(N, np.int8), np.zeros(N, np.int64), np.zeros((N, n), np.uint32))
    with pytest.raises(ValueError):
        h.lastcol_minors(out=host)  # host arrays where the call writes device memory
    with pytest.raises(ValueError):
        h.set_f64(torch.zeros((N, N), dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        h.set_cauchy(torch.tensor(x, device="cuda"), y)  # one device and one host operand
    rc, zk, D = h.factor()
    h.close()
    h2 = mpdet.Mpdet(N, p, lastcol=True)
    h2.set_cauchy(x, y)
    rc2, zk2, D2 = h2.factor()
    h2.close()
    assert (rc, zk) == (rc2, zk2) == (0, 0)
    assert all(np.array_equal(a, b) for a, b in zip(D, D2))
