"""The Python binding's buffer checks (CPU): every pointer it hands to the
library is a contiguous array of the element size, kind and count the call
reads or writes, in host or device memory as the call's mode says; anything
else raises before the library is called."""
import numpy as np
import pytest
import torch

import paper_1308_1536_gb300 as m


def triple(count, n):
    return (np.zeros(count, np.int8), np.full(count, m.ZEXP, np.int64), np.zeros((count, n), np.uint32))


def test_numv_accepts_the_number_triple():
    v = m._numv(triple(5, 16), 5, 16, False, "x")
    assert v.sign and v.exp and v.limbs
    # torch host tensors of the same layout, limbs as int32
    t = (torch.zeros(5, dtype=torch.int8), torch.zeros(5, dtype=torch.int64), torch.zeros((5, 16), dtype=torch.int32))
    assert m._numv(t, 5, 16, False, "x").limbs
    assert m._numv(None, 5, 16).sign is None
    assert m._numv(triple(5, 16), 4, 16, False, "x").limbs  # longer than needed is fine


@pytest.mark.parametrize("part,bad", [
    (0, np.zeros(5, np.int16)),                 # sign not int8
    (1, np.zeros(5, np.int32)),                 # exponent not int64
    (1, np.zeros(5, np.float64)),               # exponent not an integer
    (2, np.zeros((5, 16), np.float32)),         # limbs not integer
    (2, np.zeros((5, 8), np.uint32)),           # too few limbs
    (0, np.zeros(4, np.int8)),                  # too few numbers
    (2, np.zeros((16, 5), np.uint32).T),        # not contiguous
])
def test_numv_rejects_mistyped_or_short_parts(part, bad):
    t = list(triple(5, 16))
    t[part] = bad
    with pytest.raises(ValueError):
        m._numv(tuple(t), 5, 16, False, "x")


def test_ptr_checks_kind_count_and_memory():
    a = np.zeros(10, np.float64)
    assert m._ptr(a, 10, 8, True, False, "a")
    with pytest.raises(ValueError):
        m._ptr(np.zeros(10, np.int64), 10, 8, True, False, "a")  # integers where doubles are read
    with pytest.raises(ValueError):
        m._ptr(np.zeros(10, np.float32), 10, 8, True, False, "a")  # float32 where doubles are read
    with pytest.raises(ValueError):
        m._ptr(a, 11, 8, True, False, "a")
    with pytest.raises(ValueError):
        m._ptr(a, 10, 8, True, True, "a")  # host memory where the call reads device memory
    with pytest.raises(ValueError):
        m._ptr(torch.zeros(10, dtype=torch.float32), 10, 8, True, False, "a")
    with pytest.raises(TypeError):
        m._ptr([0.0] * 10, 10, 8, True, False, "a")
    assert m._ptr(None) is None
