"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every function declared in include/*.h, and rejects bad
arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mpdet_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import paper_1308_1536_gb300 as m

    return m.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mpdet_create", "mpdet_factor", "mpdet_lastcol_minors", "mpdet_free", "mpdet_set_cauchy",
                     "mpdet_factor_range"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_geometry_and_invalid_precisions(lib):
    import paper_1308_1536_gb300 as m

    assert m.geometry(512) == (16, 16, 1)
    assert m.geometry(2048) == (64, 16, 4)
    assert m.geometry(32768) == (1024, 32, 32)
    # any multiple of 32 in [64, 32768]: n = p/32 limbs in the next family's frame (W x G limbs)
    assert m.geometry(64) == (2, 4, 1)
    assert m.geometry(96) == (3, 4, 1)
    assert m.geometry(160) == (5, 8, 1)
    assert m.geometry(3072) == (96, 16, 8)
    assert m.geometry(32736) == (1023, 32, 32)
    for p in (0, 32, 100, 1000, 32800, 65536):
        with pytest.raises(m.MpdetError):
            m.geometry(p)


def test_create_rejects_bad_arguments_without_a_device(lib):
    h = ctypes.c_void_p()
    assert lib.mpdet_create(0, 512, 0, None, ctypes.byref(h)) == 1  # N < 1
    assert lib.mpdet_create(8, 100, 0, None, ctypes.byref(h)) == 1  # p not supported
    assert lib.mpdet_create(8, 512, 0x10, None, ctypes.byref(h)) == 1  # unknown flag
    assert lib.mpdet_create(8, 512, 0, None, None) == 1  # no output
    assert lib.mpdet_free(None) == 0
    assert lib.mpdet_last_error(None) == b"no handle"


def test_more_entry_points_reject_bad_arguments_without_a_device(lib):
    import paper_1308_1536_gb300 as m

    h = ctypes.c_void_p()
    ns = (ctypes.c_int64 * 2)(8, 0)
    assert lib.mpdet_batch_create(2, ns, 512, None, ctypes.byref(h)) == m.EINVAL  # N = 0 in the batch
    assert lib.mpdet_batch_create(0, ns, 512, None, ctypes.byref(h)) == m.EINVAL  # empty batch
    assert lib.mpdet_batch_create(1, ns, 100, None, ctypes.byref(h)) == m.EINVAL  # bad precision
    assert lib.mpdet_batch_free(None) == m.OK
    assert lib.mpdet_batch_tune(None, 1, 0) == m.EINVAL
    assert lib.mpdet_batch_autotune(None, 1, None, None, None, None) == m.EINVAL
    assert lib.mpdet_batch_launches(None) == -1
    assert lib.mpdet_batch(0, ns, 512, None, None, None, 0, None) == m.EINVAL  # empty batch
    assert lib.mpdet_batch(2, ns, 512, None, None, None, 0, None) == m.EINVAL  # no buffers
    assert lib.mpdet_selftest_timeout(0, 0, None) == m.EINVAL  # limit < 1
    z = m.NumV(None, None, None)
    assert lib.mpdet_factor_noalloc(0, 512, 0, z, z, z, None, None) == m.EINVAL
    assert lib.mpdet_minor_series(None, z, 0, 0) == m.EINVAL
    assert lib.mpdet_get_entries(None, 0, None, z, 0) == m.EINVAL
    assert lib.mpdet_tune(None, 1, 0) == m.EINVAL
    assert lib.mpdet_steps_done(None) == -1
    assert lib.mpdet_radii(None, 0, None, None, 0) == m.EINVAL
    h2 = ctypes.c_void_p()
    assert lib.mpdet_create(8, 512, 0x8, None, ctypes.byref(h2)) == m.EINVAL  # unknown flag next to MPDET_BALL


def test_noalloc_size_limit_without_a_device(lib):
    """Sizes beyond the static working array are refused before any device
    work: N^2 (4n + 9) alone exceeds 16 MiB at N = 1024, p = 2048."""
    import paper_1308_1536_gb300 as m

    s8, e64, l32 = ctypes.c_int8(), ctypes.c_int64(), ctypes.c_uint32()  # never dereferenced
    v = m.NumV(ctypes.cast(ctypes.byref(s8), ctypes.c_void_p), ctypes.cast(ctypes.byref(e64), ctypes.c_void_p),
               ctypes.cast(ctypes.byref(l32), ctypes.c_void_p))
    assert lib.mpdet_factor_noalloc(1024, 2048, 0, v, v, v, None, None) == m.ENOSCRATCH
    assert lib.mpdet_factor_noalloc(479, 512, 0, v, v, v, None, None) == m.ENOSCRATCH
    assert lib.mpdet_factor_noalloc(8, 96, 0, v, v, v, None, None) == m.EINVAL  # power-of-two limb counts only


def test_one_shot_batch_checks_sizes_before_pointers(lib):
    """mpdet_batch validates count and every N before it reads the pointer
    arrays: a bad size is refused even though in[] holds one entry only."""
    import paper_1308_1536_gb300 as m

    s8, e64, l32 = ctypes.c_int8(), ctypes.c_int64(), ctypes.c_uint32()  # never dereferenced
    v = m.NumV(ctypes.cast(ctypes.byref(s8), ctypes.c_void_p), ctypes.cast(ctypes.byref(e64), ctypes.c_void_p),
               ctypes.cast(ctypes.byref(l32), ctypes.c_void_p))
    one = (m.NumV * 1)(v)
    ns = (ctypes.c_int64 * 2)(4, 0)
    assert lib.mpdet_batch(2, ns, 512, one, one, None, 0, None) == m.EINVAL  # N = 0 before in[1] is read
    assert lib.mpdet_batch((1 << 30) + 1, ns, 512, one, one, None, 0, None) == m.EINVAL


def test_mulbench_rejects_bad_arguments_without_a_device(lib):
    import paper_1308_1536_gb300 as m

    z = m.NumV(None, None, None)
    assert lib.mpdet_mulbench(2, 4, 8192, z, z, z, 1, None, None) == m.EINVAL  # unknown method
    assert lib.mpdet_mulbench(0, 4, 4096, z, z, z, 1, None, None) == m.EINVAL  # precision without a Karatsuba case
    assert lib.mpdet_mulbench(1, 0, 8192, z, z, z, 1, None, None) == m.EINVAL  # no pairs
    assert lib.mpdet_mulbench(1, 4, 8192, z, z, z, 1, None, None) == m.EINVAL  # null buffers
