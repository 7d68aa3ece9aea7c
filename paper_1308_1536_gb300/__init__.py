"""mpdet: multiprecision Gaussian elimination without pivoting on a GB300.

Thin Python binding over the C ABI of ``libmpdet.so`` (include/mpdet.h):
argument marshalling only.  Every step of the computation runs in the CUDA
kernels of the library; there is no CPU fallback, and ``load()`` raises when
the compiled library is missing or cannot be loaded.

Numbers cross the boundary as structure-of-arrays triples
``(sign int8[c], exp int64[c], limbs uint32[c, n])`` with
x = (-1)^sign * limbs * 2^(exp - p); zero is (0, INT64_MIN, 0).
Host inputs are numpy arrays; device inputs are torch CUDA tensors (passed
by pointer with ``device_ptr = 1``, asynchronous on the handle's stream).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ZEXP = np.iinfo(np.int64).min
OK, EINVAL, ENOMEM, ECUDA, EZEROPIVOT, ETIMEOUT, ESTATE, EZERODIV, ENOSCRATCH = range(9)
LASTCOL = 1
HOSTMEM = 2
BALL = 4
RAD_INF = np.iinfo(np.int64).max
_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EZEROPIVOT", 5: "ETIMEOUT", 6: "ESTATE",
          7: "EZERODIV", 8: "ENOSCRATCH"}

_lib = None


class MpdetError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mpdet {_NAMES.get(code, code)}: {msg}")
        self.code = code


class NumV(ctypes.Structure):
    _fields_ = [("sign", ctypes.c_void_p), ("exp", ctypes.c_void_p), ("limbs", ctypes.c_void_p)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmpdet.so (building it in-tree if missing and nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"libmpdet not built at {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    P, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
    sig = {
        "mpdet_create": ([i64, i32, u32, P, ctypes.POINTER(P)], ctypes.c_int),
        "mpdet_set_f64": ([P, P, i64, ctypes.c_int], ctypes.c_int),
        "mpdet_set_i32": ([P, P, i64, ctypes.c_int], ctypes.c_int),
        "mpdet_set_mp": ([P, NumV, ctypes.c_int], ctypes.c_int),
        "mpdet_set_cauchy": ([P, P, P, ctypes.c_int], ctypes.c_int),
        "mpdet_factor_range": ([P, i64, i64], ctypes.c_int),
        "mpdet_factor": ([P, NumV, NumV, ctypes.POINTER(i64), ctypes.c_int], ctypes.c_int),
        "mpdet_status": ([P, ctypes.POINTER(i64)], ctypes.c_int),
        "mpdet_lastcol_minors": ([P, NumV, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "mpdet_get_minors": ([P, NumV, ctypes.c_int], ctypes.c_int),
        "mpdet_get_mp": ([P, NumV, ctypes.c_int], ctypes.c_int),
        "mpdet_minor_series": ([P, NumV, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "mpdet_get_entries": ([P, i64, P, NumV, ctypes.c_int], ctypes.c_int),
        "mpdet_resume": ([P, NumV, NumV, i64, ctypes.c_int], ctypes.c_int),
        "mpdet_steps_done": ([P], i64),
        "mpdet_free": ([P], ctypes.c_int),
        "mpdet_last_error": ([P], ctypes.c_char_p),
        "mpdet_geometry": ([i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)], ctypes.c_int),
        "mpdet_profile": ([P, ctypes.c_int], ctypes.c_int),
        "mpdet_tune": ([P, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "mpdet_batch_create": ([i64, P, i32, P, ctypes.POINTER(P)], ctypes.c_int),
        "mpdet_batch_set_f64": ([P, i64, P, i64, ctypes.c_int], ctypes.c_int),
        "mpdet_batch_set_i32": ([P, i64, P, i64, ctypes.c_int], ctypes.c_int),
        "mpdet_batch_set_cauchy": ([P, i64, P, P, ctypes.c_int], ctypes.c_int),
        "mpdet_batch_set_mp": ([P, i64, NumV, ctypes.c_int], ctypes.c_int),
        "mpdet_batch_factor": ([P, NumV, P, ctypes.c_int], ctypes.c_int),
        "mpdet_batch_launches": ([P], i64),
        "mpdet_batch_tune": ([P, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "mpdet_batch_variant_info": ([P, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                      ctypes.POINTER(i32), ctypes.POINTER(i32)], ctypes.c_int),
        "mpdet_batch_autotune": ([P, ctypes.c_int, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)], ctypes.c_int),
        "mpdet_batch_free": ([P], ctypes.c_int),
        "mpdet_batch": ([i64, P, i32, P, P, P, ctypes.c_int, P], ctypes.c_int),
        "mpdet_logabsdet_grad": ([P, P, i64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), P,
                                  ctypes.c_double, ctypes.c_int], ctypes.c_int),
        "mpdet_get_inverse": ([P, NumV, ctypes.c_int], ctypes.c_int),
        "mpdet_ops": ([ctypes.c_int, i64, i32, NumV, NumV, NumV, P], ctypes.c_int),
        "mpdet_factor_noalloc": ([i64, i32, u32, NumV, NumV, NumV, ctypes.POINTER(i64), P], ctypes.c_int),
        "mpdet_radii": ([P, ctypes.c_int, P, P, ctypes.c_int], ctypes.c_int),
        "mpdet_mulbench": ([ctypes.c_int, i64, i32, NumV, NumV, NumV, ctypes.c_int, P, ctypes.POINTER(ctypes.c_float)],
                           ctypes.c_int),
        "mpdet_selftest_timeout": ([i32, ctypes.c_int, P], ctypes.c_int),
        "mpdet_profile_read": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def geometry(p: int):
    """(n, W, G): limbs per number, limbs per lane, lanes per number."""
    lib = load()
    n, W, G = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    rc = lib.mpdet_geometry(p, ctypes.byref(n), ctypes.byref(W), ctypes.byref(G))
    if rc:
        raise MpdetError(rc, f"unsupported precision p = {p}")
    return n.value, W.value, G.value


def factor_noalloc(A, N: int, p: int, minors, lastcol=None, stream=None):
    """Elimination with no allocation (mpdet_factor_noalloc): A, minors and
    lastcol are triples of CUDA tensors (device memory); the library keeps its
    working memory in a static device array.  Returns (status, zero_k)."""
    lib = load()
    if stream is None:
        import torch

        stream = torch.cuda.current_stream().cuda_stream
    zk = ctypes.c_int64(0)
    N, n = int(N), int(p) // 32
    rc = lib.mpdet_factor_noalloc(N, int(p), LASTCOL if lastcol is not None else 0, _numv(A, N * N, n, True, "A"),
                                  _numv(minors, N, n, True, "minors"), _numv(lastcol, N, n, True, "lastcol"),
                                  ctypes.byref(zk), ctypes.c_void_p(stream or 0))
    if rc not in (OK, EZEROPIVOT):
        raise MpdetError(rc, f"factor_noalloc(N={N}, p={p})")
    return rc, int(zk.value)


def selftest_timeout(limit: int = 4096, arrive: bool = False, stream=None) -> int:
    """Run one bounded mbarrier wait (at most ``limit`` polls) on a barrier
    nothing completes (or, with ``arrive``, one the block completes itself);
    returns the status code: ETIMEOUT when the wait ran out, OK otherwise."""
    lib = load()
    if stream is None:
        import torch

        stream = torch.cuda.current_stream().cuda_stream
    rc = lib.mpdet_selftest_timeout(int(limit), int(bool(arrive)), ctypes.c_void_p(stream or 0))
    if rc not in (OK, ETIMEOUT):
        raise MpdetError(rc, "selftest_timeout")
    return rc


def ops(op: str, a, b, p: int):
    """Element-wise RN(a*b) ('mul'), RN(a-b) ('sub'), RN(a+b) ('add') or
    RN(1/a) ('recip') on the GPU; a, b host triples; returns a host triple."""
    import torch

    code = {"mul": 0, "sub": 1, "add": 2, "recip": 3}[op]
    lib = load()
    count = len(a[0])
    dev = lambda t: (torch.from_numpy(np.ascontiguousarray(t[0])).cuda(), torch.from_numpy(np.ascontiguousarray(t[1])).cuda(),
                     torch.from_numpy(np.ascontiguousarray(t[2]).view(np.int32)).cuda())
    A, B = dev(a), dev(b if b is not None else a)
    O = dev(empty(count, p))
    rc = lib.mpdet_ops(code, count, p, _numv(A), _numv(B), _numv(O), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc:
        raise MpdetError(rc, f"ops({op})")
    return (O[0].cpu().numpy(), O[1].cpu().numpy(), O[2].cpu().numpy().view(np.uint32))


def mulbench(method: str, a, b, p: int, reps: int = 1):
    """RN(a[i] * b[i]) at p bits (8192, 16384 or 32768) by the schoolbook
    ("school") or the one-level Karatsuba ("kara") product of the IMAD engine,
    each formed ``reps`` times (mpdet_mulbench).  a, b: host triples.
    Returns (products triple, device milliseconds)."""
    import torch

    lib = load()
    count = len(a[0])
    dev = lambda t: (torch.from_numpy(np.ascontiguousarray(t[0])).cuda(), torch.from_numpy(np.ascontiguousarray(t[1])).cuda(),
                     torch.from_numpy(np.ascontiguousarray(t[2]).view(np.int32)).cuda())
    A, B, O = dev(a), dev(b), dev(empty(count, p))
    ms = ctypes.c_float(0.0)
    rc = lib.mpdet_mulbench({"school": 0, "kara": 1}[method], count, p, _numv(A), _numv(B), _numv(O), int(reps),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(ms))
    if rc:
        raise MpdetError(rc, f"mulbench({method}, p={p})")
    return (O[0].cpu().numpy(), O[1].cpu().numpy(), O[2].cpu().numpy().view(np.uint32)), float(ms.value)


def empty(count: int, p: int):
    n = p // 32
    return (np.zeros(count, np.int8), np.full(count, ZEXP, np.int64), np.zeros((count, n), np.uint32))


def _is_dev(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


def _is_torch(a) -> bool:
    return hasattr(a, "data_ptr") and hasattr(a, "is_cuda")


def _ptr(a, count=None, itemsize=None, floating=None, dev=None, what="buffer"):
    """The address of a contiguous numpy array or torch tensor, checked
    against what the library will read or write there: at least ``count``
    elements of ``itemsize`` bytes, floating point or integer, and device
    memory (a CUDA tensor) when ``dev`` is True, host memory when False.
    The library trusts its pointers, so a short or mistyped buffer would be
    read or written past its end; these checks raise ValueError first."""
    if a is None:
        return None
    if _is_torch(a):  # CUDA tensor (device pointer) or pinned / CPU tensor (host pointer)
        contig, nel, isz, isf = a.is_contiguous(), a.numel(), a.element_size(), a.is_floating_point()
    elif isinstance(a, np.ndarray):
        contig, nel, isz, isf = a.flags.c_contiguous, a.size, a.itemsize, a.dtype.kind == "f"
    else:
        raise TypeError(f"{what}: a numpy array or a torch tensor, not {type(a).__name__}")
    if not contig:
        raise ValueError(f"{what}: not contiguous")
    if itemsize is not None and isz != itemsize:
        raise ValueError(f"{what}: elements of {isz} bytes, {itemsize} expected")
    if floating is not None and bool(isf) != floating:
        raise ValueError(f"{what}: {'floating-point' if floating else 'integer'} elements expected")
    if count is not None and nel < count:
        raise ValueError(f"{what}: {nel} elements, at least {count} needed")
    if dev is not None and _is_dev(a) != dev:
        raise ValueError(f"{what}: {'device (a CUDA tensor)' if dev else 'host'} memory expected")
    if _is_torch(a):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _numv(t, count=None, n=None, dev=None, what="numbers") -> NumV:
    """A (sign int8, exp int64, limbs uint32) triple as the ABI's view, each
    part checked by _ptr for ``count`` numbers of ``n`` limbs."""
    if t is None:
        return NumV(None, None, None)
    s, e, m = t
    lim = None if count is None or n is None else count * n
    return NumV(_ptr(s, count, 1, False, dev, f"{what} (sign)"), _ptr(e, count, 8, False, dev, f"{what} (exp)"),
                _ptr(m, lim, 4, False, dev, f"{what} (limbs)"))


class Mpdet:
    """One N x N matrix at p bits on the current CUDA device.

    ``lastcol=True`` keeps L in A's strict lower triangle so that the signed
    minors of the last column are available after the factorisation.
    ``hostmem=True`` keeps the N x N array in page-locked host memory that
    the GPU reads and writes in place (matrices larger than HBM).
    """

    def __init__(self, N: int, p: int, lastcol: bool = False, stream=None, hostmem: bool = False, ball: bool = False):
        self.lib = load()
        self.N, self.p, self.n = int(N), int(p), int(p) // 32
        self.lastcol = bool(lastcol)
        if stream is None:
            try:
                import torch

                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
            except Exception:  # torch without CUDA: legacy default stream
                stream = None
        self.stream = stream
        h = ctypes.c_void_p()
        flags = (LASTCOL if lastcol else 0) | (HOSTMEM if hostmem else 0) | (BALL if ball else 0)
        rc = self.lib.mpdet_create(self.N, self.p, flags, ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if rc:
            raise MpdetError(rc, f"create(N={N}, p={p})")
        self.h = h

    # -- lifetime -----------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.mpdet_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc, what, ok=(OK,)):
        if rc not in ok:
            raise MpdetError(rc, f"{what}: {self.lib.mpdet_last_error(self.h).decode(errors='replace')}")
        return rc

    # -- inputs -------------------------------------------------------------
    def set_f64(self, A, ld=None):
        dev = _is_dev(A)
        if not dev and not _is_torch(A):
            A = np.ascontiguousarray(A, np.float64)
        ld = self.N if ld is None else int(ld)
        if ld < self.N:
            raise ValueError(f"set_f64: ld = {ld} < N = {self.N}")
        A_ = _ptr(A, (self.N - 1) * ld + self.N, 8, True, dev, "set_f64: A")
        self._check(self.lib.mpdet_set_f64(self.h, A_, ld, int(dev)), "set_f64")

    def set_i32(self, A, ld=None):
        dev = _is_dev(A)
        if not dev and not _is_torch(A):
            A = np.ascontiguousarray(A, np.int32)
        ld = self.N if ld is None else int(ld)
        if ld < self.N:
            raise ValueError(f"set_i32: ld = {ld} < N = {self.N}")
        A_ = _ptr(A, (self.N - 1) * ld + self.N, 4, False, dev, "set_i32: A")
        self._check(self.lib.mpdet_set_i32(self.h, A_, ld, int(dev)), "set_i32")

    def set_cauchy(self, x, y):
        dev = _is_dev(x)
        if not dev and not _is_torch(x):
            x = np.ascontiguousarray(x, np.float64)
            y = np.ascontiguousarray(y, np.float64)
        x_ = _ptr(x, self.N, 8, True, dev, "set_cauchy: x")
        y_ = _ptr(y, self.N, 8, True, dev, "set_cauchy: y")
        self._check(self.lib.mpdet_set_cauchy(self.h, x_, y_, int(dev)), "set_cauchy")

    def set_mp(self, A):
        dev = _is_dev(A[0])
        if not dev:
            A = tuple(np.ascontiguousarray(t) for t in A)
        self._check(self.lib.mpdet_set_mp(self.h, _numv(A, self.N * self.N, self.n, dev, "set_mp: A"), int(dev)),
                    "set_mp")

    # -- elimination --------------------------------------------------------
    def factor_range(self, k0: int, k1: int):
        self._check(self.lib.mpdet_factor_range(self.h, k0, k1), "factor_range")

    def factor(self, out=None):
        """Run the remaining steps.  Host mode (out=None): returns
        (status, zero_k, minors) with minors = D_1..D_N (det = minors[-1]).
        Device mode: ``out`` is a triple of CUDA tensors for D_1..D_N; the
        call is asynchronous and returns None."""
        zk = ctypes.c_int64(0)
        if out is not None:
            self._check(self.lib.mpdet_factor(self.h, NumV(None, None, None), _numv(out, self.N, self.n, True, "factor: out"),
                                              ctypes.byref(zk), 1), "factor")
            return None
        D = empty(self.N, self.p)
        rc = self._check(self.lib.mpdet_factor(self.h, NumV(None, None, None), _numv(D), ctypes.byref(zk), 0),
                         "factor", ok=(OK, EZEROPIVOT))
        return rc, int(zk.value), D

    def status(self):
        zk = ctypes.c_int64(0)
        rc = self._check(self.lib.mpdet_status(self.h, ctypes.byref(zk)), "status", ok=(OK, EZEROPIVOT))
        return rc, int(zk.value)

    def lastcol_minors(self, normalised: bool = False, out=None):
        if out is not None:
            self._check(self.lib.mpdet_lastcol_minors(self.h, _numv(out, self.N, self.n, True, "lastcol_minors: out"),
                                                      int(normalised), 1), "lastcol_minors")
            return None
        C = empty(self.N, self.p)
        self._check(self.lib.mpdet_lastcol_minors(self.h, _numv(C), int(normalised), 0), "lastcol_minors")
        return C

    def minor_series(self, normalised: bool = False, out=None):
        """Last-column minors of every leading size n = 1..N (packed: series n
        at offset n(n-1)/2)."""
        if out is not None:
            cnt = self.N * (self.N + 1) // 2
            self._check(self.lib.mpdet_minor_series(self.h, _numv(out, cnt, self.n, True, "minor_series: out"),
                                                    int(normalised), 1), "minor_series")
            return None
        S = empty(self.N * (self.N + 1) // 2, self.p)
        self._check(self.lib.mpdet_minor_series(self.h, _numv(S), int(normalised), 0), "minor_series")
        return S

    def get_entries(self, idx):
        """Entries idx (flat row-major indices) of the in-place array."""
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        out = empty(len(idx), self.p)
        self._check(self.lib.mpdet_get_entries(self.h, len(idx), idx.ctypes.data_as(ctypes.c_void_p), _numv(out), 0),
                    "get_entries")
        return out

    def radii(self, which: str = "minors"):
        """Ball mode (ball=True): radii of the leading minors ("minors"), of
        the last mpdet_lastcol_minors result ("lastcol") or of the in-place
        array ("array"), as (mantissa uint32, exponent int64) arrays: radius
        = mantissa * 2^(exponent - 32); exponent RAD_INF: unbounded."""
        w = {"minors": 0, "lastcol": 1, "array": 2}[which]
        cnt = self.N * self.N if w == 2 else self.N
        rm, re_ = np.zeros(cnt, np.uint32), np.zeros(cnt, np.int64)
        self._check(self.lib.mpdet_radii(self.h, w, rm.ctypes.data_as(ctypes.c_void_p),
                                         re_.ctypes.data_as(ctypes.c_void_p), 0), "radii")
        return rm, re_

    def get_minors(self):
        D = empty(self.N, self.p)
        self._check(self.lib.mpdet_get_minors(self.h, _numv(D), 0), "get_minors")
        return D

    def get_mp(self):
        X = empty(self.N * self.N, self.p)
        self._check(self.lib.mpdet_get_mp(self.h, _numv(X), 0), "get_mp")
        return X

    def resume(self, X, D, k_done: int):
        X = tuple(np.ascontiguousarray(t) for t in X)
        D = tuple(np.ascontiguousarray(t) for t in D)
        self._check(self.lib.mpdet_resume(self.h, _numv(X, self.N * self.N, self.n, False, "resume: X"),
                                          _numv(D, self.N, self.n, False, "resume: D"), int(k_done), 0), "resume")

    def steps_done(self) -> int:
        return int(self.lib.mpdet_steps_done(self.h))

    # -- adjoint --------------------------------------------------------------
    def logabsdet_grad(self, A, grad: bool = True, scale: float = 1.0, out=None):
        """(sign, log|det|, G) for the binary64 matrix A (numpy or CUDA
        tensor): G = scale * A^-T rounded to binary64 (None if grad=False).
        With a CUDA tensor A the gradient is written to ``out`` (a CUDA
        float64 tensor, allocated if None) and returned."""
        dev = _is_dev(A)
        if not dev and not _is_torch(A):
            A = np.ascontiguousarray(A, np.float64)
        la, sg = ctypes.c_double(), ctypes.c_int()
        G = None
        if grad:
            if dev:
                import torch

                G = out if out is not None else torch.empty((self.N, self.N), dtype=torch.float64, device=A.device)
            else:
                G = np.empty((self.N, self.N), np.float64)
        NN = self.N * self.N
        A_ = _ptr(A, NN, 8, True, dev, "logabsdet_grad: A")
        G_ = _ptr(G, NN, 8, True, dev, "logabsdet_grad: out")
        rc = self.lib.mpdet_logabsdet_grad(self.h, A_, self.N, ctypes.byref(la), ctypes.byref(sg), G_, float(scale),
                                           int(dev))
        self._check(rc, "logabsdet_grad")
        return sg.value, la.value, G

    def get_inverse(self):
        Xi = empty(self.N * self.N, self.p)
        self._check(self.lib.mpdet_get_inverse(self.h, _numv(Xi), 0), "get_inverse")
        return Xi

    # -- tuning (bit-identical results for every setting) -------------------
    def tune(self, update_variant: int | None = None, engine: int | None = None, tc_min_rows: int | None = None,
             lookahead: bool | None = None, lookahead_reserve: int | None = None, update_geometry: int | None = None,
             karatsuba: bool | None = None):
        """update_variant: IMAD update register budget 0..3; engine: 1 tensor
        cores (p = 512, 1024, 2048), 2 the same one phase at a time (p =
        2048), 0 IMAD; tc_min_rows: update launches of fewer rows take the
        IMAD kernel; lookahead: overlap step k+1's pivot and multipliers with
        step k's update on a second stream; lookahead_reserve: SMs left to
        that stream; update_geometry: IMAD update lane geometry (0 own, 1/2
        32 limbs per lane for 4/3 blocks per SM, -1 per precision); karatsuba:
        the IMAD update's products by one Karatsuba level (p >= 8192).
        Results are bit-identical for every setting."""
        for key, val in ((1, update_variant), (2, engine), (3, tc_min_rows), (4, lookahead), (5, lookahead_reserve),
                         (6, update_geometry), (7, karatsuba)):
            if val is not None:
                self._check(self.lib.mpdet_tune(self.h, key, int(val)), "tune")

    # -- instrumentation ----------------------------------------------------
    def profile(self, enable: bool = True):
        self._check(self.lib.mpdet_profile(self.h, int(enable)), "profile")

    def profile_read(self):
        """dict(update_ms, update_launches, update_limb_macs, launches)."""
        ms, nl, macs, total = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
        self._check(self.lib.mpdet_profile_read(self.h, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(macs),
                                                ctypes.byref(total)), "profile_read")
        return dict(update_ms=ms.value, update_launches=nl.value, update_limb_macs=macs.value, launches=total.value)


def batch_once(mats, p: int, stream=None):
    """One-shot batch (mpdet_batch): ``mats`` is a list of triples of
    N_m * N_m numbers (row-major), all host arrays or all CUDA tensors;
    returns (zero_k[count], [minors triple of each matrix]) in the same kind
    of memory.  Allocates and frees the batch's device memory inside the
    call, which synchronises the stream."""
    lib = load()
    n = int(p) // 32
    Ns = np.array([int(round(len(t[0]) ** 0.5)) for t in mats], dtype=np.int64)
    dev = _is_dev(mats[0][0])
    if dev:
        import torch

        ins = [tuple(a.contiguous() for a in t) for t in mats]
        outs = [(torch.zeros(int(N), dtype=torch.int8, device=t[0].device),
                 torch.zeros(int(N), dtype=torch.int64, device=t[0].device),
                 torch.zeros((int(N), n), dtype=torch.int32, device=t[0].device)) for N, t in zip(Ns, ins)]
        zk = torch.zeros(len(mats), dtype=torch.int64, device=ins[0][0].device)
    else:
        ins = [tuple(np.ascontiguousarray(a) for a in _norm_host(t, n)) for t in mats]
        outs = [empty(int(N), p) for N in Ns]
        zk = np.zeros(len(mats), np.int64)
    in_arr = (NumV * len(mats))(*[_numv(t, int(N) * int(N), n, dev, f"batch: matrix {i}")
                                  for i, (N, t) in enumerate(zip(Ns, ins))])
    out_arr = (NumV * len(mats))(*[_numv(t) for t in outs])
    if stream is None:
        try:
            import torch

            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
        except Exception:
            stream = None
    rc = lib.mpdet_batch(len(mats), Ns.ctypes.data_as(ctypes.c_void_p), int(p), ctypes.cast(in_arr, ctypes.c_void_p),
                         ctypes.cast(out_arr, ctypes.c_void_p), _ptr(zk), int(dev), ctypes.c_void_p(stream or 0))
    if rc:
        raise MpdetError(rc, f"batch(count={len(mats)}, p={p})")
    return zk, outs


def _norm_host(t, n):
    s, e, m = t
    return (np.asarray(s, np.int8).reshape(-1), np.asarray(e, np.int64).reshape(-1),
            np.asarray(m, np.uint32).reshape(-1, n))


def tune_cache_key(device: str, p: int, Ns) -> str:
    """Key of a batch autotuner choice: the device, the precision and the
    size mix (count, and the matrices per N bucket of width 32, which is what
    the persistent kernel's load balance depends on)."""
    Ns = np.asarray(Ns, dtype=np.int64)
    hist = np.bincount(np.minimum(Ns // 32, 63), minlength=64)
    return f"{device}|p={int(p)}|count={len(Ns)}|hist32=" + ",".join(str(int(v)) for v in hist)


class TuneCache:
    """A JSON file of autotuner choices: {key: {variant, blocks_per_sm, ms,
    candidates}}.  Written whole to a temporary file and renamed."""

    def __init__(self, path: str):
        self.path = path

    def _load(self) -> dict:
        import json

        try:
            with open(self.path) as f:
                d = json.load(f)
            return d if isinstance(d, dict) else {}
        except (OSError, ValueError):
            return {}

    def get(self, key: str):
        return self._load().get(key)

    def put(self, key: str, value: dict) -> None:
        import json

        d = self._load()
        d[key] = value
        tmp = f"{self.path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


class Batch:
    """Many independent matrices of sizes Ns at p bits, factored in one
    persistent launch (det and leading minors of each)."""

    def __init__(self, Ns, p: int, stream=None):
        self.lib = load()
        self.Ns = np.ascontiguousarray(np.asarray(Ns, dtype=np.int64))
        self.p, self.n = int(p), int(p) // 32
        self.offsets = np.concatenate([[0], np.cumsum(self.Ns)]).astype(np.int64)
        if stream is None:
            try:
                import torch

                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
            except Exception:
                stream = None
        h = ctypes.c_void_p()
        rc = self.lib.mpdet_batch_create(len(self.Ns), self.Ns.ctypes.data_as(ctypes.c_void_p), self.p,
                                         ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if rc:
            raise MpdetError(rc, f"batch_create(count={len(self.Ns)}, p={p})")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.mpdet_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc:
            raise MpdetError(rc, what)

    def _size(self, m) -> int:
        m = int(m)
        if not 0 <= m < len(self.Ns):
            raise IndexError(f"matrix {m} of a batch of {len(self.Ns)}")
        return int(self.Ns[m])

    def set_cauchy(self, m, x, y):
        N = self._size(m)
        dev = _is_dev(x)
        if not dev and not _is_torch(x):
            x = np.ascontiguousarray(x, np.float64)
            y = np.ascontiguousarray(y, np.float64)
        x_ = _ptr(x, N, 8, True, dev, "batch set_cauchy: x")
        y_ = _ptr(y, N, 8, True, dev, "batch set_cauchy: y")
        self._check(self.lib.mpdet_batch_set_cauchy(self.h, int(m), x_, y_, int(dev)), "batch_set_cauchy")

    def set_i32(self, m, A):
        dev = _is_dev(A)
        if not dev and not _is_torch(A):
            A = np.ascontiguousarray(A, np.int32)
        N = self._size(m)
        self._check(self.lib.mpdet_batch_set_i32(self.h, int(m), _ptr(A, N * N, 4, False, dev, "batch set_i32: A"), N,
                                                 int(dev)), "batch_set_i32")

    def set_f64(self, m, A):
        dev = _is_dev(A)
        if not dev and not _is_torch(A):
            A = np.ascontiguousarray(A, np.float64)
        N = self._size(m)
        self._check(self.lib.mpdet_batch_set_f64(self.h, int(m), _ptr(A, N * N, 8, True, dev, "batch set_f64: A"), N,
                                                 int(dev)), "batch_set_f64")

    def set_mp(self, m, A):
        """Matrix m from N_m * N_m numbers already at p bits (a triple of host
        arrays, or of CUDA tensors for device memory), row-major, canonical."""
        dev = _is_dev(A[0])
        if not dev:
            A = tuple(np.ascontiguousarray(a) for a in _norm_host(A, self.n))
        N = self._size(m)
        self._check(self.lib.mpdet_batch_set_mp(self.h, int(m), _numv(A, N * N, self.n, dev, "batch set_mp: A"),
                                                int(dev)), "batch_set_mp")

    def factor(self, out=None, zero_k=None):
        """Host mode: returns (zero_k[count], minors triple of sum(N) numbers);
        matrix m's minors are rows offsets[m]:offsets[m+1].  Device mode:
        ``out`` (and optionally ``zero_k``) are CUDA tensors; asynchronous."""
        if out is not None:
            tot = int(self.offsets[-1])
            self._check(self.lib.mpdet_batch_factor(self.h, _numv(out, tot, self.n, True, "batch factor: out"),
                                                    _ptr(zero_k, len(self.Ns), 8, False, True, "batch factor: zero_k"), 1),
                        "batch_factor")
            return None
        D = empty(int(self.offsets[-1]), self.p)
        zk = np.zeros(len(self.Ns), np.int64)
        self._check(self.lib.mpdet_batch_factor(self.h, _numv(D), zk.ctypes.data_as(ctypes.c_void_p), 0),
                    "batch_factor")
        return zk, D

    def tune(self, variant: int | None = None, blocks_per_sm: int | None = None, graph: bool | None = None):
        """Lane-geometry variant, resident blocks per SM and CUDA-graph replay
        of the persistent launch (results are identical for every setting)."""
        if variant is not None:
            self._check(self.lib.mpdet_batch_tune(self.h, 1, int(variant)), "batch_tune(variant)")
        if blocks_per_sm is not None:
            self._check(self.lib.mpdet_batch_tune(self.h, 2, int(blocks_per_sm)), "batch_tune(blocks_per_sm)")
        if graph is not None:
            self._check(self.lib.mpdet_batch_tune(self.h, 3, int(bool(graph))), "batch_tune(graph)")

    def variants(self):
        """[(W, G, PW, PG, max_blocks_per_sm)] of every lane-geometry variant."""
        out, v = [], 0
        while True:
            a = [ctypes.c_int32() for _ in range(5)]
            if self.lib.mpdet_batch_variant_info(self.h, v, *map(ctypes.byref, a)):
                return out
            out.append(tuple(int(x.value) for x in a))
            v += 1

    def autotune(self, reps: int = 1, cache: str | None = None):
        """Time every variant (occupancy limit and half of it), keep the
        fastest: dict(variant, blocks_per_sm, ms, candidates).  With
        ``cache`` (a JSON file path) a choice stored for the same device,
        precision and size mix is applied without timing, and a new one is
        stored."""
        key = None
        if cache is not None:
            key = tune_cache_key(self._device_name(), self.p, self.Ns)
            hit = TuneCache(cache).get(key)
            if hit is not None and 0 <= hit.get("variant", -1) < len(self.variants()):
                self.tune(variant=hit["variant"], blocks_per_sm=hit["blocks_per_sm"])
                return dict(hit, cached=True)
        v, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        ms = ctypes.c_double()
        self._check(self.lib.mpdet_batch_autotune(self.h, int(reps), ctypes.byref(v), ctypes.byref(b),
                                                  ctypes.byref(ms), ctypes.byref(c)), "batch_autotune")
        res = dict(variant=v.value, blocks_per_sm=b.value, ms=ms.value, candidates=c.value)
        if key is not None:
            TuneCache(cache).put(key, res)
        return res

    @staticmethod
    def _device_name() -> str:
        try:
            import torch

            props = torch.cuda.get_device_properties(torch.cuda.current_device())
            return f"{props.name} sm_{props.major}{props.minor} x{props.multi_processor_count}"
        except Exception:
            return "unknown"

    def minors_of(self, D, m):
        a, b = int(self.offsets[m]), int(self.offsets[m + 1])
        return tuple(t[a:b] for t in D)

    def launches(self) -> int:
        return int(self.lib.mpdet_batch_launches(self.h))


_grad_handles = {}


def _handle_for(N: int, p: int, device):
    import torch

    key = (N, p, device)
    h = _grad_handles.get(key)
    if h is None:
        with torch.cuda.device(device):
            h = _grad_handles[key] = Mpdet(N, p, lastcol=True)
    return h


def mp_logabsdet(A, p: int = 4096):
    """log|det(A)| of a float64 CUDA matrix, computed at p bits, as a
    differentiable torch op: backward returns grad * A^-T from the adjoint
    kernels (the factor is recomputed in the backward pass, not stored)."""
    import torch

    class _MpLogDet(torch.autograd.Function):
        @staticmethod
        def forward(ctx, A_):
            h = _handle_for(A_.shape[0], p, A_.device)
            Ac = A_.detach().contiguous()
            s, la, _ = h.logabsdet_grad(Ac, grad=False)
            ctx.save_for_backward(Ac)
            ctx.sign = s
            return torch.tensor(la, dtype=torch.float64, device=A_.device)

        @staticmethod
        def backward(ctx, g):
            (Ac,) = ctx.saved_tensors
            h = _handle_for(Ac.shape[0], p, Ac.device)
            _, _, G = h.logabsdet_grad(Ac, grad=True, scale=float(g.item()))
            return G

    return _MpLogDet.apply(A)
