"""CPU oracle for multiprecision Gaussian elimination without pivoting.

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()``
and the benchmark's ``cpu_baseline`` / reference leg may import this package.
The product path (the CUDA library and its binding) never calls it, and the two
share no code: this package reads nothing from ``paper_1308_1536_gb300``.

The arithmetic lives in ``mpdet_oracle.c`` (plain C, compiled with gcc on
first use); this module only marshals numpy arrays.

Number format (Sec. 4.3 fixes a p-bit working precision; the format is
this library's reading of it): x = (-1)^s * m * 2^(e-p) with m in
[2^(p-1), 2^p) stored as n = p/32 little-endian uint32 limbs and e an int64;
zero is s = 0, m = 0, e = INT64_MIN.  Arrays of numbers are the triple
``(sign int8[c], exp int64[c], limbs uint32[c, n])``.

Functions and the passages they follow:

* ``mul, add, sub, recip``: RN(a*b), RN(a+b), RN(a-b), RN(1/a), round to
  nearest even at p bits (the method's arithmetic at fixed precision).
* ``from_f64, from_int``: exact lift of the matrix entries.
* ``cauchy``: A_ij = RN(1/RN(x_i + y_j)), the seeded stand-in for the
  interpolating matrix of eq. (det).
* ``ge``: Gaussian elimination without pivoting (Sec. 3, Alg. 1 as read
  from the surrounding text); the running products of the pivots are the
  leading minors D_1..D_N; ``lastcol`` applies the row operations to the
  identity block of [A I] stored in A's strict lower triangle.
* ``lastcol_minors``: C_jN = D_{N-1} * l_Nj (eq. minorsdef) and the
  normalised minors of eq. (minors).
* ``minor_series``: the last-column minors of every leading size n = 1..N
  (the series of minor arrays for N = 2, 3, ... of Sec. 3).
* ``usolve``: X = A^-1 = U^-1 L from a lastcol elimination, the adjoint of
  log|det| (d log|det| / dA = A^-T; all minors are partial derivatives of
  the determinant, Sec. 3), by right-looking back substitution.
* ``to_f64``: round numbers to binary64 (nearest even, subnormals).
* ``cauchy_ball, ge_ball, lastcol_ball``: the same values, each with a
  rigorous radius (|exact - value| <= radius; midpoint-radius intervals, the
  rigorous bounds the paper leaves to future work, Sec. 4.4).  Radii are
  pairs (m uint32, e int64) meaning m * 2^(e - 32), rounded up; e = RAD_INF
  marks an unbounded radius.  ``rad_op`` exposes their arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpdet_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmpdet_oracle.so")
_lock = threading.Lock()
_lib = None

ZEXP = np.iinfo(np.int64).min

OK, EINVAL, ENOMEM, EZEROPIVOT, EZERODIV = 0, 1, 2, 4, 7


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    """Load the oracle library.  MPDET_ORACLE_LIB, when set, names another
    build of it to load instead: the mutation tests point it at copies with a
    planted mistake to show that the pins catch them."""
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(os.environ.get("MPDET_ORACLE_LIB") or build())
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int
            lib.or_mul_v.argtypes = [i64, i32, P, P, P, P, P, P, P, P, P]
            lib.or_add_v.argtypes = [i64, i32, i32, P, P, P, P, P, P, P, P, P]
            lib.or_recip_v.argtypes = [i64, i32, P, P, P, P, P, P]
            lib.or_from_f64_v.argtypes = [i64, i32, P, P, P, P]
            lib.or_from_i64_v.argtypes = [i64, i32, P, P, P, P]
            lib.or_cauchy.argtypes = [i64, i32, P, P, P, P, P]
            lib.or_ge_range.argtypes = [i64, i32, i32, i32, i64, i64, P, P, P, P, P, P, P]
            lib.or_ge_range_div.argtypes = [i64, i32, i32, i32, i64, i64, P, P, P, P, P, P, P]
            lib.or_div_v.argtypes = [i64, i32, P, P, P, P, P, P, P, P, P]
            lib.or_lastcol.argtypes = [i64, i32, i32, P, P, P, ctypes.c_int8, i64, P, P, P, P]
            lib.or_usolve.argtypes = [i64, i32, i32, P, P, P, P, P, P]
            lib.or_to_f64_v.argtypes = [i64, i32, P, P, P, P]
            lib.or_rad_op.argtypes = [i32, ctypes.c_uint32, i64, ctypes.c_uint32, i64, P, P, P]
            lib.or_cauchy_ball.argtypes = [i64, i32, P, P, P, P, P, P, P]
            lib.or_ge_ball.argtypes = [i64, i32, i32, P, P, P, P, P, P, P, P, P, P, P]
            lib.or_lastcol_ball.argtypes = [i64, i32, i32, P, P, P, P, P, ctypes.c_int8, i64, P, ctypes.c_uint32, i64,
                                            P, P, P, P, P]
            for f in ("or_mul_v", "or_add_v", "or_recip_v", "or_from_f64_v", "or_from_i64_v", "or_cauchy",
                      "or_ge_range", "or_ge_range_div", "or_div_v", "or_lastcol", "or_usolve", "or_to_f64_v",
                      "or_rad_op", "or_cauchy_ball", "or_ge_ball", "or_lastcol_ball"):
                getattr(lib, f).restype = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def empty(count: int, p: int):
    """Array of ``count`` numbers (all +0) at p bits."""
    n = p // 32
    return (np.zeros(count, np.int8), np.full(count, ZEXP, np.int64), np.zeros((count, n), np.uint32))


def _norm(x, p):
    s, e, m = x
    n = p // 32
    s = np.ascontiguousarray(s, np.int8).reshape(-1)
    e = np.ascontiguousarray(e, np.int64).reshape(-1)
    m = np.ascontiguousarray(m, np.uint32).reshape(-1, n)
    assert s.shape[0] == e.shape[0] == m.shape[0]
    return s, e, m


def _check(st, what):
    if st != OK:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def mul(a, b, p: int):
    a, b = _norm(a, p), _norm(b, p)
    c = a[0].shape[0]
    o = empty(c, p)
    _check(_load().or_mul_v(c, p, *map(_ptr, a), *map(_ptr, b), *map(_ptr, o)), "mul")
    return o


def add(a, b, p: int, negate_b: bool = False):
    a, b = _norm(a, p), _norm(b, p)
    c = a[0].shape[0]
    o = empty(c, p)
    _check(_load().or_add_v(c, p, int(negate_b), *map(_ptr, a), *map(_ptr, b), *map(_ptr, o)), "add")
    return o


def sub(a, b, p: int):
    return add(a, b, p, negate_b=True)


def div(a, b, p: int):
    """RN(a/b) with one rounding (not the method's multiplier, which is
    RN(a * RN(1/b)); an option for accuracy comparisons)."""
    a, b = _norm(a, p), _norm(b, p)
    c = a[0].shape[0]
    o = empty(c, p)
    _check(_load().or_div_v(c, p, *map(_ptr, a), *map(_ptr, b), *map(_ptr, o)), "div")
    return o


def recip(a, p: int):
    a = _norm(a, p)
    c = a[0].shape[0]
    o = empty(c, p)
    _check(_load().or_recip_v(c, p, *map(_ptr, a), *map(_ptr, o)), "recip")
    return o


def from_f64(v, p: int):
    v = np.ascontiguousarray(v, np.float64).reshape(-1)
    o = empty(v.shape[0], p)
    _check(_load().or_from_f64_v(v.shape[0], p, _ptr(v), *map(_ptr, o)), "from_f64")
    return o


def from_int(v, p: int):
    v = np.ascontiguousarray(v, np.int64).reshape(-1)
    o = empty(v.shape[0], p)
    _check(_load().or_from_i64_v(v.shape[0], p, _ptr(v), *map(_ptr, o)), "from_int")
    return o


def cauchy(x, y, p: int):
    """A_ij = RN(1/RN(x_i + y_j)), row-major N*N numbers."""
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    N = x.shape[0]
    assert y.shape[0] == N
    o = empty(N * N, p)
    _check(_load().or_cauchy(N, p, _ptr(x), _ptr(y), *map(_ptr, o)), "cauchy")
    return o


def ge(A, N: int, p: int, lastcol: bool = False, nthreads: int = 1, k0: int = 0, k_end: int | None = None,
       D=None, divide: bool = False):
    """Eliminate the row-major N x N matrix A (copied), returning
    ``(status, zero_k, D, X)``: D holds the leading minors D_1..D_N, X the
    in-place array after steps k0+1..k_end (U in the upper triangle; L's
    strict lower part in lastcol mode).  ``divide=True`` forms the
    multipliers as correctly rounded quotients RN(a_ik / a_kk) instead of
    the method's RN(a_ik * RN(1/a_kk)) (accuracy comparisons only)."""
    S, E, M = (np.array(t, copy=True) for t in _norm(A, p))
    assert S.shape[0] == N * N
    if D is None:
        D = empty(N, p)
    else:
        D = tuple(np.array(t, copy=True) for t in _norm(D, p))
    zk = np.zeros(1, np.int64)
    k_end = N if k_end is None else k_end
    fn = _load().or_ge_range_div if divide else _load().or_ge_range
    st = fn(N, p, int(lastcol), int(nthreads), k0, k_end, _ptr(S), _ptr(E), _ptr(M),
                             *map(_ptr, D), _ptr(zk))
    if st not in (OK, EZEROPIVOT):
        raise RuntimeError(f"oracle ge failed with status {st}")
    return st, int(zk[0]), D, (S, E, M)


def lastcol_minors(X, D, N: int, p: int, normalised: bool = False):
    """Signed last-column minors C_jN (or delta_{N,j}) from a lastcol-mode
    elimination result X with leading minors D."""
    S, E, M = _norm(X, p)
    Ds, De, Dm = _norm(D, p)
    if N >= 2:
        ds, de, dm = Ds[N - 2], De[N - 2], np.ascontiguousarray(Dm[N - 2])
    else:  # D_0 = 1
        ds, de = 0, 1
        dm = np.zeros(p // 32, np.uint32)
        dm[-1] = 0x80000000
    o = empty(N, p)
    st = _load().or_lastcol(N, p, int(normalised), _ptr(S), _ptr(E), _ptr(M), int(ds), int(de), _ptr(dm),
                            *map(_ptr, o))
    _check(st, "lastcol")
    return o


def minor_series(X, D, N: int, p: int, normalised: bool = False):
    """Last-column minors of every leading size n = 1..N from one lastcol-mode
    elimination (Sec. 3: at step n, row n of L holds the minors of the leading
    n x n matrix, up to the factor D_{n-1}).  Series n, at offset n(n-1)/2 of
    the packed result, is ``lastcol_minors`` of the leading n x n block of X
    with D_1..D_n; a normalised series whose l_n1 is zero (C_1n = 0, delta
    undefined) is left all +0."""
    S, E, M = _norm(X, p)
    Ds, De, Dm = _norm(D, p)
    out = empty(N * (N + 1) // 2, p)
    for r in range(N):
        nn = r + 1
        rows = np.arange(nn)[:, None] * N + np.arange(nn)[None, :]
        blk = (S[rows].reshape(-1), E[rows].reshape(-1), M[rows.reshape(-1)])
        if normalised:
            o = empty(nn, p)
            st = _load().or_lastcol(nn, p, 1, *map(_ptr, map(np.ascontiguousarray, blk)), 0, 1, _ptr(o[2][0]),
                                    *map(_ptr, o))
            if st == EZERODIV:
                continue
            _check(st, "lastcol")
        else:
            o = lastcol_minors(blk, (Ds[:nn], De[:nn], Dm[:nn]), nn, p)
        off = r * (r + 1) // 2
        for t, u in zip(out, o):
            t[off:off + nn] = u
    return out


def usolve(X, N: int, p: int, nthreads: int = 1):
    """A^-1 (N*N numbers, row-major) from a lastcol-mode elimination X."""
    S, E, M = _norm(X, p)
    o = empty(N * N, p)
    _check(_load().or_usolve(N, p, int(nthreads), _ptr(S), _ptr(E), _ptr(M), *map(_ptr, o)), "usolve")
    return o


def to_f64(x, p: int):
    S, E, M = _norm(x, p)
    out = np.zeros(S.shape[0], np.float64)
    _check(_load().or_to_f64_v(S.shape[0], p, _ptr(S), _ptr(E), _ptr(M), _ptr(out)), "to_f64")
    return out


def logabsdet(D, N: int, p: int):
    """(sign, log|det|) from the leading minors D (det = D_N): the mantissa
    as a double times 2^(e-p), logarithm taken in binary64."""
    import math

    s, e, m = (t[N - 1] for t in _norm(D, p))
    if int(e) == ZEXP:
        return 0.0, float("-inf")
    top = int(m[-1]) * 2.0 ** -32 + int(m[-2]) * 2.0 ** -64  # m / 2^p in [1/2, 1)
    return (-1.0 if int(s) else 1.0), math.log(top) + float(int(e)) * math.log(2.0)


# ---------------------------------------------------------------------------
# ball mode (values with rigorous radii)
# ---------------------------------------------------------------------------
RAD_INF = np.iinfo(np.int64).max


def rad_zeros(count: int):
    return np.zeros(count, np.uint32), np.full(count, ZEXP, np.int64)


def rad_op(op: int, a, b):
    """Radius arithmetic: op 0 a+b up, 1 a*b up, 2 a*b down, 3 a/b up,
    4 a-b down.  a, b: (m, e) pairs.  Returns ((m, e), positive)."""
    om, oe, pos = ctypes.c_uint32(), ctypes.c_int64(), ctypes.c_int()
    _check(_load().or_rad_op(int(op), int(a[0]), int(a[1]), int(b[0]), int(b[1]), ctypes.byref(om),
                             ctypes.byref(oe), ctypes.byref(pos)), "rad_op")
    return (int(om.value), int(oe.value)), bool(pos.value)


def cauchy_ball(x, y, p: int):
    """cauchy() with the radius of every entry (x, y exact)."""
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    N = x.shape[0]
    o = empty(N * N, p)
    r = rad_zeros(N * N)
    _check(_load().or_cauchy_ball(N, p, _ptr(x), _ptr(y), *map(_ptr, o), *map(_ptr, r)), "cauchy_ball")
    return o, r


def ge_ball(A, RA, N: int, p: int, lastcol: bool = False):
    """ge() over all steps with radii: RA are the input's radii (None:
    exact input).  Returns (status, zero_k, D, X, RD, RX); the values D, X
    are bit-identical to ge()'s."""
    S, E, M = (np.array(t, copy=True) for t in _norm(A, p))
    RXm, RXe = (rad_zeros(N * N) if RA is None else (np.array(RA[0], np.uint32, copy=True),
                                                        np.array(RA[1], np.int64, copy=True)))
    D = empty(N, p)
    RD = rad_zeros(N)
    zk = np.zeros(1, np.int64)
    st = _load().or_ge_ball(N, p, int(lastcol), _ptr(S), _ptr(E), _ptr(M), _ptr(RXm), _ptr(RXe), *map(_ptr, D),
                            *map(_ptr, RD), _ptr(zk))
    if st not in (OK, EZEROPIVOT):
        raise RuntimeError(f"oracle ge_ball failed with status {st}")
    return st, int(zk[0]), D, (S, E, M), RD, (RXm, RXe)


def lastcol_ball(X, RX, D, RD, N: int, p: int, normalised: bool = False):
    """lastcol_minors() with radii (from a lastcol-mode ge_ball)."""
    S, E, M = _norm(X, p)
    Ds, De, Dm = _norm(D, p)
    if N >= 2:
        ds, de, dm = Ds[N - 2], De[N - 2], np.ascontiguousarray(Dm[N - 2])
        rdm, rde = int(RD[0][N - 2]), int(RD[1][N - 2])
    else:
        ds, de = 0, 1
        dm = np.zeros(p // 32, np.uint32)
        dm[-1] = 0x80000000
        rdm, rde = 0, ZEXP
    o = empty(N, p)
    r = rad_zeros(N)
    RXm = np.ascontiguousarray(RX[0], np.uint32)
    RXe = np.ascontiguousarray(RX[1], np.int64)
    _check(_load().or_lastcol_ball(N, p, int(normalised), _ptr(S), _ptr(E), _ptr(M), _ptr(RXm), _ptr(RXe), int(ds),
                                   int(de), _ptr(dm), rdm, rde, *map(_ptr, o), *map(_ptr, r)), "lastcol_ball")
    return o, r
