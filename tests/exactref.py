"""Exact rational reference for pinning the oracle (test helper).

Independent of both the oracle and the CUDA library: numbers are converted to
``fractions.Fraction`` and rounded back with an integer-only round-to-nearest-
even written here from the definition of the format

    x = (-1)^s * m * 2^(e-p),  2^(p-1) <= m < 2^p,  zero = (0, INT64_MIN, 0).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

ZEXP = np.iinfo(np.int64).min


def limbs_to_int(limbs) -> int:
    v = 0
    for i, w in enumerate(np.asarray(limbs, dtype=np.uint64).tolist()):
        v |= int(w) << (32 * i)
    return v


def int_to_limbs(v: int, n: int) -> np.ndarray:
    return np.array([(v >> (32 * i)) & 0xFFFFFFFF for i in range(n)], dtype=np.uint32)


def to_fraction(s, e, limbs, p: int) -> Fraction:
    if int(e) == ZEXP:
        return Fraction(0)
    m = limbs_to_int(limbs)
    assert (m >> (p - 1)) == 1, "mantissa not normalised"
    v = Fraction(m) * Fraction(2) ** (int(e) - p)
    return -v if int(s) else v


def rn(q: Fraction, p: int):
    """Round the rational q to p bits, nearest, ties to even -> (s, e, m)."""
    q = Fraction(q)
    if q == 0:
        return 0, ZEXP, 0
    s = 1 if q < 0 else 0
    a, b = abs(q.numerator), q.denominator
    # e with 2^(e-1) <= a/b < 2^e
    e = a.bit_length() - b.bit_length() + 1
    if e >= 1:
        if a < b << (e - 1):
            e -= 1
    else:
        if a << (1 - e) < b:
            e -= 1
    # scaled = a/b * 2^(p-e) in [2^(p-1), 2^p)
    sh = p - e
    num, den = (a << sh, b) if sh >= 0 else (a, b << (-sh))
    m, r = divmod(num, den)
    assert (m >> (p - 1)) == 1
    twice = 2 * r
    if twice > den or (twice == den and (m & 1)):
        m += 1
        if m == 1 << p:
            m = 1 << (p - 1)
            e += 1
    return s, e, m


def rn_tuple(q: Fraction, p: int):
    s, e, m = rn(q, p)
    return s, e, int_to_limbs(m, p // 32)


def pack(values, p: int):
    """List of Fractions -> rounded SoA triple (sign, exp, limbs)."""
    n = p // 32
    c = len(values)
    S = np.zeros(c, np.int8)
    E = np.full(c, ZEXP, np.int64)
    M = np.zeros((c, n), np.uint32)
    for i, v in enumerate(values):
        s, e, m = rn(Fraction(v), p)
        S[i], E[i] = s, e
        M[i] = int_to_limbs(m, n)
    return S, E, M


def unpack(x, p: int):
    S, E, M = x
    return [to_fraction(S[i], E[i], M[i], p) for i in range(len(S))]


def same(x, y) -> bool:
    """Bitwise equality of two SoA triples."""
    return (np.array_equal(np.asarray(x[0]), np.asarray(y[0])) and np.array_equal(np.asarray(x[1]), np.asarray(y[1]))
            and np.array_equal(np.asarray(x[2]), np.asarray(y[2])))
