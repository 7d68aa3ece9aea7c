"""GPU parity of the ball mode (MPDET_BALL): the values equal the plain
elimination's bit for bit, and every radius (of the leading minors, of the
in-place array, of the last-column and normalised minors) equals the
oracle's ball mode bit for bit, across kernel families, a precision held in a
larger frame, both modes, with and without look-ahead, and at a zero pivot
(the minors after it unbounded)."""
import numpy as np
import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RAD_INF = np.iinfo(np.int64).max


def rad_same(got, want, idx=None, what=""):
    gm, ge = (np.asarray(t) for t in got)
    wm, we = (np.asarray(t) for t in want)
    if idx is not None:
        gm, ge, wm, we = gm[idx], ge[idx], wm[idx], we[idx]
    # an unbounded radius is identified by its exponent alone
    inf_g, inf_w = ge == RAD_INF, we == RAD_INF
    assert np.array_equal(inf_g, inf_w), f"{what}: unbounded radii differ"
    ok = (gm == wm) & (ge == we) | inf_g
    bad = np.nonzero(~ok)[0]
    assert bad.size == 0, f"{what}: first radius mismatch at {int(bad[0])}"


def gpu_ball(mpdet, N, p, lastcol, kind, data, lookahead=True):
    h = mpdet.Mpdet(N, p, lastcol=lastcol, ball=True)
    h.tune(lookahead=lookahead)
    if kind == "cauchy":
        h.set_cauchy(*data)
    elif kind == "int":
        h.set_i32(data)
    else:
        h.set_f64(data)
    rc, zk, D = h.factor()
    out = dict(rc=rc, zk=zk, D=D, RD=h.radii("minors"), X=h.get_mp(), RX=h.radii("array"))
    if lastcol and rc == 0:
        out["C"] = h.lastcol_minors()
        out["RC"] = h.radii("lastcol")
        try:
            out["Cn"] = h.lastcol_minors(normalised=True)
            out["RCn"] = h.radii("lastcol")
        except mpdet.MpdetError as e:
            assert e.code == mpdet.EZERODIV
    h.close()
    return out


def oracle_ball(oracle, N, p, lastcol, kind, data):
    if kind == "cauchy":
        A, RA = oracle.cauchy_ball(*data, p)
    elif kind == "int":
        A, RA = oracle.from_int(np.asarray(data).reshape(-1), p), None
    else:
        A, RA = oracle.from_f64(np.asarray(data).reshape(-1), p), None
    st, zk, D, Xm, RD, RX = oracle.ge_ball(A, RA, N, p, lastcol=lastcol)
    out = dict(rc=st, zk=zk, D=D, RD=RD, X=Xm, RX=RX)
    if lastcol and st == 0:
        out["C"], out["RC"] = oracle.lastcol_ball(Xm, RX, D, RD, N, p)
        try:
            out["Cn"], out["RCn"] = oracle.lastcol_ball(Xm, RX, D, RD, N, p, normalised=True)
        except RuntimeError:
            pass
    return out


def check(mpdet, oracle, N, p, lastcol, kind, data, lookahead=True):
    g = gpu_ball(mpdet, N, p, lastcol, kind, data, lookahead)
    o = oracle_ball(oracle, N, p, lastcol, kind, data)
    assert (g["rc"], g["zk"]) == (o["rc"], o["zk"])
    assert X.same(g["D"], o["D"]), "leading minors"
    rad_same(g["RD"], o["RD"], what="radii of D")
    iu = None if lastcol else np.array([i * N + j for i in range(N) for j in range(i, N)], dtype=np.int64)
    if o["rc"] == 0:
        sub = (lambda t: t) if iu is None else (lambda t: tuple(np.asarray(a)[iu] for a in t))
        assert X.same(sub(g["X"]), sub(o["X"])), "in-place array"
        rad_same(g["RX"], o["RX"], idx=iu, what="radii of the array")
    for key in ("C", "Cn"):
        if key in o:
            assert X.same(g[key], o[key]), key
            rad_same(g["R" + key], o["R" + key], what="radii of " + key)


@pytest.mark.parametrize("p", [128, 512, 2048, 4096])
@pytest.mark.parametrize("kind", ["cauchy", "int", "f64"])
@pytest.mark.parametrize("lastcol", [False, True])
def test_ball_vs_oracle(mpdet, oracle_lib, p, kind, lastcol):
    g = W.rng(5000 + p + 3 * (kind == "int") + 7 * (kind == "f64") + lastcol)
    for N in (1, 2, 17, 37):
        if kind == "cauchy":
            data = W.cauchy_xy(N, int(g.integers(1 << 30)))
        elif kind == "int":
            data = W.int_matrix(N, int(g.integers(1 << 30)))
        else:
            data = g.standard_normal((N, N))
        check(mpdet, oracle_lib, N, p, lastcol, kind, data)


@pytest.mark.parametrize("p,N", [(96, 30), (32768, 6)])
def test_ball_other_frames_and_lookahead(mpdet, oracle_lib, p, N):
    x, y = W.cauchy_xy(N, 321)
    for la in (True, False):
        check(mpdet, oracle_lib, N, p, True, "cauchy", (x, y), lookahead=la)


def test_ball_zero_pivot(mpdet, oracle_lib):
    A = np.array([[1, 2, 3, 4], [2, 4, 5, 1], [1, 1, 1, 1], [3, 1, 4, 1]])
    g = gpu_ball(mpdet, 4, 256, False, "int", A)
    assert g["rc"] == mpdet.EZEROPIVOT and g["zk"] == 2
    assert np.all(g["RD"][1][2:] == RAD_INF)
    check(mpdet, oracle_lib, 4, 256, False, "int", A)
