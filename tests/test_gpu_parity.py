"""GPU parity: the CUDA path through the C ABI must equal the CPU oracle bit
for bit (integer limbs, exponents and signs), on seeded inputs that span
several tiles, ragged tails, every kernel family (p = 128 .. 32768), precisions
between the families (p = 64, 96, 160, 3072) and the degenerate cases of the method (zero pivots, N = 1, exact cancellations)."""
import numpy as np
import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def same(a, b):
    return X.same(a, b)


def first_diff(a, b):
    for i in range(len(a[0])):
        if a[0][i] != b[0][i] or a[1][i] != b[1][i] or not np.array_equal(a[2][i], b[2][i]):
            return i
    return None


def assert_same(got, want, what):
    i = first_diff(got, want)
    assert i is None, f"{what}: first mismatch at {i}: got ({got[0][i]}, {got[1][i]}) want ({want[0][i]}, {want[1][i]})"


def gpu_run(mpdet, N, p, lastcol, kind, data):
    h = mpdet.Mpdet(N, p, lastcol=lastcol)
    if kind == "cauchy":
        h.set_cauchy(*data)
    elif kind == "int":
        h.set_i32(data)
    else:
        h.set_f64(data)
    rc, zk, D = h.factor()
    Xm = h.get_mp()
    C = Cn = None
    if lastcol and rc == 0:
        C = h.lastcol_minors()
        try:
            Cn = h.lastcol_minors(normalised=True)
        except mpdet.MpdetError as e:
            assert e.code == mpdet.EZERODIV
    h.close()
    return rc, zk, D, Xm, C, Cn


def oracle_run(oracle, N, p, lastcol, kind, data):
    if kind == "cauchy":
        A = oracle.cauchy(*data, p)
    elif kind == "int":
        A = oracle.from_int(np.asarray(data).reshape(-1), p)
    else:
        A = oracle.from_f64(np.asarray(data).reshape(-1), p)
    st, zk, D, Xm = oracle.ge(A, N, p, lastcol=lastcol, nthreads=8)
    C = Cn = None
    if lastcol and st == 0:
        C = oracle.lastcol_minors(Xm, D, N, p)
        try:
            Cn = oracle.lastcol_minors(Xm, D, N, p, normalised=True)
        except RuntimeError:
            Cn = None
    return st, zk, D, Xm, C, Cn, A


def check_case(mpdet, oracle, N, p, lastcol, kind, data):
    g = gpu_run(mpdet, N, p, lastcol, kind, data)
    o = oracle_run(oracle, N, p, lastcol, kind, data)
    assert g[0] == o[0] and g[1] == o[1], (g[:2], o[:2])
    assert_same(g[2], o[2], "leading minors")
    if o[0] == 0:
        # the whole in-place array: U (and L in lastcol mode)
        if lastcol:
            assert_same(g[3], o[3], "in-place array")
        else:
            iu = np.array([i * N + j for i in range(N) for j in range(i, N)])
            sub = lambda t: tuple(a[iu] for a in t)
            assert_same(sub(g[3]), sub(o[3]), "upper triangle")
    if lastcol and o[0] == 0:
        assert_same(g[4], o[4], "last-column minors")
        if o[5] is not None:
            assert_same(g[5], o[5], "normalised minors")


@pytest.mark.parametrize("p", [128, 256, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("kind", ["cauchy", "int", "f64"])
@pytest.mark.parametrize("lastcol", [False, True])
def test_parity_small(mpdet, oracle_lib, p, kind, lastcol):
    g = W.rng(1000 + p + (kind == "int") * 7 + lastcol)
    for N in (1, 2, 3, 17, 40):
        if kind == "cauchy":
            data = W.cauchy_xy(N, int(g.integers(1 << 30)))
        elif kind == "int":
            data = W.int_matrix(N, int(g.integers(1 << 30)))
        else:
            data = g.standard_normal((N, N))
        check_case(mpdet, oracle_lib, N, p, lastcol, kind, data)


@pytest.mark.parametrize("p", [64, 96, 160, 3072])
def test_parity_any_multiple_of_32(mpdet, oracle_lib, p):
    """Precisions whose limb count is not a kernel family's (p = 64, 96, 160
    and 3072 live in frames of 4, 4, 8 and 128 limbs with the low limbs zero)
    round at p bits: every output equals the oracle's at p bits, in both
    modes, on all three kinds of input (Cauchy entries RN(1/RN(x+y)) round
    at p = 64 and 96 already)."""
    g = W.rng(2000 + p)
    for N, kind, lastcol in ((1, "f64", True), (2, "int", True), (3, "cauchy", False), (17, "cauchy", True),
                             (40, "int", False), (33, "f64", True), (29, "cauchy", False), (24, "int", True)):
        if kind == "cauchy":
            data = W.cauchy_xy(N, int(g.integers(1 << 30)))
        elif kind == "int":
            data = W.int_matrix(N, int(g.integers(1 << 30)))
        else:
            data = g.standard_normal((N, N))
        check_case(mpdet, oracle_lib, N, p, lastcol, kind, data)


@pytest.mark.parametrize("p", [96, 3072])
def test_any_multiple_of_32_series_adjoint_and_host_io(mpdet, oracle_lib, p):
    """The same precisions through the series of minor arrays, the adjoint
    and the device-buffer outputs (the frame's limbs are converted at the
    boundary in every direction)."""
    import torch

    N = 12
    A = W.rng(3000 + p).standard_normal((N, N))
    h = mpdet.Mpdet(N, p, lastcol=True)
    s, la, G = h.logabsdet_grad(A)
    Xi = h.get_inverse()
    ser = h.minor_series()
    n = p // 32
    dev = (torch.empty(N * (N + 1) // 2, dtype=torch.int8, device="cuda"),
           torch.empty(N * (N + 1) // 2, dtype=torch.int64, device="cuda"),
           torch.empty((N * (N + 1) // 2, n), dtype=torch.int32, device="cuda"))
    h.minor_series(out=dev)
    torch.cuda.synchronize()
    ser_dev = (dev[0].cpu().numpy(), dev[1].cpu().numpy(), dev[2].cpu().numpy().view(np.uint32))
    ent = h.get_entries(np.array([0, 5, N * N - 1]))
    h.close()
    st, zk, D, Xm = oracle_lib.ge(oracle_lib.from_f64(A.reshape(-1), p), N, p, lastcol=True)
    assert st == 0
    OX = oracle_lib.usolve(Xm, N, p)
    assert_same(Xi, OX, "A^-1")
    assert np.array_equal(G, oracle_lib.to_f64(OX, p).reshape(N, N).T)
    OS = oracle_lib.minor_series(Xm, D, N, p)
    assert_same(ser, OS, "series (host)")
    assert_same(ser_dev, OS, "series (device)")
    assert_same(ent, tuple(a[[0, 5, N * N - 1]] for a in Xm), "sampled entries")


@pytest.mark.parametrize("p", [8192, 16384, 32768])
def test_parity_high_precision(mpdet, oracle_lib, p):
    g = W.rng(p)
    for N, kind in ((3, "f64"), (6, "cauchy"), (5, "int")):
        if kind == "cauchy":
            data = W.cauchy_xy(N, int(g.integers(1 << 30)))
        elif kind == "int":
            data = W.int_matrix(N, int(g.integers(1 << 30)))
        else:
            data = g.standard_normal((N, N))
        check_case(mpdet, oracle_lib, N, p, True, kind, data)


def test_parity_config_cauchy_N64_p512(mpdet, oracle_lib):
    """Workload C1: Cauchy N = 64, p = 512, det, 64 leading minors, 64
    last-column minors: every output word equal."""
    N, p = W.C1["N"], W.C1["p"]
    check_case(mpdet, oracle_lib, N, p, True, "cauchy", W.cauchy_xy(N, W.C1["seed"]))


def test_parity_tiles_and_ragged_tails(mpdet, oracle_lib):
    # N = 137 at p = 1024 (G = 2): 68 groups per column tile, several row
    # blocks, ragged last tile in both directions
    N, p = 137, 1024
    check_case(mpdet, oracle_lib, N, p, True, "int", W.int_matrix(N, 77))
    check_case(mpdet, oracle_lib, N, p, False, "cauchy", W.cauchy_xy(N, 78))


def test_zero_pivots(mpdet, oracle_lib):
    p = 512
    for M in ([[0, 1], [1, 0]], [[1, 2, 3], [2, 4, 5], [1, 1, 1]], [[1, 2], [2, 4]], [[0]]):
        N = len(M)
        g = gpu_run(mpdet, N, p, True, "int", np.array(M))
        o = oracle_run(oracle_lib, N, p, True, "int", np.array(M))
        assert (g[0], g[1]) == (o[0], o[1])
        assert_same(g[2], o[2], "minors after zero pivot")
        if o[0] == 0 and N > 1:
            assert_same(g[4], o[4], "minors of a singular matrix")


def test_window_and_resume_are_bit_identical(mpdet, oracle_lib):
    N, p = 33, 1024
    A = W.int_matrix(N, 9)
    h = mpdet.Mpdet(N, p, lastcol=True)
    h.set_i32(A)
    _, _, Dref = h.factor()
    Xref = h.get_mp()
    h.set_i32(A)
    h.factor_range(0, 10)
    h.factor_range(10, 20)
    Xmid, Dmid = h.get_mp(), h.get_minors()
    h2 = mpdet.Mpdet(N, p, lastcol=True)
    h2.resume(Xmid, Dmid, 20)
    _, _, D2 = h2.factor()
    assert_same(D2, Dref, "resumed minors")
    assert_same(h2.get_mp(), Xref, "resumed array")
    h.close()
    h2.close()


def test_device_pointer_inputs_and_outputs(mpdet, oracle_lib):
    import torch

    N, p = 20, 512
    x, y = W.cauchy_xy(N, 5)
    h = mpdet.Mpdet(N, p, lastcol=True)
    h.set_cauchy(torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"))
    n = p // 32
    D = (torch.zeros(N, dtype=torch.int8, device="cuda"), torch.zeros(N, dtype=torch.int64, device="cuda"),
         torch.zeros((N, n), dtype=torch.int32, device="cuda"))
    h.factor(out=D)
    torch.cuda.synchronize()
    assert h.status() == (0, 0)
    got = (D[0].cpu().numpy(), D[1].cpu().numpy(), D[2].cpu().numpy().view(np.uint32))
    o = oracle_run(oracle_lib, N, p, True, "cauchy", (x, y))
    assert_same(got, o[2], "device-pointer minors")
    h.close()


def test_full_size_C2_sampled(mpdet, oracle_lib):
    """Workload C2 at full size (N = 1024, p = 2048, lastcol mode, the
    configuration the benchmark times): the leading minors D_1..D_K of the
    full run equal an oracle run of the leading K x K block (GE without
    pivoting never looks outside the leading block), C_NN = D_{N-1}
    bitwise, and sampled Cauchy entries equal the oracle's."""
    N, p, K = W.C2["N"], W.C2["p"], 96
    x, y = W.cauchy_xy(N, W.C2["seed"])
    g = W.rng(W.C2["seed"])
    A_int = W.int_matrix(N, W.C2["seed"] + 100)
    for kind, data, lead in (("cauchy", (x, y), (x[:K], y[:K])), ("int", A_int, A_int[:K, :K])):
        h = mpdet.Mpdet(N, p, lastcol=True)
        if kind == "cauchy":
            h.set_cauchy(*data)
            X0 = h.get_mp()
            idx = g.integers(0, N * N, 64)
            for t in idx:
                i, j = divmod(int(t), N)
                e = oracle_lib.cauchy(np.array([x[i]]), np.array([y[j]]), p)
                assert X0[0][t] == e[0][0] and X0[1][t] == e[1][0] and np.array_equal(X0[2][t], e[2][0])
        else:
            h.set_i32(data)
        rc, zk, D = h.factor()
        assert rc == 0
        C = h.lastcol_minors()
        h.close()
        o = oracle_run(oracle_lib, K, p, False, kind, lead)
        assert_same(tuple(t[:K] for t in D), o[2], f"{kind}: leading minors 1..{K}")
        assert C[0][N - 1] == D[0][N - 2] and C[1][N - 1] == D[1][N - 2] and np.array_equal(C[2][N - 1], D[2][N - 2])


@pytest.mark.parametrize("N,p,lastcol", [(70, 1024, True), (33, 8192, True), (40, 4096, False), (100, 4096, True)])
def test_host_resident_array(mpdet, oracle_lib, N, p, lastcol):
    """The N x N array in page-locked host memory (MPDET_HOSTMEM), read and
    written in place by the kernels: bit-identical to the device-resident
    array and to the oracle, windows and the last-column minors included
    (N = 100 at p = 4096: the tensor-core engine's launches of >= 64 rows
    read and write the host-resident array)."""
    x, y = W.cauchy_xy(N, 4040 + N)
    out = []
    for host in (False, True):
        h = mpdet.Mpdet(N, p, lastcol=lastcol, hostmem=host)
        h.set_cauchy(x, y)
        h.factor_range(0, N // 3)
        rc, zk, D = h.factor()
        Xm = h.get_mp()
        C = h.lastcol_minors() if lastcol else None
        h.close()
        out.append((rc, zk, D, Xm, C))
    assert out[0][:2] == out[1][:2] == (0, 0)
    assert same(out[0][2], out[1][2]) and same(out[0][3], out[1][3])
    if lastcol:
        assert same(out[0][4], out[1][4])
    st, ozk, OD, OX = oracle_lib.ge(oracle_lib.cauchy(x, y, p), N, p, lastcol=lastcol, nthreads=8)
    assert_same(out[1][2], OD, "leading minors (host-resident)")
