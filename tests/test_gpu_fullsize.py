"""Full-size bit-exact parity: the complete outputs of the workloads at their
full sizes, computed on the GPU in the benchmark's launch configuration,
against stored digests that tests/golden/fullsize.py wrote from the CPU
oracle alone (SHA-256 of each number, vector or row; equal digests mean
equal bits).  A mismatch names the first differing index.

* C2: N = 1024, p = 2048, last-column mode, the Cauchy and the integer
  matrix: D_1..D_1024, C_1N..C_NN (eq. minorsdef) and every row of the
  in-place array (U and L).
* C3: 4096 matrices of N uniform in [8, 256] at p = 1024 in one persistent
  launch (autotuned, replayed as a CUDA graph): every matrix's leading
  minors and first zero pivot; det of 64 sampled matrices as values.
* C4: N = 512, p = 4096, the nearly singular matrix: D_1..D_512, sign and
  log|det|, every row of X = A^-1 at p bits and of the binary64 gradient.
* C5: the leading 256 x 256 block of the N = 4096, p = 32768 Cauchy matrix
  (its leading minors are D_1..D_256 of the full factorisation): D_1..D_256
  and every row of the block's upper triangle after elimination.
"""
import os
import sys

import numpy as np
import pytest

from paper_1308_1536_gb300 import workloads as W

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import fullsize as F  # noqa: E402

pytestmark = pytest.mark.gpu


def _digests(field):
    return [r[1] for r in field]


def _expect_same(what, got, want):
    i = F.first_mismatch(got, want)
    assert i is None, f"{what}: first mismatch at index {i} (of {len(want)})"


@pytest.mark.parametrize("kind", ["cauchy", "int"])
def test_full_size_C2(mpdet, kind):
    want = F.read(f"c2_{kind}")
    cfg = W.C2
    N, p = cfg["N"], cfg["p"]
    h = mpdet.Mpdet(N, p, lastcol=True)
    if kind == "cauchy":
        h.set_cauchy(*W.cauchy_xy(N, cfg["seed"]))
    else:
        h.set_i32(W.int_matrix(N, cfg["seed"] + 100).astype(np.int32))  # the benchmark's matrix
    rc, zk, D = h.factor()
    st_w, zk_w = (int(v) for v in want["S"][0][1:3])
    assert (rc, zk) == (st_w, zk_w)
    _expect_same("D_k", F.num_digests(D), _digests(want["D"]))
    if st_w == 0:
        _expect_same("C_jN", F.num_digests(h.lastcol_minors()), _digests(want["C"]))
    _expect_same("rows of the in-place array", F.row_digests(h.get_mp(), N), _digests(want["R"]))
    h.close()


def test_full_size_C3(mpdet):
    import torch

    want = F.read("c3")
    cfg = W.C3
    p = cfg["p"]
    n = p // 32
    items = W.batch_inputs(cfg["count"], cfg["Nmin"], cfg["Nmax"], cfg["seed"])
    Ns = [len(d[0]) if k == "cauchy" else len(d) for k, d in items]
    b = mpdet.Batch(Ns, p)
    for m, (k, d) in enumerate(items):
        if k == "cauchy":
            b.set_cauchy(m, *d)
        else:
            b.set_i32(m, d)
    b.autotune(reps=1)
    b.tune(graph=True)
    tot = int(b.offsets[-1])
    out = (torch.empty(tot, dtype=torch.int8, device="cuda"), torch.empty(tot, dtype=torch.int64, device="cuda"),
           torch.empty((tot, n), dtype=torch.int32, device="cuda"))
    zk = torch.empty(len(Ns), dtype=torch.int64, device="cuda")
    b.factor(out=out, zero_k=zk)
    torch.cuda.synchronize()
    D = (out[0].cpu().numpy(), out[1].cpu().numpy(), out[2].cpu().numpy().view(np.uint32))
    zk = zk.cpu().numpy()
    recs = {int(r[0]): r[1:] for r in want["M"]}
    assert len(recs) == len(Ns)
    bad = []
    for m in range(len(Ns)):
        Nw, zkw, dw = int(recs[m][0]), int(recs[m][1]), recs[m][2]
        Dm = b.minors_of(D, m)
        if Nw != Ns[m] or zkw != int(zk[m]) or F.vec_digest(Dm) != dw:
            bad.append(m)
    assert not bad, f"{len(bad)} of {len(Ns)} matrices differ; first: {bad[:5]}"
    for r in want["V"]:
        m = int(r[0])
        N = Ns[m]
        Dm = b.minors_of(D, m)
        assert F.value_hex(Dm[0][N - 1], Dm[1][N - 1], Dm[2][N - 1]) == " ".join(r[1:4]), m
    b.close()


def test_full_size_C4(mpdet):
    want = F.read("c4")
    cfg = W.C4
    N, p = cfg["N"], cfg["p"]
    A = W.nearly_singular_f64(N, cfg["seed"])
    h = mpdet.Mpdet(N, p, lastcol=True)
    s, la, G = h.logabsdet_grad(A)
    Xi = h.get_inverse()
    D = h.get_minors()
    h.close()
    sw, law = float(want["L"][0][1]), float.fromhex(want["L"][0][2])
    assert s == sw and la == pytest.approx(law, rel=0, abs=1e-12)
    _expect_same("D_k", F.num_digests(D), _digests(want["D"]))
    _expect_same("rows of A^-1", F.row_digests(Xi, N), _digests(want["X"]))
    _expect_same("rows of the binary64 gradient", F.f64_row_digests(G), _digests(want["G"]))


def test_full_size_C5_leading_block(mpdet):
    want = F.read("c5")
    cfg = W.C5
    K, p = F.C5_LEAD, cfg["p"]
    x, y = W.cauchy_xy(cfg["N"], cfg["seed"])
    h = mpdet.Mpdet(K, p)
    h.set_cauchy(x[:K], y[:K])
    rc, zk, D = h.factor()
    assert (rc, zk) == tuple(int(v) for v in want["S"][0][1:3])
    _expect_same("D_k", F.num_digests(D), _digests(want["D"]))
    _expect_same("rows of U", F.row_digests(h.get_mp(), K, cols=lambda i: (i, K)), _digests(want["U"]))
    h.close()
