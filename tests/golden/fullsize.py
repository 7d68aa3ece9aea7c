"""Stored expected values of the full-size workloads, written from the CPU
oracle (and the seeded input generators) only, and the readers the GPU
parity tests use.

Each number, vector or matrix row is stored as a digest: the first 16 hex
digits of the SHA-256 of its bytes (sign int8, exponent int64, then the
limbs as little-endian uint32; a vector or a row is the concatenation of
its signs, then its exponents, then its limbs).  Equal digests mean equal
bits (a chance collision has probability 2^-64 per comparison), and a
mismatch is reported with its index.

Files (one per workload; the method is elimination without pivoting, Sec. 3
and Alg. 1, with the augmented matrix [A I] for the last-column minors):

* c2_cauchy_N1024_p2048.txt, c2_int_N1024_p2048.txt: workload C2, last-column
  mode (the integer matrix is the benchmark's: seed + 100).  Status and first
  zero pivot; D_1..D_1024; C_1N..C_NN (eq. minorsdef); one digest per row of
  the in-place array (U and L).
* c3_batch_4096_p1024.txt: workload C3, 4096 matrices of sizes N uniform in
  [8, 256], even index Cauchy, odd index integer.  Per matrix: N, first zero
  pivot and the digest of D_1..D_N; the value of det = D_N of 64 sampled
  matrices.
* c4_adjoint_N512_p4096.txt: workload C4 (the nearly singular N(0,1) matrix,
  det = 1e-30 C_1N).  D_1..D_N, sign and log|det|, one digest per row of
  X = A^-1 at p bits (right-looking back substitution) and of the binary64
  gradient d log|det| / dA = A^-T.
* c5_cauchy_lead256_p32768.txt: workload C5's leading 256 x 256 block (the
  Cauchy matrix of the 256 smallest x and y of the N = 4096 draw; the leading
  minors of a matrix depend on its leading block only, so these are D_1..D_256
  of the full N = 4096 factorisation).  D_1..D_256 and one digest per row of
  the block's upper triangle (j >= i) after elimination.

Usage: python tests/golden/fullsize.py [c2_cauchy c2_int c3 c4 c5]   (all by
default; about 1.5 hours on 8 cores).
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FILES = {
    "c2_cauchy": "c2_cauchy_N1024_p2048.txt",
    "c2_int": "c2_int_N1024_p2048.txt",
    "c3": "c3_batch_4096_p1024.txt",
    "c4": "c4_adjoint_N512_p4096.txt",
    "c5": "c5_cauchy_lead256_p32768.txt",
}
C5_LEAD = 256
C3_SAMPLED = 64


def path(key: str) -> str:
    return os.path.join(HERE, FILES[key])


# ---------------------------------------------------------------------------
# digests
# ---------------------------------------------------------------------------
def _h(*parts) -> str:
    d = hashlib.sha256()
    for q in parts:
        d.update(np.ascontiguousarray(q).tobytes())
    return d.hexdigest()[:16]


def num_digests(x) -> list[str]:
    """One digest per number of the triple (sign, exp, limbs)."""
    s, e, m = (np.asarray(t) for t in x)
    s = s.astype(np.int8).reshape(-1)
    e = e.astype(np.int64).reshape(-1)
    m = m.astype(np.uint32).reshape(s.shape[0], -1)
    return [_h(s[i:i + 1], e[i:i + 1], m[i]) for i in range(s.shape[0])]


def vec_digest(x) -> str:
    s, e, m = (np.asarray(t) for t in x)
    return _h(s.astype(np.int8).reshape(-1), e.astype(np.int64).reshape(-1), m.astype(np.uint32))


def row_digests(X, N: int, cols=None) -> list[str]:
    """Digest of each row of a row-major N x N array of numbers; cols(i)
    gives the column range (lo, hi) stored for row i (default: all)."""
    s, e, m = (np.asarray(t) for t in X)
    s = s.astype(np.int8).reshape(N, N)
    e = e.astype(np.int64).reshape(N, N)
    m = m.astype(np.uint32).reshape(N, N, -1)
    out = []
    for i in range(N):
        lo, hi = (0, N) if cols is None else cols(i)
        out.append(_h(s[i, lo:hi], e[i, lo:hi], m[i, lo:hi]))
    return out


def f64_row_digests(G) -> list[str]:
    G = np.asarray(G, np.float64)
    return [_h(np.ascontiguousarray(G[i])) for i in range(G.shape[0])]


def value_hex(s, e, limbs) -> str:
    return f"{int(s)} {int(e)} " + "".join(f"{int(v):08x}" for v in reversed(np.asarray(limbs).tolist()))


# ---------------------------------------------------------------------------
# file format: "# comment", then "<tag> <index> <fields...>" lines
# ---------------------------------------------------------------------------
def write(key: str, header: str, records):
    with open(path(key) + ".tmp", "w") as f:
        f.write(f"# {header}\n# written by tests/golden/fullsize.py from the oracle only\n")
        for r in records:
            f.write(" ".join(str(v) for v in r) + "\n")
    os.replace(path(key) + ".tmp", path(key))


def read(key: str) -> dict:
    """tag -> list of field lists, in file order."""
    out: dict = {}
    with open(path(key)) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            t = line.split()
            out.setdefault(t[0], []).append(t[1:])
    return out


def first_mismatch(got: list[str], want: list[str]):
    """Index (0-based) of the first differing digest, or None."""
    if len(got) != len(want):
        return min(len(got), len(want))
    for i, (a, b) in enumerate(zip(got, want)):
        if a != b:
            return i
    return None


# ---------------------------------------------------------------------------
# the oracle computations
# ---------------------------------------------------------------------------
def _threads():
    return os.cpu_count() or 4


def c2(kind: str):
    import oracle
    from paper_1308_1536_gb300 import workloads as W

    cfg = W.C2
    N, p = cfg["N"], cfg["p"]
    if kind == "cauchy":
        x, y = W.cauchy_xy(N, cfg["seed"])
        A = cauchy_parallel(x, y, p)
    else:  # the benchmark's integer matrix (its own seed, apart from the Cauchy draw)
        A = oracle.from_int(W.int_matrix(N, cfg["seed"] + 100).reshape(-1), p)
    st, zk, D, X = oracle.ge(A, N, p, lastcol=True, nthreads=_threads())
    recs = [("S", 0, st, zk)]
    recs += [("D", k + 1, d) for k, d in enumerate(num_digests(D))]
    if st == 0:
        C = oracle.lastcol_minors(X, D, N, p)
        recs += [("C", j + 1, d) for j, d in enumerate(num_digests(C))]
    recs += [("R", i, d) for i, d in enumerate(row_digests(X, N))]
    write(f"c2_{kind}", f"workload C2 ({kind}): N={N} p={p}, lastcol; S: status zero_k; D: D_k; C: C_jN; "
          "R: rows of the in-place array", recs)


def _c3_one(args):
    import oracle

    m, kind, d, p = args
    if kind == "cauchy":
        A = oracle.cauchy(d[0], d[1], p)
        N = len(d[0])
    else:
        A = oracle.from_int(np.asarray(d).reshape(-1), p)
        N = len(d)
    st, zk, D, _ = oracle.ge(A, N, p, nthreads=1)
    return m, N, zk, vec_digest(D), value_hex(D[0][N - 1], D[1][N - 1], D[2][N - 1])


def c3():
    import multiprocessing as mp

    from paper_1308_1536_gb300 import workloads as W

    cfg = W.C3
    p = cfg["p"]
    items = W.batch_inputs(cfg["count"], cfg["Nmin"], cfg["Nmax"], cfg["seed"])
    order = sorted(range(len(items)), key=lambda m: -(len(items[m][1][0]) if items[m][0] == "cauchy"
                                                       else len(items[m][1])))
    with mp.get_context("spawn").Pool(_threads()) as pool:
        res = pool.map(_c3_one, [(m, items[m][0], items[m][1], p) for m in order], chunksize=1)
    res.sort()
    sampled = set(np.linspace(0, len(items) - 1, C3_SAMPLED).astype(int).tolist())
    recs = [("M", m, N, zk, d) for m, N, zk, d, _ in res]
    recs += [("V", m, v) for m, N, zk, d, v in res if m in sampled]
    write("c3", f"workload C3: {cfg['count']} matrices, p={p}; M: index N zero_k digest(D_1..D_N); "
          "V: index sign exp limbs of det", recs)


def c4():
    import oracle
    from paper_1308_1536_gb300 import workloads as W

    cfg = W.C4
    N, p = cfg["N"], cfg["p"]
    A = W.nearly_singular_f64(N, cfg["seed"])
    st, zk, D, Xm = oracle.ge(oracle.from_f64(A.reshape(-1), p), N, p, lastcol=True, nthreads=_threads())
    assert st == 0, st
    Xi = oracle.usolve(Xm, N, p, nthreads=_threads())
    G = oracle.to_f64(Xi, p).reshape(N, N).T
    sg, la = oracle.logabsdet(D, N, p)
    recs = [("L", 0, repr(float(sg)), float(la).hex())]
    recs += [("D", k + 1, d) for k, d in enumerate(num_digests(D))]
    recs += [("X", i, d) for i, d in enumerate(row_digests(Xi, N))]
    recs += [("G", i, d) for i, d in enumerate(f64_row_digests(G))]
    write("c4", f"workload C4: N={N} p={p}; L: sign log|det| (float hex); D: D_k; X: rows of A^-1; "
          "G: rows of the binary64 gradient", recs)


def _c5_rows(args):
    import oracle

    i0, i1, x, y, p = args
    n = len(y)
    out = []
    for i in range(i0, i1):
        xi = oracle.from_f64(np.full(n, x[i]), p)
        yj = oracle.from_f64(np.asarray(y), p)
        out.append(oracle.recip(oracle.add(xi, yj, p), p))
    return i0, out


def cauchy_parallel(x, y, p):
    """The Cauchy matrix A_ij = RN(1/RN(x_i + y_j)) from the oracle's element
    operations, rows computed in parallel processes (the same two operations
    as oracle.cauchy, which is single-threaded)."""
    import multiprocessing as mp

    import oracle

    K = len(x)
    step = max(1, K // (8 * _threads()))
    with mp.get_context("spawn").Pool(_threads()) as pool:
        parts = pool.map(_c5_rows, [(i, min(K, i + step), x, y, p) for i in range(0, K, step)], chunksize=1)
    A = oracle.empty(K * K, p)
    for i0, rows in parts:
        for r, o in enumerate(rows):
            i = i0 + r
            for t, u in zip(A, o):
                t[i * K:(i + 1) * K] = u
    return A


def c5():
    import oracle
    from paper_1308_1536_gb300 import workloads as W

    cfg = W.C5
    p, K = cfg["p"], C5_LEAD
    x, y = W.cauchy_xy(cfg["N"], cfg["seed"])
    x, y = x[:K], y[:K]
    A = cauchy_parallel(x, y, p)
    st, zk, D, X = oracle.ge(A, K, p, nthreads=_threads())
    recs = [("S", 0, st, zk)]
    recs += [("D", k + 1, d) for k, d in enumerate(num_digests(D))]
    recs += [("U", i, d) for i, d in enumerate(row_digests(X, K, cols=lambda i: (i, K)))]
    write("c5", f"workload C5 leading {K}x{K} block: p={p}; S: status zero_k; D: D_k; "
          "U: rows of the upper triangle (j >= i) after elimination", recs)


if __name__ == "__main__":
    which = sys.argv[1:] or ["c2_cauchy", "c2_int", "c4", "c3", "c5"]
    for w in which:
        t = time.time()
        if w.startswith("c2_"):
            c2(w[3:])
        else:
            globals()[w]()
        print(f"{w}: {time.time() - t:.0f} s", flush=True)
