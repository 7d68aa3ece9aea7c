"""Write the stored expected values under tests/golden/ from the CPU oracle
(and the seeded input generators) only.

c1_cauchy_N64_p512.txt: workload C1 (Cauchy matrix A_ij = RN(1/RN(x_i+y_j)),
N = 64, p = 512, x, y seeded), elimination without pivoting in last-column
mode: the leading minors D_1..D_64 and the last-column signed minors
C_1N..C_NN, one number per line as "<name> <index> <sign> <exponent>
<limbs, most significant first, hex>".

Usage: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1308_1536_gb300 import workloads as W  # noqa: E402

GOLDEN = os.path.join(HERE, "c1_cauchy_N64_p512.txt")


def compute():
    cfg = W.C1
    N, p = cfg["N"], cfg["p"]
    x, y = W.cauchy_xy(N, cfg["seed"])
    st, zk, D, X = oracle.ge(oracle.cauchy(x, y, p), N, p, lastcol=True)
    assert st == 0
    C = oracle.lastcol_minors(X, D, N, p)
    return N, p, D, C


def lines(N, p, D, C):
    out = [f"# workload C1: Cauchy N={N} p={p}, lastcol; written by tests/golden/make_golden.py from the oracle"]
    for name, arr in (("D", D), ("C", C)):
        s, e, m = arr
        for i in range(N):
            limbs = "".join(f"{int(v):08x}" for v in reversed(m[i].tolist()))
            out.append(f"{name} {i + 1} {int(s[i])} {int(e[i])} {limbs}")
    return out


if __name__ == "__main__":
    with open(GOLDEN, "w") as f:
        f.write("\n".join(lines(*compute())) + "\n")
    print(GOLDEN)
