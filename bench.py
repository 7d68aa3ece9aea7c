#!/usr/bin/env python
"""Benchmark of multiprecision Gaussian elimination (det, leading minors and
last-column minors) on one or more GB300s.

One step = the whole hot path on the N = 1024, p = 2048 workload: for a seeded
Cauchy matrix (generated on the device, A_ij = RN(1/RN(x_i+y_j))) and a seeded
integer matrix with entries in [-1000, 1000] (lifted on the device): the
elimination without pivoting in last-column mode (pivots, reciprocals,
multipliers, Schur updates of U and L) and the last-column signed minors.

value   = algorithmic limb multiply-accumulates of the step (every p x p-bit
          product of the elimination counted as n^2 = (p/32)^2 limb MACs)
          / device time of the step, inputs resident in HBM.
e2e     = the same through the C ABI with host buffers: pinned host inputs
          copied in and minors copied out inside the timed region.
roofline: the Schur-update kernel (the dominant one), timed live with CUDA
          events around each of its launches, against the integer-multiply
          peak SMs x 32 limb-MAC/clk (64 IMAD lanes per SM, two IMAD-pipe slots
          per 32x32->64-bit product) x max SM clock.
--impl reference: the CPU oracle on this host's cores, on a bounded sample of
          the same workload (leading K x K blocks of both matrices).
With --gpus N > 1 (torchrun) every rank runs its own replica of the step on
its GPU (independent problems, no collective); value sums over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1308_1536_gb300 import shard  # noqa: E402
from paper_1308_1536_gb300 import workloads as W  # noqa: E402

METRIC = "mp elimination limb-MAC/s"
UNIT = "limb-MAC/s"
ORACLE_SAMPLE_K = 160


def elim_products(N: int, lastcol: bool) -> int:
    """p x p-bit products of one elimination: multipliers, Schur updates (full
    rows in lastcol mode), D_k and the last-column finalisation."""
    upd = sum((N - k - 1) * ((N - 1) if lastcol else (N - k - 1)) for k in range(N - 1))
    mult = N * (N - 1) // 2
    dk = N - 1
    fin = (N - 1) if lastcol else 0
    return upd + mult + dk + fin


def step_limb_macs(N: int, p: int, matrices: int = 2) -> float:
    n = p // 32
    return float(matrices) * elim_products(N, True) * n * n


def batch_products(Ns) -> int:
    """p x p-bit products of a batch (no L): multipliers, updates, D_k."""
    return int(sum(elim_products(int(N), False) for N in Ns))


def kernel_source_sha() -> str:
    """Hash of the sources of the tensor-core Schur-update kernel (its own
    file and the multiprecision device routines it inlines): a recorded DRAM
    traffic figure is used only while these are unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1308_1536_gb300", "csrc")
    for fn in ("tc_update.cu", "mpdev.cuh"):
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mpdet_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def recorded_traffic(products_per_launch: float, any_sources: bool = False):
    """DRAM bytes per Schur-update launch: the bytes per product of one ncu
    capture (profiles/k_update_traffic.json, dram__bytes_read.sum +
    dram__bytes_write.sum of a launch of known size) times this run's average
    products per timed launch.  None unless the capture was taken on the
    current kernel sources (any_sources: whatever sources it was taken on)."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "k_update_traffic.json")))
    except Exception:
        return None
    if t.get("source_sha") != kernel_source_sha() and not any_sources:
        return None
    return t["bytes_per_product"] * products_per_launch


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample(K: int = ORACLE_SAMPLE_K, threads: int = 0):
    import oracle

    oracle.build()
    cfg = W.C2
    N, p = cfg["N"], cfg["p"]
    x, y = W.cauchy_xy(N, cfg["seed"])
    A = W.int_matrix(N, cfg["seed"] + 100)
    threads = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    for kind in ("cauchy", "int"):
        M = oracle.cauchy(x[:K], y[:K], p) if kind == "cauchy" else oracle.from_int(A[:K, :K].reshape(-1), p)
        st, zk, D, X = oracle.ge(M, K, p, lastcol=True, nthreads=threads)
        oracle.lastcol_minors(X, D, K, p)
    dt = time.perf_counter() - t0
    macs = step_limb_macs(K, p, 2)
    return {"value": macs / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"leading {K}x{K} blocks of both workload matrices (Cauchy and integer), p={p}, lastcol mode, "
                      f"{threads} threads; {dt:.2f} s", "seconds": dt}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_sample(max(32, ORACLE_SAMPLE_K // 4))
    vals, secs = [], []
    for _ in range(args.steps):
        r = oracle_sample()
        vals.append(r["value"])
        secs.append(r["seconds"])
    v = statistics.median(vals)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": {"workload": "cauchy+int N=1024 p=2048 lastcol (oracle sample: leading "
                                  f"{ORACLE_SAMPLE_K}x{ORACLE_SAMPLE_K} blocks)", "N": W.C2["N"], "p": W.C2["p"]},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle", "sample": r["sample"]},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def bench_batch(args, dev, m, rank=0, world=1):
    """Workload C3: 4096 matrices, N ~ U[8, 256], half Cauchy half integer,
    p = 1024, det and leading minors of each, one persistent launch per step
    (inputs resident in HBM as p-bit numbers; the timed step copies them to
    the working array and factors), replayed as a CUDA graph, with the lane
    geometry and blocks per SM chosen by the batch autotuner.  With several
    ranks every rank factors its share of the 4096 matrices (no exchange;
    time = max over ranks).  The single-matrix path is timed on a sample of
    the same matrices at the same p for comparison."""
    import torch

    cfg = W.C3
    p = cfg["p"]
    n = p // 32
    Ns_all, kinds_all, seeds_all = W.batch_sizes(args.batch_count or cfg["count"], cfg["Nmin"], cfg["Nmax"],
                                                 cfg["seed"])
    mine = shard.batch_shard(Ns_all, rank, world)
    Ns, kinds, seeds = Ns_all[mine], kinds_all[mine], seeds_all[mine]
    b = m.Batch(Ns, p, stream=torch.cuda.current_stream(dev).cuda_stream)
    inputs = []
    torch.cuda.synchronize(dev)
    t_lift0 = time.perf_counter()
    for i in range(len(Ns)):
        N = int(Ns[i])
        if kinds[i] == "cauchy":
            d = W.cauchy_xy(N, int(seeds[i]))
            b.set_cauchy(i, *d)
        else:
            d = W.int_matrix(N, int(seeds[i]))
            b.set_i32(i, d)
        inputs.append(d)
    torch.cuda.synchronize(dev)
    t_lift = time.perf_counter() - t_lift0  # every matrix's input set from host arrays (lift or generation)
    tot = int(np.sum(Ns))
    out = (torch.empty(tot, dtype=torch.int8, device=dev), torch.empty(tot, dtype=torch.int64, device=dev),
           torch.empty((tot, n), dtype=torch.int32, device=dev))
    zk = torch.empty(len(Ns), dtype=torch.int64, device=dev)
    # lane geometry and blocks per SM picked by the batch autotuner on these
    # matrices; the timed factorisations replay a CUDA graph of the launch
    tuned = b.autotune(reps=1)
    var = b.variants()[tuned["variant"]]
    b.tune(graph=True)
    for _ in range(args.warmup):
        b.factor(out=out, zero_k=zk)
    torch.cuda.synchronize(dev)
    l0 = b.launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        b.factor(out=out, zero_k=zk)
    e1.record()
    torch.cuda.synchronize(dev)
    ms = shard.reduce_over_ranks(e0.elapsed_time(e1) / args.steps, "max", device=dev)
    launches = (b.launches() - l0) // args.steps
    b.close()
    macs = batch_products(Ns_all) * n * n
    # single-matrix path on a sample (every 16th matrix), same p, same GPU:
    # (a) lift + factor per matrix (as a user with raw inputs would call it),
    # (b) from the same p-bit inputs the batch starts from (mpdet_set_mp from
    # device buffers, then factor), like for like with the batch's timed step
    sample = list(range(0, len(Ns), 16))
    handles = {}
    lifted = {}
    for i in sample:
        N = int(Ns[i])
        h = handles.get(N)
        if h is None:
            h = handles[N] = m.Mpdet(N, p, stream=torch.cuda.current_stream(dev).cuda_stream)
        if kinds[i] == "cauchy":
            h.set_cauchy(*inputs[i])
        else:
            h.set_i32(inputs[i])
        Xl = h.get_mp()
        lifted[i] = (torch.from_numpy(Xl[0]).to(dev), torch.from_numpy(Xl[1]).to(dev),
                     torch.from_numpy(np.ascontiguousarray(Xl[2]).view(np.int32)).to(dev))
    t_single = t_single_mp = 0.0
    for rep in range(2):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for i in sample:
            N = int(Ns[i])
            h = handles[N]
            if kinds[i] == "cauchy":
                h.set_cauchy(*inputs[i])
            else:
                h.set_i32(inputs[i])
            h.factor_range(0, N)
        torch.cuda.synchronize(dev)
        t_single = time.perf_counter() - t0  # second repetition counts (handles warm)
        t0 = time.perf_counter()
        for i in sample:
            h = handles[int(Ns[i])]
            h.set_mp(lifted[i])
            h.factor_range(0, int(Ns[i]))
        torch.cuda.synchronize(dev)
        t_single_mp = time.perf_counter() - t0
    for h in handles.values():
        h.close()
    single_dets = len(sample) / t_single
    single_dets_mp = len(sample) / t_single_mp
    return {"workload": f"{len(Ns_all)} matrices N~U[8,256], half Cauchy half integer, p=1024: det + leading minors",
            "ranks": world, "matrices_per_rank": int(len(Ns)),
            "dets_per_s": len(Ns_all) / (ms / 1e3), "ms_per_step": ms, "limb_macs_per_s": macs / (ms / 1e3),
            "gpu_launches_per_step": int(launches),
            "autotuned": {"W": var[0], "G": var[1], "pivot_W": var[2], "pivot_G": var[3],
                          "blocks_per_sm": tuned["blocks_per_sm"], "candidates": tuned["candidates"],
                          "best_ms": tuned["ms"]},
            "cuda_graph": True,
            "single_path_dets_per_s": single_dets_mp,
            "vs_single_path": (len(Ns) / (ms / 1e3)) / single_dets_mp,
            "single_path_sample": f"every 16th matrix ({len(sample)}), from the same p-bit inputs as the batch "
                                  "(set_mp from device buffers + factor per matrix)",
            "with_lift_dets_per_s": len(Ns) / (t_lift + ms / 1e3),
            "single_path_with_lift_dets_per_s": single_dets,
            "vs_single_path_with_lift": (len(Ns) / (t_lift + ms / 1e3)) / single_dets}


def bench_adjoint(args, dev, m):
    """Workload C4: N = 512, p = 4096, the nearly singular Gaussian matrix:
    one gradient call = exact lift, elimination in lastcol mode, log|det|,
    back substitution X = U^-1 L and the binary64 gradient A^-T (device
    input and output).  Compared with the plain single-matrix path (lift and
    elimination for det only) at the same N and p."""
    import torch

    cfg = W.C4
    N, p = cfg["N"], cfg["p"]
    n = p // 32
    A = torch.tensor(W.nearly_singular_f64(N, cfg["seed"]), dtype=torch.float64, device=dev)
    G = torch.empty((N, N), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    h = m.Mpdet(N, p, lastcol=True, stream=stream)
    hp = m.Mpdet(N, p, lastcol=False, stream=stream)
    D = (torch.empty(N, dtype=torch.int8, device=dev), torch.empty(N, dtype=torch.int64, device=dev),
         torch.empty((N, n), dtype=torch.int32, device=dev))
    for _ in range(max(1, args.warmup // 2)):
        h.logabsdet_grad(A, grad=True, out=G)
        hp.set_f64(A)
        hp.factor(out=D)
    steps = max(1, args.steps)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        h.logabsdet_grad(A, grad=True, out=G)
    torch.cuda.synchronize(dev)
    t_grad = (time.perf_counter() - t0) / steps
    t0 = time.perf_counter()
    for _ in range(steps):
        hp.set_f64(A)
        hp.factor(out=D)
    torch.cuda.synchronize(dev)
    t_plain = (time.perf_counter() - t0) / steps
    h.close()
    hp.close()
    # products: lastcol elimination + back substitution (N rows of N, then k*N updates)
    prods = elim_products(N, True) + N * N + N * (N - 1) // 2 * N
    return {"workload": "N=512 p=4096 nearly singular N(0,1) matrix: log|det| and d log|det|/dA in binary64",
            "grad_calls_per_s": 1.0 / t_grad, "ms_per_call": t_grad * 1e3,
            "limb_macs_per_s": prods * n * n / t_grad,
            "plain_det_calls_per_s": 1.0 / t_plain, "grad_cost_vs_plain_det": t_grad / t_plain}


def bench_karatsuba(args, dev, m, peak_macs):
    """Schoolbook against one Karatsuba level on the IMAD engine's lane layout
    (mpdet_mulbench): RN(a*b) of many pairs at p = 8192, 16384, 32768, each
    product formed 8 times on operands held on chip, enough pairs to fill
    every SM.  Work is counted as n^2 limb-MACs per product for both (the
    schoolbook's), so the ratio of the rates is the speed-up."""
    import torch

    out = {}
    g = np.random.Generator(np.random.PCG64(1308))
    for p in (8192, 16384, 32768):
        n = p // 32
        G = 16 if n == 256 else 32
        count = torch.cuda.get_device_properties(dev).multi_processor_count * (128 // G) * 6
        a = (np.zeros(count, np.int8), g.integers(-50, 50, count).astype(np.int64),
             g.integers(0, 2 ** 32, (count, n), dtype=np.uint64).astype(np.uint32))
        b = (np.ones(count, np.int8), g.integers(-50, 50, count).astype(np.int64),
             g.integers(0, 2 ** 32, (count, n), dtype=np.uint64).astype(np.uint32))
        a[2][:, -1] |= 0x80000000
        b[2][:, -1] |= 0x80000000
        res = {}
        for meth in ("school", "kara"):
            m.mulbench(meth, a, b, p, reps=2)  # warm-up
            prods, ms = m.mulbench(meth, a, b, p, reps=8)
            res[meth] = (prods, ms)
        same = all(np.array_equal(x, y) for x, y in zip(res["school"][0], res["kara"][0]))
        macs = float(count) * 8 * n * n
        out[str(p)] = {"pairs": int(count), "school_ms": res["school"][1], "kara_ms": res["kara"][1],
                       "school_limb_macs_per_s": macs / (res["school"][1] / 1e3),
                       "kara_limb_macs_per_s": macs / (res["kara"][1] / 1e3),
                       "kara_speedup": res["school"][1] / res["kara"][1], "same_bits": bool(same)}
    return out


def cauchy_bit_loss(x, y, D, p: int, every: int = 64):
    """Correct bits of the leading minors D_k of the Cauchy matrix
    A_ij = 1/(x_i + y_j) against the closed form
        det_k = prod_{i<j<=k} (x_j - x_i)(y_j - y_i) / prod_{i,j<=k} (x_i + y_j),
    evaluated incrementally with Python integers truncated to p + 64 bits
    (every factor is an exact sum or difference of two doubles; at most 3k^2
    truncations, so the reference is good to about p + 40 bits at k = 1024).
    bits_k = -log2 |D_k - det_k| / det_k and the bit loss L_k = p - bits_k;
    also the least-squares slope of L_k over the k with bits_k > 16, in bits
    per row (the paper's empirical loss is 1.4 to 2.4 bits per row)."""
    import math

    P = p + 64

    def exact(v):
        f, E = math.frexp(float(v))
        return int(f * (1 << 53)), E - 53

    def add(a, b, sign=1):
        (ma, ea), (mb, eb) = a, b
        e = min(ea, eb)
        return (ma << (ea - e)) + sign * (mb << (eb - e)), e

    def trunc(m, e):
        sh = m.bit_length() - P
        return (m >> sh, e + sh) if sh > 0 else (m, e)

    X = [exact(v) for v in x]
    Y = [exact(v) for v in y]
    num, den = (1, 0), (1, 0)
    sgn, ex, limbs = D
    n = p // 32
    out, ks, ls = [], [], []
    min_bits = (float(p + 1), 0)
    for k in range(1, len(x) + 1):
        i = k - 1
        nm, ne = num
        for j in range(i):
            for d in (add(X[i], X[j], -1), add(Y[i], Y[j], -1)):
                nm, ne = trunc(nm * d[0], ne + d[1])
        num = (nm, ne)
        dm, de = den
        for j in range(k):
            d = add(X[i], Y[j])
            dm, de = trunc(dm * d[0], de + d[1])
            if j != i:
                d = add(X[j], Y[i])
                dm, de = trunc(dm * d[0], de + d[1])
        den = (dm, de)
        if int(ex[i]) == np.iinfo(np.int64).min or int(sgn[i]) != 0:
            bits = 0.0
        else:
            gm = 0
            for q in range(n - 1, -1, -1):
                gm = (gm << 32) | int(np.uint32(limbs[i, q]))
            ge = int(ex[i]) - p
            # |D - num/den| / (num/den) = |D den - num| / num, all as integers at a common exponent
            a = (gm * dm, ge + de)
            diff = add(a, num, -1)
            if diff[0] == 0:
                bits = float(p + 1)
            else:
                rel = math.log2(abs(diff[0])) + diff[1] - (math.log2(num[0]) + num[1])
                bits = max(0.0, -rel)
        if bits < min_bits[0]:
            min_bits = (bits, k)
        if k == 1 or k % every == 0 or k == len(x):
            out.append({"k": k, "bits": round(bits, 1), "loss": round(p - bits, 1)})
        if bits > 16:
            ks.append(k)
            ls.append(p - bits)
        elif k > 8 and bits == 0.0 and all(o["bits"] == 0.0 for o in out[-2:]):
            out.append({"k": k, "bits": 0.0, "loss": float(p), "note": "no correct bits from here on"})
            break
    slope = None
    if len(ks) >= 2:
        kb, lb = sum(ks) / len(ks), sum(ls) / len(ls)
        sxx = sum((a - kb) ** 2 for a in ks)
        slope = sum((a - kb) * (b - lb) for a, b in zip(ks, ls)) / sxx if sxx else None
    return {"per_k": out, "bits_per_row": None if slope is None else round(slope, 3),
            "fit_range": [ks[0], ks[-1]] if ks else None,
            "min_bits": round(min_bits[0], 1), "min_bits_k": min_bits[1]}


def _primes_below(limit: int, count: int):
    """The `count` largest primes below `limit` (trial division; limit ~ 2^31)."""
    out, c = [], limit - 1
    while len(out) < count:
        if c % 2 and all(c % d for d in range(3, int(c ** 0.5) + 1, 2)):
            out.append(c)
        c -= 1
    return out


def exact_leading_minors_int(A, kmax: int):
    """Exact leading minors D_1..D_kmax of an integer matrix by elimination
    without pivoting modulo many 31-bit primes at once and Chinese remaindering
    (enough primes for Hadamard's bound of the largest block, plus margin).
    A prime under which some pivot vanishes is dropped for that minor and the
    ones after it.  Returns Python ints."""
    import math

    A = np.asarray(A, dtype=np.int64)[:kmax, :kmax]
    norms = np.sqrt((A.astype(np.float64) ** 2).sum(axis=1))
    bound_bits = float(np.sum(np.log2(np.maximum(norms, 1.0)))) + 2
    P = _primes_below(2 ** 31, int(bound_bits / 30.9) + 8)
    Pv = np.array(P, dtype=np.int64)
    M = np.mod(A[None, :, :], Pv[:, None, None])
    ok = np.ones(len(P), dtype=bool)
    dets = np.ones(len(P), dtype=np.int64)
    residues = []
    for k in range(kmax):
        piv = M[:, k, k].copy()
        ok &= piv != 0
        dets = (dets * piv) % Pv
        residues.append((dets.copy(), ok.copy()))
        if k + 1 == kmax:
            break
        inv = np.array([pow(int(v), int(q) - 2, int(q)) if v else 0 for v, q in zip(piv, P)], dtype=np.int64)
        f = (M[:, k + 1:, k] * inv[:, None]) % Pv[:, None]
        M[:, k + 1:, k + 1:] = (M[:, k + 1:, k + 1:] - (f[:, :, None] * M[:, k, None, k + 1:]) % Pv[:, None, None]) % Pv[:, None, None]
    out = []
    for r, okk in residues:
        x, mod = 0, 1
        for v, q, good in zip(r.tolist(), P, okk.tolist()):
            if not good:
                continue
            # x = x + mod * ((v - x) * mod^-1 mod q)
            t = ((v - x) * pow(mod, -1, q)) % q
            x += mod * t
            mod *= q
        out.append(x - mod if x > mod // 2 else x)
    return out


def integer_bit_loss(A, D, p: int, kmax: int = 256, every: int = 32):
    """Correct bits of the leading minors D_k of an integer matrix against
    their exact values (multi-modular), k = 1..kmax; bit loss L_k = p - bits
    and its least-squares slope in bits per row."""
    import math

    exact = exact_leading_minors_int(A, kmax)
    sgn, ex, limbs = D
    n = p // 32
    out, ks, ls = [], [], []
    for i, e in enumerate(exact):
        k = i + 1
        if int(ex[i]) == np.iinfo(np.int64).min:
            bits = float(p + 1) if e == 0 else 0.0
        elif e == 0:
            bits = 0.0
        else:
            gm = 0
            for q in range(n - 1, -1, -1):
                gm = (gm << 32) | int(np.uint32(limbs[i, q]))
            ge = int(ex[i]) - p
            g = -gm if int(sgn[i]) else gm
            # |g 2^ge - e| / |e| with integers at a common scale
            if ge >= 0:
                diff = abs(g * (1 << ge) - e)
                rel = (math.log2(diff) - math.log2(abs(e))) if diff else None
            else:
                diff = abs(g - e * (1 << -ge))
                rel = (math.log2(diff) + ge - math.log2(abs(e))) if diff else None
            bits = float(p + 1) if rel is None else max(0.0, -rel)
        if k == 1 or k % every == 0 or k == len(exact):
            out.append({"k": k, "bits": round(bits, 1), "loss": round(p - bits, 1)})
        if bits > 16:
            ks.append(k)
            ls.append(p - bits)
    slope = None
    if len(ks) >= 2:
        kb, lb = sum(ks) / len(ks), sum(ls) / len(ls)
        sxx = sum((a - kb) ** 2 for a in ks)
        slope = sum((a - kb) * (b - lb) for a, b in zip(ks, ls)) / sxx if sxx else None
    return {"per_k": out, "bits_per_row": None if slope is None else round(slope, 3)}


def tcl_mma_macs_per_product(p: int) -> int:
    """bf16 multiply-accumulates the large-precision tensor engine issues per
    product at p = 4096 .. 32768 (its tile K ranges; the lower half of the
    convolution below 32 limbs under the rounding point is not formed).  The
    schoolbook count of the same 8-bit x 4-bit convolution is 32 n^2."""
    n = p // 32
    KD, KB, R0, T = 4 * n, 8 * n, 8 * n - 256, n // 32 + 1
    tot = 0
    for tau in range(T):
        rho = R0 + 256 * tau
        lo = (KD - 1 - min((rho + 255) // 2, KD - 1)) // 16
        hi = (KD - 1 - ((rho - KB + 1) // 2 if rho > KB else 0)) // 16 + 1
        tot += (hi - lo) * 16 * 256
    return tot


def bench_large(args, dev, m, peak_macs):
    """Workload C5 at full size: Cauchy N = 4096, p = 32768 (1024 limbs,
    68.9 GB in HBM), det and leading minors.  A window of its heaviest steps
    is timed here (the matrix is generated on the device, step 1 runs untimed
    as warm-up, steps 2..1+w are timed with CUDA events on the handle's
    stream) on the tensor-core engine, and two steps on the IMAD engine with
    schoolbook and with Karatsuba products for comparison; the whole run is
    bench.py --large-full.  The Schur-update launches inside the window are
    timed one by one against the tensor and integer-multiply peaks."""
    import torch

    cfg = W.C5
    N, p, w = cfg["N"], cfg["p"], 8
    n = p // 32
    x, y = W.cauchy_xy(N, cfg["seed"])
    st = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def window(engine, steps, karatsuba=False, profile=False):
        h = m.Mpdet(N, p, lastcol=False, stream=st.cuda_stream)
        h.tune(engine=engine, karatsuba=karatsuba)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h.set_cauchy(x, y)
        torch.cuda.synchronize(dev)
        tg = time.perf_counter() - t0
        h.factor_range(0, 1)
        torch.cuda.synchronize(dev)
        if profile:
            h.profile(True)
        e0.record(st)
        h.factor_range(1, 1 + steps)
        e1.record(st)
        torch.cuda.synchronize(dev)
        pr = h.profile_read() if profile else None
        assert h.status()[0] == 0
        h.close()
        return e0.elapsed_time(e1), tg, pr

    ms, t_gen, pr = window(1, w, profile=True)
    ms_imad, _, _ = window(0, 2)
    ms_kara, _, _ = window(0, 2, karatsuba=True)
    prods = sum((N - k - 1) ** 2 + (N - k - 1) + 1 for k in range(1, 1 + w))
    prods2 = sum((N - k - 1) ** 2 + (N - k - 1) + 1 for k in range(1, 3))
    rate = prods * n * n / (ms / 1e3)
    upd = pr["update_limb_macs"] / (pr["update_ms"] / 1e3)
    # tensor roofline of the update kernel: the bf16 MMA work it issues per
    # product against the measured sustained bf16 rate (a kernel inside a
    # long step)
    mma_flops = 2.0 * tcl_mma_macs_per_product(p) * (pr["update_limb_macs"] / (n * n))
    tflops = mma_flops / (pr["update_ms"] / 1e3) / 1e12
    try:
        tpeak = float(measured_peaks()["bf16_tflops_sustained"])
    except Exception:
        tpeak = 1700.0
    total = elim_products(N, False) * n * n
    # Whole-run projection: a step's cost depends on its trailing size R =
    # N - k - 1 (and p), not on the steps before it, so steps of smaller
    # leading blocks of the same matrix stand in for the late steps of the
    # full run; the step time is interpolated linearly between the sampled R
    # (in R^2, the work) and summed over R = 0..N-1.
    samples = [(N - 1 - (1 + w) / 2, ms / w)]
    for Rs in (2048, 1024, 512, 256, 128, 64, 16):
        Ns = Rs + 2
        hs = m.Mpdet(Ns, p, lastcol=False, stream=st.cuda_stream)
        hs.set_cauchy(x[:Ns], y[:Ns])
        hs.factor_range(0, 1)
        e0.record(st)
        hs.factor_range(1, 3)
        e1.record(st)
        torch.cuda.synchronize(dev)
        samples.append((Rs, e0.elapsed_time(e1) / 2))
        hs.close()
    samples.sort()
    rs = np.array([s_[0] for s_ in samples], dtype=np.float64)
    ts = np.array([s_[1] for s_ in samples], dtype=np.float64)
    Rall = np.arange(N, dtype=np.float64)
    t_all = np.interp(Rall ** 2, rs ** 2, ts, left=ts[0])  # ms per step at trailing size R
    proj_s = float(t_all.sum()) / 1e3
    return {"workload": f"Cauchy N={N} p={p} (68.9 GB in HBM), det + leading minors: steps 2..{1 + w} "
                        "timed (the heaviest; bench.py --large-full runs them all)",
            "engine": "tensor (8-bit x 4-bit digit convolution on tcgen05)",
            "window_ms": ms, "limb_macs_per_s": rate, "frac_of_imad_peak": rate / peak_macs,
            "imad_window_ms_2_steps": ms_imad, "imad_limb_macs_per_s": prods2 * n * n / (ms_imad / 1e3),
            "imad_karatsuba_window_ms_2_steps": ms_kara,
            "imad_karatsuba_limb_macs_per_s": prods2 * n * n / (ms_kara / 1e3),
            "tensor_vs_imad": (prods * n * n / (ms / 1e3)) / (prods2 * n * n / (ms_imad / 1e3)),
            "update_kernel": {"kernel": "k_update_tcl<1024>", "achieved": upd / 1e12, "peak": peak_macs / 1e12,
                              "unit": "Tlimb-MAC/s", "frac": upd / peak_macs, "launches": int(pr["update_launches"]),
                              "tensor": {"achieved": tflops, "peak": tpeak, "unit": "TFLOP/s",
                                         "frac": tflops / tpeak,
                                         "basis": "bf16 MMA flops issued (tcl_mma_macs_per_product x 2 per "
                                                  "product) / CUDA-event time, against MEASURED_PEAKS "
                                                  "bf16_tflops_sustained (of measured)"}},
            "cauchy_generation_s": t_gen,
            "step_ms_by_trailing_size": {str(int(a)): round(b, 3) for a, b in samples},
            "projected_full_factorisation_s": proj_s,
            "projected_full_limb_macs_per_s": total / proj_s,
            "projected_full_frac_of_imad_peak": total / proj_s / peak_macs}


def run_large_full(args):
    """One complete factorisation of workload C5 (Cauchy N = 4096, p = 32768,
    68.9 GB in HBM): every step, in windows of --window steps timed with CUDA
    events on the handle's stream, nvidia-smi clocks sampled per window.  The
    leading minors D_1..D_N are saved (numpy .npz) for the checks that run
    on the host afterwards: D_1..D_256 against the stored oracle digests and
    every D_k against the closed-form Cauchy determinant.  Prints one JSON
    line with the whole-run time and its fraction of the IMAD peak."""
    import torch

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import paper_1308_1536_gb300 as m

    m.load()
    cfg = W.C5
    N, p = cfg["N"], cfg["p"]
    n = p // 32
    x, y = W.cauchy_xy(N, cfg["seed"])
    if args.large_n:  # the leading large_n x large_n block of the same matrix
        N = args.large_n
        x, y = x[:N], y[:N]
    st = torch.cuda.current_stream(dev)
    h = m.Mpdet(N, p, lastcol=False, stream=st.cuda_stream)
    if args.karatsuba:
        h.tune(karatsuba=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    h.set_cauchy(x, y)
    torch.cuda.synchronize(dev)
    t_gen = time.perf_counter() - t0
    props = torch.cuda.get_device_properties(dev)
    windows = []
    total_ms = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h.profile(True)
    upd_ms = upd_macs = 0.0
    t_wall = time.perf_counter()
    for k0 in range(0, N, args.window):
        k1 = min(N, k0 + args.window)
        with Clocks(0) as clk:
            e0.record(st)
            h.factor_range(k0, k1)
            e1.record(st)
            torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        pr = h.profile_read()
        upd_ms += pr["update_ms"]
        upd_macs += pr["update_limb_macs"]
        h.profile(True)
        total_ms += ms
        prods = sum((N - k - 1) ** 2 + (N - k - 1) + 1 for k in range(k0, k1))
        c = clk.summary()
        windows.append({"steps": [k0 + 1, k1], "ms": round(ms, 3), "limb_macs_per_s": prods * n * n / (ms / 1e3),
                        "sm_mhz": c.get("sm_mhz"), "reasons": c.get("reasons")})
        print(json.dumps({"window": windows[-1]}), file=sys.stderr, flush=True)
    wall = time.perf_counter() - t_wall
    rc, zk = h.status()
    D = h.get_minors()
    h.close()
    os.makedirs(os.path.dirname(os.path.abspath(args.save)), exist_ok=True)
    np.savez(args.save, sign=D[0], exp=D[1], limbs=D[2])
    fmax = max((w["sm_mhz"] or 0) for w in windows) or 2070.0
    smax = 2070.0
    peak = props.multi_processor_count * 32 * smax * 1e6
    total = elim_products(N, False) * n * n
    reasons = sorted({r for w in windows for r in (w["reasons"] or [])})
    out = {"metric": METRIC, "workload": f"Cauchy N={N} p={p} ({N * N * (4 * n + 9) / 1e9:.1f} GB in HBM), det + {N} "
                                         "leading minors: the whole factorisation"
                                         + (f" of the leading {N} x {N} block of the N = {cfg['N']} matrix"
                                            if N != cfg["N"] else ""), "status": rc, "zero_k": zk,
           "device_ms": total_ms, "wall_s": wall, "cauchy_generation_s": t_gen,
           "limb_macs": total, "limb_macs_per_s": total / (total_ms / 1e3),
           "frac_of_imad_peak": total / (total_ms / 1e3) / peak,
           "peak_basis": f"{props.multi_processor_count} SMs x 32 limb-MAC/clk x {smax:.0f} MHz",
           "update_kernel": {"ms": upd_ms, "limb_macs_per_s": upd_macs / (upd_ms / 1e3),
                             "frac": upd_macs / (upd_ms / 1e3) / peak,
                             "tensor_tflops": 2.0 * tcl_mma_macs_per_product(p) * upd_macs / (n * n) / (upd_ms / 1e3)
                             / 1e12 if p >= 4096 else None,
                             "tensor_frac_of_sustained_bf16": 2.0 * tcl_mma_macs_per_product(p) * upd_macs / (n * n)
                             / (upd_ms / 1e3) / 1e12 / float(measured_peaks().get("bf16_tflops_sustained", 1700.0))
                             if p >= 4096 else None},
           "window_steps": args.window, "windows": windows, "clock_reasons_seen": reasons,
           "update_products": "karatsuba (one level)" if args.karatsuba else "schoolbook",
           "sm_mhz_median_of_windows": statistics.median([w["sm_mhz"] for w in windows if w["sm_mhz"]] or [0]),
           "saved": args.save}
    print(json.dumps(out))
    return 0 if rc == 0 else 1


def factor_window(N: int, p: int, k1: int) -> int:
    """Profiling aid: steps [0, k1) of the seeded Cauchy matrix of size N at
    precision p, look-ahead off (each step: pivot, multipliers, one update
    launch), on cuda:0.  Prints the status."""
    import torch

    import paper_1308_1536_gb300 as m

    m.load()
    x, y = W.cauchy_xy(N, 11)
    h = m.Mpdet(N, p, lastcol=False)
    h.tune(lookahead=0)
    h.set_cauchy(x, y)
    h.factor_range(0, k1)
    torch.cuda.synchronize()
    rc = h.status()
    h.close()
    print(json.dumps({"factor_window": [N, p, k1], "status": list(rc)}))
    return 0 if rc[0] == 0 else 1


def engine_table(p: int, Ns, reps: int = 2, thresholds=(64, 256, 512)) -> int:
    """Tuning aid: whole eliminations of the seeded Cauchy matrix (lastcol
    mode, look-ahead on) at precision p for each N, on the IMAD engine and on
    the tensor engine with update launches of at least each row threshold;
    best of ``reps`` wall times around the factorisation (which synchronises),
    and whether both engines give the same bits.  One JSON line per N."""
    import torch

    import paper_1308_1536_gb300 as m

    m.load()

    def run(N, engine, thr):
        x, y = W.cauchy_xy(N, 1310)
        h = m.Mpdet(N, p, lastcol=True)
        h.tune(engine=engine)
        if thr is not None:
            h.tune(tc_min_rows=thr)
        best, D = float("inf"), None
        for _ in range(reps):
            h.set_cauchy(x, y)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, _, D = h.factor()
            best = min(best, time.perf_counter() - t0)
        h.close()
        return best * 1e3, D

    for N in Ns:
        ref_ms, Dref = run(N, 0, None)
        rec = {"engine_table": {"p": p, "N": N}, "imad_ms": round(ref_ms, 2)}
        for thr in thresholds:
            if thr >= N:
                continue
            ms, D = run(N, 1, thr)
            rec[f"tensor_min_rows_{thr}_ms"] = round(ms, 2)
            rec[f"tensor_min_rows_{thr}_same_bits"] = all(np.array_equal(a, b) for a, b in zip(D, Dref))
        print(json.dumps(rec), flush=True)
    return 0


def check_large(path: str, lead: int = 256):
    """Host checks of the leading minors saved by --large-full (no GPU):
    D_1..D_lead against the digests the CPU oracle wrote for the leading
    lead x lead block (tests/golden/c5_cauchy_lead256_p32768.txt; the
    leading minors of a matrix depend only on its leading block), and every
    D_k against the closed-form Cauchy determinant (correct bits per k, the
    fewest over all k, the loss in bits per row)."""
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import fullsize as F

    z = np.load(path)
    D = (z["sign"], z["exp"], z["limbs"])
    cfg = W.C5
    N, p = len(D[0]), cfg["p"]
    x, y = W.cauchy_xy(cfg["N"], cfg["seed"])
    x, y = x[:N], y[:N]
    out = {"what": f"leading minors of the saved run ({path}), N = {N}, p = {p}"}
    try:
        want = [r[1] for r in F.read("c5")["D"]]
        got = F.num_digests((D[0][:lead], D[1][:lead], D[2][:lead]))
        bad = F.first_mismatch(got, want[:lead])
        out["oracle_leading"] = {"k": [1, lead], "bit_exact": bad is None,
                                 "first_mismatch_k": None if bad is None else bad + 1}
    except FileNotFoundError:
        out["oracle_leading"] = {"skipped": "no stored oracle values"}
    t0 = time.perf_counter()
    out["closed_form"] = cauchy_bit_loss(x, y, D, p, every=256)
    out["closed_form_s"] = time.perf_counter() - t0
    print(json.dumps(out))
    ok = out["oracle_leading"].get("bit_exact", True) and out["closed_form"]["min_bits"] > 0
    return 0 if ok else 1


def bench_hostmem(args, dev, m, peak_macs):
    """The N x N array in page-locked host memory that the GPU reads and
    writes in place (MPDET_HOSTMEM), for matrices larger than HBM such as the
    paper's N = 12000 at 32768 bits (590 GB).  Cauchy N = 2048, p = 32768
    (17.2 GB): steps 2..3 timed with the array host-resident and
    device-resident; the whole N = 12000 factorisation is projected from the
    host-resident step time (a step's work grows as its trailing size
    squared, measured down to R = 256 on the device-resident path)."""
    import torch

    N, p, w = 2048, 32768, 2
    n = p // 32
    need = N * N * (4 * n + 9)
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = 0
    if avail < 3 * need:
        return {"skipped": f"host memory: {avail / 1e9:.0f} GB free, {3 * need / 1e9:.0f} GB wanted"}
    x, y = W.cauchy_xy(N, W.C5["seed"])
    st = torch.cuda.current_stream(dev)
    out = {"workload": f"Cauchy N={N} p={p} ({need / 1e9:.1f} GB), det + leading minors: steps 2..{1 + w} timed"}
    for host in (True, False):
        h = m.Mpdet(N, p, lastcol=False, stream=st.cuda_stream, hostmem=host)
        h.set_cauchy(x, y)
        h.factor_range(0, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(st)
        h.factor_range(1, 1 + w)
        e1.record(st)
        torch.cuda.synchronize(dev)
        assert h.status()[0] == 0
        h.close()
        out["host_ms" if host else "device_ms"] = e0.elapsed_time(e1)
    prods = sum((N - k - 1) ** 2 + (N - k - 1) + 1 for k in range(1, 1 + w))
    rate = prods * n * n / (out["host_ms"] / 1e3)
    out["host_limb_macs_per_s"] = rate
    out["host_frac_of_imad_peak"] = rate / peak_macs
    out["host_vs_device"] = out["device_ms"] / out["host_ms"]
    Nb = 12000
    total = elim_products(Nb, False) * n * n
    out["projected_N12000_p32768_s"] = total / rate
    out["projected_N12000_p32768_array_bytes"] = Nb * Nb * (4 * n + 9)
    return out


def guarded(fn, *a):
    """Run one optional part of the benchmark; an exception is reported in
    the JSON line (as {"error": ...}) instead of losing the whole line."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"[:300]}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1308_1536_gb300 as m

    m.load()
    cfg = W.C2
    N, p = args.N or cfg["N"], args.p or cfg["p"]
    n = p // 32
    x, y = W.cauchy_xy(N, cfg["seed"])
    A = W.int_matrix(N, cfg["seed"] + 100).astype(np.int32)
    xd, yd = torch.tensor(x, device=dev), torch.tensor(y, device=dev)
    Ad = torch.tensor(A, device=dev)
    stream = torch.cuda.current_stream(dev)
    # the two matrices run on two streams, so one's serial pivot overlaps the
    # other's Schur update
    sa, sb = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    hc = m.Mpdet(N, p, lastcol=True, stream=sa.cuda_stream)
    hi = m.Mpdet(N, p, lastcol=True, stream=sb.cuda_stream)
    if args.update_variant >= 0:
        hc.tune(update_variant=args.update_variant)
        hi.tune(update_variant=args.update_variant)
    if args.engine >= 0:
        hc.tune(engine=args.engine)
        hi.tune(engine=args.engine)

    def dev_out():
        return (torch.empty(N, dtype=torch.int8, device=dev), torch.empty(N, dtype=torch.int64, device=dev),
                torch.empty((N, n), dtype=torch.int32, device=dev))

    Dc, Cc, Di, Ci = dev_out(), dev_out(), dev_out(), dev_out()

    def step():
        ev = torch.cuda.Event()
        ev.record(stream)
        sa.wait_event(ev)
        sb.wait_event(ev)
        hc.set_cauchy(xd, yd)
        hc.factor(out=Dc)
        hc.lastcol_minors(out=Cc)
        hi.set_i32(Ad)
        hi.factor(out=Di)
        hi.lastcol_minors(out=Ci)
        ea, eb = torch.cuda.Event(), torch.cuda.Event()
        ea.record(sa)
        eb.record(sb)
        stream.wait_event(ea)
        stream.wait_event(eb)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    barrier()
    l0 = hc.profile_read()["launches"] + hi.profile_read()["launches"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1) / args.steps
    launches = (hc.profile_read()["launches"] + hi.profile_read()["launches"] - l0) // args.steps
    assert hc.status()[0] == 0 and hi.status()[0] == 0
    # roofline pass: one more step with the two matrices one after the other
    # (no overlap between their kernels), CUDA events around every launch of
    # the Schur-update kernel on its stream
    hc.profile(True)
    hi.profile(True)
    torch.cuda.synchronize(dev)
    t_serial = time.perf_counter()
    hc.set_cauchy(xd, yd)
    hc.factor(out=Dc)
    hc.lastcol_minors(out=Cc)
    pc = hc.profile_read()
    hi.set_i32(Ad)
    hi.factor(out=Di)
    hi.lastcol_minors(out=Ci)
    pi = hi.profile_read()
    serial_ms = (time.perf_counter() - t_serial) * 1e3
    hc.profile(False)
    hi.profile(False)
    ms = shard.reduce_over_ranks(ms, "max", device=dev)
    macs = step_limb_macs(N, p, 2)
    value = macs * world / (ms / 1e3)

    # end-to-end through the C ABI with host buffers (pinned inputs)
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.from_numpy(y).pin_memory()
    Ah = torch.from_numpy(A).pin_memory()

    def step_e2e():
        hc.set_cauchy(xh, yh)
        rc1, _, D1 = hc.factor()
        C1 = hc.lastcol_minors()
        hi.set_i32(Ah)
        rc2, _, D2 = hi.factor()
        C2 = hi.lastcol_minors()
        return D1, C1, D2, C2

    step_e2e()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        outs = step_e2e()
    barrier()
    e2e_ms = shard.reduce_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, "max", device=dev)
    h2d = x.nbytes + y.nbytes + A.nbytes
    d2h = sum(a.nbytes for o in outs for a in o)

    # the batch workload runs on every rank (its share of the matrices)
    extras = set() if args.no_extras else set(args.extras.split(","))
    batch = guarded(bench_batch, args, dev, m, rank, world) if "batch" in extras or "all" in extras else None
    if rank == 0:
        props = torch.cuda.get_device_properties(dev)
        nsm = props.multi_processor_count
        clocks = clk.summary()
        peaks = measured_peaks()
        fmax = float(clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0)
        peak = nsm * 32 * fmax * 1e6
        upd_ms = pc["update_ms"] + pi["update_ms"]
        upd_macs = pc["update_limb_macs"] + pi["update_limb_macs"]
        upd_launches = pc["update_launches"] + pi["update_launches"]
        achieved = upd_macs / (upd_ms / 1e3)
        tensor = (p == 2048 and args.engine != 0)  # the default engine per precision
        # the recorded bytes per product belong to the tensor-core kernel at p = 2048
        per_launch = upd_macs / (n * n) / max(upd_launches, 1)
        tr = recorded_traffic(per_launch) if tensor and p == 2048 else None
        # the last capture's figure when the sources have changed since (the
        # "traffic" key stays null then)
        tr_old = recorded_traffic(per_launch, any_sources=True) if tensor and p == 2048 and tr is None else None
        if tensor:
            # exact digit convolution on the tensor cores: one limb-MAC is 16 products of 8-bit digits,
            # 32 flops; peak = measured bf16 dense throughput (sustained: the kernel runs inside a long step)
            tpeak = float(peaks.get("bf16_tflops_sustained") or 1700.0)
            roof = {"bound": "tensor", "kernel": "k_update_tcp (Schur update, tcgen05 digit convolution)",
                    "achieved": achieved * 32 / 1e12, "peak": tpeak, "unit": "TFLOP/s",
                    "frac": achieved * 32 / 1e12 / tpeak, "traffic": tr,
                    "peak_basis": "MEASURED_PEAKS bf16_tflops_sustained (of measured)",
                    "imad_equivalent": {"achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tlimb-MAC/s",
                                        "frac": achieved / peak,
                                        "peak_basis": f"{nsm} SMs x 32 limb-MAC/clk x {fmax:.0f} MHz"}}
        else:
            roof = {"bound": "alu", "kernel": "k_update (Schur update, IMAD)", "achieved": achieved / 1e12,
                    "peak": peak / 1e12, "unit": "Tlimb-MAC/s", "frac": achieved / peak, "traffic": tr,
                    "peak_basis": f"{nsm} SMs x 32 limb-MAC/clk x {fmax:.0f} MHz"}
        if tr_old is not None:
            roof["traffic_last_capture"] = {
                "bytes": tr_old, "source": "profiles/k_update_traffic.json",
                "recorded_source_sha": json.load(open(os.path.join(ROOT, "profiles", "k_update_traffic.json")))
                .get("source_sha"), "current_source_sha": kernel_source_sha(),
                "note": "captured on earlier sources of the kernel files, not recaptured since"}
        roof["update_share"] = upd_ms / serial_ms
        roof["launches"] = int(upd_launches)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"cauchy+int N={N} p={p} lastcol: det, {N} leading minors and {N} "
                                   "last-column minors of two matrices per step",
                       "N": N, "p": p, "matrices": 2, "parallelism": f"replica x{world}",
                       "engine": "tensor" if tensor else "imad",
                       "l2": "inputs larger than L2 (each matrix %.0f MB in HBM)" % (N * N * (4 * n + 9) / 1e6)},
            "e2e": {"value": macs * world / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms},
            "gpu_launches": int(launches * args.steps),
            "roofline": roof,
            "clocks": clocks,
        }
        want = lambda k: "all" in extras or k in extras  # noqa: E731
        if want("accuracy"):
            def acc_cauchy():
                Dh = (Dc[0].cpu().numpy(), Dc[1].cpu().numpy(), Dc[2].cpu().numpy().view(np.uint32))
                return {"what": f"leading minors D_k of the N={N} Cauchy matrix (GPU results of the timed step) "
                                "against the closed-form Cauchy determinant at every k", **cauchy_bit_loss(x, y, Dh, p)}

            def acc_int():
                Dih = (Di[0].cpu().numpy(), Di[1].cpu().numpy(), Di[2].cpu().numpy().view(np.uint32))
                return {"what": "leading minors D_1..D_128 of the integer matrix (GPU results of the timed step) "
                                "against their exact values (multi-modular)",
                        **integer_bit_loss(A, Dih, p, kmax=128, every=16)}

            out["accuracy"] = guarded(acc_cauchy)
            out["accuracy_int"] = guarded(acc_int)
        if batch is not None:
            out["batch"] = batch
        if want("adjoint"):
            out["adjoint"] = guarded(bench_adjoint, args, dev, m)
        if want("karatsuba"):
            out["karatsuba"] = guarded(bench_karatsuba, args, dev, m, peak)
        if want("large"):
            out["large"] = guarded(bench_large, args, dev, m, peak)
        if want("hostmem"):
            out["hostmem"] = guarded(bench_hostmem, args, dev, m, peak)
        if world == 1 and not args.no_cpu_baseline:
            cb = guarded(oracle_sample)
            cb.pop("seconds", None)
            # the same oracle on one thread, on a smaller sample (the work per
            # second is the comparable figure)
            one = guarded(oracle_sample, ORACLE_SAMPLE_K // 2, 1)
            one.pop("seconds", None)
            cb["one_thread"] = one
            out["cpu_baseline"] = cb
        print(json.dumps(out))
    hc.close()
    hi.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mpdet", choices=["mpdet", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the accuracy, batch, adjoint and large workloads")
    ap.add_argument("--extras", default="all",
                    help="comma list of accuracy,batch,adjoint,karatsuba,large,hostmem (default all)")
    ap.add_argument("--batch-count", type=int, default=0,
                    help="profiling aid: matrices in the batch workload (default: the workload's 4096)")
    ap.add_argument("--N", type=int, default=0, help="profiling aid: override N (default: the workload's 1024)")
    ap.add_argument("--p", type=int, default=0, help="profiling aid: override p (default: the workload's 2048)")
    ap.add_argument("--update-variant", type=int, default=-1, help="tuning aid: Schur-update register budget 0..3")
    ap.add_argument("--engine", type=int, default=-1, help="tuning aid: 0 IMAD, 1 tensor pipelined, 2 tensor serial")
    ap.add_argument("--factor-window", type=int, nargs=3, metavar=("N", "P", "K1"),
                    help="profiling aid: steps [0, K1) of the seeded N x N Cauchy matrix at p bits, look-ahead off")
    ap.add_argument("--engine-table", type=int, nargs="+", metavar=("P", "N"),
                    help="tuning aid: whole eliminations at precision P for each N, IMAD against tensor engine")
    ap.add_argument("--check-large", default="", metavar="NPZ",
                    help="host checks (no GPU) of the leading minors a --large-full run saved")
    ap.add_argument("--large-full", action="store_true",
                    help="the whole N=4096 p=32768 factorisation in timed windows (about an hour); not the bench line")
    ap.add_argument("--window", type=int, default=64, help="--large-full: steps per timed window")
    ap.add_argument("--large-n", type=int, default=0,
                    help="--large-full: factor the leading N x N block of the N=4096 matrix instead (its steps cost "
                         "what the full run's last N steps cost; its minors are the full run's D_1..D_N)")
    ap.add_argument("--save", default="c5_minors.npz", help="--large-full: where the leading minors go")
    ap.add_argument("--karatsuba", action="store_true",
                    help="--large-full: the IMAD update's products by one Karatsuba level")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.check_large:
        return check_large(args.check_large)
    if args.factor_window:
        return factor_window(*args.factor_window)
    if args.engine_table:
        if len(args.engine_table) < 2:
            ap.error("--engine-table P N [N ...]")
        return engine_table(args.engine_table[0], args.engine_table[1:])
    if args.large_full:
        return run_large_full(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
