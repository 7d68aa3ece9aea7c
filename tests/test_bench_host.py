"""Host-side logic of the benchmark (no GPU): the closed-form accuracy report
of the Cauchy leading minors against exact rational arithmetic, and the
work counts behind the limb-MAC/s figures."""
from fractions import Fraction
import math

import pytest

import exactref as X
from paper_1308_1536_gb300 import workloads as W

pytestmark = pytest.mark.usefixtures("oracle_lib")


def test_cauchy_bit_loss_matches_exact_rationals(oracle_lib):
    import bench

    N, p = 40, 256
    x, y = W.cauchy_xy(N, W.C1["seed"])
    st, zk, D, _ = oracle_lib.ge(oracle_lib.cauchy(x, y, p), N, p)
    r = bench.cauchy_bit_loss(x, y, D, p, every=1)
    fx = [Fraction(float(v)) for v in x]
    fy = [Fraction(float(v)) for v in y]
    num = den = Fraction(1)
    Dv = X.unpack(D, p)
    got = {o["k"]: o["bits"] for o in r["per_k"]}
    for k in range(1, N + 1):
        i = k - 1
        for j in range(i):
            num *= (fx[i] - fx[j]) * (fy[i] - fy[j])
        for j in range(k):
            den *= (fx[i] + fy[j]) * ((fx[j] + fy[i]) if j != i else 1)
        ex = num / den
        rel = abs(Dv[i] - ex) / ex
        bits = max(0.0, -(math.log2(rel.numerator) - math.log2(rel.denominator))) if rel else p + 1
        if k in got:
            assert abs(got[k] - bits) <= 0.11, (k, got[k], bits)
    assert 2.0 < r["bits_per_row"] < 12.0


def test_work_counts():
    import bench

    # plain elimination: S(N) = (N-1)N(2N-1)/6 Schur products, N(N-1)/2 multipliers, N-1 pivot products
    for N in (1, 2, 5, 64):
        assert bench.elim_products(N, False) == (N - 1) * N * (2 * N - 1) // 6 + N * (N - 1) // 2 + (N - 1)
    # lastcol: full rows, (N-1)^2 N / 2 update products, plus the N-1 last-column products
    for N in (2, 5, 64):
        assert bench.elim_products(N, True) == (N - 1) ** 2 * N // 2 + N * (N - 1) // 2 + 2 * (N - 1)


def test_exact_integer_minors_and_bit_loss(oracle_lib):
    """The multi-modular exact leading minors equal exact rational
    determinants (condensation), and the oracle's minors of an integer matrix
    keep almost all their bits against them."""
    import bench
    import test_oracle_ge as T

    A = W.int_matrix(14, 21)
    ex = bench.exact_leading_minors_int(A, 14)
    assert [int(v) for v in ex] == [int(v) for v in T.exact_leading_minors(A.tolist())]
    N, p = 48, 512
    A = W.int_matrix(N, 22)
    st, zk, D, _ = oracle_lib.ge(oracle_lib.from_int(A.reshape(-1), p), N, p)
    r = bench.integer_bit_loss(A, D, p, kmax=N, every=8)
    assert all(o["bits"] >= p - 40 for o in r["per_k"]), r
    assert r["per_k"][0]["bits"] == p + 1  # D_1 = a_11 exactly


def test_batch_tune_cache_roundtrip(tmp_path):
    """The batch autotuner's choice cache: keys separate devices, precisions
    and size mixes; a stored choice reads back; a damaged file reads as empty."""
    from paper_1308_1536_gb300 import TuneCache, tune_cache_key

    Ns, _, _ = W.batch_sizes(4096, 8, 256, 1311)
    k1 = tune_cache_key("GB300 sm_103 x152", 1024, Ns)
    assert k1 != tune_cache_key("GB300 sm_103 x152", 2048, Ns)
    assert k1 != tune_cache_key("B200 sm_100 x148", 1024, Ns)
    assert k1 != tune_cache_key("GB300 sm_103 x152", 1024, Ns[:4000])
    assert k1 == tune_cache_key("GB300 sm_103 x152", 1024, list(Ns))
    c = TuneCache(str(tmp_path / "tune.json"))
    assert c.get(k1) is None
    c.put(k1, {"variant": 3, "blocks_per_sm": 4, "ms": 1425.5, "candidates": 8})
    c.put("other", {"variant": 0, "blocks_per_sm": 2, "ms": 1.0, "candidates": 1})
    assert TuneCache(str(tmp_path / "tune.json")).get(k1)["variant"] == 3
    (tmp_path / "bad.json").write_text("{not json")
    assert TuneCache(str(tmp_path / "bad.json")).get(k1) is None


def test_recorded_traffic_scales_with_the_launch():
    """The DRAM traffic recorded from one ncu capture of the tensor update
    kernel is used only while the kernel's sources hash to the recorded value,
    and then scales with the products of the launch."""
    import json
    import os

    import bench

    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "k_update_traffic.json")))
    cap = rec["capture"]
    products = 765 * 766
    assert abs(rec["bytes_per_product"] - (cap["dram_bytes_read"] + cap["dram_bytes_write"]) / products) < 0.1
    t = bench.recorded_traffic(1000.0)
    if rec["source_sha"] == bench.kernel_source_sha():
        assert t == rec["bytes_per_product"] * 1000.0
    else:
        assert t is None


def test_guarded_optional_parts():
    import bench

    assert bench.guarded(lambda a, b: a + b, 2, 3) == 5
    r = bench.guarded(lambda: {}["missing"])
    assert set(r) == {"error"} and r["error"].startswith("KeyError")


def test_recorded_traffic_is_keyed_by_the_kernel_sources():
    """The bench line's DRAM traffic comes from the ncu record only while the
    record's source hash is the current one; the last capture's figure is
    still available, marked as such, when the sources have changed."""
    import json
    import os

    import bench

    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "k_update_traffic.json")))
    same = rec["source_sha"] == bench.kernel_source_sha()
    assert bench.recorded_traffic(1000.0, any_sources=True) == rec["bytes_per_product"] * 1000.0
    assert bench.recorded_traffic(1000.0) == (rec["bytes_per_product"] * 1000.0 if same else None)
    # the record the bench line carries beside a null traffic (the same expressions)
    last = {"bytes": bench.recorded_traffic(1000.0, any_sources=True), "source": "profiles/k_update_traffic.json",
            "recorded_source_sha": json.load(open(os.path.join(bench.ROOT, "profiles", "k_update_traffic.json")))
            .get("source_sha"), "current_source_sha": bench.kernel_source_sha()}
    assert json.loads(json.dumps(last)) == last
