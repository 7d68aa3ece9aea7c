"""The several-GPU host logic on CPU: two gloo ranks (processes) split a
batch of matrices, each eliminates its share (with the CPU oracle standing
in for a GPU), rank 0 gathers the shares and the result must equal one
process eliminating the whole batch bit for bit; the timing reduction takes
the max over ranks; shards partition the batch and balance its work."""
import os
import socket

import numpy as np
import pytest

from paper_1308_1536_gb300 import shard
from paper_1308_1536_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _items(count, p):
    g = W.rng(4242)
    Ns = g.integers(1, 13, count)
    mats = []
    for m, N in enumerate(Ns):
        if m % 2 == 0:
            mats.append(("cauchy", W.cauchy_xy(int(N), 100 + m)))
        else:
            mats.append(("int", W.int_matrix(int(N), 100 + m)))
    return Ns, mats


def _eliminate(oracle, kind, d, N, p):
    A = oracle.cauchy(*d, p) if kind == "cauchy" else oracle.from_int(np.asarray(d).reshape(-1), p)
    st, zk, D, _ = oracle.ge(A, N, p)
    return zk, tuple(np.asarray(t) for t in D)


def _rank_main(rank, world, port, count, p, outdir):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist

    import oracle

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        Ns, mats = _items(count, p)
        mine = shard.batch_shard(Ns, rank, world)
        res = {int(m): _eliminate(oracle, *mats[m], int(Ns[m]), p) for m in mine}
        gathered = [None] * world if rank == 0 else None
        dist.gather_object(res, gathered, dst=0)
        t = shard.reduce_over_ranks(float(rank + 1) * 1.5, "max")
        s = shard.reduce_over_ranks(float(rank + 1), "sum")
        if rank == 0:
            allres = {}
            for part in gathered:
                assert not set(part) & set(allres), "a matrix was eliminated on two ranks"
                allres.update(part)
            np.save(os.path.join(outdir, "reduce.npy"), np.array([t, s]))
            keys = sorted(allres)
            np.save(os.path.join(outdir, "keys.npy"), np.array(keys))
            for k in keys:
                zk, D = allres[k]
                np.savez(os.path.join(outdir, f"m{k}.npz"), zk=zk, s=D[0], e=D[1], m=D[2])
    finally:
        dist.destroy_process_group()


def test_batch_shard_partitions_and_balances():
    Ns, _, _ = W.batch_sizes(W.C3["count"], W.C3["Nmin"], W.C3["Nmax"], W.C3["seed"])
    for world in (1, 2, 3, 4, 8):
        parts = [shard.batch_shard(Ns, r, world) for r in range(world)]
        allidx = np.concatenate(parts)
        assert len(allidx) == len(Ns) and len(np.unique(allidx)) == len(Ns)
        work = shard.shard_work(Ns, world)
        assert work.sum() == shard.shard_work(Ns, 1)[0]
        assert work.max() / work.mean() < 1.01, (world, work)
    with pytest.raises(ValueError):
        shard.batch_shard(Ns, 2, 2)


def test_reduce_without_group_is_identity():
    assert shard.reduce_over_ranks(3.25, "max") == 3.25


def test_two_gloo_ranks_split_a_batch(tmp_path, oracle_lib):
    import torch.multiprocessing as mp

    count, p, world = 14, 128, 2
    mp.start_processes(_rank_main, args=(world, _free_port(), count, p, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    t, s = np.load(tmp_path / "reduce.npy")
    assert t == 3.0 and s == 3.0
    Ns, mats = _items(count, p)
    keys = np.load(tmp_path / "keys.npy")
    assert list(keys) == list(range(count))
    for m in range(count):
        zk, D = _eliminate(oracle_lib, *mats[m], int(Ns[m]), p)
        f = np.load(tmp_path / f"m{m}.npz")
        assert int(f["zk"]) == zk
        for a, b in zip((f["s"], f["e"], f["m"]), D):
            assert np.array_equal(a, b), m
