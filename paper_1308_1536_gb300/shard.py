"""Host logic for one process per GPU on one node.

The method's work comes in independent problems (whole factorisations, the
matrices of a batch), so several GPUs need no exchange on the data path: a
batch is split across ranks, each rank factors its share in its own
persistent launch, and the only collectives are the benchmark's timing
reduction and the gathering of results on rank 0.  (A single factorisation
too large for one GPU would need the paper's row-cyclic pivot-row broadcast
(Sec. 4.2); that path is not built.)
"""
from __future__ import annotations

import numpy as np


def batch_shard(Ns, rank: int, world: int) -> np.ndarray:
    """Indices of the batch matrices that ``rank`` of ``world`` owns.

    The matrices are ordered by decreasing N (stable) and dealt in snake
    order (0, 1, ..., world-1, world-1, ..., 0, ...), which balances the
    O(N^3) work of uneven sizes; every matrix has exactly one owner.  The
    returned indices are ascending."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of world {world}")
    Ns = np.asarray(Ns, dtype=np.int64)
    order = np.argsort(-Ns, kind="stable")
    pos = np.arange(len(order))
    lap, r = np.divmod(pos, world)
    owner = np.where(lap % 2 == 0, r, world - 1 - r)
    return np.sort(order[owner == rank])


def shard_work(Ns, world: int) -> np.ndarray:
    """Products of Gaussian elimination (sum over steps of (N-k-1)^2 + (N-k-1)
    + 1) per rank under ``batch_shard``."""
    Ns = np.asarray(Ns, dtype=np.int64)
    w = (Ns - 1) * Ns * (2 * Ns - 1) // 6 + Ns * (Ns - 1) // 2 + (Ns - 1)
    return np.array([int(w[batch_shard(Ns, r, world)].sum()) for r in range(world)], dtype=np.int64)


def reduce_over_ranks(value: float, op: str = "max", device=None) -> float:
    """All-reduce one float over the default process group (max or sum);
    the value itself when no group is initialised.  ``device``: where the
    reduction tensor lives (a CUDA device for NCCL, None = CPU for gloo)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())
