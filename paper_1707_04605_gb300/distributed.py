"""Multi-GPU use of the path: one process per GPU, shots sharded.

Shots are independent given (mesh, eps, dt), so the forward and the tangent
shard with no exchange; the gradient J^T w is a sum over shots, so each
rank's per-cell gradient is summed across ranks with one all-reduce of
(cells of the level) doubles.
"""
from __future__ import annotations

import numpy as np

from .api import Shots


def shard(shots, rank: int, world: int) -> tuple[Shots, np.ndarray]:
    """Round-robin shard of a shot batch: shots rank, rank+world, ...
    Returns the rank's Shots and the indices of its shots in the batch."""
    sh = Shots.of(shots)
    idx = np.arange(rank, sh.n_shots, world, dtype=np.int64)
    recs = [sh.rec[sh.rec_ptr[i]:sh.rec_ptr[i + 1]] for i in idx]
    ptr = np.concatenate([[0], np.cumsum([len(r) for r in recs])]).astype(np.int64)
    rec = np.concatenate(recs).astype(np.int32) if recs else np.zeros(0, np.int32)
    return Shots(sh.src[idx], ptr, rec), idx


def trace_rows(shots, idx) -> np.ndarray:
    """Rows of the full batch's trace array that belong to shots idx."""
    sh = Shots.of(shots)
    return np.concatenate([np.arange(sh.rec_ptr[i], sh.rec_ptr[i + 1]) for i in idx]
                          ).astype(np.int64) if len(idx) else np.zeros(0, np.int64)


def gradient_allreduce(g, group=None):
    """Sum a rank's per-cell gradient over all ranks, in place (torch tensor;
    CPU with gloo, CUDA with NCCL)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return g
