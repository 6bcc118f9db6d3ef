"""Column-block sharding of the fused reductions across ranks.

Element-wise evaluation needs no exchange.  With a column-major matrix cut
into blocks of whole columns, one block per rank:
  * sum(A, 0) of each block is that block's slice of the result, so the
    column sums only need gathering;
  * accu, the sum of squares behind norm2 / "fro", and min / max need one
    all-reduce of an FP64 scalar per result (sum, sum, min, max);
  * sum(A, 1) needs one all-reduce (sum) of an n_rows FP64 vector.

`local` computes a rank's results on its block (on the GPU through the coot
calls, see `gpu_local`); `combine` does the exchange with torch.distributed
(any backend: NCCL between GPUs, gloo between CPU processes).  Partial sums
cross ranks in FP64, and an all-reduce adds them in an order fixed by the
backend's algorithm for a given world size.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def column_block(n_cols: int, rank: int, world: int) -> tuple[int, int]:
    """[first, last) columns of rank's block: contiguous, sizes differing by
    at most one."""
    base, extra = divmod(n_cols, world)
    first = rank * base + min(rank, extra)
    return first, first + base + (1 if rank < extra else 0)


@dataclass
class LocalResults:
    """One rank's reductions over its column block."""
    accu: float
    sumsq: float
    min: float
    max: float
    count: int              # elements in the block
    col_sums: np.ndarray    # sum(block, 0): one per column of the block
    row_sums: np.ndarray    # sum(block, 1): one per row (n_rows)


def combine(local: LocalResults, n_cols: int, group=None) -> dict:
    """Global results from every rank's LocalResults (collective: every rank
    of `group` must call it)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    s = torch.tensor([local.accu, local.sumsq], dtype=torch.float64)
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    # an empty block contributes the neutral elements of min and max
    lo = torch.tensor([local.min if local.count else np.inf], dtype=torch.float64)
    hi = torch.tensor([local.max if local.count else -np.inf], dtype=torch.float64)
    dist.all_reduce(lo, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(hi, op=dist.ReduceOp.MAX, group=group)
    nan = torch.tensor([1.0 if (np.isnan(local.min) or np.isnan(local.max)) and local.count else 0.0],
                       dtype=torch.float64)
    dist.all_reduce(nan, op=dist.ReduceOp.MAX, group=group)
    rows = torch.from_numpy(np.ascontiguousarray(local.row_sums, dtype=np.float64))
    dist.all_reduce(rows, op=dist.ReduceOp.SUM, group=group)
    # column sums: blocks have different widths, so pad to the widest
    width = max(column_block(n_cols, r, world)[1] - column_block(n_cols, r, world)[0] for r in range(world))
    mine = torch.zeros(width, dtype=torch.float64)
    mine[:local.col_sums.size] = torch.from_numpy(np.asarray(local.col_sums, dtype=np.float64))
    parts = [torch.zeros(width, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    cols = np.concatenate([parts[r].numpy()[:column_block(n_cols, r, world)[1] - column_block(n_cols, r, world)[0]]
                           for r in range(world)])
    has_nan = nan.item() > 0
    return {"accu": s[0].item(), "norm_fro": float(np.sqrt(s[1].item())),
            "min": float("nan") if has_nan else lo.item(), "max": float("nan") if has_nan else hi.item(),
            "sum_dim0": cols, "sum_dim1": rows.numpy()}


def gpu_local(tree: bytes, ins, ws=None) -> LocalResults:
    """A rank's LocalResults on its own GPU block through the coot calls
    (ins: the rank's column blocks as coot Mats on its device)."""
    import torch

    import paper_2308_03120_gb300 as coot
    r, c = ins[0].n_rows, ins[0].n_cols
    n = r * c
    heads = coot.HEAD_SUM | coot.HEAD_SUMSQ | coot.HEAD_MIN | coot.HEAD_MAX
    if n:
        res = coot.coot_expr_reduce(tree, ins, heads, ws=ws).cpu().numpy()
    else:
        res = np.array([0.0, 0.0, np.inf, -np.inf])
    col = torch.empty(max(c, 1), dtype=torch.float64, device="cuda")
    row = torch.empty(max(r, 1), dtype=torch.float64, device="cuda")
    if c:
        coot.coot_sum_dim(tree, ins, 0, coot.Mat(col, 1, c, 1), ws=ws)
    if r:
        coot.coot_sum_dim(tree, ins, 1, coot.Mat(row, r, 1, r), ws=ws)
    return LocalResults(float(res[0]), float(res[1]), float(res[2]), float(res[3]), n,
                        col.cpu().numpy()[:c], row.cpu().numpy()[:r] if c else np.zeros(r))
