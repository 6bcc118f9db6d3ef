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


# ---------------------------------------------------------------- statistics along a dim

@dataclass
class LocalStats:
    """One rank's statistics over its column block: for every row the
    block's count, sum, sum of squared deviations from the block's row mean
    (M2), min and max; for each of the block's columns its six statistics
    (sum, mean, var, stddev, min, max), which need no exchange."""
    width: int                 # columns in the block
    row_sum: np.ndarray
    row_m2: np.ndarray
    row_min: np.ndarray
    row_max: np.ndarray
    col_stats: np.ndarray      # 6 x width


def _chan(n_a, mean_a, m2_a, n_b, mean_b, m2_b):
    """Merge two sets' (count, mean, M2) (Chan, Golub and LeVeque's pairwise
    update; exact in real arithmetic)."""
    n = n_a + n_b
    delta = mean_b - mean_a
    mean = mean_a + delta * (n_b / n)
    m2 = m2_a + m2_b + delta * delta * (n_a * n_b / n)
    return n, mean, m2


def merge_stats(parts, n_rows: int, norm_type: int = 0) -> dict:
    """Statistics of the whole matrix from its column blocks' LocalStats, in
    block order: rows merge the blocks' (count, mean, M2) (so the result
    does not depend on timing; min / max propagate NaN), columns are
    concatenated."""
    n, mean, m2 = 0, np.zeros(n_rows), np.zeros(n_rows)
    lo, hi = np.full(n_rows, np.inf), np.full(n_rows, -np.inf)
    total = np.zeros(n_rows)
    with np.errstate(invalid="ignore"):
        for p in parts:
            if p.width == 0:
                continue
            if n == 0:
                n, mean, m2 = p.width, p.row_sum / p.width, p.row_m2
            else:
                n, mean, m2 = _chan(n, mean, m2, p.width, p.row_sum / p.width, p.row_m2)
            total = total + p.row_sum
            lo, hi = np.minimum(lo, p.row_min), np.maximum(hi, p.row_max)
    d = n - 1 + norm_type
    with np.errstate(invalid="ignore", divide="ignore"):
        if n == 0:
            var = np.full(n_rows, np.nan)
        elif d == 0:
            var = np.where(np.isfinite(total), 0.0, np.nan)
        else:
            var = np.maximum(m2 / d, 0.0)
    cols = np.concatenate([np.asarray(p.col_stats, dtype=np.float64).reshape(6, p.width) for p in parts], axis=1)
    return {"rows": {"sum": total, "mean": mean if n else np.full(n_rows, np.nan), "var": var,
                     "stddev": np.sqrt(var), "min": lo, "max": hi},
            "cols": dict(zip(("sum", "mean", "var", "stddev", "min", "max"), cols))}


def combine_stats(local: LocalStats, n_rows: int, n_cols: int, norm_type: int = 0, group=None) -> dict:
    """merge_stats over every rank's LocalStats (collective: each rank's
    block is gathered, then merged in rank order on every rank)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    widths = [column_block(n_cols, r, world)[1] - column_block(n_cols, r, world)[0] for r in range(world)]
    width = max(widths)
    mine = torch.zeros(4 * n_rows + 6 * width, dtype=torch.float64)
    rows = np.stack([local.row_sum, local.row_m2, local.row_min, local.row_max]).astype(np.float64)
    mine[:4 * n_rows] = torch.from_numpy(np.ascontiguousarray(rows.ravel()))
    cols = np.zeros((6, width))
    cols[:, :local.width] = np.asarray(local.col_stats, dtype=np.float64).reshape(6, local.width)
    mine[4 * n_rows:] = torch.from_numpy(cols.ravel())
    gathered = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(gathered, mine, group=group)
    parts = []
    for r in range(world):
        g = gathered[r].numpy()
        rs = g[:4 * n_rows].reshape(4, n_rows)
        cs = g[4 * n_rows:].reshape(6, width)[:, :widths[r]]
        parts.append(LocalStats(widths[r], rs[0], rs[1], rs[2], rs[3], cs))
    return merge_stats(parts, n_rows, norm_type)


def gpu_local_stats(tree: bytes, ins, norm_type: int = 0, ws=None) -> LocalStats:
    """A rank's LocalStats on its own GPU block through coot_stats_dim (ins:
    the rank's column blocks as coot Mats on its device)."""
    import torch

    import paper_2308_03120_gb300 as coot
    r, c = ins[0].n_rows, ins[0].n_cols
    rows = [torch.empty(max(r, 1), dtype=torch.float64, device="cuda") for _ in range(4)]
    if r and c:
        # sum, var with divisor N (so M2 = var * N), min, max of each row
        coot.coot_stats_dim(tree, ins, 1, coot.STAT_SUM | coot.STAT_VAR | coot.STAT_MIN | coot.STAT_MAX,
                            [coot.Mat(t, r, 1, r) for t in rows], norm_type=1, ws=ws)
    cols = [torch.empty(max(c, 1), dtype=torch.float64, device="cuda") for _ in range(6)]
    if c and r:
        coot.coot_stats_dim(tree, ins, 0, 0x3F, [coot.Mat(t, 1, c, 1) for t in cols], norm_type=norm_type, ws=ws)
    h = [t.cpu().numpy()[:r] for t in rows]
    col = np.stack([t.cpu().numpy()[:c] for t in cols]) if c else np.zeros((6, 0))
    if not c:
        h = [np.zeros(r), np.zeros(r), np.full(r, np.inf), np.full(r, -np.inf)]
    return LocalStats(c, h[0], h[1] * c, h[2], h[3], col)
