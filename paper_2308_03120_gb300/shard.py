"""Column-block sharding of the fused reductions across ranks.

Element-wise evaluation needs no exchange.  With a column-major matrix cut
into blocks of whole columns, one block per rank:
  * sum(A, 0) of each block is that block's slice of the result, so the
    column sums only need gathering;
  * accu, the sum of squares behind norm2 / "fro", and min / max need one
    all-reduce of an FP64 scalar per result (sum, sum, min, max);
  * sum(A, 1) needs one all-reduce (sum) of an n_rows FP64 vector.

Every partial is an FP64 torch tensor and stays on the device that the
group's backend exchanges: the rank's GPU for NCCL (tested on one GPU as a
world-size-1 group; multi-GPU NCCL runs are unmeasured on hardware here),
the host for gloo (tested with world sizes 2 and 3).  `gpu_local` computes a
rank's partials through the coot calls and leaves them on its GPU;
`combine` moves them to the exchange device (a no-op when they are there
already) and does the exchange with torch.distributed.  An all-reduce adds
the partials in an order fixed by the backend's algorithm for a given world
size.
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


def exchange_device(group=None):
    """The device whose tensors the group's collectives take: the current
    GPU for NCCL, the host otherwise."""
    import torch
    import torch.distributed as dist
    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


@dataclass
class LocalResults:
    """One rank's reductions over its column block, as FP64 tensors on one
    device."""
    heads: object      # [accu, sum of squares, min, max]; an empty block holds 0, 0, +inf, -inf
    count: int         # elements in the block
    col_sums: object   # sum(block, 0): one per column of the block
    row_sums: object   # sum(block, 1): one per row (n_rows)

    @staticmethod
    def from_values(accu, sumsq, mn, mx, count, col_sums, row_sums, device="cpu") -> "LocalResults":
        """LocalResults from host numbers and arrays."""
        import torch
        t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device=device)  # noqa: E731
        return LocalResults(t([accu, sumsq, mn, mx]), int(count), t(col_sums), t(row_sums))


def combine(local: LocalResults, n_cols: int, group=None) -> dict:
    """Global results from every rank's LocalResults (collective: every rank
    of `group` must call it).  Returns FP64 tensors on the exchange device:
    accu, norm_fro, min, max (0-d) and sum_dim0, sum_dim1."""
    import torch
    import torch.distributed as dist
    dev = exchange_device(group)
    world = dist.get_world_size(group)
    h = local.heads.to(dev, torch.float64)
    s = h[0:2].clone()
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    # an empty block contributes the neutral elements of min and max; a NaN
    # travels as a flag (collectives' min / max need not propagate it)
    has = local.count > 0
    inf = torch.tensor([float("inf")], dtype=torch.float64, device=dev)
    lo = h[2:3].clone() if has else inf.clone()
    hi = h[3:4].clone() if has else -inf
    nan = (torch.isnan(h[2:3]) | torch.isnan(h[3:4])).to(torch.float64) if has else torch.zeros_like(inf)
    lo = torch.nan_to_num(lo, nan=float("inf"))
    hi = torch.nan_to_num(hi, nan=float("-inf"))
    dist.all_reduce(lo, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(hi, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(nan, op=dist.ReduceOp.MAX, group=group)
    rows = local.row_sums.to(dev, torch.float64).contiguous().clone()
    dist.all_reduce(rows, op=dist.ReduceOp.SUM, group=group)
    # column sums: blocks have different widths, so pad to the widest
    widths = [column_block(n_cols, r, world)[1] - column_block(n_cols, r, world)[0] for r in range(world)]
    width = max(widths)
    mine = torch.zeros(width, dtype=torch.float64, device=dev)
    mine[:local.col_sums.numel()] = local.col_sums.to(dev, torch.float64)
    parts = [torch.zeros(width, dtype=torch.float64, device=dev) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    cols = torch.cat([parts[r][:widths[r]] for r in range(world)])
    flag = nan[0] > 0
    nan0 = torch.tensor(float("nan"), dtype=torch.float64, device=dev)
    return {"accu": s[0], "norm_fro": torch.sqrt(s[1]),
            "min": torch.where(flag, nan0, lo[0]), "max": torch.where(flag, nan0, hi[0]),
            "sum_dim0": cols, "sum_dim1": rows}


def gpu_local(tree: bytes, ins, ws=None) -> LocalResults:
    """A rank's LocalResults on its own GPU block through the coot calls
    (ins: the rank's column blocks as coot Mats on its device); the partials
    stay on that device."""
    import torch

    import paper_2308_03120_gb300 as coot
    r, c = ins[0].n_rows, ins[0].n_cols
    n = r * c
    heads = coot.HEAD_SUM | coot.HEAD_SUMSQ | coot.HEAD_MIN | coot.HEAD_MAX
    if n:
        res = coot.coot_expr_reduce(tree, ins, heads, ws=ws)
    else:
        res = torch.tensor([0.0, 0.0, float("inf"), float("-inf")], dtype=torch.float64, device="cuda")
    col = torch.zeros(max(c, 1), dtype=torch.float64, device="cuda")
    row = torch.zeros(max(r, 1), dtype=torch.float64, device="cuda")
    if n:
        coot.coot_sum_dim(tree, ins, 0, coot.Mat(col, 1, c, 1), ws=ws)
        coot.coot_sum_dim(tree, ins, 1, coot.Mat(row, r, 1, r), ws=ws)
    return LocalResults(res, n, col[:c], row[:r])


# ---------------------------------------------------------------- statistics along a dim

@dataclass
class LocalStats:
    """One rank's statistics over its column block, FP64 tensors on one
    device: for every row the block's sum, sum of squared deviations from
    the block's row mean (M2), min and max; for each of the block's columns
    its six statistics (sum, mean, var, stddev, min, max), which need no
    exchange."""
    width: int          # columns in the block
    row_sum: object
    row_m2: object
    row_min: object
    row_max: object
    col_stats: object   # 6 x width

    @staticmethod
    def from_values(width, row_sum, row_m2, row_min, row_max, col_stats, device="cpu") -> "LocalStats":
        import torch
        t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device=device)  # noqa: E731
        return LocalStats(int(width), t(row_sum), t(row_m2), t(row_min), t(row_max),
                          t(np.asarray(col_stats, dtype=np.float64).reshape(6, int(width))))


def merge_stats(parts, n_rows: int, norm_type: int = 0) -> dict:
    """Statistics of the whole matrix from its column blocks' LocalStats, in
    block order, on the blocks' device: rows merge the blocks' (count, mean,
    M2) with the pairwise update of Chan, Golub and LeVeque
    (mean = mean_a + d n_b / n, M2 = M2_a + M2_b + d^2 n_a n_b / n, d the
    difference of the means), so the result does not depend on timing
    (min / max propagate NaN); columns are concatenated."""
    import torch
    dev = parts[0].row_sum.device if parts else torch.device("cpu")
    f = dict(dtype=torch.float64, device=dev)
    n = 0
    mean, m2 = torch.zeros(n_rows, **f), torch.zeros(n_rows, **f)
    lo, hi = torch.full((n_rows,), float("inf"), **f), torch.full((n_rows,), float("-inf"), **f)
    total = torch.zeros(n_rows, **f)
    for p in parts:
        if p.width == 0:
            continue
        mean_b = p.row_sum / p.width
        if n == 0:
            n, mean, m2 = p.width, mean_b, p.row_m2.clone()
        else:
            nn = n + p.width
            d = mean_b - mean
            mean = mean + d * (p.width / nn)
            m2 = m2 + p.row_m2 + d * d * (n * p.width / nn)
            n = nn
        total = total + p.row_sum
        lo = torch.where(torch.isnan(lo) | torch.isnan(p.row_min), torch.full_like(lo, float("nan")),
                         torch.minimum(lo, p.row_min))
        hi = torch.where(torch.isnan(hi) | torch.isnan(p.row_max), torch.full_like(hi, float("nan")),
                         torch.maximum(hi, p.row_max))
    dd = n - 1 + norm_type
    if n == 0:
        var = torch.full((n_rows,), float("nan"), **f)
    elif dd == 0:
        var = torch.where(torch.isfinite(total), torch.zeros_like(total), torch.full_like(total, float("nan")))
    else:
        var = torch.clamp(m2 / dd, min=0.0)
    cols = torch.cat([p.col_stats.reshape(6, p.width) for p in parts], dim=1) if parts else torch.zeros(6, 0, **f)
    return {"rows": {"sum": total, "mean": mean if n else torch.full((n_rows,), float("nan"), **f), "var": var,
                     "stddev": torch.sqrt(var), "min": lo, "max": hi},
            "cols": dict(zip(("sum", "mean", "var", "stddev", "min", "max"), cols))}


def combine_stats(local: LocalStats, n_rows: int, n_cols: int, norm_type: int = 0, group=None) -> dict:
    """merge_stats over every rank's LocalStats (collective: each rank's
    block is gathered on the exchange device, then merged in rank order on
    every rank)."""
    import torch
    import torch.distributed as dist
    dev = exchange_device(group)
    world = dist.get_world_size(group)
    widths = [column_block(n_cols, r, world)[1] - column_block(n_cols, r, world)[0] for r in range(world)]
    width = max(widths)
    mine = torch.zeros(4 * n_rows + 6 * width, dtype=torch.float64, device=dev)
    rows = torch.stack([local.row_sum, local.row_m2, local.row_min, local.row_max]).to(dev, torch.float64)
    mine[:4 * n_rows] = rows.reshape(-1)
    cols = torch.zeros(6, width, dtype=torch.float64, device=dev)
    cols[:, :local.width] = local.col_stats.to(dev, torch.float64).reshape(6, local.width)
    mine[4 * n_rows:] = cols.reshape(-1)
    gathered = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(gathered, mine, group=group)
    parts = []
    for r in range(world):
        g = gathered[r]
        rs = g[:4 * n_rows].reshape(4, n_rows)
        cs = g[4 * n_rows:].reshape(6, width)[:, :widths[r]]
        parts.append(LocalStats(widths[r], rs[0], rs[1], rs[2], rs[3], cs))
    return merge_stats(parts, n_rows, norm_type)


def gpu_local_stats(tree: bytes, ins, norm_type: int = 0, ws=None) -> LocalStats:
    """A rank's LocalStats on its own GPU block through coot_stats_dim (ins:
    the rank's column blocks as coot Mats on its device); the partials stay
    on that device."""
    import torch

    import paper_2308_03120_gb300 as coot
    r, c = ins[0].n_rows, ins[0].n_cols
    f = dict(dtype=torch.float64, device="cuda")
    if not (r and c):
        return LocalStats(c, torch.zeros(r, **f), torch.zeros(r, **f), torch.full((r,), float("inf"), **f),
                          torch.full((r,), float("-inf"), **f), torch.zeros(6, c, **f))
    rows = [torch.empty(r, **f) for _ in range(4)]
    # sum, var with divisor N (so M2 = var * N), min, max of each row
    coot.coot_stats_dim(tree, ins, 1, coot.STAT_SUM | coot.STAT_VAR | coot.STAT_MIN | coot.STAT_MAX,
                        [coot.Mat(t, r, 1, r) for t in rows], norm_type=1, ws=ws)
    cols = torch.empty(6, c, **f)
    coot.coot_stats_dim(tree, ins, 0, 0x3F, [coot.Mat(cols[k], 1, c, 1) for k in range(6)], norm_type=norm_type,
                        ws=ws)
    return LocalStats(c, rows[0], rows[1] * c, rows[2], rows[3], cols)
