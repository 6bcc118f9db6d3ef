"""Exhaustive launch-shape tuning.

For one call (a closure that issues coot calls on the current stream) and
one kernel kind, every launch shape of a grid is set with
coot_set_launch_config, compiled on first use, and timed with CUDA events
(median over repetitions, inputs larger than L2 or an L2 flush between
repetitions when asked).  The fastest shape is the tuner's answer; the
whole table is the data the learned launch-shape model trains on.

    python -m paper_2308_03120_gb300.tune            # the matrix workload's four calls
    python -m paper_2308_03120_gb300.tune stats      # per-dim statistics
    python -m paper_2308_03120_gb300.tune batched    # batched evaluation
"""
from __future__ import annotations

import itertools
import json
import statistics
import sys

from . import (KIND_BATCHED, KIND_COLSTATS, KIND_COLSUM, KIND_MAP, KIND_MULTI, KIND_REDUCE,  # noqa: F401
               KIND_ROWSTATS, KIND_ROWSUM)

GRIDS = {
    KIND_MAP: dict(block=[128, 256, 512], vec=[0, 2, 1], unroll=[1, 2, 4, 8], blocks_per_sm=[0], split=[0]),
    KIND_REDUCE: dict(block=[128, 256, 512], vec=[0, 2, 1], unroll=[1, 2, 4, 8, 16], blocks_per_sm=[0], split=[0]),
    KIND_COLSUM: dict(block=[128, 256, 512], vec=[0], unroll=[1, 2, 4, 8], blocks_per_sm=[0], split=[0, 1, 2, 4]),
    KIND_ROWSUM: dict(block=[64, 128, 256, 512], vec=[0], unroll=[2, 4, 8, 16], blocks_per_sm=[0],
                      split=[0, 8, 16, 32, 64]),
    KIND_BATCHED: dict(block=[128, 256, 512], vec=[0], unroll=[1, 2, 4, 8], blocks_per_sm=[0, 2, 4], split=[0]),
    KIND_COLSTATS: dict(block=[128, 256, 512], vec=[0, 2], unroll=[2, 4, 8], blocks_per_sm=[0], split=[0, 1, 2, 4]),
    KIND_ROWSTATS: dict(block=[64, 128, 256], vec=[0, 2, 1], unroll=[2, 4, 8], blocks_per_sm=[0],
                        split=[0, 8, 16, 32]),
    KIND_MULTI: dict(block=[128, 256, 512], vec=[0, 2, 1], unroll=[1, 2, 4, 8], blocks_per_sm=[0], split=[0]),
}


def configs(kind: int, grid: dict | None = None):
    g = grid or GRIDS[kind]
    keys = ["block", "vec", "unroll", "blocks_per_sm", "split"]
    for vals in itertools.product(*(g[k] for k in keys)):
        yield dict(zip(keys, vals))


def time_call(fn, reps: int = 10, warmup: int = 2, flush=None) -> float:
    """Median device time of fn() in milliseconds (CUDA events on the
    current stream)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        if flush is not None:
            flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def sweep(fn, kind: int, grid: dict | None = None, reps: int = 10, flush=None):
    """Time fn under every launch shape of the grid for `kind`; returns
    [(ms, config, launch actually used)] sorted by time.  The built-in
    choice is timed too (config None)."""
    import paper_2308_03120_gb300 as coot
    out = []
    try:
        coot.coot_set_launch_config(kind, 0)
        ms = time_call(fn, reps, flush=flush)
        out.append((ms, None, coot.coot_last_launch()))
        for cfg in configs(kind, grid):
            coot.coot_set_launch_config(kind, **cfg)
            ms = time_call(fn, reps, flush=flush)
            out.append((ms, cfg, coot.coot_last_launch()))
    finally:
        coot.coot_set_launch_config(kind, 0)
    return sorted(out, key=lambda r: r[0])


def _matrix_workload(n: int = 8192):
    import torch

    import paper_2308_03120_gb300 as coot
    import synth
    seed = synth.BASE_SEED + 1
    dev = [torch.from_numpy(synth.uniform_f32(seed + k, n * n, 0.0 if k == 3 else -1.0, 2.0 if k == 3 else 1.0))
           .cuda() for k in range(4)]
    mats = [coot.Mat(t, n, n, n) for t in dev]
    out1 = torch.empty(n * n, device="cuda")
    out2 = torch.empty(n * n, device="cuda")
    col = torch.empty(n, device="cuda")
    row = torch.empty(n, device="cuda")
    res = torch.empty(4, dtype=torch.float64, device="cuda")
    ws = coot.Workspace(n)
    t_expr = coot.serialize(synth.MAT_EXPR)
    t_chain = coot.serialize(synth.MAT_CHAIN)
    leaf = coot.serialize(synth.LEAF0)
    heads = coot.HEAD_SUM | coot.HEAD_NORM2 | coot.HEAD_MIN | coot.HEAD_MAX
    O1 = coot.Mat(out1, n, n, n)
    return {
        "expr_reduce": (KIND_MAP, 5 * n * n * 4,
                        lambda: coot.coot_expr_reduce(t_expr, mats, heads, out=O1, out_dev=res, ws=ws)),
        "expr_eval": (KIND_MAP, 5 * n * n * 4, lambda: coot.coot_expr_eval(t_chain, mats, coot.Mat(out2, n, n, n))),
        "sum_dim0": (KIND_COLSUM, n * n * 4, lambda: coot.coot_sum_dim(leaf, [O1], 0, coot.Mat(col, 1, n, 1), ws=ws)),
        "sum_dim1": (KIND_ROWSUM, n * n * 4, lambda: coot.coot_sum_dim(leaf, [O1], 1, coot.Mat(row, n, 1, n), ws=ws)),
    }


def _batched_workload(nmat: int = 4096):
    import numpy as np
    import torch

    import paper_2308_03120_gb300 as coot
    import synth
    rows = synth.loguniform_int(synth.BASE_SEED + 3, nmat, 1, 512)
    cols = synth.loguniform_int(synth.BASE_SEED + 4, nmat, 1, 512)
    sizes = (rows * cols).astype(np.int64)
    offs = np.zeros(nmat + 1, dtype=np.int64)
    offs[1:] = np.cumsum((sizes + 3) // 4 * 4)
    coff = np.zeros(nmat + 1, dtype=np.int64)
    coff[1:] = np.cumsum((cols + 3) // 4 * 4)
    bufs = [torch.from_numpy(synth.uniform_f32(synth.BASE_SEED + 10 + k, int(offs[-1]))).cuda() for k in range(3)]
    out = torch.empty(int(offs[-1]), device="cuda")
    csum = torch.empty(int(coff[-1]), device="cuda")
    items = []
    for m in range(nmat):
        r, c, o = int(rows[m]), int(cols[m]), int(offs[m])
        items.append(coot.batch_item([coot.Mat(b, r, c, r, o) for b in bufs], coot.Mat(out, r, c, r, o),
                                     coot.Mat(csum, 1, c, 1, int(coff[m]))))
    plan, n_items, n_work = coot.coot_batch_plan(items, 3)
    tree = coot.serialize(synth.BATCH_EXPR)
    nbytes = int(sizes.sum()) * 16 + int(cols.sum()) * 4
    return {"batched": (KIND_BATCHED, nbytes,
                        lambda: coot.coot_expr_eval_batched(tree, [0, 0, 0], 0, 0, plan, n_items, n_work))}


def _stats_workload(n: int = 8192):
    """All six statistics of each column / row, of a stored matrix (one
    input) and of the four-input matrix tree."""
    import torch

    import paper_2308_03120_gb300 as coot
    import synth
    seed = synth.BASE_SEED + 1
    dev = [torch.from_numpy(synth.uniform_f32(seed + k, n * n, 0.0 if k == 3 else -1.0, 2.0 if k == 3 else 1.0))
           .cuda() for k in range(4)]
    mats = [coot.Mat(t, n, n, n) for t in dev]
    ws = coot.Workspace(n)
    outs = {0: [coot.Mat(torch.empty(n, device="cuda"), 1, n, 1) for _ in range(6)],
            1: [coot.Mat(torch.empty(n, device="cuda"), n, 1, n) for _ in range(6)]}
    calls = {}
    for name, sexpr, ins in (("leaf", synth.LEAF0, mats[:1]), ("tree", synth.MAT_EXPR, mats)):
        tree = coot.serialize(sexpr)
        for dim in (0, 1):
            calls[f"{name}_dim{dim}"] = (KIND_COLSTATS if dim == 0 else KIND_ROWSTATS, len(ins) * n * n * 4,
                                         lambda t=tree, i=ins, d=dim: coot.coot_stats_dim(t, i, d, 0x3F, outs[d],
                                                                                          ws=ws))
    return calls


def _precision_workload(n: int = 1 << 28):
    """The precision workload's calls on BF16 and FP16 vectors of 2^28
    (signed lognormal values): accu + norm2 of x in one pass and dot(x, z)."""
    import numpy as np
    import torch

    import paper_2308_03120_gb300 as coot
    import synth
    ws = coot.Workspace(1)
    res = torch.empty(3, dtype=torch.float64, device="cuda")
    leaf = coot.serialize(synth.LEAF0)
    calls = {}
    for dt, tdt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        hx, _ = synth.lognormal_signed(synth.BASE_SEED + 2, n, dt)
        hz, _ = synth.lognormal_signed(synth.BASE_SEED + 3, n, dt)
        x = torch.from_numpy(hx.view(np.int16)).view(tdt).cuda()
        z = torch.from_numpy(hz.view(np.int16)).view(tdt).cuda()
        X, Z = coot.Mat(x, n, 1, n), coot.Mat(z, n, 1, n)
        calls[f"{dt}_accu_norm2"] = (KIND_REDUCE, 2 * n, lambda X=X: coot.coot_expr_reduce(
            leaf, [X], coot.HEAD_SUM | coot.HEAD_NORM2, out_dev=res[0:2], ws=ws))
        calls[f"{dt}_dot"] = (KIND_REDUCE, 4 * n, lambda X=X, Z=Z: coot.coot_dot(X, Z, out_dev=res[2:3], ws=ws))
    return calls


def main(argv=None):
    import paper_2308_03120_gb300 as coot
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    which = argv[0] if argv else "matrices"
    calls = {"batched": _batched_workload, "stats": _stats_workload,
             "precision": _precision_workload}.get(which, _matrix_workload)()
    report = {}
    for name, (kind, nbytes, fn) in calls.items():
        fn()
        res = sweep(fn, kind, reps=8)
        base = next(r for r in res if r[1] is None)
        best = res[0]
        report[name] = {"builtin_ms": round(base[0], 4), "builtin_gbs": round(nbytes / base[0] / 1e6, 1),
                        "builtin": base[2], "best_ms": round(best[0], 4), "best_gbs": round(nbytes / best[0] / 1e6, 1),
                        "best": best[1], "best_launch": best[2],
                        "top5": [(round(r[0], 4), r[1]) for r in res[:5]]}
        print(name, json.dumps(report[name]), flush=True)
    return report


if __name__ == "__main__":
    main(sys.argv[1:])
