"""Multi-rank combine of the sharded reductions, on CPU: world_size 2 (and
3) gloo processes, each rank holding a column block of the matrix.  The
per-rank results come from the FP64 oracle (the GPU computes them on a real
multi-GPU run); what is tested here is the block split and the exchange.
The combined results must equal the oracle over the whole matrix."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
from oracle import coot_oracle as O
from paper_2308_03120_gb300.shard import LocalResults, column_block, combine


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_local(tree, mats, rank, world):
    c0, c1 = column_block(mats[0].n_cols, rank, world)
    r = mats[0].n_rows
    blk = [synth.as_mat(m.buf[c0 * m.ld:c1 * m.ld].copy(), m.dtype, r, c1 - c0, m.ld) for m in mats]
    n = r * (c1 - c0)
    if n:
        v = O.evaluate(tree, blk)
        lo, hi = O.minmax(tree, blk)
        return LocalResults.from_values(O.accu(tree, blk), O._fsum(v * v), lo, hi, n, O.sum_dim(tree, blk, 0),
                                        O.sum_dim(tree, blk, 1))
    return LocalResults.from_values(0.0, 0.0, math.inf, -math.inf, 0, np.zeros(0), np.zeros(r))


def _worker(rank, world, port, shape, seed, nan_at, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, c = shape
        mats = []
        for k in range(4):
            flat = synth.uniform_f32(seed + k, r * c, 0.0 if k == 3 else -1.0, 2.0 if k == 3 else 1.0)
            if nan_at is not None and k == 0:
                flat[nan_at] = np.nan
            mats.append(synth.as_mat(flat, "f32", r, c))
        tree = O.encode(synth.MAT_EXPR)
        res = combine(_oracle_local(tree, mats, rank, world), c)
        assert all(t.device.type == "cpu" for t in res.values())   # gloo exchanges host tensors
        q.put((rank, {k: (v.item() if v.dim() == 0 else v.numpy()) for k, v in res.items()}))
    finally:
        dist.destroy_process_group()


def _run(world, shape, seed, nan_at=None):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, shape, seed, nan_at, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


@pytest.mark.parametrize("world,shape", [(2, (257, 101)), (3, (64, 7)), (2, (50, 1))])
def test_sharded_reductions_equal_the_whole(world, shape):
    seed = 4321
    out = _run(world, shape, seed)
    r, c = shape
    mats = [synth.as_mat(synth.uniform_f32(seed + k, r * c, 0.0 if k == 3 else -1.0, 2.0 if k == 3 else 1.0),
                         "f32", r, c) for k in range(4)]
    tree = O.encode(synth.MAT_EXPR)
    v = O.evaluate(tree, mats)
    want = {"accu": O.accu(tree, mats), "norm_fro": O.norm(tree, mats, "fro")}
    lo, hi = O.minmax(tree, mats)
    for rank, res in out.items():
        # every rank gets the same answer
        assert res["accu"] == out[0]["accu"] and np.array_equal(res["sum_dim1"], out[0]["sum_dim1"])
        assert res["accu"] == pytest.approx(want["accu"], rel=1e-12, abs=1e-12 * np.sum(np.abs(v)))
        assert res["norm_fro"] == pytest.approx(want["norm_fro"], rel=1e-12)
        assert (res["min"], res["max"]) == (lo, hi)
        assert res["sum_dim0"].shape == (c,)
        assert np.array_equal(res["sum_dim0"], O.sum_dim(tree, mats, 0))   # whole columns: exact
        np.testing.assert_allclose(res["sum_dim1"], O.sum_dim(tree, mats, 1), rtol=1e-12,
                                   atol=1e-12 * np.max(np.sum(np.abs(v), axis=1)))


def test_nan_on_one_rank_reaches_every_rank():
    out = _run(2, (40, 10), 99, nan_at=7 * 40 + 3)   # a NaN in the last block
    for res in out.values():
        assert math.isnan(res["min"]) and math.isnan(res["max"]) and math.isnan(res["accu"])


def test_column_blocks_cover_every_column_once():
    for n in (0, 1, 7, 100):
        for world in (1, 2, 3, 8):
            blocks = [column_block(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
            widths = [b - a for a, b in blocks]
            assert max(widths) - min(widths) <= 1


# ---------------------------------------------------------------- sharded statistics

def _oracle_local_stats(tree, mats, rank, world, norm_type):
    from paper_2308_03120_gb300.shard import LocalStats
    c0, c1 = column_block(mats[0].n_cols, rank, world)
    r, w = mats[0].n_rows, c1 - c0
    blk = [synth.as_mat(m.buf[c0 * m.ld:c1 * m.ld].copy(), m.dtype, r, w, m.ld) for m in mats]
    if w == 0:
        return LocalStats.from_values(0, np.zeros(r), np.zeros(r), np.full(r, np.inf), np.full(r, -np.inf),
                                      np.zeros((6, 0)))
    st = lambda dim, s, nt=0: O.stats_dim(tree, blk, dim, s, nt)  # noqa: E731
    cols = np.stack([st(0, s, norm_type) for s in O.STATS])
    return LocalStats.from_values(w, st(1, "sum"), st(1, "var", 1) * w, st(1, "min"), st(1, "max"), cols)


def _stats_worker(rank, world, port, shape, seed, norm_type, q):
    import torch.distributed as dist
    from paper_2308_03120_gb300.shard import combine_stats
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, c = shape
        mats = [synth.as_mat(synth.uniform_f32(seed + k, r * c, 0.0 if k == 3 else -1.0, 2.0 if k == 3 else 1.0),
                             "f32", r, c) for k in range(4)]
        tree = O.encode(synth.MAT_EXPR)
        res = combine_stats(_oracle_local_stats(tree, mats, rank, world, norm_type), r, c, norm_type)
        q.put((rank, {part: {k: v.numpy() for k, v in res[part].items()} for part in ("rows", "cols")}))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,shape,norm_type", [(2, (67, 101), 0), (3, (40, 8), 1), (3, (9, 2), 0)])
def test_sharded_statistics_equal_the_whole(world, shape, norm_type):
    """Row statistics merge the ranks' (count, mean, M2) in rank order;
    column statistics are gathered.  Against the oracle over the whole
    matrix."""
    seed = 2468
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_stats_worker, args=(r, world, port, shape, seed, norm_type, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    r, c = shape
    mats = [synth.as_mat(synth.uniform_f32(seed + k, r * c, 0.0 if k == 3 else -1.0, 2.0 if k == 3 else 1.0),
                         "f32", r, c) for k in range(4)]
    tree = O.encode(synth.MAT_EXPR)
    for rank, res in out.items():
        for s in O.STATS:
            want_rows = O.stats_dim(tree, mats, 1, s, norm_type)
            np.testing.assert_allclose(res["rows"][s], want_rows, rtol=1e-12, atol=1e-13, err_msg=s)
            assert np.array_equal(res["cols"][s], O.stats_dim(tree, mats, 0, s, norm_type)), s
            assert np.array_equal(res["rows"][s], out[0]["rows"][s])      # every rank agrees
