"""GPU parity of the batched evaluation (many small matrices of uneven
shapes in one launch) against the FP64 oracle, matrix by matrix."""
import math

import numpy as np
import pytest
import torch

import paper_2308_03120_gb300 as coot
import synth
from oracle import coot_oracle as O
from paper_2308_03120_gb300.expr import serialize
from tests.gpu_util import check_elementwise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    yield
    torch.cuda.synchronize()


def make_batch(shapes, seed, n_in=3, sum64=False, ld_pad=0):
    """Per matrix: n_in inputs (uniform [-1, 1]), an output and column sums,
    all packed in shared device buffers (the layout a Cube-like container
    would use)."""
    hosts, items, outs, sums = [], [], [], []
    bufs = []
    for k, (r, c) in enumerate(shapes):
        ld = r + ld_pad if r else 1
        ins = [synth.as_mat(synth.uniform_f32(seed + 7 * k + s, r * c), "f32", r, c, ld) for s in range(n_in)]
        hosts.append(ins)
        dev = [coot.Mat(torch.from_numpy(h.buf).cuda(), r, c, ld) for h in ins]
        out = torch.full((max(ld * c, 1),), float("nan"), device="cuda")
        cs = torch.full((max(c, 1),), float("nan"), dtype=torch.float64 if sum64 else torch.float32, device="cuda")
        bufs.append((dev, out, cs))
        items.append(coot.batch_item(dev, coot.Mat(out, r, c, ld), coot.Mat(cs, 1, c, 1)))
        outs.append(out)
        sums.append(cs)
    return hosts, items, outs, sums, bufs


def check_batch(tree, shapes, hosts, outs, sums, n_in):
    for k, (r, c) in enumerate(shapes):
        if r * c == 0:
            if c:
                assert np.all(sums[k].cpu().numpy()[:c] == 0.0)
            continue
        ld = hosts[k][0].ld
        got = synth.HostMat(outs[k].cpu().numpy()[:ld * c], "f32", r, c, ld)
        check_elementwise(tree, hosts[k], got)
        v, bound, _ = O.error_bound(tree, hosts[k])
        want = O.sum_dim(tree, hosts[k], 0)
        gs = sums[k].cpu().numpy()[:c].astype(np.float64)
        tol = 1e-6 * np.abs(want) + 6.0 * np.sqrt(np.sum(bound * bound, axis=0)) + 1e-9 * np.sum(np.abs(v), axis=0)
        tol += np.abs(want) * 2.0 ** -24
        assert np.all(np.abs(gs - want) <= tol), (k, r, c)


def test_batch_of_uneven_matrices():
    n = 300
    rows = synth.loguniform_int(11, n, 1, 512)
    cols = synth.loguniform_int(12, n, 1, 512)
    shapes = list(zip(rows.tolist(), cols.tolist()))
    tree = serialize(synth.BATCH_EXPR)
    hosts, items, outs, sums, bufs = make_batch(shapes, 100, 3)
    plan, n_items, n_work = coot.coot_batch_plan(items, 3)
    coot.coot_expr_eval_batched(tree, [0, 0, 0], 0, 0, plan, n_items, n_work)
    torch.cuda.synchronize()
    check_batch(tree, shapes, hosts, outs, sums, 3)


@pytest.mark.parametrize("shapes", [
    [(1, 1), (31, 2), (32, 3), (33, 4), (0, 5), (7, 0), (512, 512), (2, 100), (16, 33)],
    [(r, 1 + r % 7) for r in range(1, 70)],
])
def test_edge_shapes(shapes):
    tree = serialize(synth.BATCH_EXPR)
    hosts, items, outs, sums, bufs = make_batch(shapes, 7, 3)
    plan, n_items, n_work = coot.coot_batch_plan(items, 3)
    coot.coot_expr_eval_batched(tree, [0, 0, 0], 0, 0, plan, n_items, n_work)
    torch.cuda.synchronize()
    check_batch(tree, shapes, hosts, outs, sums, 3)


def test_fp64_sums_ld_and_graph_replay():
    shapes = [(5, 7), (100, 3), (513, 2), (1, 40)]
    tree = serialize(("mul", synth.X(0), synth.X(1)))
    hosts, items, outs, sums, bufs = make_batch(shapes, 3, 2, sum64=True, ld_pad=3)
    plan, n_items, n_work = coot.coot_batch_plan(items, 2)
    coot.coot_expr_eval_batched(tree, [0, 0], 0, 3, plan, n_items, n_work)   # compile outside the capture
    torch.cuda.synchronize()
    for o in outs:
        o.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            coot.coot_expr_eval_batched(tree, [0, 0], 0, 3, plan, n_items, n_work, stream=s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for k, (r, c) in enumerate(shapes):
        ld = r + 3
        got = synth.HostMat(outs[k].cpu().numpy()[:ld * c], "f32", r, c, ld)
        check_elementwise(tree, hosts[k], got)
        want = O.sum_dim(tree, hosts[k], 0)
        assert np.allclose(sums[k].cpu().numpy()[:c], want, rtol=1e-6, atol=1e-9)


def test_plan_rejects_bad_items():
    t = torch.zeros(16, device="cuda")
    it = coot.batch_item([coot.Mat(t, 4, 4, 4)], None, None)
    it.in_[0] = None
    with pytest.raises(coot.CootError):
        coot.coot_batch_plan([it], 1)
    it2 = coot.batch_item([coot.Mat(t, 4, 4, 4)], None, None)
    it2.ld_in[0] = 2
    with pytest.raises(coot.CootError):
        coot.coot_batch_plan([it2], 1)


def test_config_size_batch_sampled():
    """4096 matrices with rows and cols log-uniform in [1, 512] (the batching
    workload), one launch; 64 matrices checked against the oracle."""
    n = 4096
    rows = synth.loguniform_int(synth.BASE_SEED + 3, n, 1, 512)
    cols = synth.loguniform_int(synth.BASE_SEED + 4, n, 1, 512)
    shapes = list(zip(rows.tolist(), cols.tolist()))
    tree = serialize(synth.BATCH_EXPR)
    hosts, items, outs, sums, bufs = make_batch(shapes, 5000, 3)
    plan, n_items, n_work = coot.coot_batch_plan(items, 3)
    coot.coot_expr_eval_batched(tree, [0, 0, 0], 0, 0, plan, n_items, n_work)
    torch.cuda.synchronize()
    pick = sorted(set(np.linspace(0, n - 1, 64).astype(int).tolist()))
    check_batch(tree, [shapes[k] for k in pick], [hosts[k] for k in pick], [outs[k] for k in pick],
                [sums[k] for k in pick], 3)
