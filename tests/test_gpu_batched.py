"""GPU parity of the batched evaluation (many small matrices of uneven
shapes in one launch) against the FP64 oracle, matrix by matrix."""
import ctypes
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


def test_batch_paths_bf16_four_inputs_and_misaligned():
    """BF16 inputs (staged, values kept apart from the 2-byte inputs), four
    FP32 inputs (two units do not fit in shared memory: the register path)
    and matrices that start off a 16-byte boundary (the global path)."""
    shapes = [(r, 1 + (r * 7) % 40) for r in (1, 3, 17, 32, 100, 257, 511)]
    # BF16 (the device tensors stay referenced in `keep`: the items hold
    # raw pointers)
    hosts, items, outs, sums, keep = [], [], [], [], []
    for k, (r, c) in enumerate(shapes):
        ins = []
        for s in range(3):
            x = (synth.uniform_f32(800 + 7 * k + s, r * c) * np.float32(4.0)).astype(np.float32)
            bits = (x.view(np.uint32) >> np.uint32(16)).astype(np.uint16)   # truncate to BF16 bits
            ins.append(synth.as_mat(bits, "bf16", r, c))
        hosts.append(ins)
        dev = [coot.Mat(torch.from_numpy(h.buf.view(np.int16).copy()).view(torch.bfloat16).cuda(), r, c, r)
               for h in ins]
        out = torch.full((r * c,), float("nan"), device="cuda")
        cs = torch.full((c,), float("nan"), device="cuda")
        items.append(coot.batch_item(dev, coot.Mat(out, r, c, r), coot.Mat(cs, 1, c, 1)))
        keep.append(dev)
        outs.append(out)
        sums.append(cs)
    tree = serialize(synth.BATCH_EXPR)
    plan, n_items, n_work = coot.coot_batch_plan(items, 3)
    coot.coot_expr_eval_batched(tree, [1, 1, 1], 0, 0, plan, n_items, n_work)
    torch.cuda.synchronize()
    check_batch(tree, shapes, hosts, outs, sums, 3)
    # four FP32 inputs
    tree4 = serialize(("add", synth.BATCH_EXPR, ("mul", synth.X(3), synth.X(3))))
    hosts, items, outs, sums, bufs = make_batch(shapes, 810, 4)
    plan, n_items, n_work = coot.coot_batch_plan(items, 4)
    coot.coot_expr_eval_batched(tree4, [0, 0, 0, 0], 0, 0, plan, n_items, n_work)
    torch.cuda.synchronize()
    check_batch(tree4, shapes, hosts, outs, sums, 4)
    # operands one element off a 16-byte boundary
    hosts, items, outs, sums = [], [], [], []
    for k, (r, c) in enumerate(shapes):
        ins = [synth.as_mat(synth.uniform_f32(820 + 7 * k + s, r * c), "f32", r, c) for s in range(3)]
        hosts.append(ins)
        dev = [coot.Mat(torch.cat([torch.zeros(1), torch.from_numpy(h.buf)]).cuda(), r, c, r, 1) for h in ins]
        out = torch.full((r * c + 1,), float("nan"), device="cuda")
        cs = torch.full((c,), float("nan"), device="cuda")
        items.append(coot.batch_item(dev, coot.Mat(out, r, c, r, 1), coot.Mat(cs, 1, c, 1)))
        keep.append(dev)
        outs.append(out[1:])
        sums.append(cs)
    plan, n_items, n_work = coot.coot_batch_plan(items, 3)
    coot.coot_expr_eval_batched(tree, [0, 0, 0], 0, 0, plan, n_items, n_work)
    torch.cuda.synchronize()
    check_batch(tree, shapes, hosts, outs, sums, 3)


def test_bounded_wait_reports_a_timeout(monkeypatch):
    """A staged unit whose copy is never started (the status test hook):
    every wait gives up after about a second, the kernel records
    COOT_ERR_TIMEOUT, and the next batch runs normally."""
    shapes = [(64, 8)] * 400
    tree = serialize(synth.BATCH_EXPR)
    hosts, items, outs, sums, bufs = make_batch(shapes, 830, 3)
    plan, n_items, n_work = coot.coot_batch_plan(items, 3)
    coot.coot_expr_eval_batched(tree, [0, 0, 0], 0, 0, plan, n_items, n_work)   # compile, status clean
    torch.cuda.synchronize()
    status = ctypes.c_int(-1)
    from paper_2308_03120_gb300 import _abi
    _abi.call("coot_device_status", ctypes.byref(status))
    assert status.value == 0
    monkeypatch.setenv("COOT_FAULT", "batched_wait")
    coot.coot_expr_eval_batched(tree, [0, 0, 0], 0, 0, plan, n_items, n_work)
    torch.cuda.synchronize()
    _abi.call("coot_device_status", ctypes.byref(status))
    assert _abi.STATUS[status.value] == "COOT_ERR_TIMEOUT"
    monkeypatch.delenv("COOT_FAULT")
    for o in outs:
        o.fill_(float("nan"))
    coot.coot_expr_eval_batched(tree, [0, 0, 0], 0, 0, plan, n_items, n_work)
    torch.cuda.synchronize()
    _abi.call("coot_device_status", ctypes.byref(status))
    assert status.value == 0
    check_batch(tree, shapes, hosts, outs, sums, 3)
