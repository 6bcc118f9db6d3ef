"""The canonical form on the GPU: results with canonical forms on and off are
bit-for-bit equal element-wise (the rewrites are exact), match the oracle on
the original tree, and operands passed twice are read once (dot(x, x))."""
import numpy as np
import pytest
import torch

import paper_2308_03120_gb300 as coot
import synth
from oracle import coot_oracle as O
from paper_2308_03120_gb300.expr import serialize
from tests.gpu_util import Out, assert_sum_close, check_elementwise, host_mats, to_dev
from tests.test_canonical_host import _inject

pytestmark = pytest.mark.gpu

X0, X1, X2, C = synth.X(0), synth.X(1), synth.X(2), synth.C


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    yield
    coot.coot_set_canonical(True)
    torch.cuda.synchronize()


def _eval(tree, dev, r, c, canonical):
    coot.coot_set_canonical(canonical)
    try:
        out = Out(r, c)
        coot.coot_expr_eval(tree, dev, out.mat)
        torch.cuda.synchronize()
        out.check()
        return out
    finally:
        coot.coot_set_canonical(True)


@pytest.mark.parametrize("seed", range(12))
def test_canonical_and_original_trees_agree_bitwise(seed):
    n_in = 1 + seed % 3
    e = _inject(synth.random_tree(9000 + seed, 2 + seed % 6, n_in), iter(synth.uniform01(9100 + seed, 4096).tolist()))
    tree = serialize(e, n_inputs=n_in)
    r, c = 2049, 33
    ins = host_mats([("f32", r, c, None, -2.0, 2.0)] * n_in, 9200 + seed)
    dev = [to_dev(h) for h in ins]
    on = _eval(tree, dev, r, c, True)
    off = _eval(tree, dev, r, c, False)
    a, b = on.t.cpu().numpy(), off.t.cpu().numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32)) or np.array_equal(a, b, equal_nan=True)
    check_elementwise(tree, ins, on.host(), max_skip_frac=0.05)


def test_repeated_operands_are_read_once():
    # large enough (5.7 M elements, dense, so one flat run) that the built-in
    # shape keeps its unroll (4 blocks per SM of 8192-element tiles and
    # more), so the unroll shows the operand count
    r, c = 8195, 700
    ins = host_mats([("f32", r, c, None, -1.0, 1.0), ("f32", r, c, None, -1.0, 1.0)], 9301)
    A, B = (to_dev(h) for h in ins)
    # x0 % x1 + x2 with (A, A, B): the kernel reads A once
    tree = serialize(("add", ("mul", X0, X1), X2))
    out = Out(r, c)
    coot.coot_expr_eval(tree, [A, A, B], out.mat)
    torch.cuda.synchronize()
    out.check()
    check_elementwise(tree, [ins[0], ins[0], ins[1]], out.host())
    last = coot.coot_last_launch()
    assert last["unroll"] == 8      # two operands now: the built-in unroll for fewer than 3 inputs
    # dot(x, x) = norm(x)^2
    n = 1_000_003
    x = host_mats([("f32", n, 1, None, -1.0, 1.0)], 9302)[0]
    X = to_dev(x)
    d = coot.coot_dot(X, X).item()
    v = O.logical(x).ravel()
    assert_sum_close(d, O.dot(x, x), v * v, np.zeros(n), "dot(x, x)")
    coot.coot_set_canonical(False)
    try:
        d_off = coot.coot_dot(X, X).item()
    finally:
        coot.coot_set_canonical(True)
    assert_sum_close(d_off, O.dot(x, x), v * v, np.zeros(n), "dot(x, x) without canonical forms")


def test_reductions_and_unfused_with_redundant_trees():
    r, c = 3001, 17
    ins = host_mats([("f32", r, c, None, -1.0, 1.0), ("f32", r, c, None, -1.0, 1.0)], 9401)
    dev = [to_dev(h) for h in ins]
    e = ("add", ("neg", ("neg", ("mul", X0, C(1.0)))), ("mul", C(2.0), ("mul", C(4.0), ("sub", X1, C(0.0)))))
    tree = serialize(e)
    v, err, _ = O.error_bound(tree, ins)
    assert_sum_close(coot.coot_accu(tree, dev).item(), O.accu(tree, ins), v.ravel(), err.ravel(), "accu")
    outs = []
    for canonical in (True, False):
        coot.coot_set_canonical(canonical)
        try:
            out = Out(r, c)
            coot.coot_unfused_eval(tree, dev, out.mat)
            torch.cuda.synchronize()
            outs.append(out.t.cpu().numpy())
        finally:
            coot.coot_set_canonical(True)
    assert np.array_equal(outs[0], outs[1])
    check_elementwise(tree, ins, synth.HostMat(outs[0][64:64 + r * c], "f32", r, c, r))


def test_constant_tree_fills_the_output():
    r, c = 1000, 3
    h = host_mats([("f32", r, c, None, -1.0, 1.0)], 9501)[0]
    tree = serialize(("mul", ("add", C(1.0), C(2.0)), ("sqrt", C(4.0))), n_inputs=1)
    out = Out(r, c)
    coot.coot_expr_eval(tree, [to_dev(h)], out.mat)
    torch.cuda.synchronize()
    assert np.all(O.logical(out.host()) == 6.0)
