"""GPU parity of relational nodes (Table 5's "A < x" and the other
relational expressions) and of the all / any reductions against the FP64
oracle.  A relational node is exact (1 or 0) wherever its decision is
certain; the oracle's error bound marks the elements where rounding could
flip it, and those are skipped and counted."""
import math

import numpy as np
import pytest
import torch

import paper_2308_03120_gb300 as coot
import synth
from oracle import coot_oracle as O
from paper_2308_03120_gb300.expr import serialize
from tests.gpu_util import Out, assert_sum_close, check_elementwise, host_mats, to_dev

pytestmark = pytest.mark.gpu

X0, X1, C = synth.X(0), synth.X(1), synth.C


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    yield
    torch.cuda.synchronize()


def _f32(r, c, lo=-1.0, hi=1.0):
    return ("f32", r, c, None, lo, hi)


RELATIONAL_TREES = [
    ("lt", X0, C(0.5)),
    ("ge", X0, X1),
    ("mul", ("gt", X0, C(0.0)), X0),                              # positive part
    ("add", ("le", X0, X1), ("mul", ("ne", X0, C(0.25)), C(2.0))),
    ("eq", ("abs", X0), X0),                                      # 1 where x >= 0
    ("gt", ("mul", X0, X1), C(0.125)),                            # inexact operand: some skips
]


@pytest.mark.parametrize("sexpr", RELATIONAL_TREES)
@pytest.mark.parametrize("shape", [(100_003, 1), (257, 129)])
def test_relational_trees_elementwise(sexpr, shape):
    r, c = shape
    ins = host_mats([_f32(r, c), _f32(r, c)], 301)
    n_in = synth.tree_inputs(sexpr)
    tree = serialize(sexpr, n_inputs=n_in)
    out = Out(r, c)
    coot.coot_expr_eval(tree, [to_dev(h) for h in ins[:n_in]], out.mat)
    torch.cuda.synchronize()
    out.check()
    rep = check_elementwise(tree, ins[:n_in], out.host())
    if sexpr[0] in ("lt", "ge") or sexpr[1][0] == "gt":
        assert rep["skipped"] == 0


def test_relational_with_nan_and_bf16():
    a = np.array([-1.0, 0.0, 0.5, 1.0, np.nan, 0.5], dtype=np.float32)
    ins = [synth.as_mat(a, "f32", 6, 1)]
    for name in ("lt", "le", "gt", "ge", "eq", "ne"):
        tree = serialize((name, X0, C(0.5)))
        out = Out(6, 1)
        coot.coot_expr_eval(tree, [to_dev(ins[0])], out.mat)
        torch.cuda.synchronize()
        assert O.logical(out.host()).ravel().tolist() == O.evaluate(tree, ins).ravel().tolist(), name
    h = host_mats([("bf16", 4096, 3, None, 0, 0)], 307)
    tree = serialize(("lt", X0, C(1.0)))
    out = Out(4096, 3, "bf16")
    coot.coot_expr_eval(tree, [to_dev(h[0])], out.mat)
    torch.cuda.synchronize()
    check_elementwise(tree, h, out.host())


@pytest.mark.parametrize("shape", [(1_000_003, 1), (1037, 605), (1, 1)])
def test_all_any_against_the_oracle(shape):
    r, c = shape
    ins = host_mats([_f32(r, c)], 311)
    dev = [to_dev(ins[0])]
    lo, hi = O.minmax(serialize(synth.LEAF0), ins)
    # thresholds below, inside and above the data, and exactly at min / max
    for k in (lo - 0.5, lo, (lo + hi) / 2, hi, hi + 0.5):
        k = float(np.float32(k))
        for name in ("lt", "le", "gt", "ge"):
            tree = serialize((name, X0, C(k)))
            got = coot.coot_all_any(tree, dev).tolist()
            assert got == [float(O.all_(tree, ins)), float(O.any_(tree, ins))], (name, k, got)
    leaf = serialize(synth.LEAF0)
    assert coot.coot_all_any(leaf, dev).tolist() == [float(O.all_(leaf, ins)), float(O.any_(leaf, ins))]


def test_all_any_special_values():
    leaf = serialize(synth.LEAF0)
    cases = [[1.0, -2.0, 0.5], [1.0, 0.0, 0.5], [0.0, -0.0, 0.0], [0.0, np.nan, 0.0], [np.nan], [np.inf, -np.inf]]
    for vals in cases:
        a = np.array(vals, dtype=np.float32)
        ins = [synth.as_mat(a, "f32", a.size, 1)]
        got = coot.coot_all_any(leaf, [to_dev(ins[0])]).tolist()
        assert got == [float(O.all_(leaf, ins)), float(O.any_(leaf, ins))], vals
    empty = coot.Mat(torch.zeros(4, device="cuda"), 0, 3, 1)
    assert coot.coot_all_any(leaf, [empty]).tolist() == [1.0, 0.0]
    # a value that is nonzero in FP64 but rounds to zero in FP32 compute
    tiny = np.array([1e-10, 1.0], dtype=np.float64)
    ins = [synth.as_mat(tiny, "f64", 2, 1)]
    tree = serialize(("mul", X0, C(1e-40)))
    assert coot.coot_all_any(tree, [to_dev(ins[0])]).tolist() == [float(O.all_(tree, ins)), float(O.any_(tree, ins))]


def test_count_and_heads_in_one_pass():
    """accu(x < 0.5) counts the elements; all / any / sum / max heads share
    one pass with the stored relational values."""
    r, c = 40_000, 33
    ins = host_mats([_f32(r, c)], 313)
    dev = [to_dev(ins[0])]
    tree = serialize(("lt", X0, C(0.5)))
    count = coot.coot_accu(tree, dev).item()
    assert count == O.accu(tree, ins) == float(np.sum(O.logical(ins[0]) < np.float32(0.5)))
    heads = coot.HEAD_SUM | coot.HEAD_MAX | coot.HEAD_ALL | coot.HEAD_ANY
    out = Out(r, c)
    res = coot.coot_expr_reduce(tree, dev, heads, out=out.mat).tolist()
    torch.cuda.synchronize()
    out.check()
    check_elementwise(tree, ins, out.host())
    assert res == [count, 1.0, float(O.all_(tree, ins)), float(O.any_(tree, ins))]
    # a masked sum: accu((x > 0) % x) is the sum of the positive part
    pos = serialize(("mul", ("gt", X0, C(0.0)), X0))
    v, e, _ = O.error_bound(pos, ins)
    assert_sum_close(coot.coot_accu(pos, dev).item(), O.accu(pos, ins), v.ravel(), e.ravel(), "positive part")
