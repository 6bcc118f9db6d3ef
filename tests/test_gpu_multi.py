"""GPU parity of coot_expr_multi (several trees over the same operands in one
pass) against the FP64 oracle and against the single-tree calls: each stored
tree equals coot_expr_eval's result element for element (the same tree
function per element), and each tree's heads agree with the oracle within
the reduction tolerances of the parity tests (tests/gpu_util)."""
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

X0, X1, X2 = synth.X(0), synth.X(1), synth.X(2)
ORDER = [coot.HEAD_SUM, coot.HEAD_SUMSQ, coot.HEAD_NORM2, coot.HEAD_SUMABS, coot.HEAD_MIN, coot.HEAD_MAX,
         coot.HEAD_MINABS, coot.HEAD_MAXABS, coot.HEAD_ALL, coot.HEAD_ANY]


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    yield
    coot.coot_set_launch_config(coot.KIND_MULTI, 0)
    torch.cuda.synchronize()


def _f32(r, c, ld=None, lo=-1.0, hi=1.0):
    return ("f32", r, c, ld, lo, hi)


def _check_heads(tree, ins, heads, got, what):
    """One tree's results (head-bit order) against the oracle."""
    v, e, unsafe = O.error_bound(tree, ins)
    assert not unsafe.any()
    t, e = v.ravel(order="F"), e.ravel(order="F")
    leaf = not np.any(e)
    k = 0
    for bit in ORDER:
        if not heads & bit:
            continue
        g = float(got[k])
        k += 1
        if bit == coot.HEAD_SUM:
            assert_sum_close(g, O.accu(tree, ins), t, e, f"{what} sum")
        elif bit == coot.HEAD_NORM2:
            o = O.norm(tree, ins, "fro")
            sq_err = 2.0 * np.abs(t) * e + e * e
            assert abs(g * g - o * o) <= 1e-6 * o * o + 6.0 * math.sqrt(float(np.sum(sq_err ** 2))), (what, g, o)
        elif bit in (coot.HEAD_MIN, coot.HEAD_MAX):
            lo, hi = O.minmax(tree, ins)
            o = lo if bit == coot.HEAD_MIN else hi
            slack = 0.0 if leaf else 2.0 * float(np.max(e))
            assert abs(g - o) <= slack, (what, bit, g, o)
        elif bit in (coot.HEAD_ALL, coot.HEAD_ANY):
            r32 = O.round_to_format(v, "f32") if O.decode(tree).compute == "f32" else v
            nz = (r32 != 0) | np.isnan(r32)
            o = float(nz.all()) if bit == coot.HEAD_ALL else float(nz.any())
            assert g == o, (what, bit, g, o)
        else:
            raise AssertionError(f"no check for head {bit}")
    assert k == len(got)


def _run(sexprs, ins, heads, stored, out_dtypes=None, offset=0, out_ld=None):
    """coot_expr_multi over the host inputs: returns (Out or None per tree,
    per-tree result lists)."""
    n_in = max(synth.tree_inputs(s) for s in sexprs)
    trees = [serialize(s, n_inputs=synth.tree_inputs(s)) for s in sexprs]
    dev = [to_dev(h, offset) for h in ins[:n_in]]
    r, c = ins[0].n_rows, ins[0].n_cols
    out_dtypes = out_dtypes or ["f32"] * len(trees)
    outs = [Out(r, c, out_dtypes[k], ld=out_ld, offset=offset) if stored[k] else None for k in range(len(trees))]
    res = coot.coot_expr_multi(trees, dev, [o.mat if o else None for o in outs], heads, ws=coot.Workspace(1))
    torch.cuda.synchronize()
    per, k = [], 0
    vals = res.cpu().numpy() if res is not None else np.zeros(0)
    for h in heads:
        m = bin(h).count("1")
        per.append(vals[k:k + m])
        k += m
    for o in outs:
        if o is not None:
            o.check()
    return trees, dev, outs, per


def _same_as_single(tree, dev, out, out_dtype="f32"):
    """The stored tree equals coot_expr_eval's result element for element."""
    single = Out(out.n_rows, out.n_cols, out_dtype, ld=out.ld)
    coot.coot_expr_eval(tree, dev, single.mat)
    torch.cuda.synchronize()
    a, b = O.logical(out.host()), O.logical(single.host())
    assert np.array_equal(a, b, equal_nan=True)


@pytest.mark.parametrize("n", [1_000_000, 1_000_003, 1, 7])
def test_the_vector_step_in_one_pass(n):
    """Task 1 and 2 of the paper in one launch: y = 2x + 3z stored, accu(x % z)
    and norm2(x)."""
    ins = host_mats([_f32(n, 1), _f32(n, 1)], synth.BASE_SEED)
    sexprs = [synth.AXPY_2X_3Z, synth.SCHUR_XZ, synth.LEAF0]
    heads = [0, coot.HEAD_SUM, coot.HEAD_NORM2]
    trees, dev, outs, per = _run(sexprs, ins, heads, [True, False, False])
    rep = check_elementwise(trees[0], ins, outs[0].host())
    assert rep["skipped"] == 0
    _same_as_single(trees[0], dev, outs[0])
    _check_heads(trees[1], ins, heads[1], per[1], "accu(x % z)")
    _check_heads(trees[2], ins[:1], heads[2], per[2], "norm2(x)")


@pytest.mark.parametrize("shape", [(1037, 605), (3, 4099), (4099, 3)])
def test_two_matrix_trees_share_the_pass(shape):
    """The matrix tree with accu, norm2, min and max, and the exp/sqrt chain,
    both stored, from one read of the four operands."""
    r, c = shape
    ins = host_mats([_f32(r, c), _f32(r, c), _f32(r, c), _f32(r, c, lo=0.0, hi=2.0)], 61)
    heads = [coot.HEAD_SUM | coot.HEAD_NORM2 | coot.HEAD_MIN | coot.HEAD_MAX, 0]
    trees, dev, outs, per = _run([synth.MAT_EXPR, synth.MAT_CHAIN], ins, heads, [True, True])
    for k in range(2):
        check_elementwise(trees[k], ins, outs[k].host())
        _same_as_single(trees[k], dev, outs[k])
    _check_heads(trees[0], ins, heads[0], per[0], "matrix tree")


def test_four_trees_with_mixed_storage_and_heads():
    """Four trees over BF16 operands (FP32 arithmetic): a BF16 and an FP32
    output, heads of every kind of combine (sum, min / max, all / any)."""
    r, c = 2049, 37
    ins = host_mats([("bf16", r, c, None, 0, 0), ("bf16", r, c, None, 0, 0)], 91)
    sexprs = [("add", X0, X1), ("mul", X0, X1), ("abs", X0), ("lt", X0, X1)]
    heads = [coot.HEAD_MAX, coot.HEAD_SUM | coot.HEAD_NORM2, 0, coot.HEAD_ALL | coot.HEAD_ANY | coot.HEAD_SUM]
    trees, dev, outs, per = _run(sexprs, ins, heads, [True, False, True, False], out_dtypes=["bf16", "f32", "f32",
                                                                                           "f32"])
    check_elementwise(trees[0], ins, outs[0].host())
    _same_as_single(trees[0], dev, outs[0], "bf16")
    check_elementwise(trees[2], ins[:1], outs[2].host())
    for k in (0, 1, 3):
        _check_heads(trees[k], ins[:synth.tree_inputs(sexprs[k])], heads[k], per[k], f"tree {k}")


def test_strided_and_misaligned_operands():
    r, c, ld = 1031, 67, 1040
    for offset in (0, 1):
        ins = host_mats([_f32(r, c, ld), _f32(r, c, ld), _f32(r, c, ld)], 101)
        sexprs = [synth.BATCH_EXPR, ("sub", X0, X2)]
        heads = [coot.HEAD_SUM, coot.HEAD_MIN | coot.HEAD_MAX]
        trees, dev, outs, per = _run(sexprs, ins, heads, [True, True], offset=offset, out_ld=ld + 3)
        for k in range(2):
            check_elementwise(trees[k], ins[:synth.tree_inputs(sexprs[k])], outs[k].host())
            _check_heads(trees[k], ins[:synth.tree_inputs(sexprs[k])], heads[k], per[k], f"tree {k}")


def test_an_output_identical_to_an_input_reads_the_old_values():
    """Tree 0 = 2 x0 + x1 stored over x0 itself; tree 1 = x0 % x1 must see the
    old x0 (every element's operands are read before any value is stored)."""
    r, c = 777, 13
    ins = host_mats([_f32(r, c), _f32(r, c)], 111)
    dev = [to_dev(h) for h in ins]
    t0 = serialize(("add", ("mul", synth.C(2.0), X0), X1))
    t1 = serialize(synth.SCHUR_XZ)
    res = coot.coot_expr_multi([t0, t1], dev, [dev[0], None], [0, coot.HEAD_SUM], ws=coot.Workspace(1))
    torch.cuda.synchronize()
    got = synth.HostMat(dev[0].buf.cpu().numpy().copy(), "f32", r, c, r)
    check_elementwise(t0, ins, got)
    _check_heads(t1, ins, coot.HEAD_SUM, res.cpu().numpy(), "accu(old x0 % x1)")


def test_empty_operands():
    ins = [coot.Mat(torch.empty(0, device="cuda"), 0, 5, 1)] * 2
    t0, t1 = serialize(synth.SCHUR_XZ), serialize(synth.LEAF0)
    res = coot.coot_expr_multi([t0, t1], ins, None, [coot.HEAD_SUM | coot.HEAD_ANY, coot.HEAD_ALL | coot.HEAD_NORM2],
                               ws=coot.Workspace(1))
    torch.cuda.synchronize()
    assert res.tolist() == [0.0, 0.0, 0.0, 1.0]
    with pytest.raises(coot.CootError) as e:
        coot.coot_expr_multi([t0, t1], ins, None, [coot.HEAD_SUM, coot.HEAD_MIN], ws=coot.Workspace(1))
    assert e.value.status_name == "COOT_ERR_EMPTY"


@pytest.mark.parametrize("cfg", [dict(block=128, vec=1, unroll=1), dict(block=512, vec=2, unroll=8)])
def test_launch_shapes_keep_results(cfg):
    r, c = 1037, 605
    ins = host_mats([_f32(r, c), _f32(r, c), _f32(r, c), _f32(r, c, lo=0.0, hi=2.0)], 121)
    heads = [coot.HEAD_SUM | coot.HEAD_MAX, coot.HEAD_NORM2]
    coot.coot_set_launch_config(coot.KIND_MULTI, cfg["block"], cfg["vec"], cfg["unroll"], 0, 0)
    try:
        trees, dev, outs, per = _run([synth.MAT_EXPR, synth.MAT_CHAIN], ins, heads, [True, False])
        last = coot.coot_last_launch()
        assert last["block"] == cfg["block"] and last["unroll"] == cfg["unroll"]
    finally:
        coot.coot_set_launch_config(coot.KIND_MULTI, 0)
    _same_as_single(trees[0], dev, outs[0])
    for k in range(2):
        _check_heads(trees[k], ins, heads[k], per[k], f"tree {k}")
