"""GPU parity of coot_expr_multi_dims: sums along a dimension (Table 6,
sum(A, 0) and sum(A, 1)) formed in the same pass that stores the trees and
takes their full heads.  Column and row sums are checked against the FP64
oracle's sums with the tolerance of the sum tests (gpu_util.check_dim_sums),
stored trees element by element against the single-tree call, and heads as
in the several-tree tests; shapes span many row segments and column chunks
and end in ragged tails, with strided, misaligned, BF16 and FP64-compute
operands, launch-shape overrides, the route for shapes whose partials do not
fit the workspace, empty objects and the argument errors."""
import numpy as np
import pytest
import torch

import paper_2308_03120_gb300 as coot
import synth
from oracle import coot_oracle as O
from paper_2308_03120_gb300.expr import serialize
from tests.gpu_util import Out, check_dim_sums, check_elementwise, host_mats, to_dev
from tests.test_gpu_multi import _check_heads

pytestmark = pytest.mark.gpu

CS, RS = coot.HEAD_COLSUM, coot.HEAD_ROWSUM
HEADS4 = coot.HEAD_SUM | coot.HEAD_NORM2 | coot.HEAD_MIN | coot.HEAD_MAX


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    yield
    coot.coot_set_launch_config(coot.KIND_DIMS, 0)
    torch.cuda.synchronize()


def _f32(r, c, ld=None, lo=-1.0, hi=1.0):
    return ("f32", r, c, ld, lo, hi)


def _mat_specs(r, c, ld=None, dt="f32"):
    if dt == "f32":
        return [_f32(r, c, ld), _f32(r, c, ld), _f32(r, c, ld), _f32(r, c, ld, 0.0, 2.0)]
    return [(dt, r, c, ld, 0, 0)] * 4


def _run(sexprs, ins, heads, stored, sum_dtype="f32", offset=0, out_ld=None, compute="f32", out_dtype="f32"):
    """coot_expr_multi_dims over the host inputs; returns (trees, device
    inputs, stored Outs, per-tree head results, column-sum Outs, row-sum
    Outs)."""
    n_in = max(synth.tree_inputs(s) for s in sexprs)
    trees = [serialize(s, n_inputs=synth.tree_inputs(s), compute=compute) for s in sexprs]
    dev = [to_dev(h, offset) for h in ins[:n_in]]
    r, c = ins[0].n_rows, ins[0].n_cols
    outs = [Out(r, c, out_dtype, ld=out_ld, offset=offset) if stored[k] else None for k in range(len(trees))]
    cols = [Out(1, c, sum_dtype, ld=3) if h & CS else None for h in heads]
    rows = [Out(r, 1, sum_dtype) if h & RS else None for h in heads]
    res = coot.coot_expr_multi_dims(trees, dev, [o.mat if o else None for o in outs], heads,
                                    [o.mat if o else None for o in cols], [o.mat if o else None for o in rows],
                                    ws=coot.Workspace(r))
    torch.cuda.synchronize()
    per, k = [], 0
    vals = res.cpu().numpy() if res is not None else np.zeros(0)
    for h in heads:
        m = bin(h & 0x3FF).count("1")
        per.append(vals[k:k + m])
        k += m
    for o in outs + cols + rows:
        if o is not None:
            o.check()
    return trees, dev, outs, per, cols, rows


def _check_all(sexprs, ins, heads, stored, **kw):
    trees, dev, outs, per, cols, rows = _run(sexprs, ins, heads, stored, **kw)
    for k, tree in enumerate(trees):
        mine = ins[:synth.tree_inputs(sexprs[k])]
        if outs[k] is not None:
            check_elementwise(tree, mine, outs[k].host())
        if heads[k] & 0x3FF:
            _check_heads(tree, mine, heads[k] & 0x3FF, per[k], f"tree {k}")
        if cols[k] is not None:
            check_dim_sums(tree, mine, 0, O.logical(cols[k].host()).ravel())
        if rows[k] is not None:
            check_dim_sums(tree, mine, 1, O.logical(rows[k].host()).ravel())
    return trees, dev, outs, per, cols, rows


@pytest.mark.parametrize("shape", [(1037, 605), (4096, 3), (3, 4099), (1, 10007), (100003, 1), (4097, 7),
                                   (513, 2049), (8192, 64)])
def test_matrix_step_in_one_pass(shape):
    """The matrix step's results in one launch: (A % B + 2C) / (1 + |D|)
    stored with accu, norm2, min, max and both sums; the exp/sqrt chain
    stored."""
    r, c = shape
    ins = host_mats(_mat_specs(r, c), 401)
    _check_all([synth.MAT_EXPR, synth.MAT_CHAIN], ins, [HEADS4 | CS | RS, 0], [True, True])


@pytest.mark.parametrize("sexpr", [synth.LEAF0, synth.SCHUR_XZ, synth.MAT_CHAIN])
def test_sums_only(sexpr):
    """Only the sums (nothing stored, no full heads), each dimension alone
    and both."""
    r, c = 2049, 333
    ins = host_mats(_mat_specs(r, c), 403)
    for h in (CS, RS, CS | RS):
        _check_all([sexpr], ins, [h], [False])


def test_every_tree_its_own_sums():
    """Four trees, each with its own sums and heads."""
    r, c = 777, 129
    ins = host_mats(_mat_specs(r, c), 405)
    sexprs = [synth.MAT_EXPR, synth.MAT_CHAIN, synth.LEAF0, synth.SCHUR_XZ]
    heads = [CS | RS | coot.HEAD_SUM, RS, CS | coot.HEAD_MAX, CS | RS]
    _check_all(sexprs, ins, heads, [True, False, True, False])


@pytest.mark.parametrize("ld_pad", [1, 5])
def test_strided_operands(ld_pad):
    r, c = 1500, 41
    ins = host_mats(_mat_specs(r, c, r + ld_pad), 407)
    _check_all([synth.MAT_EXPR], ins, [HEADS4 | CS | RS], [True], out_ld=r + 2 * ld_pad)


@pytest.mark.parametrize("offset", [1, 3])
def test_misaligned_operands(offset):
    r, c = 999, 17
    ins = host_mats(_mat_specs(r, c), 409)
    _check_all([synth.MAT_EXPR], ins, [CS | RS | coot.HEAD_SUM], [True], offset=offset)


@pytest.mark.parametrize("dt", ["bf16", "f16"])
def test_low_precision_operands(dt):
    """BF16 / FP16 inputs and stored output, FP32 arithmetic and sums."""
    r, c = 2050, 77
    ins = host_mats([(dt, r, c, None, 0, 0)] * 2, 411)
    _check_all([synth.AXPY_2X_3Z], ins, [CS | RS | coot.HEAD_SUM | coot.HEAD_NORM2], [True], out_dtype=dt)


def test_fp64_compute_and_sums():
    r, c = 700, 45
    ins = host_mats([("f64", r, c, None, -1.0, 1.0)] * 3 + [("f64", r, c, None, 0.0, 2.0)], 413)
    trees, dev, outs, per, cols, rows = _run([synth.MAT_CHAIN], ins, [CS | RS | coot.HEAD_SUM], [True],
                                             sum_dtype="f64", compute="f64", out_dtype="f64")
    tree = trees[0]
    for dim, o in ((0, cols[0]), (1, rows[0])):
        got = O.logical(o.host()).ravel()
        want = O.sum_dim(tree, ins, dim)
        assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want) + 1e-13), dim


@pytest.mark.parametrize("cfg", [dict(unroll=1, split=1), dict(unroll=2, split=3), dict(unroll=4, split=64),
                                 dict(block=512, unroll=2), dict(block=64, vec=1, unroll=3, split=7)])
def test_launch_shapes_keep_results(cfg):
    """One segment per column or many, one chunk or many: every launch shape
    gives results within the tolerances (row segments of 32 x vec x unroll
    rows, split = column chunks)."""
    r, c = 3001, 203
    ins = host_mats(_mat_specs(r, c), 415)
    coot.coot_set_launch_config(coot.KIND_DIMS, cfg.get("block", 256), cfg.get("vec", 0), cfg.get("unroll", 0), 0,
                                cfg.get("split", 0))
    try:
        _check_all([synth.MAT_EXPR, synth.MAT_CHAIN], ins, [HEADS4 | CS | RS, RS], [True, False])
        last = coot.coot_last_launch()
        if cfg.get("split") in (1, 3):
            assert last["split"] == cfg["split"]
    finally:
        coot.coot_set_launch_config(coot.KIND_DIMS, 0)


def test_wide_matrix_takes_the_split_route():
    """More columns than the workspace has counters, with several row
    segments: the sums come from the column / row sum kernels before the
    storing pass; the results are the same within rounding."""
    r, c = 600, 17000
    ins = host_mats(_mat_specs(r, c), 417)
    _check_all([synth.MAT_EXPR], ins, [HEADS4 | CS | RS], [True])


def test_in_place_with_sums():
    """A stored tree identical to its input (B = B + 3A) with the sums of
    that tree: every sum is of the values before the store."""
    r, c = 1111, 37
    ins = host_mats([_f32(r, c), _f32(r, c)], 419)
    e = ("add", synth.X(0), ("mul", synth.C(3.0), synth.X(1)))
    tree = serialize(e)
    dev = [to_dev(h) for h in ins]
    col = Out(1, c)
    row = Out(r, 1)
    coot.coot_expr_multi_dims([tree], dev, [dev[0]], [CS | RS], [col.mat], [row.mat], ws=coot.Workspace(r))
    torch.cuda.synchronize()
    check_dim_sums(tree, ins, 0, O.logical(col.host()).ravel())
    check_dim_sums(tree, ins, 1, O.logical(row.host()).ravel())
    got = dev[0].buf.cpu().numpy()[:r * c]
    want = O.evaluate(tree, ins)
    assert np.allclose(got.reshape(c, r).T, want, rtol=1e-6, atol=1e-6)


def test_deterministic():
    r, c = 4099, 1031
    ins = host_mats(_mat_specs(r, c), 421)
    a = _run([synth.MAT_EXPR], ins, [HEADS4 | CS | RS], [False])
    b = _run([synth.MAT_EXPR], ins, [HEADS4 | CS | RS], [False])
    assert np.array_equal(a[3][0], b[3][0])
    assert np.array_equal(a[4][0].host().buf, b[4][0].host().buf)
    assert np.array_equal(a[5][0].host().buf, b[5][0].host().buf)


@pytest.mark.parametrize("shape", [(0, 5), (5, 0), (0, 0)])
def test_empty_objects(shape):
    """Sums of an empty object are zeros (one per column or row); the full
    heads follow coot_expr_reduce's rules."""
    r, c = shape
    ins = host_mats([_f32(r, c)], 3)
    dev = [to_dev(h) for h in ins]
    col = Out(1, c)
    row = Out(r, 1)
    col.t.fill_(float("nan"))
    row.t.fill_(float("nan"))
    res = coot.coot_expr_multi_dims([serialize(synth.LEAF0)], dev, None, [CS | RS | coot.HEAD_SUM], [col.mat],
                                    [row.mat], ws=coot.Workspace(max(r, 1)))
    torch.cuda.synchronize()
    assert res.item() == 0.0
    assert np.all(O.logical(col.host()) == 0.0) and np.all(O.logical(row.host()) == 0.0)


def test_argument_errors():
    r, c = 64, 8
    ins = host_mats([_f32(r, c)], 5)
    dev = [to_dev(h) for h in ins]
    leaf = serialize(synth.LEAF0)
    ws = coot.Workspace(r)
    col, row = Out(1, c), Out(r, 1)
    with pytest.raises(coot.CootError) as e:   # no output for the requested sums
        coot.coot_expr_multi_dims([leaf], dev, None, [CS], None, None, ws=ws)
    assert e.value.status_name == "COOT_ERR_INVALID_ARG"
    with pytest.raises(coot.CootError) as e:   # wrong shape
        coot.coot_expr_multi_dims([leaf], dev, None, [RS], None, [col.mat], ws=ws)
    assert e.value.status_name == "COOT_ERR_SHAPE"
    ti = torch.zeros(c, dtype=torch.int32, device="cuda")
    with pytest.raises(coot.CootError) as e:   # integer sums
        coot.coot_expr_multi_dims([leaf], dev, None, [CS], [coot.Mat(ti, 1, c, 1)], None, ws=ws)
    assert e.value.status_name == "COOT_ERR_DTYPE"
    with pytest.raises(coot.CootError) as e:   # a sum over an input
        coot.coot_expr_multi_dims([leaf], dev, None, [RS], None, [coot.Mat(dev[0].buf, r, 1, r, dev[0].offset)],
                                  ws=ws)
    assert e.value.status_name == "COOT_ERR_ALIAS"
    with pytest.raises(coot.CootError) as e:   # dimension bits are not coot_expr_multi heads
        coot.coot_expr_multi([leaf], dev, None, [CS], ws=ws)
    assert e.value.status_name == "COOT_ERR_INVALID_ARG"
    coot.coot_expr_multi_dims([leaf], dev, None, [CS | RS], [col.mat], [row.mat], ws=ws)
    torch.cuda.synchronize()
