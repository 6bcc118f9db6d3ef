"""GPU parity of the statistics along a dimension (coot_stats_dim: sum,
mean, var, stddev, min, max of each column or row in one pass) against the
FP64 oracle, with the tolerances derived from the kernels' arithmetic:

  * sum: as the column / row sums (1e-6 |o|, the cancellation floor
    1e-9 sum|t|, six standard deviations of the element errors), plus the
    rounding of the stored result;
  * mean: the sum's tolerance / N, plus the stored rounding;
  * var: 1e-6 |o| + 12 u sum (v - K)^2 / (N - 1 + norm_type) (the shifted
    one-pass formula: K the line's first value, u the compute type's unit
    roundoff) + (2 sum |v - mean| E + sum E^2) / (N - 1 + norm_type) for the
    element errors E, plus the stored rounding;
  * stddev: the same bound on stddev^2;
  * min / max: exact for leaves, within 2 max E for trees.
"""
import math

import numpy as np
import pytest
import torch

import paper_2308_03120_gb300 as coot
import synth
from oracle import coot_oracle as O
from paper_2308_03120_gb300.expr import serialize
from tests.gpu_util import Out, host_mats, sum_tolerance, to_dev

pytestmark = pytest.mark.gpu

NAMES = ["sum", "mean", "var", "stddev", "min", "max"]
ALL = 0x3F


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    yield
    for kind in (5, 6):
        coot.coot_set_launch_config(kind, 0)
    torch.cuda.synchronize()


def _f32(r, c, ld=None, lo=-1.0, hi=1.0):
    return ("f32", r, c, ld, lo, hi)


def _inputs(sexpr, specs, seed, compute="f32"):
    ins = host_mats(specs, seed)
    n_in = synth.tree_inputs(sexpr)
    return serialize(sexpr, compute=compute, n_inputs=n_in), ins[:n_in], [to_dev(h) for h in ins[:n_in]]


def run_stats(tree, dev, dim, mask, out_dtype="f32", norm_type=0, out_ld=None):
    r, c = dev[0].n_rows, dev[0].n_cols
    names = [n for b, n in enumerate(NAMES) if mask >> b & 1]
    outs = [Out(1, c, out_dtype, ld=out_ld) if dim == 0 else Out(r, 1, out_dtype) for _ in names]
    coot.coot_stats_dim(tree, dev, dim, mask, [o.mat for o in outs], norm_type)
    torch.cuda.synchronize()
    got = {}
    for n, o in zip(names, outs):
        o.check()
        got[n] = O.logical(o.host()).ravel()
    return got


def check_stats(tree, ins, dim, got, norm_type=0, out_dtype="f32"):
    t = O.decode(tree)
    v, E, unsafe = O.error_bound(t, ins)
    assert not unsafe.any()
    lines_v = v if dim == 0 else v.T           # column k holds line k
    lines_E = E if dim == 0 else E.T
    N = lines_v.shape[0]
    u = 2.0 ** -24 if t.compute == "f32" else 2.0 ** -53
    store = 2.0 ** -24 if out_dtype == "f32" else 2.0 ** -53
    leaf = not np.any(E)
    for name, g in got.items():
        want = O.stats_dim(t, ins, dim, name, norm_type)
        assert g.shape == want.shape, name
        for k in range(want.size):
            o, gk = float(want[k]), float(g[k])
            x, e = lines_v[:, k], lines_E[:, k]
            if math.isnan(o):
                assert math.isnan(gk), (name, k, gk)
                continue
            if math.isinf(o):
                assert gk == o, (name, k, gk, o)
                continue
            if name == "sum":
                tol = sum_tolerance(o, x, e) + abs(o) * store
            elif name == "mean":
                tol = sum_tolerance(o * N, x, e) / N + abs(o) * store
            elif name in ("var", "stddev"):
                d = N - 1 + norm_type
                var_o = o if name == "var" else o * o
                if d == 0:
                    assert gk == 0.0, (name, k, gk)
                    continue
                mu = float(np.mean(x))
                arith = 12.0 * u * float(np.sum((x - x[0]) ** 2)) / d
                elem = (2.0 * float(np.sum(np.abs(x - mu) * e)) + float(np.sum(e * e))) / d
                tol_var = 1e-6 * abs(var_o) + arith + elem + 2.0 * store * abs(var_o)
                if name == "var":
                    tol = tol_var
                else:
                    err = abs(gk * gk - var_o)
                    assert err <= tol_var + 4.0 * store * var_o, (name, k, gk, o, err, tol_var)
                    continue
            else:
                tol = (0.0 if leaf else 2.0 * float(np.max(e))) + (abs(o) * store if t.compute != out_dtype else 0.0)
            assert abs(gk - o) <= tol, f"{name}[{k}] (dim {dim}): got {gk!r}, oracle {o!r}, tol {tol:.3e}"


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (7, 1), (33, 17), (1000, 3), (3, 1000), (4099, 37), (131, 1029)])
@pytest.mark.parametrize("sexpr", [synth.LEAF0, synth.MAT_EXPR])
@pytest.mark.parametrize("dim", [0, 1])
def test_all_six_statistics_match_the_oracle(shape, sexpr, dim):
    r, c = shape
    specs = [_f32(r, c), _f32(r, c), _f32(r, c), _f32(r, c, lo=0.0, hi=2.0)]
    tree, ins, dev = _inputs(sexpr, specs, 211)
    check_stats(tree, ins, dim, run_stats(tree, dev, dim, ALL))


@pytest.mark.parametrize("dim,shape", [(0, (200_003, 3)), (1, (700, 5001))])
def test_split_lines_match_the_oracle(dim, shape):
    """Tall few columns split each column over several warps; short wide
    matrices split each row over several column chunks."""
    r, c = shape
    tree, ins, dev = _inputs(synth.LEAF0, [_f32(r, c)], 223)
    got = run_stats(tree, dev, dim, ALL)
    last = coot.coot_last_launch()
    assert last["split"] > 1, last
    check_stats(tree, ins, dim, got)


@pytest.mark.parametrize("mask", [0x4, 0x8 | 0x10, 0x1 | 0x20, 0x2 | 0x4, 0x10 | 0x20, 0x1])
@pytest.mark.parametrize("norm_type", [0, 1])
def test_subsets_of_statistics_and_norm_type(mask, norm_type):
    r, c = 517, 29
    specs = [_f32(r, c), _f32(r, c), _f32(r, c), _f32(r, c, lo=0.0, hi=2.0)]
    tree, ins, dev = _inputs(synth.MAT_CHAIN, specs, 227)
    for dim in (0, 1):
        check_stats(tree, ins, dim, run_stats(tree, dev, dim, mask, norm_type=norm_type), norm_type)


def test_variance_with_a_large_mean():
    """Values 1000 + U[0, 1]: mean / stddev is about 3500, where the plain
    one-pass formula sum(v^2) - sum(v)^2 / N would lose about ten digits.
    The shifted sums keep the variance within a few units of 1e-7."""
    for dim, (r, c) in ((0, (5000, 7)), (1, (7, 5000))):
        tree, ins, dev = _inputs(synth.LEAF0, [_f32(r, c, lo=1000.0, hi=1001.0)], 229)
        got = run_stats(tree, dev, dim, 0x4 | 0x2, out_dtype="f64")
        check_stats(tree, ins, dim, got, out_dtype="f64")
        want = O.stats_dim(serialize(synth.LEAF0), ins, dim, "var")
        rel = np.max(np.abs(got["var"] - want) / want)
        assert rel < 2e-6, rel


def test_fp64_outputs_with_ld_and_bf16_inputs():
    r, c = 1500, 41
    ins = host_mats([("bf16", r, c, None, 0, 0)], 233)
    tree = serialize(synth.LEAF0)
    dev = [to_dev(ins[0])]
    check_stats(tree, ins, 0, run_stats(tree, dev, 0, ALL, out_dtype="f64", out_ld=3), out_dtype="f64")
    check_stats(tree, ins, 1, run_stats(tree, dev, 1, ALL, out_dtype="f64"), out_dtype="f64")


def test_strided_inputs():
    r, c, ld = 1001, 23, 1013
    specs = [_f32(r, c, ld), _f32(r, c, ld + 8), _f32(r, c), _f32(r, c, lo=0.0, hi=2.0)]
    tree, ins, dev = _inputs(synth.MAT_EXPR, specs, 239)
    for dim in (0, 1):
        check_stats(tree, ins, dim, run_stats(tree, dev, dim, ALL))


def test_fp64_compute():
    r, c = 777, 19
    specs = [("f64", r, c, None, -1.0, 1.0), ("f64", r, c, None, -1.0, 1.0), ("f64", r, c, None, -1.0, 1.0),
             ("f64", r, c, None, 0.0, 2.0)]
    tree, ins, dev = _inputs(synth.MAT_EXPR, specs, 241, compute="f64")
    for dim in (0, 1):
        check_stats(tree, ins, dim, run_stats(tree, dev, dim, ALL, out_dtype="f64"), out_dtype="f64")


def test_degenerate_lines():
    leaf = serialize(synth.LEAF0)
    # one element per column: var 0, mean the value
    ins = host_mats([_f32(1, 9)], 251)
    dev = [to_dev(ins[0])]
    got = run_stats(leaf, dev, 0, ALL)
    assert got["var"].tolist() == [0.0] * 9 and got["stddev"].tolist() == [0.0] * 9
    assert got["mean"].tolist() == O.logical(ins[0]).ravel().tolist()
    check_stats(leaf, ins, 0, run_stats(leaf, dev, 0, 0x4, norm_type=1), norm_type=1)
    # columns of length 0: sums 0, mean / var NaN, min / max refused
    empty = coot.Mat(torch.zeros(8, device="cuda"), 0, 5, 1)
    got = run_stats(leaf, [empty], 0, 0x1 | 0x2 | 0x4)
    assert got["sum"].tolist() == [0.0] * 5
    assert np.isnan(got["mean"]).all() and np.isnan(got["var"]).all()
    with pytest.raises(coot.CootError) as e:
        run_stats(leaf, [empty], 0, 0x10)
    assert e.value.status_name == "COOT_ERR_EMPTY"
    # no lines at all: nothing to do
    assert run_stats(leaf, [empty], 1, ALL)["sum"].size == 0


def test_nan_stays_in_its_line():
    r, c = 300, 6
    a = synth.uniform_f32(257, r * c)
    a[2 * r + 17] = np.nan                   # column 2, row 17
    ins = [synth.as_mat(a, "f32", r, c)]
    leaf = serialize(synth.LEAF0)
    got = run_stats(leaf, [to_dev(ins[0])], 0, ALL)
    for name in NAMES:
        assert np.isnan(got[name][2]), name
        assert not np.isnan(np.delete(got[name], 2)).any(), name
    got = run_stats(leaf, [to_dev(ins[0])], 1, ALL)
    for name in NAMES:
        assert np.isnan(got[name][17]) and np.isnan(got[name]).sum() == 1, name


def test_results_are_reproducible():
    r, c = 20_001, 13
    specs = [_f32(r, c), _f32(r, c), _f32(r, c), _f32(r, c, lo=0.0, hi=2.0)]
    tree, ins, dev = _inputs(synth.MAT_EXPR, specs, 263)
    for dim in (0, 1):
        a = run_stats(tree, dev, dim, ALL)
        b = run_stats(tree, dev, dim, ALL)
        for n in NAMES:
            assert np.array_equal(a[n], b[n], equal_nan=True), n


@pytest.mark.parametrize("kind,block,unroll,split", [(5, 128, 2, 0), (5, 512, 8, 3), (6, 64, 2, 0),
                                                     (6, 256, 8, 5), (6, 512, 4, 1)])
def test_launch_shape_overrides(kind, block, unroll, split):
    r, c = 3001, 211
    specs = [_f32(r, c), _f32(r, c), _f32(r, c), _f32(r, c, lo=0.0, hi=2.0)]
    tree, ins, dev = _inputs(synth.MAT_EXPR, specs, 269)
    coot.coot_set_launch_config(kind, block, 0, unroll, 0, split)
    try:
        got = run_stats(tree, dev, kind - 5, ALL)
        last = coot.coot_last_launch()
        assert last["block"] == min(block, 256) if kind == 6 else last["block"] == block
        assert last["unroll"] == unroll
    finally:
        coot.coot_set_launch_config(kind, 0)
    check_stats(tree, ins, kind - 5, got)


def test_column_blocks_merge_to_the_whole():
    """Three column blocks' statistics computed on the GPU (shard.gpu_local_stats)
    and merged in block order (shard.merge_stats) equal the oracle over the
    whole matrix: the per-rank half of a sharded run."""
    from paper_2308_03120_gb300 import shard
    r, c = 1001, 103
    specs = [_f32(r, c), _f32(r, c), _f32(r, c), _f32(r, c, lo=0.0, hi=2.0)]
    tree, ins, dev = _inputs(synth.MAT_EXPR, specs, 277)
    parts = []
    for k in range(3):
        c0, c1 = shard.column_block(c, k, 3)
        blocks = [m.cols(c0, c1 - 1) for m in dev]
        parts.append(shard.gpu_local_stats(tree, blocks))
    merged = shard.merge_stats(parts, r, 0)
    assert merged["rows"]["sum"].is_cuda        # merged on the device that holds the blocks
    merged = {part: {k: v.cpu().numpy() for k, v in merged[part].items()} for part in ("rows", "cols")}
    for s in NAMES:
        want_rows = O.stats_dim(tree, ins, 1, s)
        np.testing.assert_allclose(merged["rows"][s], want_rows, rtol=2e-6, atol=1e-6, err_msg=s)
        np.testing.assert_allclose(merged["cols"][s], O.stats_dim(tree, ins, 0, s), rtol=2e-6, atol=1e-6, err_msg=s)
