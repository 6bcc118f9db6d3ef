"""GPU parity of Table 7's pow, log10 and trigonometric functions, of the
integer storage types (read into FP32 / FP64 trees, and stored with
truncation and saturation) and of the unfused baseline on the new nodes,
against the FP64 oracle.  Element-wise tolerances are those of gpu_util
(the oracle's error bound uses the documented ulp figures of CUDA's
functions, taken at their upper end); integer outputs must equal the
oracle's truncation wherever the element's error interval does not straddle
an integer boundary."""
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


def _spec(dt, r, c, lo, hi):
    return (dt, r, c, None, lo, hi)


# (tree, range of x0, range of x1)
OP_CASES = [
    (("sin", X0), (-10.0, 10.0), None),
    (("cos", X0), (-10.0, 10.0), None),
    (("tan", X0), (-1.5, 1.5), None),
    (("tan", X0), (-30.0, 30.0), None),
    (("asin", X0), (-1.0, 1.0), None),
    (("acos", X0), (-1.0, 1.0), None),
    (("atan", X0), (-50.0, 50.0), None),
    (("log10", X0), (0.0, 100.0), None),
    (("pow", X0, X1), (0.0, 4.0), (-3.0, 3.0)),
    (("pow", X0, C(3.0)), (-2.0, 2.0), None),
    (("pow", X0, C(0.5)), (-1.0, 1.0), None),               # negative bases give NaN
    (("add", ("sin", ("mul", X0, X1)), ("cos", X0)), (-3.0, 3.0), (-3.0, 3.0)),
    (("atan", ("div", X0, X1)), (-1.0, 1.0), (-1.0, 1.0)),
    (("pow", ("add", ("abs", X0), C(0.5)), X1), (-2.0, 2.0), (-2.0, 2.0)),
    (("mul", ("log10", ("add", C(1.0), ("abs", X0))), ("asin", ("mul", C(0.5), X1))), (-9.0, 9.0), (-1.0, 1.0)),
]


@pytest.mark.parametrize("case", range(len(OP_CASES)))
@pytest.mark.parametrize("compute", ["f32", "f64"])
def test_table7_functions_elementwise(case, compute):
    sexpr, r0, r1 = OP_CASES[case]
    n = 300_007
    dt = "f32" if compute == "f32" else "f64"
    specs = [_spec(dt, n, 1, *r0)] + ([_spec(dt, n, 1, *r1)] if r1 else [])
    ins = host_mats(specs, 401 + case)
    n_in = synth.tree_inputs(sexpr)
    tree = serialize(sexpr, compute=compute, n_inputs=n_in)
    out = Out(n, 1, dt)
    coot.coot_expr_eval(tree, [to_dev(h) for h in ins[:n_in]], out.mat)
    torch.cuda.synchronize()
    out.check()
    rep = check_elementwise(tree, ins[:n_in], out.host(), max_skip_frac=0.01)
    if sexpr[0] in ("sin", "cos", "asin", "acos", "atan", "log10") and sexpr[1] == X0:
        assert rep["skipped"] == 0


def test_table7_functions_in_reductions_and_sums():
    r, c = 3001, 57
    ins = host_mats([_spec("f32", r, c, -2.0, 2.0), _spec("f32", r, c, -2.0, 2.0)], 421)
    dev = [to_dev(h) for h in ins]
    tree = serialize(("add", ("sin", ("mul", X0, X1)), ("pow", ("add", C(1.0), ("abs", X0)), X1)))
    v, e, unsafe = O.error_bound(tree, ins)
    assert not unsafe.any()
    assert_sum_close(coot.coot_accu(tree, dev).item(), O.accu(tree, ins), v.ravel(), e.ravel(), "accu")
    col = Out(1, c)
    coot.coot_sum_dim(tree, dev, 0, col.mat)
    torch.cuda.synchronize()
    got = O.logical(col.host()).ravel()
    want = O.sum_dim(tree, ins, 0)
    for k in range(c):
        assert_sum_close(got[k], want[k], v[:, k], e[:, k], f"column {k}")


def _int_mat(seed, n, dtype, lo, hi):
    u = synth.uniform01(seed, n)
    a = np.floor(lo + u * (hi - lo))
    return synth.as_mat(a.astype(np.int32 if dtype == "i32" else np.uint32), dtype, n, 1)


def _int_dev(h):
    t = torch.from_numpy(h.buf.view(np.int32).copy())
    if h.dtype == "u32":
        t = t.view(torch.uint32)
    return coot.Mat(t.cuda(), h.n_rows, h.n_cols, h.ld)


@pytest.mark.parametrize("dtype,lo,hi", [("i32", -2.0 ** 31, 2.0 ** 31), ("i32", -1000.0, 1000.0),
                                         ("u32", 0.0, 2.0 ** 32)])
@pytest.mark.parametrize("compute", ["f32", "f64"])
def test_integer_inputs(dtype, lo, hi, compute):
    """Integers are rounded to the nearest FP32 on load for an FP32 tree
    (exact below 2^24) and are exact in FP64; the fused conversion feeds
    the tree and the reductions directly."""
    n = 200_003
    h = _int_mat(431, n, dtype, lo, hi)
    dev = [_int_dev(h)]
    tree = serialize(("add", ("mul", C(2.0), X0), C(1.0)), compute=compute)
    out_dt = "f32" if compute == "f32" else "f64"
    out = Out(n, 1, out_dt)
    coot.coot_expr_eval(tree, dev, out.mat)
    torch.cuda.synchronize()
    out.check()
    check_elementwise(tree, [h], out.host())
    leaf = serialize(X0, compute=compute)
    v, e, _ = O.error_bound(leaf, [h])
    assert_sum_close(coot.coot_accu(leaf, dev).item(), O.accu(leaf, [h]), v.ravel(), e.ravel(), "accu")
    lo_g, hi_g = coot.coot_minmax(leaf, dev).tolist()
    assert (lo_g, hi_g) == O.minmax(leaf, [h])


def _check_integer_output(tree, ins, g, dtype):
    t = O.decode(tree)
    v, e, unsafe = O.error_bound(t, ins)
    v, e, unsafe = v.ravel(), e.ravel(), unsafe.ravel()
    want = O.to_integer(v, dtype)
    # the truncation is certain when both ends of the error interval
    # truncate (and saturate) to the same integer
    certain = ~unsafe & ((np.isnan(v)) | (O.to_integer(v - e, dtype) == O.to_integer(v + e, dtype)))
    assert certain.mean() > 0.97, certain.mean()
    bad = certain & (g != want)
    assert not bad.any(), (np.flatnonzero(bad)[:5], g[bad][:5], want[bad][:5])


@pytest.mark.parametrize("dtype", ["i32", "u32"])
@pytest.mark.parametrize("compute", ["f32", "f64"])
def test_integer_outputs_truncate_and_saturate(dtype, compute):
    n = 100_003
    ins = host_mats([_spec("f32", n, 1, -1000.0, 1000.0)], 441)
    a = ins[0].buf.copy()
    a[::997] = np.nan
    a[5], a[6] = np.inf, -np.inf
    a[7], a[8] = 1e12, -1e12                   # far outside both ranges: saturate
    a[9], a[10] = 7e8, -7e8                    # x 3.5 + 0.25: beyond int32, inside uint32 for the positive
    ins = [synth.as_mat(a, "f32", n, 1)]
    tree = serialize(("add", ("mul", X0, C(3.5)), C(0.25)), compute=compute)
    tdt = torch.int32 if dtype == "i32" else torch.uint32
    out = torch.full((n,), 12345, dtype=torch.int32, device="cuda").view(tdt)
    coot.coot_expr_eval(tree, [to_dev(ins[0])], coot.Mat(out, n, 1, n))
    torch.cuda.synchronize()
    raw = out.view(torch.int32).cpu().numpy()
    g = raw.astype(np.float64) if dtype == "i32" else raw.view(np.uint32).astype(np.float64)
    _check_integer_output(tree, ins, g, dtype)
    assert g[5] == (2.0 ** 31 - 1 if dtype == "i32" else 2.0 ** 32 - 1) and g[0] == 0.0  # inf saturates, NaN -> 0


def test_integer_sums_are_refused():
    h = _int_mat(451, 64, "i32", 0, 10)
    dev = [_int_dev(h)]
    out = coot.Mat(torch.zeros(1, dtype=torch.int32, device="cuda"), 1, 1, 1)
    with pytest.raises(coot.CootError) as e:
        coot.coot_sum_dim(serialize(X0), dev, 0, out)
    assert e.value.status_name == "COOT_ERR_DTYPE"


@pytest.mark.parametrize("sexpr", [("sin", ("mul", X0, X1)), ("pow", ("add", C(1.0), ("abs", X0)), X1),
                                   ("add", ("lt", X0, X1), ("atan", X0)), ("log10", ("add", C(2.0), X0))])
def test_unfused_baseline_matches_on_the_new_nodes(sexpr):
    r, c = 1023, 77
    ins = host_mats([_spec("f32", r, c, -1.0, 1.0), _spec("f32", r, c, -1.0, 1.0)], 461)
    n_in = synth.tree_inputs(sexpr)
    tree = serialize(sexpr, n_inputs=n_in)
    out = Out(r, c)
    coot.coot_unfused_eval(tree, [to_dev(h) for h in ins[:n_in]], out.mat)
    torch.cuda.synchronize()
    out.check()
    check_elementwise(tree, ins[:n_in], out.host())


def test_bf16_inputs_through_trig():
    h = host_mats([("bf16", 65_536, 3, None, 0, 0)], 471)
    tree = serialize(("atan", X0))
    out = Out(65_536, 3, "bf16")
    coot.coot_expr_eval(tree, [to_dev(h[0])], out.mat)
    torch.cuda.synchronize()
    check_elementwise(tree, h, out.host())
