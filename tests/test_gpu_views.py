"""Submatrix views as leaves and as outputs (Table 1: .rows, .cols, .submat,
.row, .col, .diag): every entry point on views of larger matrices against
the oracle on the same views, the elements outside an output view left
untouched, disjoint views of one matrix allowed as in and out, overlapping
ones refused, and batched work lists over views (ld > rows)."""
import numpy as np
import pytest
import torch

import paper_2308_03120_gb300 as coot
import synth
from oracle import coot_oracle as O
from paper_2308_03120_gb300.expr import serialize
from tests.gpu_util import assert_sum_close, check_elementwise

pytestmark = pytest.mark.gpu

X0, X1, C = synth.X(0), synth.X(1), synth.C
R, COLS = 1000, 300


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    yield
    torch.cuda.synchronize()


def _parent(seed, lo=-1.0, hi=1.0):
    h = synth.uniform_f32(seed, R * COLS, lo, hi)
    return h, coot.Mat(torch.from_numpy(h.copy()).cuda(), R, COLS, R)


def _host_view(buf, v: coot.Mat):
    """The oracle's matrix for a view: the parent buffer from the view's
    first element, with the view's shape and ld."""
    return synth.HostMat(np.ascontiguousarray(buf[v.offset:]), "f32", v.n_rows, v.n_cols, v.ld)


def _touched(before, after, v: coot.Mat):
    """Indices of the parent that changed, and whether all lie in view v."""
    changed = np.flatnonzero(before.view(np.uint32) != after.view(np.uint32))
    rel = changed - v.offset
    inside = (rel >= 0) & (rel % v.ld < v.n_rows) & (rel // v.ld < v.n_cols)
    return changed, bool(inside.all())


@pytest.mark.parametrize("view", ["submat", "rows", "cols", "row", "col"])
def test_elementwise_on_views(view):
    ha, A = _parent(601)
    hb, B = _parent(602)
    args = {"submat": (17, 5, 900, 250), "rows": (3, 998), "cols": (11, 299), "row": (37,), "col": (123,)}[view]
    va, vb = getattr(A, view)(*args), getattr(B, view)(*args)
    hout, OUT = _parent(603)
    vo = getattr(OUT, view)(*args)
    tree = serialize(synth.AXPY_2X_3Z)
    coot.coot_expr_eval(tree, [va, vb], vo)
    torch.cuda.synchronize()
    after = OUT.buf.cpu().numpy()
    changed, inside = _touched(hout, after, vo)
    assert inside and changed.size > 0
    check_elementwise(tree, [_host_view(ha, va), _host_view(hb, vb)], _host_view(after, vo))


def test_disjoint_views_of_one_matrix_in_and_out():
    """A.rows(0, 499) = 2 A.rows(500, 999) + A.rows(0, 499) (in place on
    the first half, reading the second)."""
    ha, A = _parent(611)
    top, bottom = A.rows(0, 499), A.rows(500, 999)
    tree = serialize(("add", ("mul", C(2.0), X0), X1))
    coot.coot_expr_eval(tree, [bottom, top], top)
    torch.cuda.synchronize()
    after = A.buf.cpu().numpy()
    check_elementwise(tree, [_host_view(ha, bottom), _host_view(ha, top)], _host_view(after, top))
    assert np.array_equal(after.reshape(COLS, R)[:, 500:], ha.reshape(COLS, R)[:, 500:])
    # an output identical to input 0 that overlaps input 1 (rows 250..749
    # against 0..499) is refused
    with pytest.raises(coot.CootError) as e:
        coot.coot_expr_eval(tree, [A.rows(250, 749), top], A.rows(250, 749))
    assert e.value.status_name == "COOT_ERR_ALIAS"


def test_partially_overlapping_output_is_refused():
    _, A = _parent(612)
    tree = serialize(("mul", C(2.0), X0))
    with pytest.raises(coot.CootError) as e:
        coot.coot_expr_eval(tree, [A.rows(0, 499)], A.rows(250, 749))
    assert e.value.status_name == "COOT_ERR_ALIAS"


def test_reductions_sums_and_statistics_on_views():
    ha, A = _parent(621)
    v = A.submat(100, 20, 899, 279)
    hv = _host_view(ha, v)
    tree = serialize(("add", ("mul", X0, X0), C(0.5)))
    vals, e, _ = O.error_bound(tree, [hv])
    assert_sum_close(coot.coot_accu(tree, [v]).item(), O.accu(tree, [hv]), vals.ravel(), e.ravel(), "accu")
    assert coot.coot_minmax(serialize(X0), [v]).tolist() == list(O.minmax(serialize(X0), [hv]))
    for dim in (0, 1):
        n = v.n_cols if dim == 0 else v.n_rows
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        om = coot.Mat(out, 1, n, 1) if dim == 0 else coot.Mat(out, n, 1, n)
        coot.coot_sum_dim(tree, [v], dim, om)
        got = out.cpu().numpy()
        want = O.sum_dim(tree, [hv], dim)
        terms = vals if dim == 0 else vals.T
        for k in range(n):
            assert_sum_close(got[k], want[k], terms[:, k], np.zeros(terms.shape[0]), f"sum {dim} [{k}]")
        outs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(2)]
        oms = [coot.Mat(t, 1, n, 1) if dim == 0 else coot.Mat(t, n, 1, n) for t in outs]
        coot.coot_stats_dim(serialize(X0), [v], dim, coot.STAT_MEAN | coot.STAT_MAX, oms)
        np.testing.assert_allclose(outs[0].cpu().numpy(), O.stats_dim(serialize(X0), [hv], dim, "mean"),
                                   rtol=1e-6, atol=1e-9)
        assert outs[1].cpu().numpy().tolist() == O.stats_dim(serialize(X0), [hv], dim, "max").tolist()


@pytest.mark.parametrize("k", [0, 5, -7])
def test_diagonal_views(k):
    ha, A = _parent(631)
    d = A.diag(k)
    hd = _host_view(ha, d)
    # accu of the diagonal = trace (k = 0); 2 * diag written into B's diagonal
    leaf = serialize(X0)
    vals = O.logical(hd).ravel()
    assert_sum_close(coot.coot_accu(leaf, [d]).item(), float(np.sum(vals.astype(np.float64))), vals,
                     np.zeros(vals.size), "trace")
    assert vals.size == min(R - max(-k, 0), COLS - max(k, 0))
    hb, B = _parent(632)
    db = B.diag(k)
    tree = serialize(("mul", C(2.0), X0))
    coot.coot_expr_eval(tree, [d], db)
    torch.cuda.synchronize()
    after = B.buf.cpu().numpy()
    changed, inside = _touched(hb, after, db)
    assert inside
    check_elementwise(tree, [hd], _host_view(after, db))


def test_batched_work_lists_over_views():
    """Each batch item is a different window of three large matrices (ld =
    1000): the work list follows every item's ld."""
    ha, A = _parent(641)
    hb, B = _parent(642)
    hc, Cm = _parent(643)
    hout, OUT = _parent(644)
    csum = torch.zeros(64 * COLS, device="cuda")
    windows = [(0, 0, 9, 9), (10, 3, 600, 40), (999, 0, 999, 149), (5, 100, 300, 100), (200, 150, 999, 299),
               (950, 120, 950, 120), (400, 41, 431, 90)]
    items, sums = [], []
    for i, (r0, c0, r1, c1) in enumerate(windows):
        views = [m.submat(r0, c0, r1, c1) for m in (A, B, Cm)]
        cs = coot.Mat(csum, 1, c1 - c0 + 1, 1, i * COLS)
        items.append(coot.batch_item(views, OUT.submat(r0, c0, r1, c1), cs))
        sums.append(cs)
    # the windows are disjoint in OUT
    tree = serialize(synth.BATCH_EXPR)
    plan, n_items, n_work = coot.coot_batch_plan(items, 3)
    coot.coot_expr_eval_batched(tree, [0, 0, 0], 0, 0, plan, n_items, n_work)
    torch.cuda.synchronize()
    after = OUT.buf.cpu().numpy()
    csh = csum.cpu().numpy()
    for i, (r0, c0, r1, c1) in enumerate(windows):
        vo = OUT.submat(r0, c0, r1, c1)
        hv = [_host_view(h, m.submat(r0, c0, r1, c1)) for h, m in ((ha, A), (hb, B), (hc, Cm))]
        check_elementwise(tree, hv, _host_view(after, vo))
        want = O.sum_dim(tree, hv, 0)
        np.testing.assert_allclose(csh[i * COLS:i * COLS + (c1 - c0 + 1)], want, rtol=1e-5, atol=1e-6)
