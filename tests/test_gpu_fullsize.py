"""Parity at the workloads' full sizes, through the same calls and launch
shapes the benchmark times: every stored element, every column and row sum
and the full reductions of the 8192 x 8192 matrix step, sums taken exactly
by the oracle (math.fsum), and the 2^28-element precision workload.  The
oracle works on column blocks so that host memory stays a few GB."""
import math

import numpy as np
import pytest
import torch

import paper_2308_03120_gb300 as coot
import synth
from oracle import coot_oracle as O
from paper_2308_03120_gb300.expr import serialize
from tests.gpu_util import assert_sum_close, check_elementwise

pytestmark = pytest.mark.gpu

N = 8192
BLOCK_COLS = 512


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    yield
    torch.cuda.synchronize()


def _sub(mats, idx_rows, idx_cols):
    """Host sub-matrices (rows idx_rows x cols idx_cols) as dense HostMats."""
    out = []
    for m in mats:
        full = m.buf.reshape(m.n_cols, m.ld).T  # (rows, cols) view of a dense column-major buffer
        blk = np.ascontiguousarray(full[np.ix_(idx_rows, idx_cols)].ravel(order="F"))
        out.append(synth.as_mat(blk, m.dtype, len(idx_rows), len(idx_cols)))
    return out


def test_matrix_workload_8192():
    """(A % B + 2C) / (1 + abs(D)) with accu, norm2, min, max in one pass,
    the exp/sqrt chain, and sum(out, 0), sum(out, 1): the benchmark step."""
    seed = synth.BASE_SEED + 1
    host = [synth.as_mat(synth.uniform_f32(seed + k, N * N, 0.0 if k == 3 else -1.0, 2.0 if k == 3 else 1.0),
                         "f32", N, N) for k in range(4)]
    dev = [coot.Mat(torch.from_numpy(h.buf).cuda(), N, N, N) for h in host]
    t_expr = serialize(synth.MAT_EXPR)
    t_chain = serialize(synth.MAT_CHAIN)
    leaf = serialize(synth.LEAF0)
    out1 = torch.empty(N * N, device="cuda")
    out2 = torch.empty(N * N, device="cuda")
    col = torch.empty(N, device="cuda")
    row = torch.empty(N, device="cuda")
    ws = coot.Workspace(N)
    O1 = coot.Mat(out1, N, N, N)
    res = coot.coot_expr_reduce(t_expr, dev, coot.HEAD_SUM | coot.HEAD_NORM2 | coot.HEAD_MIN | coot.HEAD_MAX,
                                out=O1, ws=ws)
    coot.coot_expr_eval(t_chain, dev, coot.Mat(out2, N, N, N), ws=ws)
    coot.coot_sum_dim(leaf, [O1], 0, coot.Mat(col, 1, N, 1), ws=ws)
    coot.coot_sum_dim(leaf, [O1], 1, coot.Mat(row, N, 1, N), ws=ws)
    torch.cuda.synchronize()
    s, n2, lo, hi = res.tolist()

    # every result over all 67M elements, evaluated by column blocks: the
    # full reductions, every column sum, every row sum (exact per-block
    # partials of each row, then their sum) and every element of both
    # stored trees
    allr = np.arange(N)
    o1 = out1.view(N, N).T.cpu().numpy()  # (rows, cols)
    o2m = out2.view(N, N).T.cpu().numpy()
    gc = col.cpu().numpy().astype(np.float64)
    gr = row.cpu().numpy().astype(np.float64)
    vals, sq, e2, s_abs = [], [], 0.0, 0.0
    olo, ohi, emax = math.inf, -math.inf, 0.0
    row_part = np.zeros((N // BLOCK_COLS, N))
    row_abs, row_e2 = np.zeros(N), np.zeros(N)
    for b, c0 in enumerate(range(0, N, BLOCK_COLS)):
        cidx = np.arange(c0, c0 + BLOCK_COLS)
        blk = _sub(host, allr, cidx)
        v, bound, unsafe = O.error_bound(t_expr, blk)
        assert not unsafe.any()
        vals.append(v.ravel())
        sq.append((v * v).ravel())
        s_abs += float(np.sum(np.abs(v)))
        e2 += float(np.sum(bound * bound))
        emax = max(emax, float(bound.max()))
        r32 = O.round_to_format(v, "f32")
        olo, ohi = min(olo, float(r32.min())), max(ohi, float(r32.max()))
        # the stored tree: within 1e-5 |v| + 2 E of the oracle, element by element
        err = np.abs(o1[:, cidx].astype(np.float64) - v)
        assert np.all(err <= 1e-5 * np.abs(v) + 2.0 * bound), f"stored tree, columns {c0}.."
        # the sums take the stored FP32 values: each term's bound grows by
        # its own rounding to FP32
        errs = np.hypot(bound, v * 2.0 ** -24)
        want_c = np.array([O._fsum(v[:, j]) for j in range(BLOCK_COLS)])
        abs_c = np.sum(np.abs(v), axis=0)
        tol = 1e-6 * np.abs(want_c) + np.where(np.abs(want_c) < 1e-3 * abs_c, 1e-9 * abs_c, 0.0)
        tol += 6.0 * np.sqrt(np.sum(errs * errs, axis=0))
        bad = np.abs(gc[cidx] - want_c) > tol
        assert not bad.any(), f"column sums {cidx[bad][:4]}"
        row_part[b] = [O._fsum(v[i, :]) for i in range(N)]
        row_abs += np.sum(np.abs(v), axis=1)
        row_e2 += np.sum(errs * errs, axis=1)
        # the exp/sqrt chain, stored: the oracle's own tolerance
        got2 = np.ascontiguousarray(o2m[:, cidx].ravel(order="F"))
        check_elementwise(t_chain, blk, synth.as_mat(got2, "f32", N, BLOCK_COLS))
    # (the tolerance needs only sum |t| and sqrt(sum E^2))
    assert_sum_close(s, O._fsum(vals), np.array([s_abs]), np.array([math.sqrt(e2)]), "accu")
    o2 = math.sqrt(O._fsum(sq))
    assert abs(n2 - o2) <= 1e-6 * o2
    assert abs(lo - olo) <= 2 * emax and abs(hi - ohi) <= 2 * emax
    del vals, sq
    want_r = np.array([O._fsum(row_part[:, i]) for i in range(N)])
    tol = 1e-6 * np.abs(want_r) + np.where(np.abs(want_r) < 1e-3 * row_abs, 1e-9 * row_abs, 0.0)
    tol += 6.0 * np.sqrt(row_e2)
    bad = np.abs(gr - want_r) > tol
    assert not bad.any(), f"row sums {np.nonzero(bad)[0][:4]}"


@pytest.mark.parametrize("dt", ["bf16", "f16"])
def test_precision_workload_2_28(dt):
    """n = 2^28 stored as BF16 / FP16: y = 2x + 3z stored in the same type,
    accu(x) and norm2(x) in one pass, dot(x, z); the error of each result
    against the FP64 oracle is printed."""
    n = 1 << 28
    seed = synth.BASE_SEED + 2
    hx, rx = synth.lognormal_signed(seed, n, dt)
    hz, rz = synth.lognormal_signed(seed + 1, n, dt)
    tdt = torch.bfloat16 if dt == "bf16" else torch.float16

    def dev(h):
        return (torch.from_numpy(h.view(np.int16)).view(tdt) if dt == "bf16" else torch.from_numpy(h)).cuda()
    x, z = dev(hx), dev(hz)
    y = torch.empty(n, dtype=tdt, device="cuda")
    X, Z = coot.Mat(x, n, 1, n), coot.Mat(z, n, 1, n)
    ws = coot.Workspace(1)
    coot.coot_expr_eval(serialize(synth.AXPY_2X_3Z), [X, Z], coot.Mat(y, n, 1, n))
    r = coot.coot_expr_reduce(serialize(synth.LEAF0), [X], coot.HEAD_SUM | coot.HEAD_NORM2, ws=ws).tolist()
    d = coot.coot_dot(X, Z, ws=ws).item()
    torch.cuda.synchronize()

    step = 1 << 24
    chunks = range(0, n, step)
    vx = lambda i: O.decode_storage(hx[i:i + step], dt)  # noqa: E731
    vz = lambda i: O.decode_storage(hz[i:i + step], dt)  # noqa: E731
    acc = O._fsum(vx(i) for i in chunks)
    # magnitudes for the tolerance only: an ordinary FP64 sum is accurate enough
    s_abs = float(sum(np.sum(np.abs(vx(i))) for i in chunks))
    nrm = math.sqrt(O._fsum(vx(i) ** 2 for i in chunks))
    dot = O._fsum(vx(i) * vz(i) for i in chunks)
    s_abs_dot = float(sum(np.sum(np.abs(vx(i) * vz(i))) for i in chunks))
    sq_dot = float(sum(np.sum((vx(i) * vz(i)) ** 2) for i in chunks))
    print(f"\n{dt} n=2^28 (FP16 redraws {rx}+{rz}): accu rel err {abs(r[0] - acc) / abs(acc):.3e}, "
          f"norm2 rel err {abs(r[1] - nrm) / nrm:.3e}, dot rel err {abs(d - dot) / abs(dot):.3e}")
    # sums of exactly representable terms: 1e-6 |o|, or the cancellation floor
    for got, want, sabs, what in ((r[0], acc, s_abs, "accu"), (d, dot, s_abs_dot, "dot")):
        tol = 1e-6 * abs(want) + (1e-9 * sabs if abs(want) < 1e-3 * sabs else 0.0)
        if what == "dot":
            tol += 6.0 * 2.0 ** -24 * math.sqrt(sq_dot)  # FP32 rounding of each product
        assert abs(got - want) <= tol, (what, got, want, tol)
    assert abs(r[1] - nrm) <= 1e-6 * nrm

    # sampled elements of y
    idx = np.sort(np.random.default_rng(2).choice(n, 1 << 20, replace=False))
    ins = [synth.as_mat(hx[idx], dt, idx.size, 1), synth.as_mat(hz[idx], dt, idx.size, 1)]
    yh = y.cpu()
    yb = (yh.view(torch.int16).numpy().view(np.uint16) if dt == "bf16" else yh.numpy())[idx]
    rep = check_elementwise(serialize(synth.AXPY_2X_3Z), ins, synth.as_mat(yb, dt, idx.size, 1))
    print(f"{dt} 2x+3z: {rep}")


@pytest.mark.parametrize("sexpr", [synth.LEAF0, synth.MAT_EXPR])
def test_statistics_workload_8192(sexpr):
    """All six statistics of every column and every row of the 8192 x 8192
    inputs (a stored matrix, and the four-input tree), at the launch shapes
    the benchmark times; 48 sampled columns and 48 sampled rows (the first
    and last included) are checked against the oracle with the tolerances
    of the statistics tests."""
    from tests.test_gpu_stats import NAMES, check_stats
    seed = synth.BASE_SEED + 1
    n_in = synth.tree_inputs(sexpr)
    host = [synth.as_mat(synth.uniform_f32(seed + k, N * N, 0.0 if k == 3 else -1.0, 2.0 if k == 3 else 1.0),
                         "f32", N, N) for k in range(n_in)]
    dev = [coot.Mat(torch.from_numpy(h.buf).cuda(), N, N, N) for h in host]
    tree = serialize(sexpr)
    ws = coot.Workspace(N)
    rng = np.random.default_rng(11)
    for dim in (0, 1):
        outs = [torch.empty(N, device="cuda") for _ in NAMES]
        mats = [coot.Mat(t, 1, N, 1) if dim == 0 else coot.Mat(t, N, 1, N) for t in outs]
        coot.coot_stats_dim(tree, dev, dim, 0x3F, mats, ws=ws)
        torch.cuda.synchronize()
        idx = np.unique(np.concatenate([[0, N - 1], rng.choice(N, 46, replace=False)]))
        got = {name: outs[b].cpu().numpy()[idx].astype(np.float64) for b, name in enumerate(NAMES)}
        every = np.arange(N)
        sub = _sub(host, every, idx) if dim == 0 else _sub(host, idx, every)
        check_stats(tree, sub, dim, got)


def test_views_workload_8192():
    """The views workload: the matrix tree over the 6144 x 6144 window at
    (1024, 1024) of the 8192 x 8192 inputs (ld 8192), stored into the same
    window of an output whose other elements must stay untouched, then the
    column and row sums of the stored window, at the benchmark's launch
    shapes; sampled lines and elements against the oracle."""
    seed = synth.BASE_SEED + 1
    host = [synth.as_mat(synth.uniform_f32(seed + k, N * N, 0.0 if k == 3 else -1.0, 2.0 if k == 3 else 1.0),
                         "f32", N, N) for k in range(4)]
    full = [coot.Mat(torch.from_numpy(h.buf).cuda(), N, N, N) for h in host]
    w0, w1 = N // 8, N - N // 8 - 1
    n = w1 - w0 + 1
    mats = [m.submat(w0, w0, w1, w1) for m in full]
    out = torch.full((N * N,), float("nan"), device="cuda")
    O1 = coot.Mat(out, N, N, N).submat(w0, w0, w1, w1)
    col = torch.empty(n, device="cuda")
    row = torch.empty(n, device="cuda")
    ws = coot.Workspace(n)
    t_expr = serialize(synth.MAT_EXPR)
    leaf = serialize(synth.LEAF0)
    coot.coot_expr_eval(t_expr, mats, O1)
    coot.coot_sum_dim(leaf, [O1], 0, coot.Mat(col, 1, n, 1), ws=ws)
    coot.coot_sum_dim(leaf, [O1], 1, coot.Mat(row, n, 1, n), ws=ws)
    torch.cuda.synchronize()
    o = out.view(N, N).T.cpu().numpy()  # (rows, cols)
    assert np.isnan(o[:w0, :]).all() and np.isnan(o[w1 + 1:, :]).all()
    assert np.isnan(o[:, :w0]).all() and np.isnan(o[:, w1 + 1:]).all()

    rng = np.random.default_rng(3)
    win = np.arange(w0, w1 + 1)
    ri = np.unique(np.concatenate([[w0, w1], rng.choice(win, 62, replace=False)]))
    ci = np.unique(np.concatenate([[w0, w1], rng.choice(win, 62, replace=False)]))
    # sums of the stored window: the oracle's tree values, each with its
    # error bound and the FP32 rounding of the store
    vc, bc, unsafe = O.error_bound(t_expr, _sub(host, win, ci))
    assert not unsafe.any()
    gc = col.cpu().numpy()[ci - w0].astype(np.float64)
    for k in range(len(ci)):
        assert_sum_close(gc[k], O._fsum(vc[:, k]), vc[:, k], np.hypot(bc[:, k], vc[:, k] * 2.0 ** -24),
                         f"column {ci[k]}")
    vr, br, unsafe = O.error_bound(t_expr, _sub(host, ri, win))
    assert not unsafe.any()
    gr = row.cpu().numpy()[ri - w0].astype(np.float64)
    for k in range(len(ri)):
        assert_sum_close(gr[k], O._fsum(vr[k, :]), vr[k, :], np.hypot(br[k, :], vr[k, :] * 2.0 ** -24),
                         f"row {ri[k]}")
    got = np.ascontiguousarray(o[np.ix_(ri, ci)].ravel(order="F"))
    check_elementwise(t_expr, _sub(host, ri, ci), synth.as_mat(got, "f32", len(ri), len(ci)))


def test_convert_workload_8192():
    """The conversion workload: B = 2 A + 1 with A an 8192 x 8192 int32
    matrix (values in [-1e6, 1e6)) and B FP32, fused in one kernel and in
    two steps (convert into an FP32 temporary, then evaluate).  Every result
    is an integer below 2^24 in magnitude, so both paths must give 2 A + 1
    exactly, element for element."""
    u = synth.uniform01(synth.BASE_SEED + 5, N * N)
    ha = np.floor(-1e6 + u * 2e6).astype(np.int32)
    want = (2.0 * ha.astype(np.float64) + 1.0).astype(np.float32)
    a = torch.from_numpy(ha).cuda()
    tmp = torch.empty(N * N, device="cuda")
    out = torch.empty(N * N, device="cuda")
    A, T, B = (coot.Mat(t, N, N, N) for t in (a, tmp, out))
    expr = serialize(("add", ("mul", synth.C(2.0), synth.X(0)), synth.C(1.0)))
    coot.coot_expr_eval(expr, [A], B)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want)
    out.fill_(float("nan"))
    coot.coot_expr_eval(serialize(synth.LEAF0), [A], T)
    coot.coot_expr_eval(expr, [T], B)
    torch.cuda.synchronize()
    assert np.array_equal(tmp.cpu().numpy(), ha.astype(np.float32))
    assert np.array_equal(out.cpu().numpy(), want)
