"""Parity at the workloads' full sizes, through the same calls and launch
shapes the benchmark times: sampled outputs the oracle computes one by one,
and full reductions the oracle computes exactly (math.fsum).  The oracle
works on column blocks so that host memory stays a few GB."""
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

    # full reductions over all 67M elements, evaluated by column blocks
    allr = np.arange(N)
    vals, sq, e2, s_abs = [], [], 0.0, 0.0
    olo, ohi, emax = math.inf, -math.inf, 0.0
    row_blocks = []
    for c0 in range(0, N, BLOCK_COLS):
        blk = _sub(host, allr, np.arange(c0, c0 + BLOCK_COLS))
        v, bound, unsafe = O.error_bound(t_expr, blk)
        assert not unsafe.any()
        vals.append(v.ravel())
        sq.append((v * v).ravel())
        s_abs += float(np.sum(np.abs(v)))
        e2 += float(np.sum(bound * bound))
        emax = max(emax, float(bound.max()))
        r32 = O.round_to_format(v, "f32")
        olo, ohi = min(olo, float(r32.min())), max(ohi, float(r32.max()))
        row_blocks.append((v, bound))
    # (the tolerance needs only sum |t| and sqrt(sum E^2))
    assert_sum_close(s, O._fsum(vals), np.array([s_abs]), np.array([math.sqrt(e2)]), "accu")
    o2 = math.sqrt(O._fsum(sq))
    assert abs(n2 - o2) <= 1e-6 * o2
    assert abs(lo - olo) <= 2 * emax and abs(hi - ohi) <= 2 * emax
    del vals, sq

    # sampled row sums: the oracle's row sums over every column block
    rng = np.random.default_rng(1)
    ri = np.sort(rng.choice(N, 64, replace=False))
    ci = np.sort(rng.choice(N, 64, replace=False))
    gr = row.cpu().numpy()[ri].astype(np.float64)
    for k, i in enumerate(ri):
        terms = np.concatenate([v[i, :] for v, _ in row_blocks])
        errs = np.concatenate([np.hypot(b[i, :], v[i, :] * 2.0 ** -24) for v, b in row_blocks])
        assert_sum_close(gr[k], O._fsum(terms), terms, errs, f"row {i}")
    del row_blocks

    # sampled column sums
    cols = _sub(host, allr, ci)
    want = O.sum_dim(t_expr, cols, 0)
    vb, bb, _ = O.error_bound(t_expr, cols)
    gc = col.cpu().numpy()[ci].astype(np.float64)
    for k in range(len(ci)):
        assert_sum_close(gc[k], want[k], vb[:, k], np.hypot(bb[:, k], vb[:, k] * 2.0 ** -24), f"column {ci[k]}")

    # sampled elements of both stored results
    sub = _sub(host, ri, ci)
    o1 = out1.view(N, N).T.cpu().numpy()  # (rows, cols)
    o2m = out2.view(N, N).T.cpu().numpy()
    for tree, stored in ((t_expr, o1), (t_chain, o2m)):
        got = np.ascontiguousarray(stored[np.ix_(ri, ci)].ravel(order="F"))
        check_elementwise(tree, sub, synth.as_mat(got, "f32", len(ri), len(ci)))


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
