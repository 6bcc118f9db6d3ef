"""Helpers of the GPU parity tests: moving seeded host matrices to the
device (optionally misaligned), guarded output buffers, and the comparisons
against the FP64 oracle with their tolerances.

Tolerances (FP32 compute):
  * element-wise: |g - o| <= 1e-5 |o| + 2 E, where E is the oracle's
    first-order bound on the FP32 evaluation error of that element (zero for
    a leaf, a few units of roundoff times the operands for a well-conditioned
    tree); elements where the bound says nothing (an intermediate beyond the
    FP32 range, a log/sqrt/division operand whose error interval touches the
    domain edge) are skipped and counted;
  * stored in BF16 / FP16 (or FP32 from FP64 compute): the oracle value
    rounded to the storage type, with at most one storage ulp of difference
    and at least 99.9% of elements exact;
  * sums of n elements: 1e-6 |o|; when |o| < 1e-3 sum|t| (cancellation) the
    floor 1e-9 sum|t| is added; plus 6 sqrt(sum E_i^2), six standard
    deviations of the sum of independent element rounding errors of size at
    most E_i;
  * min / max: exact for leaves; for trees within 2 max E_i.
"""
from __future__ import annotations

import math

import numpy as np
import torch

import paper_2308_03120_gb300 as coot
import synth
from oracle import coot_oracle as O

TORCH_DT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16, "f64": torch.float64}
NP_DT = {"f32": np.float32, "bf16": np.uint16, "f16": np.float16, "f64": np.float64}
GUARD = 64


def _to_torch(buf: np.ndarray, dtype: str) -> torch.Tensor:
    if dtype == "bf16":
        return torch.from_numpy(buf.view(np.int16).copy()).view(torch.bfloat16)
    if dtype == "f16":
        return torch.from_numpy(buf.view(np.float16).copy())
    return torch.from_numpy(np.ascontiguousarray(buf))


def to_dev(h: synth.HostMat, offset: int = 0) -> coot.Mat:
    """Device copy of a host matrix; `offset` elements of padding in front
    make the data pointer misaligned by that many elements."""
    t = _to_torch(h.buf, h.dtype)
    if offset:
        pad = torch.zeros(offset, dtype=t.dtype)
        t = torch.cat([pad, t])
    return coot.Mat(t.cuda(), h.n_rows, h.n_cols, h.ld, offset)


class Out:
    """An output matrix inside a buffer with guard bands; every element of
    the buffer starts as a sentinel, and check() verifies the guards and the
    padding rows were left alone."""

    def __init__(self, n_rows, n_cols, dtype="f32", ld=None, offset=0):
        self.dtype = dtype
        self.n_rows, self.n_cols = n_rows, n_cols
        self.ld = max(n_rows, 1) if ld is None else ld
        size = self.ld * n_cols if n_rows * n_cols else 0
        self.lo = GUARD + offset
        total = self.lo + size + GUARD
        self.t = torch.empty(total, dtype=TORCH_DT[dtype], device="cuda")
        self.t.view(torch.uint8).fill_(0x7F)
        self.mat = coot.Mat(self.t, n_rows, n_cols, self.ld, self.lo)
        self.size = size

    def host(self) -> synth.HostMat:
        t = self.t.cpu()
        if self.dtype == "bf16":
            buf = t.view(torch.int16).numpy().view(np.uint16)
        else:
            buf = t.numpy()
        return synth.HostMat(buf[self.lo:self.lo + self.size].copy(), self.dtype, self.n_rows, self.n_cols, self.ld)

    def check(self):
        raw = self.t.view(torch.uint8).cpu().numpy()
        es = self.t.element_size()
        assert np.all(raw[:self.lo * es] == 0x7F), "guard band before the output was written"
        assert np.all(raw[(self.lo + self.size) * es:] == 0x7F), "guard band after the output was written"
        if self.ld > self.n_rows and self.n_cols and self.size:
            body = raw[self.lo * es:(self.lo + self.size) * es].reshape(self.n_cols, self.ld * es)
            assert np.all(body[:, self.n_rows * es:] == 0x7F), "padding rows were written"


def ulp_of(v: np.ndarray, fmt: str) -> np.ndarray:
    p, emin, emax = O.FORMATS[fmt]
    a = np.abs(v)
    _, ex = np.frexp(np.where(a > 0, a, 1.0))
    e = np.maximum(ex - 1, emin)
    return np.ldexp(1.0, e - (p - 1))


def check_elementwise(tree: bytes, ins, out: synth.HostMat, max_skip_frac=0.02):
    """Compare a stored element-wise result with the oracle (see module
    docstring).  Returns a small report dict."""
    t = O.decode(tree)
    v, bound, unsafe = O.error_bound(t, ins)
    g = O.logical(out)
    assert g.shape == v.shape
    safe = ~unsafe
    n = v.size
    report = {"n": n, "skipped": int(unsafe.sum())}
    assert unsafe.sum() <= max_skip_frac * max(n, 1) + 2, report
    compute = t.compute
    same_type = (out.dtype == compute)
    nan_v, nan_g = np.isnan(v), np.isnan(g)
    assert np.array_equal(nan_v[safe], nan_g[safe]), "NaN pattern differs"
    inf_v = np.isinf(v) & safe
    assert np.array_equal(v[inf_v], g[inf_v]), "infinities differ"
    fin = safe & np.isfinite(v)
    if same_type:
        rel = 1e-5 if compute == "f32" else 1e-13
        # the oracle's own FP64 rounding matters only for FP64 compute
        own = 0.0 if compute == "f32" else 4e-16 * np.abs(v[fin])
        err = np.abs(g[fin] - v[fin])
        tol = rel * np.abs(v[fin]) + 2.0 * bound[fin] + own
        bad = err > tol
        report["max_rel"] = float(np.max(err / np.maximum(np.abs(v[fin]), 1e-300))) if err.size else 0.0
        report["outside_pure_rel"] = int(np.sum(err > rel * np.abs(v[fin])))
        assert not bad.any(), (f"{int(bad.sum())} elements outside tolerance; worst at "
                               f"{np.argmax(err - tol)}: got {g[fin][np.argmax(err - tol)]} "
                               f"want {v[fin][np.argmax(err - tol)]}")
    else:
        ref = O.round_to_format(v, out.dtype)
        fin2 = fin & np.isfinite(ref)
        diff = np.abs(g[fin2] - ref[fin2])
        ulp = ulp_of(ref[fin2], out.dtype)
        assert np.all(diff <= ulp * 1.0000001), "more than one storage ulp off"
        exact = float(np.mean(diff == 0)) if diff.size else 1.0
        report["exact_frac"] = exact
        assert exact >= 0.999, report
        ovf = fin & ~np.isfinite(ref)
        assert np.all(np.isinf(g[ovf]) | (np.abs(g[ovf]) >= np.finfo(np.float16).max)), "overflow differs"
    return report


def sum_tolerance(o: float, terms: np.ndarray, errs: np.ndarray) -> float:
    """Tolerance of a GPU sum against the oracle's (module docstring)."""
    s_abs = float(np.sum(np.abs(terms)))
    tol = 1e-6 * abs(o)
    if abs(o) < 1e-3 * s_abs:
        tol += 1e-9 * s_abs
    tol += 6.0 * math.sqrt(float(np.sum(errs * errs)))
    return tol


def assert_sum_close(g: float, o: float, terms, errs, what=""):
    if math.isnan(o):
        assert math.isnan(g), what
        return
    if math.isinf(o):
        assert g == o, what
        return
    tol = sum_tolerance(o, terms, errs)
    assert abs(g - o) <= tol, f"{what}: got {g!r}, oracle {o!r}, |diff| {abs(g - o):.3e} > tol {tol:.3e}"


def check_dim_sums(tree: bytes, ins, dim: int, got: np.ndarray, what: str = ""):
    """Sums along dim (0: each column, 1: each row), stored in FP32, against
    the oracle's: the sum tolerance of each line over its terms, plus one
    FP32 rounding of the result."""
    v, bound, unsafe = O.error_bound(tree, ins)
    assert not unsafe.any()
    want = O.sum_dim(tree, ins, dim)
    assert got.shape == want.shape, (got.shape, want.shape)
    terms = v if dim == 0 else v.T          # column k of `terms` feeds result k
    errs = bound if dim == 0 else bound.T
    s_abs = np.sum(np.abs(terms), axis=0)
    tol = 1e-6 * np.abs(want) + np.where(np.abs(want) < 1e-3 * s_abs, 1e-9 * s_abs, 0.0)
    tol += 6.0 * np.sqrt(np.sum(errs * errs, axis=0))
    tol += np.abs(want) * 2.0 ** -24
    bad = np.abs(got - want) > tol
    assert not bad.any(), (what, dim, int(np.argmax(bad)), got[bad][:3], want[bad][:3])
    return float(np.max(np.abs(got - want) / np.maximum(np.abs(want), 1e-300))) if want.size else 0.0


def host_mats(specs, seed):
    """Seeded inputs: specs = [(dtype, n_rows, n_cols, ld, lo, hi)]."""
    out = []
    for k, (dt, r, c, ld, lo, hi) in enumerate(specs):
        n = r * c
        if dt == "f32":
            flat = synth.uniform_f32(seed + k, n, lo, hi)
        elif dt == "f64":
            flat = synth.uniform01(seed + k, n) * (hi - lo) + lo
        elif dt in ("bf16", "f16"):
            flat, _ = synth.lognormal_signed(seed + k, n, dt)
        out.append(synth.as_mat(flat, dt, r, c, ld))
    return out
