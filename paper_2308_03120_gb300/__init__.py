"""Fused element-wise expression + reduction engine for GB300 (sm_103a).

A thin binding over libcoot.so (include/coot.h).  PyTorch supplies device
memory and streams; every computation happens inside the library's CUDA
kernels.  The functions below carry the ABI's names and take torch-backed
`Mat` operands:

    import paper_2308_03120_gb300 as coot
    from paper_2308_03120_gb300.expr import var, exp
    x, z = var(0), var(1)
    coot.coot_init(0)
    coot.coot_expr_eval((2 * x + 3 * z).tree(), [X, Z], Y)    # Y = 2X + 3Z
    s = coot.coot_accu((x % z).tree(), [X, Z])                # accu(X % Z)

There is no CPU path: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import _abi
from ._abi import (COOT_BF16, COOT_F16, COOT_F32, COOT_F64, COOT_I32, COOT_NORM_FRO, COOT_NORM_INF, COOT_NORM_NEG_INF,
                   COOT_U32,
                   HEAD_ALL, HEAD_ANY, HEAD_MAX, HEAD_MAXABS, HEAD_MIN, HEAD_MINABS, HEAD_NORM2, HEAD_SUM,
                   HEAD_SUMABS, HEAD_SUMSQ, HEAD_COLSUM, HEAD_ROWSUM, KIND_BATCHED, KIND_COLSTATS, KIND_COLSUM,
                   KIND_DIMS, KIND_MAP, KIND_REDUCE, KIND_MULTI, KIND_ROWSTATS, KIND_ROWSUM, STAT_MAX, STAT_MEAN, STAT_MIN, STAT_STDDEV, STAT_SUM, STAT_VAR,
                   CootError, coot_mat)
from .expr import (Expr, abs_, acos, asin, atan, const, cos, eq, exp, log, log10, ne, pow_, serialize, sin, sqrt,
                   square, tan, var)

__all__ = [
    "Mat", "Workspace", "CootError", "coot_init", "coot_finalize", "coot_workspace_size", "coot_tree_check",
    "coot_tree_source", "coot_tree_compile", "coot_expr_eval", "coot_accu", "coot_sum_dim", "coot_dot",
    "coot_norm", "coot_minmax", "coot_all_any", "coot_stats_dim", "coot_expr_reduce", "coot_expr_multi",
    "coot_expr_multi_dims", "coot_unfused_eval",
    "coot_unfused_tmp_count", "Expr", "var", "const", "exp", "log", "sqrt", "square", "abs_", "eq", "ne",
    "pow_", "log10", "sin", "cos", "tan", "asin", "acos", "atan", "serialize",
    "batch_item", "coot_batch_plan", "coot_expr_eval_batched",
]

_TORCH_DTYPES = None


def _dtype_code(t) -> int:
    global _TORCH_DTYPES
    import torch
    if _TORCH_DTYPES is None:
        _TORCH_DTYPES = {torch.float32: COOT_F32, torch.bfloat16: COOT_BF16, torch.float16: COOT_F16,
                         torch.float64: COOT_F64, torch.int32: COOT_I32}
        if hasattr(torch, "uint32"):
            _TORCH_DTYPES[torch.uint32] = COOT_U32
    try:
        return _TORCH_DTYPES[t.dtype]
    except KeyError:
        raise TypeError(f"unsupported element type {t.dtype}") from None


@dataclass
class Mat:
    """A column-major n_rows x n_cols matrix over torch storage: element
    (i, j) is buf[offset + i + j * ld] (buf flattened).  `base`, when not 0,
    is the device address of buf's first element (pinned host storage
    reached over NVLink-C2C; see mapped())."""
    buf: object
    n_rows: int
    n_cols: int
    ld: int
    offset: int = 0
    base: int = 0

    @staticmethod
    def of(t, n_rows: int | None = None, n_cols: int | None = None, ld: int | None = None) -> "Mat":
        """Wrap a tensor.  1-D: an n x 1 column (or the given shape);
        2-D: must be column-major (stride(0) == 1), e.g. torch.empty(c, r).t()."""
        if t.dim() == 2 and n_rows is None:
            if t.shape[0] > 1 and t.stride(0) != 1:
                raise ValueError("2-D tensors must be column-major (stride(0) == 1)")
            return Mat(t, t.shape[0], t.shape[1], max(t.stride(1), t.shape[0], 1), 0)
        if n_rows is None:
            n_rows, n_cols = t.numel(), 1
        n_cols = 1 if n_cols is None else n_cols
        ld = max(n_rows, 1) if ld is None else ld
        return Mat(t, n_rows, n_cols, ld, 0)

    def c(self) -> coot_mat:
        t = self.buf
        ptr = (self.base or t.data_ptr()) + self.offset * t.element_size()
        return coot_mat(ptr, _dtype_code(t), 0, self.n_rows, self.n_cols, self.ld)

    def mapped(self) -> "Mat":
        """The same matrix over pinned host storage, addressed through its
        device mapping (coot_host_device_pointer): kernels then read and
        write host memory directly, with no copy.  Raises CootError for
        pageable storage."""
        dev = ctypes.c_void_p()
        _abi.call("coot_host_device_pointer", ctypes.c_void_p(self.buf.data_ptr()), ctypes.byref(dev))
        return Mat(self.buf, self.n_rows, self.n_cols, self.ld, self.offset, dev.value)

    # ---- submatrix views (coot_submat / coot_diag; Table 1)
    def _view(self, v: coot_mat) -> "Mat":
        es = self.buf.element_size()
        return Mat(self.buf, v.n_rows, v.n_cols, v.ld, (v.ptr - (self.base or self.buf.data_ptr())) // es, self.base)

    def submat(self, r0: int, c0: int, r1: int, c1: int) -> "Mat":
        """Rows r0..r1 and columns c0..c1 (inclusive), sharing storage."""
        src, v = self.c(), coot_mat()
        _abi.call("coot_submat", ctypes.byref(src), r0, c0, r1, c1, ctypes.byref(v))
        return self._view(v)

    def rows(self, a: int, b: int) -> "Mat":
        return self.submat(a, 0, b, self.n_cols - 1)

    def cols(self, c: int, d: int) -> "Mat":
        return self.submat(0, c, self.n_rows - 1, d)

    def row(self, i: int) -> "Mat":
        return self.submat(i, 0, i, self.n_cols - 1)

    def col(self, j: int) -> "Mat":
        return self.submat(0, j, self.n_rows - 1, j)

    def diag(self, k: int = 0) -> "Mat":
        """The k-th diagonal as a 1 x n view (ld + 1 apart)."""
        src, v = self.c(), coot_mat()
        _abi.call("coot_diag", ctypes.byref(src), k, ctypes.byref(v))
        return self._view(v)


def _mats(ms):
    arr = (coot_mat * len(ms))(*[m.c() for m in ms])
    return arr, len(ms)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Workspace:
    """Zero-filled device workspace sized by coot_workspace_size."""

    def __init__(self, max_rows: int, device="cuda"):
        import torch
        self.bytes = coot_workspace_size(max_rows)
        self.buf = torch.zeros(self.bytes, dtype=torch.uint8, device=device)

    @property
    def ptr(self):
        return ctypes.c_void_p(self.buf.data_ptr())


_default_ws = {}


def _ws(ws, rows):
    if ws is not None:
        return ws
    import torch
    dev = torch.cuda.current_device()
    cur = _default_ws.get(dev)
    if cur is None or cur.bytes < coot_workspace_size(rows):
        cur = Workspace(max(rows, 1 << 14), device=f"cuda:{dev}")
        _default_ws[dev] = cur
    return cur


# ---------------------------------------------------------------- set-up / host-only

def coot_init(device: int = 0, flags: int = 0) -> None:
    """Bind the library to CUDA device `device` (the runtime set-up of
    Section 3); every device call needs it first."""
    _abi.call("coot_init", device, flags)


def coot_finalize() -> None:
    """Drop the compiled-kernel cache and the device binding."""
    _abi.call("coot_finalize")


def coot_workspace_size(max_rows: int) -> int:
    """Bytes of workspace the reductions and sums need for operands of up to
    `max_rows` rows (row sums keep partials per row)."""
    n = ctypes.c_size_t()
    _abi.call("coot_workspace_size", max_rows, ctypes.byref(n))
    return n.value


def coot_tree_check(tree: bytes):
    """Validate serialised tree bytes; returns (inputs, compute type code,
    FNV-1a hash of the bytes)."""
    n_in, comp, h = ctypes.c_int(), ctypes.c_int(), ctypes.c_uint64()
    _abi.call("coot_tree_check", tree, len(tree), ctypes.byref(n_in), ctypes.byref(comp), ctypes.byref(h))
    return n_in.value, comp.value, h.value


def coot_tree_source(tree: bytes, kind: int = 0) -> str:
    """The CUDA source generated for a tree and kernel kind (host only)."""
    n = ctypes.c_size_t()
    _abi.call("coot_tree_source", tree, len(tree), kind, None, 0, ctypes.byref(n))
    buf = ctypes.create_string_buffer(n.value + 1)
    _abi.call("coot_tree_source", tree, len(tree), kind, buf, n.value + 1, ctypes.byref(n))
    return buf.value.decode()


def coot_tree_compile(tree: bytes, kind: int = 0, in_dtype: int = COOT_F32, out_dtype: int = COOT_F32,
                      heads: int = 0, arch: str = "sm_103a") -> int:
    """Compile a tree's kernel with NVRTC for `arch` without loading it (no
    GPU needed); returns the cubin size in bytes."""
    n = ctypes.c_size_t()
    _abi.call("coot_tree_compile", tree, len(tree), kind, in_dtype, out_dtype, heads, arch.encode(),
              ctypes.byref(n))
    return n.value


def coot_unfused_tmp_count(tree: bytes) -> int:
    """Temporaries the unfused baseline needs for a tree (one per inner
    node, reused once dead)."""
    n = ctypes.c_int()
    _abi.call("coot_unfused_tmp_count", tree, len(tree), ctypes.byref(n))
    return n.value


# ---------------------------------------------------------------- device calls

def _result(out_dev, n):
    import torch
    if out_dev is None:
        out_dev = torch.empty(n, dtype=torch.float64, device="cuda")
    return out_dev


def coot_expr_eval(tree: bytes, ins, out: Mat, ws=None, stream=None) -> None:
    """out = tree(ins...) element-wise in one fused kernel, no temporaries
    (delayed evaluation at assignment, Section 7).  `out` may be identical
    to an input."""
    arr, n = _mats(ins)
    o = out.c()
    _abi.call("coot_expr_eval", tree, len(tree), arr, n, ctypes.byref(o), None, 0, _stream(stream))


def coot_expr_reduce(tree: bytes, ins, heads: int, out: Mat | None = None, out_dev=None, ws=None, stream=None):
    """Several reductions (HEAD_* mask) in one pass; returns the FP64 device
    tensor of results (one per set bit, increasing bit order)."""
    arr, n = _mats(ins)
    w = _ws(ws, 0)
    res = _result(out_dev, bin(heads).count("1"))
    o = ctypes.byref(out.c()) if out is not None else None
    _abi.call("coot_expr_reduce", tree, len(tree), arr, n, heads, o, ctypes.c_void_p(res.data_ptr()), w.ptr,
              w.bytes, _stream(stream))
    return res


def coot_expr_multi(trees, ins, outs=None, heads=None, out_dev=None, ws=None, stream=None):
    """Several trees over the same operands in one pass: tree k is stored
    into outs[k] (a Mat, or None) and reduced by heads[k] (a HEAD_* mask, or
    0).  Returns the FP64 device tensor of results (tree 0's heads in
    increasing bit order, then tree 1's, ...), or None without heads."""
    nt = len(trees)
    keep = [ctypes.create_string_buffer(bytes(t), len(t)) for t in trees]
    tp = (ctypes.c_void_p * nt)(*[ctypes.cast(b, ctypes.c_void_p) for b in keep])
    tl = (ctypes.c_size_t * nt)(*[len(t) for t in trees])
    arr, n = _mats(ins)
    o_arr = None
    if outs is not None:
        o_arr = (coot_mat * nt)(*[m.c() if m is not None else coot_mat() for m in outs])
    hs = list(heads) if heads is not None else [0] * nt
    h_arr = (ctypes.c_uint * nt)(*hs)
    total = sum(bin(h).count("1") for h in hs)
    res = _result(out_dev, total) if total else None
    w = _ws(ws, 0)
    _abi.call("coot_expr_multi", tp, tl, nt, arr, n, o_arr, h_arr,
              ctypes.c_void_p(res.data_ptr()) if res is not None else None, w.ptr, w.bytes, _stream(stream))
    return res


def coot_expr_multi_dims(trees, ins, outs=None, heads=None, colsums=None, rowsums=None, out_dev=None, ws=None,
                         stream=None):
    """coot_expr_multi plus sums along a dimension in the same pass: heads[k]
    may hold HEAD_COLSUM (tree k's column sums into colsums[k], a 1 x n_cols
    Mat) and HEAD_ROWSUM (its row sums into rowsums[k], an n_rows x 1 Mat).
    Returns the FP64 device tensor of the full heads, or None without."""
    nt = len(trees)
    keep = [ctypes.create_string_buffer(bytes(t), len(t)) for t in trees]
    tp = (ctypes.c_void_p * nt)(*[ctypes.cast(b, ctypes.c_void_p) for b in keep])
    tl = (ctypes.c_size_t * nt)(*[len(t) for t in trees])
    arr, n = _mats(ins)

    def mats(ms):
        if ms is None:
            return None
        return (coot_mat * nt)(*[m.c() if m is not None else coot_mat() for m in ms])
    hs = list(heads) if heads is not None else [0] * nt
    h_arr = (ctypes.c_uint * nt)(*hs)
    total = sum(bin(h & 0x3FF).count("1") for h in hs)
    res = _result(out_dev, total) if total else None
    w = _ws(ws, ins[0].n_rows)
    _abi.call("coot_expr_multi_dims", tp, tl, nt, arr, n, mats(outs), h_arr,
              ctypes.c_void_p(res.data_ptr()) if res is not None else None, mats(colsums), mats(rowsums), w.ptr,
              w.bytes, _stream(stream))
    return res


def coot_accu(tree: bytes, ins, out_dev=None, ws=None, stream=None):
    """accu(tree(ins...)): the sum of every element (Table 5), one pass;
    returns a 1-element FP64 device tensor."""
    arr, n = _mats(ins)
    w = _ws(ws, 0)
    res = _result(out_dev, 1)
    _abi.call("coot_accu", tree, len(tree), arr, n, ctypes.c_void_p(res.data_ptr()), w.ptr, w.bytes,
              _stream(stream))
    return res


def coot_sum_dim(tree: bytes, ins, dim: int, out: Mat, ws=None, stream=None) -> None:
    """sum(tree(ins...), dim) into `out` (Table 6): dim 0 sums each column
    (out is 1 x n_cols), dim 1 each row (out is n_rows x 1)."""
    arr, n = _mats(ins)
    w = _ws(ws, ins[0].n_rows if dim == 1 else 0)
    o = out.c()
    _abi.call("coot_sum_dim", tree, len(tree), arr, n, dim, ctypes.byref(o), w.ptr, w.bytes, _stream(stream))


def coot_dot(a: Mat, b: Mat, out_dev=None, ws=None, stream=None):
    """dot(a, b) over equal element counts (Table 5); returns a 1-element
    FP64 device tensor."""
    w = _ws(ws, 0)
    res = _result(out_dev, 1)
    ca, cb = a.c(), b.c()
    _abi.call("coot_dot", ctypes.byref(ca), ctypes.byref(cb), ctypes.c_void_p(res.data_ptr()), w.ptr, w.bytes,
              _stream(stream))
    return res


def coot_norm(tree: bytes, ins, p, out_dev=None, ws=None, stream=None):
    """p: 1, 2, "inf", "-inf" or "fro"."""
    code = {"inf": COOT_NORM_INF, "-inf": COOT_NORM_NEG_INF, "fro": COOT_NORM_FRO}.get(p, p)
    arr, n = _mats(ins)
    w = _ws(ws, 0)
    res = _result(out_dev, 1)
    _abi.call("coot_norm", tree, len(tree), arr, n, int(code), ctypes.c_void_p(res.data_ptr()), w.ptr, w.bytes,
              _stream(stream))
    return res


def coot_minmax(tree: bytes, ins, out_dev=None, ws=None, stream=None):
    """[min, max] over every element of tree(ins...) (Table 6); NaN
    propagates; returns a 2-element FP64 device tensor."""
    arr, n = _mats(ins)
    w = _ws(ws, 0)
    res = _result(out_dev, 2)
    _abi.call("coot_minmax", tree, len(tree), arr, n, ctypes.c_void_p(res.data_ptr()), w.ptr, w.bytes,
              _stream(stream))
    return res


def coot_all_any(tree: bytes, ins, out_dev=None, ws=None, stream=None):
    """[all, any] of the tree's elements as 1.0 / 0.0 (FP64 device tensor)."""
    arr, n = _mats(ins)
    w = _ws(ws, 0)
    res = _result(out_dev, 2)
    _abi.call("coot_all_any", tree, len(tree), arr, n, ctypes.c_void_p(res.data_ptr()), w.ptr, w.bytes,
              _stream(stream))
    return res


def coot_stats_dim(tree: bytes, ins, dim: int, stats: int, outs, norm_type: int = 0, ws=None, stream=None) -> None:
    """Statistics (STAT_* mask) of each column (dim 0) or row (dim 1) in one
    pass; `outs` holds one Mat per set bit, in increasing bit order."""
    arr, n = _mats(ins)
    w = _ws(ws, ins[0].n_rows if dim == 1 else 0)
    o_arr, n_out = _mats(outs)
    if n_out != bin(stats & 0x3F).count("1"):
        raise ValueError("one output per statistic")
    _abi.call("coot_stats_dim", tree, len(tree), arr, n, dim, stats, norm_type, o_arr, w.ptr, w.bytes,
              _stream(stream))


def coot_unfused_eval(tree: bytes, ins, out: Mat, tmp=None, stream=None) -> None:
    """The baseline: one kernel per tree node with HBM temporaries (the
    apply() chain of Section 7), for measuring what fusion gains."""
    import torch
    arr, n = _mats(ins)
    k = coot_unfused_tmp_count(tree)
    _, comp, _ = coot_tree_check(tree)
    esize = 8 if comp == COOT_F64 else 4
    need = k * ins[0].n_rows * ins[0].n_cols * esize
    if tmp is None or tmp.numel() * tmp.element_size() < need:
        tmp = torch.empty(max(need, 16), dtype=torch.uint8, device="cuda")
    o = out.c()
    _abi.call("coot_unfused_eval", tree, len(tree), arr, n, ctypes.byref(o), ctypes.c_void_p(tmp.data_ptr()),
              tmp.numel() * tmp.element_size(), _stream(stream))
    return tmp


# ---------------------------------------------------------------- batched evaluation

def batch_item(ins, out: Mat | None = None, colsum: Mat | None = None) -> _abi.coot_batch_item:
    """One matrix of a batch: inputs (Mats of equal shape), optional
    element-wise output and optional 1 x n_cols column-sum output."""
    it = _abi.coot_batch_item()
    r, c = ins[0].n_rows, ins[0].n_cols
    for k, m in enumerate(ins):
        cm = m.c()
        it.in_[k] = cm.ptr
        it.ld_in[k] = cm.ld
    for k in range(len(ins), 4):
        it.ld_in[k] = max(r, 1)
    if out is not None:
        co = out.c()
        it.out, it.ld_out = co.ptr, co.ld
    else:
        it.ld_out = max(r, 1)
    if colsum is not None:
        cs = colsum.c()
        it.colsum, it.ld_colsum = cs.ptr, cs.ld if colsum.n_rows == 1 else 1
    else:
        it.ld_colsum = 1
    it.n_rows, it.n_cols = r, c
    # the item holds raw pointers: keep the storage alive with it
    it._keep = [m.buf for m in ins] + [m.buf for m in (out, colsum) if m is not None]
    return it


def coot_batch_plan(items, n_inputs: int, device="cuda"):
    """Build the plan of a batch on the host and copy it to the device once.
    Returns (plan tensor, n_items, n_work)."""
    import torch
    arr = (_abi.coot_batch_item * len(items))(*items)
    nbytes, n_work = ctypes.c_size_t(), ctypes.c_int64()
    _abi.call("coot_batch_plan_size", arr, len(items), ctypes.byref(nbytes), ctypes.byref(n_work))
    host = torch.empty(max(nbytes.value, 16), dtype=torch.uint8)
    _abi.call("coot_batch_plan_build", arr, len(items), n_inputs, ctypes.c_void_p(host.data_ptr()), nbytes.value)
    plan = host.to(device)
    # the plan holds the items' raw pointers: it keeps their storage alive
    plan._keep = [getattr(it, "_keep", None) for it in items]
    return plan, len(items), n_work.value


def coot_expr_eval_batched(tree: bytes, in_dtypes, out_dtype: int, colsum_dtype: int, plan, n_items: int,
                           n_work: int, stream=None) -> None:
    """One persistent launch over a batch plan (coot_batch_plan): every
    item's element-wise output and column sums."""
    dts = (ctypes.c_int32 * 4)(*(list(in_dtypes) + [0] * (4 - len(in_dtypes))))
    _abi.call("coot_expr_eval_batched", tree, len(tree), dts, out_dtype, colsum_dtype,
              ctypes.c_void_p(plan.data_ptr()), n_items, n_work, _stream(stream))


def coot_sum_rows_f32_static(a: Mat, out: Mat, stream=None) -> None:
    """sum(a, 1) of an FP32 matrix with the library's own scratch (no
    workspace, no allocation); n_rows <= 32768."""
    ca, co = a.c(), out.c()
    _abi.call("coot_sum_rows_f32_static", ctypes.byref(ca), ctypes.byref(co), _stream(stream))


# ---------------------------------------------------------------- launch shapes

def coot_set_canonical(enable: bool) -> None:
    """Canonical forms of the trees of the calls that follow on this thread
    (on by default)."""
    _abi.call("coot_set_canonical", int(bool(enable)))


def coot_tree_canonical(tree: bytes) -> bytes:
    """The canonical form of a tree (exact rewrites; host-only)."""
    n = ctypes.c_size_t()
    _abi.call("coot_tree_canonical", tree, len(tree), None, 0, ctypes.byref(n))
    buf = ctypes.create_string_buffer(n.value)
    _abi.call("coot_tree_canonical", tree, len(tree), buf, n.value, ctypes.byref(n))
    return buf.raw[:n.value]


def coot_set_launch_config(kind: int, block: int = 0, vec: int = 0, unroll: int = 0, blocks_per_sm: int = 0,
                           split: int = 0) -> None:
    """Launch shape for the kernels of `kind` on this thread (block = 0
    restores the built-in choice)."""
    _abi.call("coot_set_launch_config", kind, block, vec, unroll, blocks_per_sm, split)


def coot_last_launch() -> dict:
    b, v, u = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    g, s = ctypes.c_int64(), ctypes.c_int64()
    _abi.call("coot_last_launch", ctypes.byref(b), ctypes.byref(v), ctypes.byref(u), ctypes.byref(g), ctypes.byref(s))
    return {"block": b.value, "vec": v.value, "unroll": u.value, "grid": g.value, "split": s.value}
