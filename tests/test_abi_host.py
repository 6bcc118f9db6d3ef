"""Host-side checks of the C ABI (no GPU): the library loads and exports
every function include/coot.h declares, the C tree validator agrees with the
oracle's independent decoder, the Python serializer agrees with the oracle's
encoder, every kernel kind compiles with NVRTC for sm_103a, injected
faults and argument errors come back as status codes."""
import ctypes
import os
import re
import struct

import pytest

import synth
from oracle import coot_oracle as O
import paper_2308_03120_gb300 as coot
from paper_2308_03120_gb300 import _abi
from paper_2308_03120_gb300.expr import as_expr, serialize, var, exp, sqrt, log, abs_

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2308_03120_gb300 import build
    build.build()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "coot.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(coot_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound():
    names = declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(_abi.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
        assert n in _abi.SIGNATURES, n


def test_version_and_status_strings():
    L = _abi.lib()
    assert L.coot_version() >= 100
    assert L.coot_status_string(0) == b"COOT_OK"
    assert L.coot_status_string(12) == b"COOT_ERR_WORKSPACE"


def _hdr(n_nodes, n_inputs=1, compute=0, version=1, magic=b"COOT", r0=0, r1=0):
    return struct.pack("<4sHHBBHI", magic, version, n_nodes, n_inputs, compute, r0, r1)


def _node(op, a=0, b=0, imm=0.0, z0=0, z1=0):
    return struct.pack("<BBHHHd", op, z0, a, b, z1, imm)


MALFORMED = [
    _hdr(1, magic=b"COOX") + _node(0), _hdr(1, version=2) + _node(0), _hdr(0), _hdr(65) + _node(0) * 65,
    _hdr(1, n_inputs=0) + _node(0), _hdr(1, n_inputs=5) + _node(0), _hdr(1, compute=1) + _node(0),
    _hdr(1, r0=1) + _node(0), _hdr(2) + _node(0), _hdr(1) + _node(200), _hdr(1) + _node(0, a=1),
    _hdr(2) + _node(0) + _node(2, a=1), _hdr(2) + _node(0) + _node(8, a=0, b=2),
    _hdr(2) + _node(0) + _node(2, a=0, b=1), _hdr(1) + _node(1, a=1, imm=1.0), _hdr(1) + _node(0, z0=1),
    b"COOT",
]


@pytest.mark.parametrize("raw", MALFORMED)
def test_validator_rejects_what_the_oracle_rejects(raw):
    with pytest.raises(O.TreeError):
        O.decode(raw)
    with pytest.raises(coot.CootError) as e:
        coot.coot_tree_check(raw)
    assert e.value.status_name == "COOT_ERR_BAD_TREE"


def _trees():
    out = [synth.AXPY_2X_3Z, synth.SCHUR_XZ, synth.LEAF0, synth.MAT_EXPR, synth.MAT_CHAIN, synth.BATCH_EXPR]
    out += [synth.random_tree(77 + s, 2 + s % 11, 1 + s % 4) for s in range(30)]
    return out


@pytest.mark.parametrize("sexpr", _trees())
def test_serializer_matches_oracle_encoder(sexpr):
    for compute in ("f32", "f64"):
        n_in = synth.tree_inputs(sexpr)
        b = serialize(sexpr, compute=compute, n_inputs=n_in)
        assert b == O.encode(sexpr, n_inputs=n_in, compute=compute)
        n, comp, h = coot.coot_tree_check(b)
        assert n == n_in and comp == {"f32": 0, "f64": 3}[compute]
        assert O.to_sexpr(O.decode(b)) == O.to_sexpr(O.decode(O.encode(sexpr, n_inputs=n_in, compute=compute)))


def test_operator_overloading_builds_the_workload_trees():
    x, z = var(0), var(1)
    A, B, C, D = var(0), var(1), var(2), var(3)
    assert (2 * x + 3 * z).sexpr() == synth.AXPY_2X_3Z
    assert (x % z).sexpr() == synth.SCHUR_XZ
    assert ((A % B + 2 * C) / (1 + abs(D))).sexpr() == synth.MAT_EXPR
    assert (exp(-abs_(A % B + 2 * C)) / sqrt(1 + abs(D))).sexpr() == synth.MAT_CHAIN
    assert (exp(-abs(A)) % B + 0.5 * C).sexpr() == synth.BATCH_EXPR
    assert (1 - x).sexpr() == ("sub", ("c", 1.0), ("x", 0))
    assert (x / 4).sexpr() == ("div", ("x", 0), ("c", 4.0))
    with pytest.raises(TypeError):
        x * z
    assert as_expr(synth.MAT_CHAIN).sexpr() == synth.MAT_CHAIN


def test_tree_hash_is_stable_and_content_addressed():
    a = serialize(synth.MAT_EXPR)
    b = serialize(synth.MAT_CHAIN)
    assert coot.coot_tree_check(a)[2] == coot.coot_tree_check(a)[2]
    assert coot.coot_tree_check(a)[2] != coot.coot_tree_check(b)[2]


def test_generated_source_inlines_the_tree():
    src = coot.coot_tree_source(serialize(synth.MAT_CHAIN), 0)
    assert "expf(" in src and "sqrtf(" in src and "fabsf(" in src
    assert "#define COOT_NIN 4" in src
    src64 = coot.coot_tree_source(serialize(synth.MAT_CHAIN, compute="f64"), 1)
    assert "exp(" in src64 and "#define COOT_REAL double" in src64


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("dt", [0, 1, 2, 3])
def test_every_kernel_kind_compiles_for_sm103a(kind, dt):
    t = serialize(synth.MAT_CHAIN, compute="f64" if dt == 3 else "f32")
    heads = {1: 0x3FF, 5: 0x3F, 6: 0x3F, 7: 0x3FF, 8: 0x3FF}.get(kind, 0)
    out_dt = dt if kind < 5 or kind >= 7 else (3 if dt == 3 else 0)
    n = coot.coot_tree_compile(t, kind=kind, in_dtype=dt, out_dtype=out_dt, heads=heads)
    assert n > 1000


@pytest.mark.parametrize("dims", [1 << 10, 1 << 11, 3 << 10])
@pytest.mark.parametrize("heads", [0, 0x3FF])
def test_dimension_sum_variants_compile(dims, heads):
    """Kind 8 with column sums only, row sums only and both, with and
    without full heads."""
    n = coot.coot_tree_compile(serialize(synth.MAT_EXPR), kind=8, heads=heads | dims)
    assert n > 1000


def test_relational_trees_compile():
    x = coot.var(0)
    t = ((x < 0.5) % x + coot.eq(x, 1.0) - (x >= -1.0)).tree()
    src = coot.coot_tree_source(t, 0)
    assert " < " in src and " == " in src and " >= " in src
    assert coot.coot_tree_compile(t, kind=1, heads=0x300) > 1000


def test_injected_compile_failure_is_a_status(monkeypatch):
    monkeypatch.setenv("COOT_FAULT", "nvrtc_fail")
    with pytest.raises(coot.CootError) as e:
        coot.coot_tree_compile(serialize(synth.AXPY_2X_3Z))
    assert e.value.status_name == "COOT_ERR_COMPILE"
    assert "injected" in str(e.value)


def _fake(n_rows, n_cols, ld=None, ptr=1 << 20, dtype=0):
    return _abi.coot_mat(ptr, dtype, 0, n_rows, n_cols, ld if ld is not None else max(n_rows, 1))


def _call(name, *args):
    L = _abi.lib()
    return getattr(L, name)(*args), (L.coot_last_error() or b"").decode()


def test_argument_errors_are_reported_before_any_device_work():
    t = serialize(synth.AXPY_2X_3Z)
    ins = (_abi.coot_mat * 2)(_fake(10, 3), _fake(10, 4, ptr=1 << 24))
    out = _fake(10, 3, ptr=1 << 28)
    st, msg = _call("coot_expr_eval", t, len(t), ins, 2, ctypes.byref(out), None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_SHAPE" and "equal sizes" in msg
    ins = (_abi.coot_mat * 2)(_fake(10, 3), _fake(10, 3, ptr=1 << 24))
    st, _ = _call("coot_expr_eval", t, len(t), ins, 1, ctypes.byref(out), None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG"
    # partial overlap with input 0 (shifted by one element)
    bad = _fake(10, 3, ptr=(1 << 20) + 4)
    st, msg = _call("coot_expr_eval", t, len(t), ins, 2, ctypes.byref(bad), None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_ALIAS"
    # ld < n_rows
    st, _ = _call("coot_expr_eval", t, len(t), (_abi.coot_mat * 2)(_fake(10, 3, ld=5), _fake(10, 3)), 2,
                  ctypes.byref(out), None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG"
    # unknown dtype
    st, _ = _call("coot_expr_eval", t, len(t), (_abi.coot_mat * 2)(_fake(10, 3, dtype=9), _fake(10, 3)), 2,
                  ctypes.byref(out), None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_DTYPE"


def test_reduction_argument_errors():
    leaf = serialize(synth.LEAF0)
    m = (_abi.coot_mat * 1)(_fake(30, 40))
    res = ctypes.c_void_p(1 << 30)
    st, msg = _call("coot_norm", leaf, len(leaf), m, 1, 2, res, ctypes.c_void_p(1 << 32), 1 << 22, None)
    assert _abi.STATUS[st] == "COOT_ERR_UNSUPPORTED" and "spectral" in msg
    st, _ = _call("coot_norm", leaf, len(leaf), m, 1, 7, res, ctypes.c_void_p(1 << 32), 1 << 22, None)
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG"
    empty = (_abi.coot_mat * 1)(_fake(0, 5))
    st, _ = _call("coot_minmax", leaf, len(leaf), empty, 1, res, ctypes.c_void_p(1 << 32), 1 << 22, None)
    assert _abi.STATUS[st] == "COOT_ERR_EMPTY"
    st, _ = _call("coot_accu", leaf, len(leaf), m, 1, res, None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_WORKSPACE"
    out = _fake(1, 41, ptr=1 << 28)
    st, msg = _call("coot_sum_dim", leaf, len(leaf), m, 1, 0, ctypes.byref(out), None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_SHAPE"
    st, _ = _call("coot_sum_dim", leaf, len(leaf), m, 1, 2, ctypes.byref(out), None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG"
    a, b = _fake(1, 6), _fake(5, 1, ptr=1 << 24)
    st, _ = _call("coot_dot", ctypes.byref(a), ctypes.byref(b), res, None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_SHAPE"
    st, msg = _call("coot_expr_reduce", leaf, len(leaf), m, 1, 1 << 10, None, res, None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG" and "head" in msg


def test_multi_tree_argument_errors():
    """coot_expr_multi (several trees in one pass) rejects bad calls before
    any device work."""
    t1, t2 = serialize(synth.AXPY_2X_3Z), serialize(synth.SCHUR_XZ)
    ins = (_abi.coot_mat * 2)(_fake(10, 3), _fake(10, 3, ptr=1 << 24))
    res = ctypes.c_void_p(1 << 30)
    ws = ctypes.c_void_p(1 << 32)

    def call(trees, n_in=2, outs=None, heads=None, w=ws, wb=1 << 22, nt=None):
        keep = [ctypes.create_string_buffer(bytes(t), len(t)) for t in trees]
        tp = (ctypes.c_void_p * max(len(trees), 1))(*[ctypes.cast(b, ctypes.c_void_p) for b in keep])
        tl = (ctypes.c_size_t * max(len(trees), 1))(*[len(t) for t in trees])
        o = (_abi.coot_mat * len(outs))(*outs) if outs is not None else None
        h = (ctypes.c_uint * len(heads))(*heads) if heads is not None else None
        return _call("coot_expr_multi", tp, tl, len(trees) if nt is None else nt, ins, n_in, o, h, res, w, wb, None)

    st, _ = call([t1], nt=0)
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG"
    st, _ = call([t1] * 5)
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG"
    # a tree with neither an output nor heads
    st, msg = call([t1, t2], heads=[1, 0])
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG" and "tree 1" in msg
    # a tree reading more operands than given
    st, msg = call([t1], n_in=1, heads=[1])
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG" and "inputs" in msg
    # compute types differ
    st, _ = call([t1, serialize(synth.SCHUR_XZ, compute="f64")], heads=[1, 1])
    assert _abi.STATUS[st] == "COOT_ERR_DTYPE"
    st, msg = call([t1, t2], heads=[1, 1 << 10])
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG" and "head" in msg
    # two stored trees on the same memory; an output of another shape
    o = _fake(10, 3, ptr=1 << 28)
    st, _ = call([t1, t2], outs=[o, o])
    assert _abi.STATUS[st] == "COOT_ERR_ALIAS"
    st, _ = call([t1], outs=[_fake(10, 4, ptr=1 << 28)])
    assert _abi.STATUS[st] == "COOT_ERR_SHAPE"
    # an output overlapping an input without being identical to it
    st, _ = call([t1], outs=[_fake(10, 3, ptr=(1 << 20) + 4)])
    assert _abi.STATUS[st] == "COOT_ERR_ALIAS"
    # heads need a workspace
    st, _ = call([t1, t2], heads=[1, 4], w=None, wb=0)
    assert _abi.STATUS[st] == "COOT_ERR_WORKSPACE"
    # heads need a result pointer; 1 to 4 operands
    keep = [ctypes.create_string_buffer(bytes(t1), len(t1))]
    tp = (ctypes.c_void_p * 1)(ctypes.cast(keep[0], ctypes.c_void_p))
    tl = (ctypes.c_size_t * 1)(len(t1))
    h = (ctypes.c_uint * 1)(1)
    st, msg = _call("coot_expr_multi", tp, tl, 1, ins, 2, None, h, None, ws, 1 << 22, None)
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG" and "result" in msg
    for n_in in (0, 5):
        st, _ = _call("coot_expr_multi", tp, tl, 1, ins, n_in, None, h, res, ws, 1 << 22, None)
        assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG"


def test_stats_argument_errors():
    leaf = serialize(synth.LEAF0)
    m = (_abi.coot_mat * 1)(_fake(30, 40))
    ws = ctypes.c_void_p(1 << 32)

    def stats(dim, mask, outs, norm_type=0, ins=m):
        arr = (_abi.coot_mat * len(outs))(*outs)
        st, msg = _call("coot_stats_dim", leaf, len(leaf), ins, 1, dim, mask, norm_type, arr, ws, 1 << 22, None)
        return _abi.STATUS[st], msg

    row = lambda k, dt=0: _fake(1, 40, ptr=(1 << 28) + k * 4096, dtype=dt)  # noqa: E731
    assert stats(0, 0, [row(0)])[0] == "COOT_ERR_INVALID_ARG"                  # no statistic
    assert stats(0, 1 << 6, [row(0)])[0] == "COOT_ERR_INVALID_ARG"             # unknown bit
    assert stats(2, 1, [row(0)])[0] == "COOT_ERR_INVALID_ARG"                  # dim
    assert stats(0, 1, [row(0)], norm_type=2)[0] == "COOT_ERR_INVALID_ARG"     # norm_type
    assert stats(1, 1, [row(0)])[0] == "COOT_ERR_SHAPE"                        # dim 1 wants 30 x 1
    assert stats(0, 1, [row(0, dt=1)])[0] == "COOT_ERR_DTYPE"                  # BF16 statistics
    assert stats(0, 3, [row(0), row(1, dt=3)])[0] == "COOT_ERR_DTYPE"          # mixed dtypes
    st, msg = stats(0, 3, [row(0), _fake(1, 40, ptr=(1 << 28) + 8)])
    assert st == "COOT_ERR_ALIAS"                                               # outputs overlap
    assert stats(0, 1, [_fake(1, 40, ptr=(1 << 20) + 64)])[0] == "COOT_ERR_ALIAS"  # overlaps the input
    empty = (_abi.coot_mat * 1)(_fake(0, 5))
    st, _ = stats(0, 16, [_fake(1, 5, ptr=1 << 28)], ins=empty)
    assert st == "COOT_ERR_EMPTY"

def test_device_calls_need_init():
    # valid arguments that reach the kernel cache: refused without coot_init
    t = serialize(synth.AXPY_2X_3Z)
    ins = (_abi.coot_mat * 2)(_fake(10, 3), _fake(10, 3, ptr=1 << 24))
    out = _fake(10, 3, ptr=1 << 28)
    st, msg = _call("coot_expr_eval", t, len(t), ins, 2, ctypes.byref(out), None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_NOT_INIT"


def test_workspace_size_grows_with_rows():
    a = coot.coot_workspace_size(1)
    b = coot.coot_workspace_size(1 << 20)
    assert 65536 < a < b
    assert b >= 64 * (1 << 20) * 8


def test_views_of_one_matrix_alias_by_rows_and_columns():
    """Disjoint submatrices of one parent (same ld) pass the alias check (the
    call then stops at the uninitialised device); overlapping ones fail."""
    t = serialize(("mul", synth.C(2.0), synth.X(0)))
    parent = _fake(1000, 300, ptr=1 << 24)
    top, bottom, mid = (_abi.coot_mat() for _ in range(3))
    L = _abi.lib()
    assert L.coot_submat(ctypes.byref(parent), 0, 0, 499, 299, ctypes.byref(top)) == 0
    assert L.coot_submat(ctypes.byref(parent), 500, 0, 999, 299, ctypes.byref(bottom)) == 0
    assert L.coot_submat(ctypes.byref(parent), 250, 0, 749, 299, ctypes.byref(mid)) == 0
    assert (top.ld, bottom.ld, bottom.ptr - parent.ptr) == (1000, 1000, 500 * 4)
    ins = (_abi.coot_mat * 1)(bottom)
    st, _ = _call("coot_expr_eval", t, len(t), ins, 1, ctypes.byref(top), None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_NOT_INIT"
    st, _ = _call("coot_expr_eval", t, len(t), ins, 1, ctypes.byref(mid), None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_ALIAS"
    # columns 0..9 against columns 10..19 of the same rows: disjoint
    a, b = _abi.coot_mat(), _abi.coot_mat()
    L.coot_submat(ctypes.byref(parent), 0, 0, 999, 9, ctypes.byref(a))
    L.coot_submat(ctypes.byref(parent), 0, 10, 999, 19, ctypes.byref(b))
    st, _ = _call("coot_expr_eval", t, len(t), (_abi.coot_mat * 1)(a), 1, ctypes.byref(b), None, 0, None)
    assert _abi.STATUS[st] == "COOT_ERR_NOT_INIT"
    # out of bounds
    assert L.coot_submat(ctypes.byref(parent), 0, 0, 1000, 0, ctypes.byref(a)) == 3   # COOT_ERR_SHAPE
    d = _abi.coot_mat()
    assert L.coot_diag(ctypes.byref(parent), -2, ctypes.byref(d)) == 0
    assert (d.n_rows, d.n_cols, d.ld, d.ptr - parent.ptr) == (1, 300, 1001, 2 * 4)


def test_header_compiles_as_c99_and_cpp(tmp_path):
    """include/coot.h is a plain C header: it compiles as pedantic C99 and
    as C++17 with every warning on."""
    import shutil
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "use.c"
    src.write_text('#include "coot.h"\nint main(void) { return coot_version() > 0 ? 0 : 1; }\n')
    for cc, flags in (("gcc", ["-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror"]),
                      ("g++", ["-std=c++17", "-Wall", "-Wextra", "-Werror", "-x", "c++"])):
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not found")
        r = subprocess.run([cc, *flags, "-I", os.path.join(root, "include"), "-c", str(src), "-o",
                            str(tmp_path / f"use_{cc}.o")], capture_output=True, text=True)
        assert r.returncode == 0, (cc, r.stderr)


def test_batched_work_list_cuts_whole_aligned_columns():
    """The batch plan (host only): items copied first, then one work unit
    {item, col0, n_cols} per ~2048 elements of whole columns, cut so that a
    unit of a 16-byte aligned FP32 matrix starts 16-byte aligned (col0 *
    n_rows a multiple of 4); a column longer than 2048 rows is a unit of its
    own."""
    shapes = [(512, 9), (300, 13), (301, 11), (2, 5000), (3000, 3), (1, 1), (7, 0), (0, 6)]
    items = []
    for k, (r, c) in enumerate(shapes):
        it = _abi.coot_batch_item()
        for i in range(3):
            it.in_[i] = (1 << 30) + (k << 24) + (i << 20)
            it.ld_in[i] = max(r, 1)
        it.ld_in[3] = max(r, 1)
        it.out, it.ld_out = (1 << 40) + (k << 24), max(r, 1)
        it.n_rows, it.n_cols = r, c
        items.append(it)
    arr = (_abi.coot_batch_item * len(items))(*items)
    nbytes, n_work = ctypes.c_size_t(), ctypes.c_int64()
    st, _ = _call("coot_batch_plan_size", arr, len(items), ctypes.byref(nbytes), ctypes.byref(n_work))
    assert _abi.STATUS[st] == "COOT_OK"
    buf = ctypes.create_string_buffer(nbytes.value)
    st, _ = _call("coot_batch_plan_build", arr, len(items), 3, buf, nbytes.value)
    assert _abi.STATUS[st] == "COOT_OK"
    raw = buf.raw
    assert raw[:112 * len(items)] == bytes(arr)  # the items, as given
    units = [struct.unpack_from("<4i", raw, 112 * len(items) + 16 * u) for u in range(n_work.value)]
    assert len(units) == n_work.value and nbytes.value == 112 * len(items) + 16 * len(units)
    for k, (r, c) in enumerate(shapes):
        mine = [(c0, nc) for item, c0, nc, _ in units if item == k]
        # every column exactly once, in order, whole
        cols = [c0 + j for c0, nc in mine for j in range(nc)]
        assert cols == list(range(c)), (r, c, mine)
        for c0, nc in mine:
            assert nc * r <= 2048 or nc == 1, (r, c0, nc)
            assert (c0 * r) % 4 == 0, (r, c0)  # aligned start
        if c and r:
            # whole-column units are as large as the rule allows
            full = max(1, 2048 // r)
            m = 1 if r % 4 == 0 else (2 if r % 2 == 0 else 4)
            expect = full - full % m if full >= m else full
            assert max(nc for _, nc in mine) == min(expect, c), (r, c, mine)


def test_several_tree_source_defines_every_slot():
    """Kind 7 with one tree: coot_ft0 holds the tree, coot_ft1..3 are
    constant stubs no code path reads, and the per-tree macros say one tree,
    stored, with the given heads."""
    t = serialize(synth.MAT_EXPR)
    src = coot.coot_tree_source(t, 7)
    assert "#define COOT_KIND 7" in src and "#define COOT_NT 1" in src
    assert "#define COOT_ENTRY coot_multi" in src
    body = src[src.index("COOT_REAL coot_ft0("):src.index("COOT_REAL coot_ft1(")]
    assert "x[3]" in body and "fabsf(" in body
    for k in (1, 2, 3):
        assert f"COOT_REAL coot_ft{k}(const COOT_REAL* x) {{ return (COOT_REAL)0; }}" in src
    assert "#define COOT_STORE_0 1" in src and "#define COOT_STORE_1 0" in src
    assert "#define COOT_HEADS_1 0u" in src


def test_host_device_pointer_refuses_what_it_cannot_map():
    """A NULL pointer, and host memory the CUDA runtime does not know as
    pinned (here: a plain ctypes buffer), are refused with
    COOT_ERR_INVALID_ARG and a message; no address is returned."""
    dev = ctypes.c_void_p(0)
    st, msg = _call("coot_host_device_pointer", None, ctypes.byref(dev))
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG" and msg and dev.value is None
    buf = ctypes.create_string_buffer(4096)
    st, msg = _call("coot_host_device_pointer", ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(dev))
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG" and msg and dev.value is None
    st, _ = _call("coot_host_device_pointer", ctypes.cast(buf, ctypes.c_void_p), None)
    assert _abi.STATUS[st] == "COOT_ERR_INVALID_ARG"
