"""Pins for the FP64 oracle: closed forms, identities, special cases that
reduce to a library routine, hand-written byte fixtures and brute force on
tiny inputs.  CPU only; nothing here touches the CUDA path."""
import ast
import math
import os
import struct
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import coot_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def vec(values, dtype="f32"):
    a = np.asarray(values, dtype={"f32": np.float32, "f64": np.float64, "f16": np.float16}[dtype])
    return synth.as_mat(a, dtype, a.size, 1)


def mat(m2d, dtype="f32", ld=None):
    m2d = np.asarray(m2d)
    r, c = m2d.shape
    flat = np.asarray(m2d, dtype=np.float32 if dtype == "f32" else np.float64).ravel(order="F")
    return synth.as_mat(flat, dtype, r, c, ld)


X0, X1, X2, X3 = (synth.X(k) for k in range(4))


# ---------------------------------------------------------------- tree format

def _golden_trees():
    out = []
    with open(os.path.join(GOLDEN, "trees.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, hexs, sexpr, cite = [p.strip() for p in line.split("|")]
            out.append((name, bytes.fromhex(hexs.replace(" ", "")), ast.literal_eval(sexpr), cite))
    return out


@pytest.mark.parametrize("name,raw,sexpr,cite", _golden_trees())
def test_golden_tree_bytes(name, raw, sexpr, cite):
    tree = O.decode(raw)
    assert O.to_sexpr(tree) == sexpr
    compute = tree.compute
    assert O.encode(sexpr, n_inputs=tree.n_inputs, compute=compute) == raw


def _hdr(n_nodes, n_inputs=1, compute=0, version=1, magic=b"COOT", r0=0, r1=0):
    return struct.pack("<4sHHBBHI", magic, version, n_nodes, n_inputs, compute, r0, r1)


def _node(op, a=0, b=0, imm=0.0, z0=0, z1=0):
    return struct.pack("<BBHHHd", op, z0, a, b, z1, imm)


@pytest.mark.parametrize("raw", [
    b"",
    _hdr(1, magic=b"COOX") + _node(0),
    _hdr(1, version=2) + _node(0),
    _hdr(0),
    _hdr(65) + _node(0) * 65,
    _hdr(1, n_inputs=0) + _node(0),
    _hdr(1, n_inputs=5) + _node(0),
    _hdr(1, compute=1) + _node(0),
    _hdr(1, r0=1) + _node(0),
    _hdr(2) + _node(0),                       # length mismatch
    _hdr(1) + _node(200),                     # unknown op
    _hdr(1) + _node(0, a=1),                  # slot >= n_inputs
    _hdr(2) + _node(0) + _node(2, a=1),       # self reference
    _hdr(2) + _node(0) + _node(8, a=0, b=2),  # forward reference
    _hdr(2) + _node(0) + _node(2, a=0, b=1),  # unary with a second operand
    _hdr(1) + _node(1, a=1, imm=1.0),         # constant with an operand
    _hdr(1) + _node(0, z0=1),                 # reserved byte set
])
def test_decode_rejects_malformed(raw):
    with pytest.raises(O.TreeError):
        O.decode(raw)


def test_shared_subexpression_is_one_node():
    e = ("add", ("exp", X0), ("exp", X0))
    t = O.decode(O.encode(e))
    assert len(t.nodes) == 3


# ---------------------------------------------------------------- element-wise ops

@pytest.mark.parametrize("sexpr,x,expect", [
    (("neg", X0), 3.0, -3.0),
    (("abs", X0), -2.5, 2.5),
    (("exp", X0), 1.0, math.e),
    (("log", X0), math.e, 1.0),
    (("sqrt", X0), 2.0, math.sqrt(2.0)),
    (("square", X0), -3.0, 9.0),
    (("sub", X0, synth.C(5.0)), 3.0, -2.0),      # A - k
    (("sub", synth.C(5.0), X0), 3.0, 2.0),       # k - A
    (("div", X0, synth.C(4.0)), 1.0, 0.25),      # A / k
    (("div", synth.C(4.0), X0), 1.0, 4.0),       # k / A
    (("add", synth.C(1.5), X0), 2.0, 3.5),       # k + A
    (("mul", synth.C(3.0), X0), 2.0, 6.0),       # k * A
])
def test_each_operator(sexpr, x, expect):
    """Each opcode against its textbook value (Table 2 scalar forms, Table 7)."""
    v = O.evaluate(O.encode(sexpr, compute="f64"), [vec([x], "f64")])
    assert v.shape == (1, 1)
    assert v[0, 0] == pytest.approx(expect, rel=1e-15, abs=0)


def test_binary_operand_order():
    a = vec([3.0, 8.0], "f64")
    b = vec([5.0, 2.0], "f64")
    ms = [a, b]
    assert O.evaluate(O.encode(("sub", X0, X1), compute="f64"), ms).ravel().tolist() == [-2.0, 6.0]
    assert O.evaluate(O.encode(("div", X0, X1), compute="f64"), ms).ravel().tolist() == [0.6, 4.0]
    assert O.evaluate(O.encode(("mul", X0, X1), compute="f64"), ms).ravel().tolist() == [15.0, 16.0]


def test_2x_plus_3z_with_ones_is_five():
    ones = vec(np.ones(17))
    v = O.evaluate(O.encode(synth.AXPY_2X_3Z), [ones, ones])
    assert np.all(v == 5.0)


def test_exp_log_roundtrip():
    x = vec(np.linspace(0.01, 50.0, 101), "f64")
    v = O.evaluate(O.encode(("exp", ("log", X0)), compute="f64"), [x])
    assert np.allclose(v.ravel(), O.logical(x).ravel(), rtol=1e-14, atol=0)


def test_constants_round_to_compute_type():
    x = vec([1.0])
    v32 = O.evaluate(O.encode(("mul", synth.C(0.1), X0), compute="f32"), [x])[0, 0]
    v64 = O.evaluate(O.encode(("mul", synth.C(0.1), X0), compute="f64"), [vec([1.0], "f64")])[0, 0]
    assert v32 == float(np.float32(0.1)) and v32 != 0.1
    assert v64 == 0.1


def test_brute_force_rational():
    """+, -, %, / trees on small dyadic inputs against exact rationals."""
    ops = ["add", "sub", "mul", "div"]
    rng = np.random.default_rng(7)
    for trial in range(200):
        leaves = [X0, X1, X2, synth.C(float(rng.integers(-4, 5)) / 2 or 0.5)]
        def build(d):
            if d == 0 or rng.random() < 0.25:
                return leaves[int(rng.integers(0, 4))]
            return (ops[int(rng.integers(0, 4))], build(d - 1), build(d - 1))
        e = build(4)
        if e[0] in ("x", "c"):
            e = ("add", e, X0)
        vals = [rng.integers(1, 64, size=6) / 8.0 * rng.choice([-1, 1], size=6) for _ in range(3)]
        ms = [vec(v, "f64") for v in vals]
        t = O.encode(e, n_inputs=3, compute="f64")
        got = O.evaluate(t, ms).ravel()
        for i in range(6):
            env = {k: Fraction(float(vals[k][i])) for k in range(3)}
            try:
                ex = O.evaluate_exact(O.to_sexpr(O.decode(t)), env)
            except ZeroDivisionError:
                continue
            if not math.isfinite(got[i]):
                continue
            assert got[i] == pytest.approx(float(ex), rel=1e-12, abs=1e-300), (e, i)


# ---------------------------------------------------------------- reductions: closed forms

@pytest.mark.parametrize("n", [1, 2, 10, 1000, (1 << 20) + 3])
def test_accu_one_to_n(n):
    x = vec(np.arange(1, n + 1, dtype=np.float64))
    assert O.accu(O.encode(X0), [x]) == n * (n + 1) / 2


def test_accu_ones_with_padding():
    r, c, ld = 37, 11, 45          # padding rows hold NaN
    m = synth.as_mat(np.ones(r * c, dtype=np.float32), "f32", r, c, ld)
    assert O.accu(O.encode(X0), [m]) == r * c


@pytest.mark.parametrize("n", [1, 3, 1000, 100003])
def test_dot_one_to_n(n):
    x = vec(np.arange(1, n + 1, dtype=np.float64))
    assert O.dot(x, x) == n * (n + 1) * (2 * n + 1) / 6


def test_dot_needs_equal_counts_not_shapes():
    a = synth.as_mat(np.arange(1, 7, dtype=np.float32), "f32", 1, 6)
    b = synth.as_mat(np.ones(6, dtype=np.float32), "f32", 6, 1)
    assert O.dot(a, b) == 21.0
    with pytest.raises(ValueError):
        O.dot(a, vec(np.ones(5)))


@pytest.mark.parametrize("k", [3.0, -0.5])
def test_norms_of_constants(k):
    n = 1000
    x = vec(np.full(n, k))
    t = O.encode(X0)
    assert O.norm(t, [x], 2) == pytest.approx(abs(k) * math.sqrt(n), rel=1e-15)
    assert O.norm(t, [x], 1) == abs(k) * n
    assert O.norm(t, [x], "inf") == abs(k)
    assert O.norm(t, [x], "-inf") == abs(k)
    r, c = 30, 40
    m = mat(np.full((r, c), k))
    assert O.norm(t, [m], "fro") == pytest.approx(abs(k) * math.sqrt(r * c), rel=1e-15)
    with pytest.raises(O.UnsupportedError):
        O.norm(t, [m], 2)


def test_norm_inf_picks_magnitudes():
    x = vec([-5.0, 2.0, -0.25, 3.0])
    t = O.encode(X0)
    assert O.norm(t, [x], "inf") == 5.0
    assert O.norm(t, [x], "-inf") == 0.25
    assert O.norm(t, [x], 1) == 10.25


def test_sum_dim_orientation():
    """M[i, j] = i + 1000 j: column sums and row sums have distinct closed
    forms, so a transposed or swapped dim fails."""
    r, c = 7, 5
    i = np.arange(r)[:, None]
    j = np.arange(c)[None, :]
    m = mat(i + 1000.0 * j, ld=9)
    t = O.encode(X0)
    col = O.sum_dim(t, [m], 0)
    row = O.sum_dim(t, [m], 1)
    assert col.shape == (c,) and row.shape == (r,)
    assert col.tolist() == [r * (r - 1) / 2 + 1000.0 * jj * r for jj in range(c)]
    assert row.tolist() == [c * ii + 1000.0 * c * (c - 1) / 2 for ii in range(r)]


def test_sum_ones():
    r, c = 13, 6
    m = mat(np.ones((r, c)))
    t = O.encode(X0)
    assert O.sum_dim(t, [m], 0).tolist() == [r] * c
    assert O.sum_dim(t, [m], 1).tolist() == [c] * r


def test_minmax_linspace_endpoints():
    x = vec(np.linspace(-3.0, 7.0, 1001))
    assert O.minmax(O.encode(X0), [x]) == (-3.0, 7.0)


def test_minmax_nan_propagates_and_empty_raises():
    x = vec([1.0, float("nan"), 3.0])
    lo, hi = O.minmax(O.encode(X0), [x])
    assert math.isnan(lo) and math.isnan(hi)
    with pytest.raises(O.EmptyError):
        O.minmax(O.encode(X0), [vec([])])


def test_empty_reductions_are_zero():
    e = vec([])
    t = O.encode(X0)
    assert O.accu(t, [e]) == 0.0
    assert O.dot(e, e) == 0.0
    assert O.norm(t, [e], 2) == 0.0
    assert O.sum_dim(t, [synth.as_mat(np.zeros(0, np.float32), "f32", 0, 4)], 0).tolist() == [0.0] * 4


def test_minmax_rounds_elements_to_f32():
    # 1/3 in FP64 vs its FP32 rounding: the oracle reports the FP32 value
    x = vec([3.0])
    lo, hi = O.minmax(O.encode(("div", synth.C(1.0), X0)), [x])
    assert lo == hi == float(np.float32(1.0 / 3.0))


# ---------------------------------------------------------------- identities

def _rand_mats(seed, r, c, k=4):
    out = []
    for s in range(k):
        flat = synth.uniform_f32(seed + s, r * c)
        out.append(synth.as_mat(flat, "f32", r, c))
    return out


def test_identities():
    ms = _rand_mats(11, 33, 21)
    t = O.encode(synth.MAT_EXPR)
    a = O.accu(t, ms)
    assert math.fsum(O.sum_dim(t, ms, 0)) == pytest.approx(a, rel=1e-14)
    assert math.fsum(O.sum_dim(t, ms, 1)) == pytest.approx(a, rel=1e-14)
    x, z = ms[0], ms[1]
    assert O.dot(x, x) == pytest.approx(O.norm(O.encode(X0), [x], "fro") ** 2, rel=1e-14)
    # products of FP32 values are exact in FP64, so both sides are the same correctly rounded sum
    assert O.accu(O.encode(synth.SCHUR_XZ), [x, z]) == O.dot(x, z)
    assert O.accu(O.encode(("mul", synth.C(4.0), X0)), [x]) == 4.0 * O.accu(O.encode(X0), [x])
    lo, hi = O.minmax(O.encode(X0), [x])
    nlo, nhi = O.minmax(O.encode(("neg", X0)), [x])
    assert hi == -nlo and lo == -nhi


def test_row_sums_are_column_sums_of_transpose():
    r, c = 19, 23
    m2 = np.asarray(synth.uniform_f32(5, r * c)).reshape((r, c), order="F")
    m = mat(m2)
    mt = mat(m2.T)
    t = O.encode(X0)
    assert O.sum_dim(t, [m], 1).tolist() == O.sum_dim(t, [mt], 0).tolist()


def test_accu_uniform_statistics():
    n = 1_000_000
    x = vec(synth.uniform_f32(3, n))
    a = O.accu(O.encode(X0), [x])
    assert abs(a) < 5.0 * math.sqrt(n / 3.0)
    assert O.accu(O.encode(("abs", X0)), [x]) == pytest.approx(n / 2.0, rel=5e-3)


def test_delayed_evaluation_reads_old_values():
    """B = B + 3A (Task 2, B += 3*A): the value is computed from the inputs
    before anything is stored."""
    a = vec([1.0, 2.0])
    b = vec([10.0, 20.0])
    v = O.evaluate(O.encode(("add", X1, ("mul", synth.C(3.0), X0))), [a, b])
    assert v.ravel().tolist() == [13.0, 26.0]


# ---------------------------------------------------------------- storage types

def test_decode_storage_bits():
    bf = np.array([0x3F80, 0xC000, 0x0001, 0x7F80, 0xFF80], dtype=np.uint16)
    assert O.decode_storage(bf, "bf16").tolist() == [1.0, -2.0, 2.0 ** -133, math.inf, -math.inf]
    hf = np.array([0x3C00, 0x0001, 0x7BFF, 0x8400], dtype=np.uint16).view(np.float16)
    assert O.decode_storage(hf, "f16").tolist() == [1.0, 2.0 ** -24, 65504.0, -(2.0 ** -14)]


def _window(fmt, e0, e1):
    """Every representable value of a format in [2**e0, 2**(e1 + 1)], by
    enumeration (normal numbers only), or in [0, 2**emin] for e0 = None
    (the subnormal range)."""
    p, emin, emax = O.FORMATS[fmt]
    if e0 is None:
        return np.array([m * 2.0 ** (emin - p + 1) for m in range(0, 2 ** (p - 1) + 1)])
    vals = [(1 + m / 2 ** (p - 1)) * 2.0 ** e for e in range(e0, e1 + 1) for m in range(2 ** (p - 1))]
    vals.append(2.0 ** (e1 + 1))
    return np.array(vals)


@pytest.mark.parametrize("window", [(None, None), (-126, -124), (-2, 1), (125, 126)])
def test_round_to_bf16_brute_force(window):
    grid = _window("bf16", *window)
    rng = np.random.default_rng(1)
    x = rng.uniform(grid[0], grid[-1], 20000)
    got = O.round_to_format(x, "bf16")
    idx = np.clip(np.searchsorted(grid, x), 1, grid.size - 1)
    lo, hi = grid[idx - 1], grid[idx]
    nearest = np.where(x - lo < hi - x, lo, hi)
    tie = (x - lo) == (hi - x)
    assert np.all((got == nearest) | (tie & ((got == lo) | (got == hi))))


def test_round_to_f16_matches_numpy_and_f32_matches_numpy():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.standard_normal(50000) * 10.0 ** rng.uniform(-9, 5, 50000),
                        [65504.0, 65519.99, 65520.0, -65520.0, 2.0 ** -25, 3 * 2.0 ** -26, 0.0, -0.0]])
    assert np.array_equal(O.round_to_format(x, "f16"), x.astype(np.float16).astype(np.float64))
    y = rng.standard_normal(50000) * 10.0 ** rng.uniform(-45, 38, 50000)
    assert np.array_equal(O.round_to_format(y, "f32"), y.astype(np.float32).astype(np.float64))


def test_round_ties_to_even():
    # halfway between 1 and 1 + 2**-7 in BF16 rounds to the even neighbour 1
    assert O.round_to_format([1.0 + 2.0 ** -8], "bf16")[0] == 1.0
    assert O.round_to_format([1.0 + 3 * 2.0 ** -8], "bf16")[0] == 1.0 + 2.0 ** -6


# ---------------------------------------------------------------- error bound

def _eval_f32_numpy(sexpr, xs32):
    """An independent FP32 evaluation (numpy float32, one rounding per node)."""
    name = sexpr[0]
    with np.errstate(all="ignore"):
        if name == "x":
            return xs32[sexpr[1]]
        if name == "c":
            return np.float32(sexpr[1])
        if name in O.UNARY:
            a = _eval_f32_numpy(sexpr[1], xs32)
            return {"neg": np.negative, "abs": np.abs, "exp": np.exp, "log": np.log,
                    "sqrt": np.sqrt, "square": np.square}[name](a).astype(np.float32)
        a = _eval_f32_numpy(sexpr[1], xs32)
        b = _eval_f32_numpy(sexpr[2], xs32)
        return {"add": np.add, "sub": np.subtract, "mul": np.multiply, "div": np.divide}[name](a, b).astype(np.float32)


@pytest.mark.parametrize("seed", range(40))
def test_error_bound_covers_an_fp32_evaluation(seed):
    n_in = 1 + seed % 4
    e = synth.random_tree(1000 + seed, 2 + seed % 11, n_in)
    r, c = 64, 8
    ms = _rand_mats(50 + seed, r, c, n_in)
    t = O.encode(e, n_inputs=n_in)
    v, bound, unsafe = O.error_bound(t, ms)
    xs32 = [O.logical(m).astype(np.float32) for m in ms]
    g = np.broadcast_to(_eval_f32_numpy(e, xs32), v.shape).astype(np.float64)
    safe = ~unsafe
    fin = safe & np.isfinite(v)
    # numpy's FP32 exp/log are not guaranteed to be CUDA's, so allow a factor 2
    assert np.all(np.abs(g[fin] - v[fin]) <= 2.0 * bound[fin] + 1e-30), e
    nonfin = safe & ~np.isfinite(v)
    assert np.array_equal(np.isnan(g[nonfin]), np.isnan(v[nonfin]))
    assert unsafe.mean() < 0.25


def test_error_bound_is_not_vacuous():
    ms = _rand_mats(9, 128, 4)
    v, bound, unsafe = O.error_bound(O.encode(synth.MAT_EXPR), ms)
    assert not unsafe.any()
    # a handful of roundings of O(1) values: a few FP32 units of the operands
    assert np.max(bound) < 1e-5


# ---------------------------------------------------------------- generator

def test_splitmix64_reference_outputs():
    """SplitMix64 seeded with 0 (the published reference stream)."""
    z = synth.splitmix64(0, 0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_generator_is_chunk_independent():
    a = synth.uniform_f32(42, 10)
    b = synth.uniform01(42, 5, start=5)
    assert np.array_equal(a[5:], (-1.0 + 2.0 * b).astype(np.float32))
