"""FP64 CPU oracle for fused element-wise expressions and their reductions.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check in
`__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import
this module.  It shares no code with the CUDA path: it decodes the tree
byte format itself, from the format's written definition, and computes every
result from the plain definitions below, slowly and in FP64.

What it follows (Bandicoot, arXiv 2308.03120):
  * element-wise operators and scalar operators: Table 2 ("A + k", "k - A",
    "A * k", "A + B", "A - B", "A % B" element-wise product, "A / B"
    element-wise division);
  * element-wise functions exp, log, sqrt, square, pow, log10: Table 7
    ("misc(A)"); cos, sin, tan, acos, asin, atan: Table 7 ("trig(A)"); abs
    and negation are the unary forms of the same family;
  * storage types: FP32, BF16, FP16, FP64 and the integer types int32 and
    uint32 (Section 7's conversion example reads an integer matrix into a
    float expression);
  * relational operators inside expressions ("A < x" and the other
    relational expressions of Table 5's all/any rows);
  * reductions: Table 5 (accu = sum of all elements, dot of two objects with
    equal element counts, norm(A, p), all(A) / any(A) = whether all / any
    elements are nonzero) and Table 6 (sum/min/max along dim 0 = per
    column, dim 1 = per row, and the statistics mean/stddev/var along a
    dim);
  * column-major element order ("(i)" walks the matrix column by column,
    Table 1);
  * delayed evaluation (Section 7): the destination receives the value of
    the whole expression, so an output that aliases an input still sees the
    input's old values.

Readings where the paper is silent (each is listed with its reason in the
design notes of the repository):
  * immediates are stored as FP64 in the tree and rounded to the compute
    type before use (for FP32 compute: nearest FP32), on both sides;
  * an input is converted to the compute type when it is read: FP64, int32
    and uint32 values are rounded to the nearest FP32 for an FP32 tree
    (exact up to 2^24 for the integers); every type is exact in FP64;
  * an integer output receives the value rounded toward zero, saturated to
    the type's range, with NaN stored as 0;
  * pow(a, b) follows C's pow (IEEE 754 pown/powr special cases: pow(x, 0)
    = 1 even for NaN x, a negative base with a non-integer exponent is NaN);
  * min/max propagate NaN; for FP32 compute each element value is rounded to
    FP32 before the extremum is taken (a comparison adds no rounding);
  * norm with p = 2 of a matrix (more than one row and more than one column)
    is the spectral norm, which needs an SVD and is rejected; p = "fro" is
    the Frobenius norm; on a vector p = 2 is the Euclidean norm;
  * empty inputs: accu, dot, norm and sums are 0; min/max raise EmptyError;
    all() of nothing is true and any() of nothing is false;
  * a relational node is 1 where the relation holds and 0 elsewhere, in the
    compute type; NaN is unordered (every relation false except "!=");
  * all/any test each element value, rounded to the compute type, against
    zero (NaN is nonzero);
  * var(A, norm_type, dim) divides by N - 1 (norm_type 0, the default) or by
    N (norm_type 1), N the number of elements reduced; with N = 1 and
    norm_type 0 it is 0; stddev is its square root; mean, var and stddev of
    N = 0 elements are NaN; per-dim min/max round each element to the
    compute type first, like the full min/max.

Sums use math.fsum (the correctly rounded sum of the FP64 element values),
so the only error in an oracle reduction is the rounding of each element's
FP64 value and of the final sum.
"""
from __future__ import annotations

import itertools
import math
import struct
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

# --------------------------------------------------------------------------
# Tree byte format (restated from its definition; little-endian)
#
#   header, 16 bytes: "COOT" | u16 version=1 | u16 n_nodes (1..64)
#                     | u8 n_inputs (1..4) | u8 compute type (0 FP32, 3 FP64)
#                     | u16 0 | u32 0
#   node i, 16 bytes at offset 16 + 16 i:
#                     u8 op | u8 0 | u16 a | u16 b | u16 0 | f64 imm
#   ops:  0 input slot a | 1 constant imm | 2 neg a | 3 abs a | 4 exp a
#         5 log a | 6 sqrt a | 7 square a | 8 a + b | 9 a - b
#         10 a % b (element-wise product) | 11 a / b
#         12 a < b | 13 a <= b | 14 a > b | 15 a >= b | 16 a == b | 17 a != b
#            (1 where the relation holds, else 0)
#         18 pow(a, b) | 19 log10 a | 20 sin a | 21 cos a | 22 tan a
#         23 asin a | 24 acos a | 25 atan a
#   Operands name earlier nodes (a, b < i); the last node is the root.
# --------------------------------------------------------------------------

MAGIC = b"COOT"
VERSION = 1
MAX_NODES = 64
MAX_INPUTS = 4

OP_NAMES = {0: "x", 1: "c", 2: "neg", 3: "abs", 4: "exp", 5: "log", 6: "sqrt",
            7: "square", 8: "add", 9: "sub", 10: "mul", 11: "div",
            12: "lt", 13: "le", 14: "gt", 15: "ge", 16: "eq", 17: "ne",
            18: "pow", 19: "log10", 20: "sin", 21: "cos", 22: "tan", 23: "asin", 24: "acos", 25: "atan"}
NAME_OPS = {v: k for k, v in OP_NAMES.items()}
UNARY = {"neg", "abs", "exp", "log", "sqrt", "square", "log10", "sin", "cos", "tan", "asin", "acos", "atan"}
RELATIONAL = {"lt", "le", "gt", "ge", "eq", "ne"}
BINARY = {"add", "sub", "mul", "div", "pow"} | RELATIONAL
_NUMPY_UNARY = {"log10": np.log10, "sin": np.sin, "cos": np.cos, "tan": np.tan, "asin": np.arcsin,
                "acos": np.arccos, "atan": np.arctan}
COMPUTE = {0: "f32", 3: "f64"}


class TreeError(ValueError):
    pass


class EmptyError(ValueError):
    pass


class UnsupportedError(ValueError):
    pass


@dataclass
class Tree:
    nodes: list          # (name, a, b, imm)
    n_inputs: int
    compute: str         # "f32" or "f64"


def decode(buf: bytes) -> Tree:
    """Parse and validate a serialised tree."""
    buf = bytes(buf)
    if len(buf) < 16:
        raise TreeError("shorter than the header")
    magic, version, n_nodes, n_inputs, compute, r0, r1 = struct.unpack_from("<4sHHBBHI", buf, 0)
    if magic != MAGIC:
        raise TreeError("bad magic")
    if version != VERSION:
        raise TreeError("unknown version")
    if not (1 <= n_nodes <= MAX_NODES):
        raise TreeError("node count out of range")
    if not (1 <= n_inputs <= MAX_INPUTS):
        raise TreeError("input count out of range")
    if compute not in COMPUTE:
        raise TreeError("unknown compute type")
    if r0 or r1:
        raise TreeError("reserved header bytes are not zero")
    if len(buf) != 16 + 16 * n_nodes:
        raise TreeError("length does not match node count")
    nodes = []
    for i in range(n_nodes):
        op, z0, a, b, z1, imm = struct.unpack_from("<BBHHHd", buf, 16 + 16 * i)
        if op not in OP_NAMES:
            raise TreeError(f"node {i}: unknown op {op}")
        if z0 or z1:
            raise TreeError(f"node {i}: reserved bytes are not zero")
        name = OP_NAMES[op]
        if name == "x":
            if a >= n_inputs or b != 0:
                raise TreeError(f"node {i}: bad input slot")
        elif name == "c":
            if a or b:
                raise TreeError(f"node {i}: constant with operands")
        elif name in UNARY:
            if a >= i or b != 0:
                raise TreeError(f"node {i}: bad operand")
        else:
            if a >= i or b >= i:
                raise TreeError(f"node {i}: bad operand")
        nodes.append((name, a, b, imm))
    return Tree(nodes, n_inputs, COMPUTE[compute])


def encode(sexpr, n_inputs: int | None = None, compute: str = "f32") -> bytes:
    """Serialise a nested-tuple expression; equal subexpressions share one
    node.  n_inputs defaults to the largest slot used + 1."""
    nodes = []
    index = {}

    def key(t):
        if t[0] in ("x", "c"):
            return t
        return (t[0],) + tuple(key(c) for c in t[1:])

    def visit(t):
        k = key(t)
        if k in index:
            return index[k]
        name = t[0]
        if name == "x":
            rec = (NAME_OPS["x"], int(t[1]), 0, 0.0)
        elif name == "c":
            rec = (NAME_OPS["c"], 0, 0, float(t[1]))
        elif name in UNARY:
            rec = (NAME_OPS[name], visit(t[1]), 0, 0.0)
        elif name in BINARY:
            a = visit(t[1])
            b = visit(t[2])
            rec = (NAME_OPS[name], a, b, 0.0)
        else:
            raise TreeError(f"unknown op {name!r}")
        nodes.append(rec)
        index[k] = len(nodes) - 1
        return index[k]

    visit(sexpr)
    slots = [a for (op, a, b, imm) in nodes if op == 0]
    if n_inputs is None:
        n_inputs = (max(slots) + 1) if slots else 1
    code = {"f32": 0, "f64": 3}[compute]
    out = struct.pack("<4sHHBBHI", MAGIC, VERSION, len(nodes), n_inputs, code, 0, 0)
    for op, a, b, imm in nodes:
        out += struct.pack("<BBHHHd", op, 0, a, b, 0, imm)
    return out


def to_sexpr(tree: Tree):
    """The nested-tuple form of a decoded tree (shared nodes are repeated)."""
    built = []
    for name, a, b, imm in tree.nodes:
        if name == "x":
            built.append(("x", a))
        elif name == "c":
            built.append(("c", imm))
        elif name in UNARY:
            built.append((name, built[a]))
        else:
            built.append((name, built[a], built[b]))
    return built[-1]


# --------------------------------------------------------------------------
# Storage types
# --------------------------------------------------------------------------

# (significant bits incl. the implicit one, minimum normal exponent, maximum exponent)
FORMATS = {"f32": (24, -126, 127), "bf16": (8, -126, 127), "f16": (11, -14, 15), "f64": (53, -1022, 1023)}


def decode_storage(buf: np.ndarray, dtype: str) -> np.ndarray:
    """Storage elements -> exact FP64 values."""
    if dtype == "f32":
        return buf.astype(np.float64)
    if dtype == "f64":
        return buf.astype(np.float64)
    if dtype == "f16":
        return buf.view(np.float16).astype(np.float64)
    if dtype == "bf16":
        # a BF16 number is the upper half of the FP32 number with the same bits
        return (buf.view(np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
    if dtype == "i32":
        return buf.view(np.int32).astype(np.float64)
    if dtype == "u32":
        return buf.view(np.uint32).astype(np.float64)
    raise ValueError(dtype)


INT_RANGE = {"i32": (-2.0 ** 31, 2.0 ** 31 - 1), "u32": (0.0, 2.0 ** 32 - 1)}


def to_integer(v64, dtype: str) -> np.ndarray:
    """FP64 values -> the integer storage type: rounded toward zero,
    saturated to the type's range, NaN -> 0 (the values as FP64)."""
    lo, hi = INT_RANGE[dtype]
    v = np.asarray(v64, dtype=np.float64)
    with np.errstate(invalid="ignore"):
        t = np.trunc(v)
        t = np.where(np.isnan(v), 0.0, np.clip(t, lo, hi))
    return t


def round_to_format(v, fmt: str) -> np.ndarray:
    """Round FP64 values to the nearest number of a binary format, ties to
    even, with gradual underflow and overflow to infinity (IEEE 754
    roundTiesToEven)."""
    p, emin, emax = FORMATS[fmt]
    v = np.array(v, dtype=np.float64, copy=True)
    out = v.copy()
    fin = np.isfinite(v) & (v != 0.0)
    a = np.abs(v[fin])
    _, ex = np.frexp(a)                     # a = m * 2**ex, m in [0.5, 1)
    e = np.maximum(ex - 1, emin)            # exponent of the leading bit, floored at emin
    q = np.ldexp(1.0, e - (p - 1))          # spacing of the format at that exponent
    r = np.rint(a / q) * q                  # a / q is exact (power-of-two scale)
    largest = (2.0 - 2.0 ** (1 - p)) * 2.0 ** emax
    r = np.where(r > largest, np.inf, r)
    out[fin] = np.copysign(r, v[fin])
    return out


def encode_storage(v64: np.ndarray, dtype: str) -> np.ndarray:
    """FP64 values (already representable) -> storage elements."""
    if dtype == "f32":
        return v64.astype(np.float32)
    if dtype == "f64":
        return v64.astype(np.float64)
    if dtype == "f16":
        return v64.astype(np.float16)
    if dtype == "bf16":
        f = v64.astype(np.float32).view(np.uint32)
        return (f >> np.uint32(16)).astype(np.uint16)
    if dtype in ("i32", "u32"):
        return to_integer(v64, dtype).astype(np.int32 if dtype == "i32" else np.uint32)
    raise ValueError(dtype)


def logical(mat) -> np.ndarray:
    """The (n_rows, n_cols) FP64 matrix held by a column-major buffer:
    element (i, j) is buf[i + j * ld]."""
    i = np.arange(mat.n_rows, dtype=np.int64)[:, None]
    j = np.arange(mat.n_cols, dtype=np.int64)[None, :]
    vals = decode_storage(np.asarray(mat.buf), mat.dtype)
    if mat.n_rows == 0 or mat.n_cols == 0:
        return np.zeros((mat.n_rows, mat.n_cols))
    return vals[i + j * mat.ld]


# --------------------------------------------------------------------------
# Evaluation (Table 2, Table 7; Section 7 delayed evaluation)
# --------------------------------------------------------------------------

def _tree(t) -> Tree:
    return t if isinstance(t, Tree) else decode(t)


def _check_shapes(tree: Tree, mats):
    if len(mats) != tree.n_inputs:
        raise TreeError("input count does not match the tree")
    shape = (mats[0].n_rows, mats[0].n_cols)
    for m in mats:
        if (m.n_rows, m.n_cols) != shape:
            raise ValueError("element-wise operands must have equal sizes")
    return shape


def constant(tree: Tree, imm: float) -> float:
    """An immediate as the compute type sees it."""
    return float(np.float32(imm)) if tree.compute == "f32" else float(imm)


def evaluate(tree, mats) -> np.ndarray:
    """Value of the expression at every element, in FP64."""
    tree = _tree(tree)
    shape = _check_shapes(tree, mats)
    xs = [leaf_values(tree, m) for m in mats]
    vals = []
    with np.errstate(all="ignore"):
        for name, a, b, imm in tree.nodes:
            if name == "x":
                v = xs[a]
            elif name == "c":
                v = np.full(shape, constant(tree, imm))
            elif name == "neg":
                v = -vals[a]
            elif name == "abs":
                v = np.abs(vals[a])
            elif name == "exp":
                v = np.exp(vals[a])
            elif name == "log":
                v = np.log(vals[a])
            elif name == "sqrt":
                v = np.sqrt(vals[a])
            elif name == "square":
                v = vals[a] * vals[a]
            elif name == "add":
                v = vals[a] + vals[b]
            elif name == "sub":
                v = vals[a] - vals[b]
            elif name == "mul":
                v = vals[a] * vals[b]
            elif name == "div":
                v = vals[a] / vals[b]
            elif name in RELATIONAL:
                v = np.where(_relate(name, vals[a], vals[b]), 1.0, 0.0)
            elif name == "pow":
                v = np.power(vals[a], vals[b])
            elif name in _NUMPY_UNARY:
                v = _NUMPY_UNARY[name](vals[a])
            vals.append(v)
    return vals[-1]


def leaf_values(tree: Tree, mat) -> np.ndarray:
    """An input as the compute type reads it: storage types wider than FP32's
    24-bit significand (FP64, int32, uint32) are rounded to the nearest FP32
    for an FP32 tree; everything is exact in FP64."""
    v = logical(mat)
    if tree.compute == "f32" and mat.dtype in ("f64", "i32", "u32"):
        v = round_to_format(v, "f32")
    return v


def _relate(name, x, y):
    """The relation of a relational node (numpy comparisons are IEEE:
    unordered operands make every relation false except !=)."""
    return {"lt": np.less, "le": np.less_equal, "gt": np.greater, "ge": np.greater_equal,
            "eq": np.equal, "ne": np.not_equal}[name](x, y)


def evaluate_exact(sexpr, env: dict):
    """Exact rational value of a +, -, %, / expression over Fraction inputs
    (brute-force check of `evaluate` on tiny inputs)."""
    name = sexpr[0]
    if name == "x":
        return env[sexpr[1]]
    if name == "c":
        return Fraction(sexpr[1])
    if name == "neg":
        return -evaluate_exact(sexpr[1], env)
    if name == "abs":
        return abs(evaluate_exact(sexpr[1], env))
    if name == "square":
        v = evaluate_exact(sexpr[1], env)
        return v * v
    a = evaluate_exact(sexpr[1], env)
    b = evaluate_exact(sexpr[2], env)
    if name == "add":
        return a + b
    if name == "sub":
        return a - b
    if name == "mul":
        return a * b
    if name == "div":
        return a / b
    if name in RELATIONAL:
        return Fraction(int({"lt": a < b, "le": a <= b, "gt": a > b, "ge": a >= b, "eq": a == b,
                             "ne": a != b}[name]))
    raise ValueError(f"no exact form for {name}")


# --------------------------------------------------------------------------
# Forward error bound of a compute-type evaluation (used for tolerances)
# --------------------------------------------------------------------------

# accuracy of the device functions, in units in the last place of the result,
# as documented for CUDA's single and double precision maths (without fast
# maths: IEEE-rounded add, multiply, divide and square root)
# (taken at or above the documented figures: where a figure is not certain
# the larger one is used, which only widens the tolerance)
ULPS = {"f32": {"exp": 2.0, "log": 1.0, "sqrt": 0.5, "op": 0.5, "log10": 2.0, "sin": 2.0, "cos": 2.0,
                "tan": 4.0, "asin": 4.0, "acos": 4.0, "atan": 2.0, "pow": 8.0},
        "f64": {"exp": 1.0, "log": 1.0, "sqrt": 0.5, "op": 0.5, "log10": 2.0, "sin": 2.0, "cos": 2.0,
                "tan": 2.0, "asin": 2.0, "acos": 2.0, "atan": 2.0, "pow": 2.0}}


def error_bound(tree, mats):
    """First-order bound on |fl(expr) - expr| for an evaluation in the
    compute type that rounds every node once (or fuses a multiply-add, which
    only removes a rounding).

    Returns (value, bound, unsafe) arrays.  `unsafe` marks elements where the
    bound says nothing: an intermediate beyond the compute type's range, or a
    log/sqrt/division whose operand's error interval reaches the edge of its
    domain.  Non-finite results that every evaluation must reproduce (for
    example log of a clearly negative number) are safe with bound 0."""
    tree = _tree(tree)
    shape = _check_shapes(tree, mats)
    fmt = tree.compute
    p, emin, emax = FORMATS[fmt]
    u = 2.0 ** -p                                   # unit roundoff
    eta = 2.0 ** (emin - p + 1)                     # subnormal spacing
    big = (2.0 - 2.0 ** (1 - p)) * 2.0 ** emax
    ulp = ULPS[fmt]
    xs = [leaf_values(tree, m) for m in mats]
    vals, errs = [], []
    unsafe = np.zeros(shape, dtype=bool)

    def rnd(v, k=0.5, underflow=True):
        # k ulps of |v|: one ulp is at most 2u|v|, or the subnormal spacing
        # for results that can underflow (a sum or difference that lands in
        # the subnormal range is exact, so add and sub pass underflow=False)
        return (2.0 * k) * u * np.abs(v) + (k * 2.0 * eta if underflow else 0.0)

    with np.errstate(all="ignore"):
        for name, a, b, imm in tree.nodes:
            if name == "x":
                v, e = xs[a], np.zeros(shape)
            elif name == "c":
                v, e = np.full(shape, constant(tree, imm)), np.zeros(shape)
            elif name == "neg":
                v, e = -vals[a], errs[a]
            elif name == "abs":
                v, e = np.abs(vals[a]), errs[a]
            elif name == "square":
                x, ex = vals[a], errs[a]
                v = x * x
                e = 2.0 * np.abs(x) * ex + ex * ex + rnd(v, ulp["op"])
            elif name in ("add", "sub"):
                x, y = vals[a], vals[b]
                v = x + y if name == "add" else x - y
                e = errs[a] + errs[b] + rnd(v, ulp["op"], underflow=False)
            elif name == "mul":
                x, y, ex, ey = vals[a], vals[b], errs[a], errs[b]
                v = x * y
                e = np.abs(x) * ey + np.abs(y) * ex + ex * ey + rnd(v, ulp["op"])
            elif name == "div":
                x, y, ex, ey = vals[a], vals[b], errs[a], errs[b]
                v = x / y
                ay = np.abs(y)
                ok = ay > ey
                e = np.where(ok, (np.abs(x) * ey + ay * ex) / (ay * np.maximum(ay - ey, 1e-300)), np.inf)
                e = e + rnd(v, ulp["op"])
                exact_zero = (y == 0) & (ey == 0) & ((np.abs(x) > ex) | ((x == 0) & (ex == 0)))
                exact_zero |= np.isnan(x) | np.isnan(y)       # NaN in, NaN out
                e = np.where(exact_zero, 0.0, e)
                unsafe |= ~ok & ~exact_zero
            elif name == "exp":
                x, ex = vals[a], errs[a]
                v = np.exp(x)
                e = v * np.expm1(ex) + rnd(v, ulp["exp"])
            elif name == "log":
                x, ex = vals[a], errs[a]
                v = np.log(x)
                ok = x - ex > 0
                certain_nan = (x + ex < 0) | np.isnan(x)
                certain_zero = (x == 0) & (ex == 0)
                e = np.where(ok, -np.log1p(-np.minimum(ex / np.where(ok, x, 1.0), 0.5)), 0.0)
                e = np.where(ok & (ex > 0.5 * x), np.inf, e) + np.where(ok, rnd(v, ulp["log"]), 0.0)
                unsafe |= ~(ok | certain_nan | certain_zero)
            elif name == "sqrt":
                x, ex = vals[a], errs[a]
                v = np.sqrt(x)
                ok = x - ex >= 0
                certain_nan = (x + ex < 0) | np.isnan(x)
                e = np.where(ok, ex / (np.sqrt(np.abs(x)) + np.sqrt(np.maximum(x - ex, 0.0)) + 1e-300), 0.0)
                e = np.where(ok & (ex == 0), 0.0, e) + np.where(ok, rnd(v, ulp["sqrt"]), 0.0)
                unsafe |= ~(ok | certain_nan)
            elif name == "log10":
                x, ex = vals[a], errs[a]
                v = np.log10(x)
                ok = x - ex > 0
                certain_nan = (x + ex < 0) | np.isnan(x)
                certain_zero = (x == 0) & (ex == 0)
                e = np.where(ok, -np.log1p(-np.minimum(ex / np.where(ok, x, 1.0), 0.5)) / math.log(10.0), 0.0)
                e = np.where(ok & (ex > 0.5 * x), np.inf, e) + np.where(ok, rnd(v, ulp["log10"]), 0.0)
                unsafe |= ~(ok | certain_nan | certain_zero)
            elif name in ("sin", "cos"):
                # both are 1-Lipschitz and bounded by 1
                x, ex = vals[a], errs[a]
                v = np.sin(x) if name == "sin" else np.cos(x)
                e = np.minimum(ex, 2.0) + rnd(v, ulp[name])
            elif name == "tan":
                # the operand's interval must not reach a pole pi/2 + k pi;
                # tan is monotonic between poles, so its slope 1 + tan^2 is
                # largest at an end of the interval
                x, ex = vals[a], errs[a]
                v = np.tan(x)
                k_lo = np.floor((x - ex) / np.pi - 0.5)
                k_hi = np.floor((x + ex) / np.pi - 0.5)
                ok = (k_lo == k_hi) | (ex == 0)
                slope = 1.0 + np.maximum(np.tan(x - ex) ** 2, np.tan(x + ex) ** 2)
                e = np.where(ok, ex * slope, 0.0) + rnd(v, ulp["tan"])
                unsafe |= ~(ok | np.isnan(x))
            elif name in ("asin", "acos"):
                # slope 1 / sqrt(1 - x^2): the interval must stay inside
                # (-1, 1) unless the operand is exact
                x, ex = vals[a], errs[a]
                v = np.arcsin(x) if name == "asin" else np.arccos(x)
                ax = np.abs(x)
                ok = ax + ex < 1.0
                exact = (ex == 0) & (ax <= 1.0)
                certain_nan = (ax - ex > 1.0) | np.isnan(x)
                slope = 1.0 / np.sqrt(np.maximum(1.0 - (ax + ex) ** 2, 1e-300))
                e = np.where(ok, ex * slope, 0.0) + np.where(ok | exact, rnd(v, ulp[name]), 0.0)
                unsafe |= ~(ok | exact | certain_nan)
            elif name == "atan":
                x, ex = vals[a], errs[a]
                v = np.arctan(x)
                e = ex / (1.0 + np.maximum(np.abs(x) - ex, 0.0) ** 2) + rnd(v, ulp["atan"])
            elif name == "pow":
                # x^y = exp(y ln|x|) (sign from an integer y): relative
                # perturbations multiply it by at most
                # exp(|y| ex / (|x| - ex) + |ln|x|| ey)
                x, y, ex, ey = vals[a], vals[b], errs[a], errs[b]
                v = np.power(x, y)
                ax = np.abs(x)
                y_int = (ey == 0) & (np.floor(y) == y)
                base_ok = (ax - ex > 0) & ((x > 0) | y_int)
                exact = (ex == 0) & (ey == 0)
                zero_base = (x == 0) & (ex == 0) & ((y - ey > 0) | (y + ey < 0))
                rel = np.abs(y) * ex / np.where(base_ok, ax - ex, 1.0) + \
                    np.abs(np.log(np.where(base_ok, ax, 1.0))) * ey
                e = np.where(base_ok & ~exact, np.abs(v) * np.expm1(np.minimum(rel, 700.0)), 0.0)
                e = e + rnd(v, ulp["pow"])
                unsafe |= ~(base_ok | exact | zero_base | np.isnan(x) | np.isnan(y))
            elif name in RELATIONAL:
                # the result is exactly 0 or 1; it is certain where the
                # operands' error intervals do not reach each other (or both
                # operands are exact)
                x, y, ex, ey = vals[a], vals[b], errs[a], errs[b]
                v = np.where(_relate(name, x, y), 1.0, 0.0)
                e = np.zeros(shape)
                exact = (ex == 0) & (ey == 0)
                apart = np.abs(x - y) > ex + ey
                unsafe |= ~(exact | apart | np.isnan(x) | np.isnan(y))
            # values beyond the compute type's range overflow there but not here
            fin = np.isfinite(v)
            unsafe |= fin & (np.abs(v) > big)
            # non-finite values arise here only from non-finite inputs or from
            # the domain cases above that are certain, and IEEE arithmetic
            # reproduces them in every precision
            e = np.where(fin, e, 0.0)
            unsafe |= fin & ~np.isfinite(e)
            vals.append(v)
            errs.append(e)
    return vals[-1], errs[-1], unsafe


# --------------------------------------------------------------------------
# Reductions (Table 5, Table 6)
# --------------------------------------------------------------------------

def _fsum(x) -> float:
    """Correctly rounded sum of FP64 values: one math.fsum over every value
    (an array, or an iterable of arrays fed one after the other), so the
    values stream through a single exact summation without materialising a
    Python list of all of them."""
    parts = [np.asarray(x, dtype=np.float64).ravel()] if isinstance(x, np.ndarray) else \
        [np.asarray(p, dtype=np.float64).ravel() for p in x]
    if sum(p.size for p in parts) == 0:
        return 0.0
    if not all(np.all(np.isfinite(p)) for p in parts):
        # fsum raises on inf - inf; IEEE summation gives NaN there
        return float(sum(np.sum(p) for p in parts))
    step = 1 << 20
    return math.fsum(itertools.chain.from_iterable(p[i:i + step].tolist() for p in parts
                                                   for i in range(0, p.size, step)))


def accu(tree, mats) -> float:
    """accu(expr): the sum of all elements (Table 5)."""
    return _fsum(evaluate(tree, mats))


def sum_dim(tree, mats, dim: int) -> np.ndarray:
    """sum(expr, dim): dim = 0 gives the sum of each column (a 1 x n_cols
    result), dim = 1 the sum of each row (an n_rows x 1 result) (Table 6)."""
    v = evaluate(tree, mats)
    if dim == 0:
        return np.array([_fsum(v[:, j]) for j in range(v.shape[1])])
    if dim == 1:
        return np.array([_fsum(v[i, :]) for i in range(v.shape[0])])
    raise ValueError("dim must be 0 or 1")


def dot(a, b) -> float:
    """dot(A, B) for objects with equal element counts, taken in column-major
    element order (Table 5)."""
    va = logical(a).ravel(order="F")
    vb = logical(b).ravel(order="F")
    if va.size != vb.size:
        raise ValueError("dot needs equal element counts")
    return _fsum(va * vb)


def norm(tree, mats, p) -> float:
    """norm(expr, p) (Table 5).  p = 2 on a vector and p = "fro" on anything:
    square root of the sum of squares; p = 1: sum of magnitudes; p = "inf":
    largest magnitude; p = "-inf": smallest magnitude (vector norms).  p = 2
    of a matrix is the spectral norm and is not supported."""
    tree = _tree(tree)
    v = evaluate(tree, mats)
    is_vec = v.shape[0] == 1 or v.shape[1] == 1
    if p == "fro" or (p == 2 and is_vec):
        return math.sqrt(_fsum(v * v)) if v.size else 0.0
    if p == 2:
        raise UnsupportedError("p = 2 of a matrix is the spectral norm")
    if not is_vec:
        raise UnsupportedError("p = 1, inf, -inf are vector norms here")
    if v.size == 0:
        return 0.0
    if p == 1:
        return _fsum(np.abs(v))
    if p == "inf":
        return float(np.max(np.abs(v)))
    if p == "-inf":
        return float(np.min(np.abs(v)))
    raise ValueError(f"unknown p {p!r}")


def minmax(tree, mats) -> tuple[float, float]:
    """(min, max) over all elements (Table 6's min/max over both dims).
    Each element is first rounded to the compute type; NaN propagates."""
    tree = _tree(tree)
    v = evaluate(tree, mats)
    if v.size == 0:
        raise EmptyError("min/max of an empty object")
    if tree.compute == "f32":
        v = round_to_format(v, "f32")
    return float(np.min(v)), float(np.max(v))


def _compute_values(tree: Tree, mats) -> np.ndarray:
    """Element values rounded to the compute type (what a comparison with
    zero or an extremum sees)."""
    v = evaluate(tree, mats)
    return round_to_format(v, "f32") if tree.compute == "f32" else v


def all_(tree, mats) -> bool:
    """all(expr): whether every element is nonzero (Table 5); NaN is
    nonzero; true for an empty object."""
    tree = _tree(tree)
    return bool(np.all(_compute_values(tree, mats) != 0.0))


def any_(tree, mats) -> bool:
    """any(expr): whether some element is nonzero (Table 5); false for an
    empty object."""
    tree = _tree(tree)
    return bool(np.any(_compute_values(tree, mats) != 0.0))


STATS = ("sum", "mean", "var", "stddev", "min", "max")


def stats_dim(tree, mats, dim: int, stat: str, norm_type: int = 0) -> np.ndarray:
    """A statistic of each column (dim = 0, a 1 x n_cols result) or of each
    row (dim = 1, an n_rows x 1 result) of expr (Table 6): sum, mean, var,
    stddev, min or max.  var = sum((v - mean)^2) / (N - 1 + norm_type) with
    the mean taken first (two passes), N the elements of the line."""
    tree = _tree(tree)
    if stat not in STATS:
        raise ValueError(f"unknown statistic {stat!r}")
    if dim not in (0, 1):
        raise ValueError("dim must be 0 or 1")
    if norm_type not in (0, 1):
        raise ValueError("norm_type must be 0 or 1")
    v = evaluate(tree, mats)
    lines = [v[:, j] for j in range(v.shape[1])] if dim == 0 else [v[i, :] for i in range(v.shape[0])]
    n = v.shape[0] if dim == 0 else v.shape[1]
    if stat in ("min", "max"):
        if n == 0 and lines:
            raise EmptyError("min/max along a dim of length 0")
        if tree.compute == "f32":
            lines = [round_to_format(x, "f32") for x in lines]
        f = np.min if stat == "min" else np.max
        return np.array([float(f(x)) for x in lines])
    out = []
    for x in lines:
        if stat == "sum":
            out.append(_fsum(x))
            continue
        if n == 0:
            out.append(math.nan)
            continue
        mean = _fsum(x) / n
        if stat == "mean":
            out.append(mean)
            continue
        if n == 1 and norm_type == 0:
            var = 0.0 if np.isfinite(x).all() else math.nan
        else:
            var = _fsum((x - mean) ** 2) / (n - 1 + norm_type)
        out.append(var if stat == "var" else math.sqrt(var) if var >= 0 else math.nan)
    return np.array(out, dtype=np.float64)
