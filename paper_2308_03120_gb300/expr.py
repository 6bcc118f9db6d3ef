"""Armadillo-style expression building (delayed evaluation).

Operators build a tree instead of computing anything, as Bandicoot's
expression templates do (Section 7 of arXiv 2308.03120); `tree()` turns the
tree into the serialised form of include/coot.h, which one library call
evaluates in one fused kernel.  The operators mirror the paper's Table 2:

    x + y, x - y, k + x, x - k, k - x     element-wise / scalar sums
    k * x, x * k                          scalar multiple
    x % y                                 element-wise (Schur) product
    x / y, x / k, k / x                   element-wise division
    -x
and Table 7's element-wise functions exp, log, sqrt, square, pow (also
x ** y), log10, sin, cos, tan, asin, acos, atan, plus abs.
Relational expressions (Table 5's "A < x" inside all/any) build 1/0
nodes: x < y, x <= y, x > y, x >= y, and eq(x, y), ne(x, y) (Python's ==
and != keep their usual meaning on expression objects).
`x * y` of two expressions is a matrix product in Armadillo and is refused
here (matrix multiplication is not an element-wise operation).
"""
from __future__ import annotations

import struct

_OPS = {"x": 0, "c": 1, "neg": 2, "abs": 3, "exp": 4, "log": 5, "sqrt": 6, "square": 7,
        "add": 8, "sub": 9, "mul": 10, "div": 11,
        "lt": 12, "le": 13, "gt": 14, "ge": 15, "eq": 16, "ne": 17,
        "pow": 18, "log10": 19, "sin": 20, "cos": 21, "tan": 22, "asin": 23, "acos": 24, "atan": 25}
_BINARY = ("add", "sub", "mul", "div", "lt", "le", "gt", "ge", "eq", "ne", "pow")
_UNARY = ("neg", "abs", "exp", "log", "sqrt", "square", "log10", "sin", "cos", "tan", "asin", "acos", "atan")


class Expr:
    """A node of an expression tree built with Armadillo's operators (Table
    2): `+`, `-`, `%` (Schur product), `/`, scalar `*`, unary `-`, `abs()`,
    `**`, and the relational operators.  `A * B` between two expressions is
    a matrix product and raises.  `tree()` serialises the tree."""
    __slots__ = ("op", "args", "value")

    def __init__(self, op: str, args=(), value=None):
        self.op = op
        self.args = tuple(args)
        self.value = value

    # ---- construction
    @staticmethod
    def _wrap(v) -> "Expr":
        if isinstance(v, Expr):
            return v
        if isinstance(v, (int, float)):
            return Expr("c", value=float(v))
        raise TypeError(f"cannot use {type(v).__name__} in an expression")

    def __add__(self, o):
        return Expr("add", (self, Expr._wrap(o)))

    def __radd__(self, o):
        return Expr("add", (Expr._wrap(o), self))

    def __sub__(self, o):
        return Expr("sub", (self, Expr._wrap(o)))

    def __rsub__(self, o):
        return Expr("sub", (Expr._wrap(o), self))

    def __mul__(self, o):
        if isinstance(o, Expr):
            raise TypeError("A * B is a matrix product; use A % B for the element-wise product")
        return Expr("mul", (self, Expr._wrap(o)))

    def __rmul__(self, o):
        if isinstance(o, Expr):
            raise TypeError("A * B is a matrix product; use A % B for the element-wise product")
        return Expr("mul", (Expr._wrap(o), self))

    def __mod__(self, o):
        return Expr("mul", (self, Expr._wrap(o)))

    def __rmod__(self, o):
        return Expr("mul", (Expr._wrap(o), self))

    def __truediv__(self, o):
        return Expr("div", (self, Expr._wrap(o)))

    def __rtruediv__(self, o):
        return Expr("div", (Expr._wrap(o), self))

    def __neg__(self):
        return Expr("neg", (self,))

    def __abs__(self):
        return Expr("abs", (self,))

    def __lt__(self, o):
        return Expr("lt", (self, Expr._wrap(o)))

    def __le__(self, o):
        return Expr("le", (self, Expr._wrap(o)))

    def __gt__(self, o):
        return Expr("gt", (self, Expr._wrap(o)))

    def __ge__(self, o):
        return Expr("ge", (self, Expr._wrap(o)))

    def __pow__(self, o):
        return Expr("pow", (self, Expr._wrap(o)))

    def __rpow__(self, o):
        return Expr("pow", (Expr._wrap(o), self))

    # ---- nested-tuple form and serialisation
    def sexpr(self):
        if self.op == "x":
            return ("x", self.value)
        if self.op == "c":
            return ("c", self.value)
        return (self.op,) + tuple(a.sexpr() for a in self.args)

    def n_inputs(self) -> int:
        if self.op == "x":
            return self.value + 1
        if self.op == "c":
            return 0
        return max(a.n_inputs() for a in self.args)

    def tree(self, compute: str = "f32", n_inputs: int | None = None) -> bytes:
        return serialize(self.sexpr(), compute=compute, n_inputs=n_inputs)


def var(k: int) -> Expr:
    """Input slot k (0..3)."""
    if not 0 <= k < 4:
        raise ValueError("input slots are 0..3")
    return Expr("x", value=int(k))


def const(v: float) -> Expr:
    """A constant leaf (stored as FP64, rounded to the compute type)."""
    return Expr("c", value=float(v))


def exp(e):
    """exp(e), element-wise (Table 7)."""
    return Expr("exp", (Expr._wrap(e),))


def log(e):
    """Natural log(e), element-wise (Table 7)."""
    return Expr("log", (Expr._wrap(e),))


def sqrt(e):
    """sqrt(e), element-wise (Table 7)."""
    return Expr("sqrt", (Expr._wrap(e),))


def square(e):
    """e * e, element-wise (Table 7)."""
    return Expr("square", (Expr._wrap(e),))


def abs_(e):
    """|e|, element-wise (Table 7)."""
    return Expr("abs", (Expr._wrap(e),))


def pow_(a, b):
    """pow(a, b), element-wise (Table 7)."""
    return Expr("pow", (Expr._wrap(a), Expr._wrap(b)))


def log10(e):
    """log10(e), element-wise (Table 7)."""
    return Expr("log10", (Expr._wrap(e),))


def sin(e):
    """sin(e), element-wise (Table 7)."""
    return Expr("sin", (Expr._wrap(e),))


def cos(e):
    """cos(e), element-wise (Table 7)."""
    return Expr("cos", (Expr._wrap(e),))


def tan(e):
    """tan(e), element-wise (Table 7)."""
    return Expr("tan", (Expr._wrap(e),))


def asin(e):
    """asin(e), element-wise (Table 7)."""
    return Expr("asin", (Expr._wrap(e),))


def acos(e):
    """acos(e), element-wise (Table 7)."""
    return Expr("acos", (Expr._wrap(e),))


def atan(e):
    """atan(e), element-wise (Table 7)."""
    return Expr("atan", (Expr._wrap(e),))


def eq(a, b):
    """1 where a == b, else 0."""
    return Expr("eq", (Expr._wrap(a), Expr._wrap(b)))


def ne(a, b):
    """1 where a != b (NaN included), else 0."""
    return Expr("ne", (Expr._wrap(a), Expr._wrap(b)))


def as_expr(sexpr) -> Expr:
    """Expr from the nested-tuple form (("x", k), ("c", v), (op, a[, b]))."""
    op = sexpr[0]
    if op == "x":
        return var(sexpr[1])
    if op == "c":
        return const(sexpr[1])
    return Expr(op, tuple(as_expr(a) for a in sexpr[1:]))


def serialize(sexpr, compute: str = "f32", n_inputs: int | None = None) -> bytes:
    """Nested-tuple expression -> tree bytes (include/coot.h layout).  Equal
    subexpressions become one shared node."""
    nodes: list[tuple[int, int, int, float]] = []
    seen: dict = {}

    def walk(t) -> int:
        if t in seen:
            return seen[t]
        op = t[0]
        if op == "x":
            rec = (_OPS["x"], int(t[1]), 0, 0.0)
        elif op == "c":
            rec = (_OPS["c"], 0, 0, float(t[1]))
        elif op in _UNARY:
            rec = (_OPS[op], walk(t[1]), 0, 0.0)
        elif op in _BINARY:
            a = walk(t[1])
            b = walk(t[2])
            rec = (_OPS[op], a, b, 0.0)
        else:
            raise ValueError(f"unknown operator {op!r}")
        nodes.append(rec)
        seen[t] = len(nodes) - 1
        return seen[t]

    walk(_hashable(sexpr))
    if n_inputs is None:
        slots = [a for (op, a, _, _) in nodes if op == 0]
        n_inputs = max(slots) + 1 if slots else 1
    head = struct.pack("<4sHHBBHI", b"COOT", 1, len(nodes), n_inputs, {"f32": 0, "f64": 3}[compute], 0, 0)
    return head + b"".join(struct.pack("<BBHHHd", op, 0, a, b, 0, imm) for op, a, b, imm in nodes)


def _hashable(t):
    if t[0] in ("x", "c"):
        return (t[0], t[1])
    return (t[0],) + tuple(_hashable(a) for a in t[1:])
