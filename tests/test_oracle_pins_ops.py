"""Pins for the oracle's Table 7 functions pow, log10, sin, cos, tan, asin,
acos, atan, its integer storage types and its input conversion: values by
hand, C's special cases of pow, trigonometric identities, an independent
FP32 evaluation inside the error bound, and integer rounding by hand.  CPU
only."""
import math

import numpy as np
import pytest

import synth
from oracle import coot_oracle as O

X0, X1, C = synth.X(0), synth.X(1), synth.C


def vec(values, dtype="f64"):
    a = np.asarray(values, dtype={"f32": np.float32, "f64": np.float64, "i32": np.int32, "u32": np.uint32}[dtype])
    return synth.as_mat(a, dtype, a.size, 1)


def ev(sexpr, *cols, compute="f64", dtype="f64"):
    return O.evaluate(O.encode(sexpr, n_inputs=max(1, len(cols)), compute=compute),
                      [vec(c, dtype) for c in cols]).ravel()


# ---------------------------------------------------------------- values by hand

def test_trig_and_log10_at_known_points():
    pi = math.pi
    assert ev(("sin", X0), [pi / 6, 0.0, -pi / 2]) == pytest.approx([0.5, 0.0, -1.0], rel=1e-15, abs=1e-16)
    assert ev(("cos", X0), [0.0, pi, pi / 3]) == pytest.approx([1.0, -1.0, 0.5], rel=1e-15)
    assert ev(("tan", X0), [pi / 4, 0.0, -pi / 4]) == pytest.approx([1.0, 0.0, -1.0], rel=1e-15, abs=1e-16)
    assert ev(("asin", X0), [1.0, -0.5, 0.0]) == pytest.approx([pi / 2, -pi / 6, 0.0], rel=1e-15)
    assert ev(("acos", X0), [-1.0, 0.5, 1.0]) == pytest.approx([pi, pi / 3, 0.0], rel=1e-15, abs=1e-16)
    assert ev(("atan", X0), [1.0, -1.0, 0.0]) == pytest.approx([pi / 4, -pi / 4, 0.0], rel=1e-15)
    assert ev(("log10", X0), [1000.0, 1.0, 0.01]).tolist() == [3.0, 0.0, -2.0]
    out = ev(("log10", X0), [0.0, -1.0])
    assert out[0] == -math.inf and math.isnan(out[1])
    assert all(math.isnan(v) for v in ev(("asin", X0), [1.5, -2.0]))
    assert all(math.isnan(v) for v in ev(("sin", X0), [math.inf, math.nan]))


def test_pow_follows_c():
    p = ("pow", X0, X1)
    assert ev(p, [2.0, 3.0, -2.0, 9.0], [10.0, 0.0, 3.0, 0.5]).tolist() == [1024.0, 1.0, -8.0, 3.0]
    assert ev(p, [math.nan], [0.0]).tolist() == [1.0]             # x^0 = 1 even for NaN x
    assert ev(p, [1.0], [math.nan]).tolist() == [1.0]             # 1^y = 1 even for NaN y
    assert math.isnan(ev(p, [-8.0], [1.0 / 3.0])[0])              # negative base, non-integer power
    assert ev(p, [0.0, -0.0, 0.0], [-1.0, -1.0, 2.0]).tolist() == [math.inf, -math.inf, 0.0]
    assert ev(p, [-2.0], [-2.0]).tolist() == [0.25]


def test_trig_identities_on_random_values():
    x = synth.uniform01(17, 2000) * 20.0 - 10.0
    s, c, t = ev(("sin", X0), x), ev(("cos", X0), x), ev(("tan", X0), x)
    np.testing.assert_allclose(s * s + c * c, 1.0, rtol=0, atol=4e-16)
    ok = np.abs(c) > 1e-3
    np.testing.assert_allclose(t[ok], s[ok] / c[ok], rtol=1e-14)
    h = synth.uniform01(18, 2000) * math.pi - math.pi / 2
    np.testing.assert_allclose(ev(("asin", ("sin", X0)), h), h, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(ev(("atan", ("tan", X0)), h * 0.999), h * 0.999, rtol=1e-13, atol=1e-15)
    q = 0.05 + synth.uniform01(19, 2000) * (math.pi - 0.1)     # acos is well conditioned away from 0 and pi
    np.testing.assert_allclose(ev(("acos", ("cos", X0)), q), q, rtol=1e-13)
    y = synth.uniform01(20, 2000) * 100.0 + 1e-3
    np.testing.assert_allclose(ev(("log10", X0), y), np.log(y) / math.log(10.0), rtol=1e-15)
    z = synth.uniform01(21, 2000) * 4.0 - 2.0
    np.testing.assert_allclose(ev(("pow", X0, X1), y, z), np.exp(z * np.log(y)), rtol=1e-13)


# ---------------------------------------------------------------- error bound of the new functions

def _f32_numpy(sexpr, xs32):
    """Independent FP32 evaluation with numpy's float32 functions."""
    name = sexpr[0]
    if name == "x":
        return xs32[sexpr[1]]
    if name == "c":
        return np.float32(sexpr[1])
    f = {"sin": np.sin, "cos": np.cos, "tan": np.tan, "asin": np.arcsin, "acos": np.arccos, "atan": np.arctan,
         "log10": np.log10, "exp": np.exp, "log": np.log, "sqrt": np.sqrt, "abs": np.abs, "neg": np.negative}
    with np.errstate(all="ignore"):
        if name in f:
            return f[name](_f32_numpy(sexpr[1], xs32)).astype(np.float32)
        a, b = _f32_numpy(sexpr[1], xs32), _f32_numpy(sexpr[2], xs32)
        g = {"add": np.add, "sub": np.subtract, "mul": np.multiply, "div": np.divide, "pow": np.power}[name]
        return g(np.float32(a), np.float32(b)).astype(np.float32)


TREES = [
    ("sin", ("mul", X0, X1)),
    ("cos", ("add", X0, ("mul", C(3.0), X1))),
    ("tan", ("mul", C(1.4), X0)),
    ("asin", ("mul", C(0.9), X0)),
    ("acos", ("mul", X0, X1)),
    ("atan", ("div", X0, ("add", C(0.1), ("abs", X1)))),
    ("log10", ("add", C(1.5), X0)),
    ("pow", ("add", C(1.5), X0), X1),
    ("pow", X0, C(3.0)),
    ("pow", ("abs", X0), ("mul", C(2.5), X1)),
    ("add", ("sin", X0), ("pow", ("cos", X1), C(2.0))),
]


@pytest.mark.parametrize("sexpr", TREES)
def test_error_bound_covers_an_fp32_evaluation_of_the_new_functions(sexpr):
    n = 4000
    xs = [synth.uniform_f32(31 + k, n) for k in range(2)]
    ms = [synth.as_mat(x, "f32", n, 1) for x in xs]
    n_in = synth.tree_inputs(sexpr)
    t = O.encode(sexpr, n_inputs=n_in)
    v, bound, unsafe = O.error_bound(t, ms[:n_in])
    g = np.asarray(_f32_numpy(sexpr, xs), dtype=np.float64) * np.ones(n)
    safe = ~unsafe
    fin = safe & np.isfinite(v)
    f = fin.ravel()
    assert np.all(np.abs(g[f] - v.ravel()[f]) <= bound.ravel()[f] + 1e-30), sexpr
    nonfin = (safe & ~np.isfinite(v)).ravel()
    assert np.array_equal(np.isnan(g[nonfin]), np.isnan(v.ravel()[nonfin]))
    assert unsafe.mean() < 0.05, (sexpr, unsafe.mean())


def test_error_bound_flags_the_domain_edges():
    # tan at a pole of its operand's interval, asin at the edge, pow of a
    # base interval around zero: unsafe; exact operands: safe
    x = synth.as_mat(np.array([np.float32(math.pi / 2), 0.5, 1.0], np.float32), "f32", 3, 1)
    # fl32(pi/2) lies 4.4e-8 above the pole; adding 1e-8 rounds by about 9e-8
    _, _, unsafe = O.error_bound(O.encode(("tan", ("add", X0, C(1e-8)))), [x])
    assert unsafe.ravel().tolist() == [True, False, False]
    _, _, unsafe = O.error_bound(O.encode(("asin", ("mul", X0, C(0.1)))), [x])
    assert not unsafe.any()
    _, _, unsafe = O.error_bound(O.encode(("asin", X0)), [x])          # exact 1.0: in the domain
    assert not unsafe.any()
    _, _, unsafe = O.error_bound(O.encode(("asin", ("mul", X0, C(1.0 / 3.0)))), [synth.as_mat(
        np.array([3.0], np.float32), "f32", 1, 1)])                         # 3 * (1/3) rounds near 1
    assert unsafe.all()
    # a base whose error interval holds zero: x * 0.1 - 0.1 at x = 1
    one = synth.as_mat(np.array([1.0], np.float32), "f32", 1, 1)
    _, _, unsafe = O.error_bound(O.encode(("pow", ("sub", ("mul", X0, C(0.1)), C(0.1)), C(0.5))), [one])
    assert unsafe.all()
    # the same base exactly zero (no rounding on the way): 0^0.5 = 0, safe
    _, _, unsafe = O.error_bound(O.encode(("pow", ("sub", X0, C(1.0)), C(0.5))), [one])
    assert not unsafe.any()


# ---------------------------------------------------------------- integer storage and conversion

def test_integer_storage_decodes_exactly():
    a = np.array([0, 1, -1, 2 ** 31 - 1, -2 ** 31], dtype=np.int32)
    assert O.decode_storage(a, "i32").tolist() == [0.0, 1.0, -1.0, 2.0 ** 31 - 1, -2.0 ** 31]
    b = np.array([0, 1, 2 ** 32 - 1], dtype=np.uint32)
    assert O.decode_storage(b, "u32").tolist() == [0.0, 1.0, 2.0 ** 32 - 1]


def test_integer_outputs_truncate_and_saturate():
    v = np.array([2.7, -2.7, 0.5, -0.5, 1e10, -1e10, math.inf, -math.inf, math.nan, 2147483647.9])
    assert O.to_integer(v, "i32").tolist() == [2.0, -2.0, 0.0, 0.0, 2.0 ** 31 - 1, -2.0 ** 31, 2.0 ** 31 - 1,
                                               -2.0 ** 31, 0.0, 2.0 ** 31 - 1]
    assert O.to_integer(v, "u32").tolist() == [2.0, 0.0, 0.0, 0.0, 2.0 ** 32 - 1, 0.0, 2.0 ** 32 - 1, 0.0, 0.0,
                                               2147483647.0]
    assert O.encode_storage(np.array([3.9, -7.2]), "i32").tolist() == [3, -7]


def test_fp32_tree_rounds_wide_inputs_on_load():
    # int32 above 2^24 and FP64 are rounded to the nearest FP32 (ties to even)
    big = np.array([2 ** 24 + 1, 2 ** 24 + 3, 2 ** 31 - 1, -(2 ** 24) - 1], dtype=np.int32)
    t32 = O.encode(X0, compute="f32")
    t64 = O.encode(X0, compute="f64")
    m = synth.as_mat(big, "i32", 4, 1)
    assert O.evaluate(t32, [m]).ravel().tolist() == [2.0 ** 24, 2.0 ** 24 + 4, 2.0 ** 31, -(2.0 ** 24)]
    assert O.evaluate(t64, [m]).ravel().tolist() == [float(x) for x in big]
    u = synth.as_mat(np.array([2 ** 32 - 1], dtype=np.uint32), "u32", 1, 1)
    assert O.evaluate(t32, [u]).ravel().tolist() == [2.0 ** 32]
    d = synth.as_mat(np.array([0.1]), "f64", 1, 1)
    assert O.evaluate(t32, [d]).ravel().tolist() == [float(np.float32(0.1))]
    assert O.evaluate(t64, [d]).ravel().tolist() == [0.1]
