"""Pins for the oracle's relational operators, all/any and per-dim
statistics: values by hand, exact rational brute force, closed forms,
Python's `statistics` module (exact rational arithmetic on floats) and
identities with the other reductions.  CPU only."""
import math
import statistics
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import coot_oracle as O

X0, X1 = synth.X(0), synth.X(1)


def vec(values, dtype="f32"):
    a = np.asarray(values, dtype=np.float32 if dtype == "f32" else np.float64)
    return synth.as_mat(a, dtype, a.size, 1)


def mat(m2d, dtype="f32"):
    m2d = np.asarray(m2d, dtype=np.float64)
    r, c = m2d.shape
    flat = np.asarray(m2d, dtype=np.float32 if dtype == "f32" else np.float64).ravel(order="F")
    return synth.as_mat(flat, dtype, r, c)


# ---------------------------------------------------------------- relational operators

@pytest.mark.parametrize("name,want", [
    ("lt", [1, 1, 0, 0, 0]), ("le", [1, 1, 1, 0, 0]), ("gt", [0, 0, 0, 1, 0]),
    ("ge", [0, 0, 1, 1, 0]), ("eq", [0, 0, 1, 0, 0]), ("ne", [1, 1, 0, 1, 1])])
def test_relational_by_hand(name, want):
    # values -1, 0, 0.5, 1, NaN against 0.5; NaN is unordered
    x = vec([-1.0, 0.0, 0.5, 1.0, math.nan])
    got = O.evaluate(O.encode((name, X0, synth.C(0.5))), [x]).ravel()
    assert got.tolist() == [float(w) for w in want]


def test_relational_operand_order():
    # a < b is not b < a: 1 < 2 holds, 2 < 1 does not
    a, b = vec([1.0, 2.0]), vec([2.0, 1.0])
    assert O.evaluate(O.encode(("lt", X0, X1)), [a, b]).ravel().tolist() == [1.0, 0.0]
    assert O.evaluate(O.encode(("gt", X0, X1)), [a, b]).ravel().tolist() == [0.0, 1.0]


def test_relational_trees_match_exact_rationals():
    rng = np.random.default_rng(5)
    for trial in range(200):
        name = ["lt", "le", "gt", "ge", "eq", "ne"][trial % 6]
        # (x0 op1 x1) relation (x1 op2 c) on small integers: exact in FP64
        op1, op2 = rng.choice(["add", "sub", "mul"], 2)
        c = float(rng.integers(-3, 4))
        sexpr = (name, (op1, X0, X1), (op2, X1, synth.C(c)))
        xs = rng.integers(-4, 5, size=(2, 8)).astype(np.float64)
        got = O.evaluate(O.encode(sexpr), [vec(xs[0]), vec(xs[1])]).ravel()
        for i in range(8):
            env = {0: Fraction(int(xs[0, i])), 1: Fraction(int(xs[1, i]))}
            assert got[i] == float(O.evaluate_exact(sexpr, env))


def test_relational_node_feeds_arithmetic():
    # (x > 0) % x keeps the positive part: the relational value is 1 or 0
    x = vec([-2.0, -0.5, 0.0, 0.25, 3.0])
    got = O.evaluate(O.encode(("mul", ("gt", X0, synth.C(0.0)), X0)), [x]).ravel()
    assert got.tolist() == [0.0, 0.0, 0.0, 0.25, 3.0]


def test_relational_error_bound_flags_uncertain_decisions():
    # x * 0.1 compared with 0.1: x = 1 is on the edge (0.1 is inexact), x = 3
    # is clearly above
    x = vec([1.0, 3.0])
    _, e, unsafe = O.error_bound(O.encode(("gt", ("mul", X0, synth.C(0.1)), synth.C(0.1))), [x])
    assert unsafe.ravel().tolist() == [True, False]
    assert e.ravel().tolist() == [0.0, 0.0]
    # exact operands: no uncertainty even at equality
    _, _, unsafe = O.error_bound(O.encode(("ge", X0, synth.C(1.0))), [x])
    assert not unsafe.any()


# ---------------------------------------------------------------- all / any

def test_all_any_by_hand():
    leaf = O.encode(X0)
    assert O.all_(leaf, [vec([1.0, -2.0, 0.5])]) is True
    assert O.all_(leaf, [vec([1.0, 0.0, 0.5])]) is False
    assert O.all_(leaf, [vec([1.0, math.nan])]) is True          # NaN is nonzero
    assert O.any_(leaf, [vec([0.0, -0.0, 0.0])]) is False
    assert O.any_(leaf, [vec([0.0, math.nan])]) is True
    empty = synth.as_mat(np.zeros(0, np.float32), "f32", 0, 3)
    assert O.all_(leaf, [empty]) is True
    assert O.any_(leaf, [empty]) is False


def test_all_any_of_a_relation_agree_with_minmax():
    rng = np.random.default_rng(7)
    for _ in range(50):
        x = vec(rng.uniform(-1, 1, 17))
        k = float(np.float32(rng.uniform(-1.2, 1.2)))
        lo, hi = O.minmax(O.encode(X0), [x])
        assert O.all_(O.encode(("lt", X0, synth.C(k))), [x]) == (hi < k)
        assert O.any_(O.encode(("lt", X0, synth.C(k))), [x]) == (lo < k)
        assert O.all_(O.encode(("ge", X0, synth.C(k))), [x]) == (lo >= k)


def test_all_tests_the_compute_type_value():
    # 1e-10 * 1e-40 is about 1e-50: nonzero in FP64, zero once rounded to FP32
    x = vec([1e-10, 1.0], "f64")
    tree32 = O.encode(("mul", X0, synth.C(1e-40)), compute="f32")
    tree64 = O.encode(("mul", X0, synth.C(1e-40)), compute="f64")
    assert O.all_(tree32, [x]) is False
    assert O.all_(tree64, [x]) is True


# ---------------------------------------------------------------- per-dim statistics

def test_stats_closed_forms_of_1_to_n():
    for n in (1, 2, 7, 100, 1001):
        col = np.arange(1, n + 1, dtype=np.float64)
        m = mat(col[:, None])
        leaf = O.encode(X0)
        assert O.stats_dim(leaf, [m], 0, "sum")[0] == n * (n + 1) / 2
        assert O.stats_dim(leaf, [m], 0, "mean")[0] == (n + 1) / 2
        if n > 1:
            assert O.stats_dim(leaf, [m], 0, "var")[0] == pytest.approx(n * (n + 1) / 12, rel=1e-15)
        assert O.stats_dim(leaf, [m], 0, "var", 1)[0] == pytest.approx((n * n - 1) / 12, rel=1e-15)
        assert O.stats_dim(leaf, [m], 0, "stddev")[0] == pytest.approx(
            math.sqrt(n * (n + 1) / 12) if n > 1 else 0.0, rel=1e-15)
        assert O.stats_dim(leaf, [m], 0, "min")[0] == 1.0
        assert O.stats_dim(leaf, [m], 0, "max")[0] == n


def test_stats_match_the_statistics_module():
    # statistics.mean / variance / pvariance / stdev work in exact rationals
    rng = np.random.default_rng(11)
    leaf = O.encode(X0)
    for trial in range(40):
        r = int(rng.integers(2, 40))
        c = int(rng.integers(1, 6))
        a = np.float32(rng.normal(rng.uniform(-5, 5), rng.uniform(0.01, 3), (r, c))).astype(np.float64)
        m = mat(a)
        for dim in (0, 1):
            lines = [a[:, j] for j in range(c)] if dim == 0 else [a[i, :] for i in range(r)]
            n = len(lines[0])
            got = {s: O.stats_dim(leaf, [m], dim, s) for s in ("mean", "var", "stddev")}
            got1 = O.stats_dim(leaf, [m], dim, "var", 1)
            for k, line in enumerate(lines):
                vals = line.tolist()
                assert got["mean"][k] == pytest.approx(statistics.mean(vals), rel=1e-14, abs=1e-14)
                if n > 1:
                    assert got["var"][k] == pytest.approx(statistics.variance(vals), rel=1e-12, abs=1e-300)
                    assert got["stddev"][k] == pytest.approx(statistics.stdev(vals), rel=1e-12, abs=1e-300)
                assert got1[k] == pytest.approx(statistics.pvariance(vals), rel=1e-12, abs=1e-300)


def test_stats_orientation_on_i_plus_1000_j():
    r, c = 5, 4
    a = np.arange(r)[:, None] + 1000.0 * np.arange(c)[None, :]
    m = mat(a)
    leaf = O.encode(X0)
    j = np.arange(c)
    i = np.arange(r)
    assert O.stats_dim(leaf, [m], 0, "mean").tolist() == ((r - 1) / 2 + 1000.0 * j).tolist()
    assert O.stats_dim(leaf, [m], 1, "mean").tolist() == (i + 1000.0 * (c - 1) / 2).tolist()
    np.testing.assert_allclose(O.stats_dim(leaf, [m], 0, "var"), r * (r + 1) / 12, rtol=1e-15)
    np.testing.assert_allclose(O.stats_dim(leaf, [m], 1, "var"), 1e6 * c * (c + 1) / 12, rtol=1e-15)
    assert O.stats_dim(leaf, [m], 0, "min").tolist() == (1000.0 * j).tolist()
    assert O.stats_dim(leaf, [m], 0, "max").tolist() == (r - 1 + 1000.0 * j).tolist()
    assert O.stats_dim(leaf, [m], 1, "min").tolist() == i.astype(float).tolist()
    assert O.stats_dim(leaf, [m], 1, "max").tolist() == (i + 1000.0 * (c - 1)).tolist()
    assert O.stats_dim(leaf, [m], 0, "sum").tolist() == O.sum_dim(leaf, [m], 0).tolist()
    assert O.stats_dim(leaf, [m], 1, "sum").tolist() == O.sum_dim(leaf, [m], 1).tolist()


def test_stats_shift_and_scale():
    # integers in columns of 32: the mean is a dyadic rational and every step
    # before the final division is exact, so var(x + 1000) == var(x) and
    # var(2 x) == 4 var(x) hold exactly
    rng = np.random.default_rng(3)
    a = rng.integers(-50, 50, size=(32, 3)).astype(np.float64)
    v = O.stats_dim(O.encode(X0), [mat(a)], 0, "var")
    assert O.stats_dim(O.encode(X0), [mat(a + 1000.0)], 0, "var").tolist() == v.tolist()
    assert O.stats_dim(O.encode(X0), [mat(2.0 * a)], 0, "var").tolist() == (4.0 * v).tolist()
    # and through a tree: var(x * 2 + 1000) from the tree equals 4 var(x)
    t = O.encode(("add", ("mul", X0, synth.C(2.0)), synth.C(1000.0)))
    assert O.stats_dim(t, [mat(a)], 0, "var").tolist() == (4.0 * v).tolist()


def test_stats_degenerate_lines():
    leaf = O.encode(X0)
    one = mat(np.array([[3.5, -1.0, 7.0]]))          # 1 x 3: a single element per column
    assert O.stats_dim(leaf, [one], 0, "var").tolist() == [0.0, 0.0, 0.0]
    assert O.stats_dim(leaf, [one], 0, "var", 1).tolist() == [0.0, 0.0, 0.0]
    assert O.stats_dim(leaf, [one], 0, "mean").tolist() == [3.5, -1.0, 7.0]
    empty_rows = synth.as_mat(np.zeros(0, np.float32), "f32", 0, 3)
    assert O.stats_dim(leaf, [empty_rows], 0, "sum").tolist() == [0.0, 0.0, 0.0]
    assert all(math.isnan(x) for x in O.stats_dim(leaf, [empty_rows], 0, "mean"))
    assert all(math.isnan(x) for x in O.stats_dim(leaf, [empty_rows], 0, "var"))
    with pytest.raises(O.EmptyError):
        O.stats_dim(leaf, [empty_rows], 0, "min")
    assert O.stats_dim(leaf, [empty_rows], 1, "mean").size == 0


def test_stats_nan_stays_in_its_line():
    a = np.array([[1.0, 2.0], [math.nan, 4.0], [3.0, 6.0]])
    leaf = O.encode(X0)
    for s in ("sum", "mean", "var", "stddev", "min", "max"):
        got = O.stats_dim(leaf, [mat(a)], 0, s)
        assert math.isnan(got[0]) and not math.isnan(got[1]), s
    assert O.stats_dim(leaf, [mat(a)], 0, "var")[1] == 4.0
