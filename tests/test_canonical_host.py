"""Canonical forms of trees (host-only): the rewrites by hand, and their
exactness -- the canonical tree gives bit-for-bit the value of the original
on random trees with redundancy injected, under the FP64 oracle and under an
independent numpy FP32 evaluation.  No GPU needed."""
import math

import numpy as np
import pytest

import paper_2308_03120_gb300 as coot
import synth
from oracle import coot_oracle as O

X0, X1, X2, C = synth.X(0), synth.X(1), synth.X(2), synth.C


def canon(sexpr, n_inputs=None, compute="f32"):
    t = O.encode(sexpr, n_inputs=n_inputs, compute=compute)
    return O.decode(coot.coot_tree_canonical(t))


@pytest.mark.parametrize("sexpr,want", [
    (("neg", ("neg", X0)), X0),
    (("mul", ("add", C(2), C(3)), X0), ("mul", C(5.0), X0)),
    (("exp", C(1.0)), ("exp", C(1.0))),                                  # library functions are not folded
    (("mul", X0, C(1)), X0),
    (("div", X0, C(-1)), ("neg", X0)),
    (("sub", X0, C(0)), X0),
    (("add", X0, C(0)), ("add", C(0.0), X0)),                          # x + 0 is kept (-0 + 0 = +0)
    (("add", X0, C(-0.0)), X0),
    (("mul", ("neg", X0), ("neg", X1)), ("mul", X0, X1)),
    (("div", ("neg", X0), ("neg", X1)), ("div", X0, X1)),
    (("sub", X0, ("neg", X1)), ("add", X0, X1)),
    (("add", ("neg", X0), X1), ("sub", X1, X0)),
    (("mul", C(4), ("mul", C(2), X0)), ("mul", C(8.0), X0)),
    (("mul", C(0.5), ("mul", C(2), X0)), ("mul", C(0.5), ("mul", C(2.0), X0))),  # not merged
    (("neg", ("mul", C(3), X0)), ("mul", C(-3.0), X0)),
    (("mul", C(3), ("neg", X0)), ("mul", C(-3.0), X0)),
    (("abs", ("neg", ("abs", X0))), ("abs", X0)),
    (("square", ("neg", X0)), ("square", X0)),
    (("lt", C(1.0), C(2.0)), C(1.0)),
    (("sqrt", C(-1.0)), None),                                           # folds to NaN
])
def test_rewrites_by_hand(sexpr, want):
    got = O.to_sexpr(canon(sexpr))
    if want is None:
        assert got[0] == "c" and math.isnan(got[1])
    else:
        assert got == want


def test_common_subexpressions_share_one_node():
    # 2 * x and x * 2 are one node, so the sum has 3 nodes: x, 2, 2x, sum
    t = canon(("add", ("mul", C(2), X0), ("mul", X0, C(2))))
    assert [n[0] for n in t.nodes] == ["c", "x", "mul", "add"] or [n[0] for n in t.nodes] == ["x", "c", "mul", "add"]
    assert t.nodes[-1][1] == t.nodes[-1][2]


def test_folding_rounds_in_the_compute_type():
    e = ("add", ("mul", C(0.1), C(3.0)), C(0.7))
    f32 = canon(e).nodes
    f64 = canon(e, compute="f64").nodes
    want32 = np.float32(np.float32(np.float32(0.1) * np.float32(3.0)) + np.float32(0.7))
    assert len(f32) == 1 and f32[0][3] == float(want32)
    assert len(f64) == 1 and f64[0][3] == 0.1 * 3.0 + 0.7


def test_dead_nodes_and_slots():
    # a hand-built tree whose node 1 is never used: dropped; the slots keep
    # their numbers (x1 stays slot 1 of 2)
    raw = O.encode(("add", X1, X1), n_inputs=2)
    t = O.decode(coot.coot_tree_canonical(raw))
    assert t.n_inputs == 2 and O.to_sexpr(t) == ("add", X1, X1)
    import struct
    hdr = struct.pack("<4sHHBBHI", b"COOT", 1, 3, 1, 0, 0, 0)
    body = (struct.pack("<BBHHHd", 0, 0, 0, 0, 0, 0.0) + struct.pack("<BBHHHd", 4, 0, 0, 0, 0, 0.0) +
            struct.pack("<BBHHHd", 3, 0, 0, 0, 0, 0.0))
    t = O.decode(coot.coot_tree_canonical(hdr + body))
    assert O.to_sexpr(t) == ("abs", X0) and len(t.nodes) == 2


# ---------------------------------------------------------------- exactness on random trees

def _inject(sexpr, u):
    """Wrap random subtrees in value-preserving redundancy."""
    if sexpr[0] in ("x", "c"):
        node = sexpr
    else:
        node = (sexpr[0],) + tuple(_inject(a, u) for a in sexpr[1:])
    r = next(u)
    if r < 0.05:
        return ("neg", ("neg", node))
    if r < 0.1:
        return ("mul", node, C(1.0))
    if r < 0.15:
        return ("sub", node, C(0.0))
    if r < 0.2:
        return ("mul", C(2.0), ("mul", C(4.0), node))
    if r < 0.25:
        return ("add", node, ("neg", ("mul", C(0.0), C(3.0))))   # + (-0)
    if r < 0.28:
        return ("abs", ("neg", node))
    if r < 0.31:
        return ("mul", ("neg", node), ("neg", ("add", C(1.0), C(0.5))))
    return node


def _f32_eval(sexpr, xs):
    """Independent FP32 evaluation (numpy float32, one rounding per node)."""
    name = sexpr[0]
    if name == "x":
        return xs[sexpr[1]]
    if name == "c":
        return np.float32(sexpr[1])
    f1 = {"neg": np.negative, "abs": np.abs, "exp": np.exp, "log": np.log, "sqrt": np.sqrt,
          "square": lambda a: a * a}
    with np.errstate(all="ignore"):
        if name in f1:
            return np.float32(f1[name](_f32_eval(sexpr[1], xs)))
        a, b = np.float32(_f32_eval(sexpr[1], xs)), np.float32(_f32_eval(sexpr[2], xs))
        return np.float32({"add": np.add, "sub": np.subtract, "mul": np.multiply, "div": np.divide}[name](a, b))


@pytest.mark.parametrize("seed", range(40))
def test_canonical_trees_give_identical_values(seed):
    n_in = 1 + seed % 3
    base = synth.random_tree(5000 + seed, 2 + seed % 6, n_in)
    u = iter(synth.uniform01(6000 + seed, 4096).tolist())
    e = _inject(base, u)
    t = O.encode(e, n_inputs=n_in)
    assert len(O.decode(t).nodes) <= 64
    c = O.decode(coot.coot_tree_canonical(t))
    assert len(c.nodes) <= len(O.decode(t).nodes)
    n = 512
    xs = [synth.uniform_f32(7000 + seed + k, n) * np.float32(3.0) for k in range(n_in)]
    xs[0][:4] = [0.0, -0.0, np.inf, np.nan]
    ms = [synth.as_mat(x, "f32", n, 1) for x in xs]
    # the same tree in FP64 compute (constants folded in FP64) through the
    # FP64 oracle: identical values, NaN where NaN
    t64 = O.encode(e, n_inputs=n_in, compute="f64")
    c64 = O.decode(coot.coot_tree_canonical(t64))
    a = O.evaluate(t64, ms).ravel()
    b = O.evaluate(c64, ms).ravel()
    assert np.array_equal(a, b, equal_nan=True)
    # an FP32 evaluation, one rounding per node: identical bits
    fa = np.asarray(_f32_eval(e, xs), dtype=np.float32) * np.ones(n, np.float32)
    fb = np.asarray(_f32_eval(O.to_sexpr(c), xs), dtype=np.float32) * np.ones(n, np.float32)
    same = (fa.view(np.uint32) == fb.view(np.uint32)) | (np.isnan(fa) & np.isnan(fb))
    assert same.all(), (e, O.to_sexpr(c))
