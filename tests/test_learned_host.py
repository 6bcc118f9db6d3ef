"""Host side of the learned launch shapes (no GPU): the library's
cost-model inference against the FP64 oracle, the feature vector against
hand computation, the candidate grid."""
import math

import numpy as np
import pytest

import synth
from oracle import mlp_oracle as M
from paper_2308_03120_gb300 import _abi, learn
from paper_2308_03120_gb300.expr import serialize


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2308_03120_gb300 import build
    build.build()


def test_host_prediction_matches_the_oracle():
    rng = np.random.default_rng(5)
    p = (rng.standard_normal(learn.n_params()) * 0.2).astype(np.float32)
    _abi.call("coot_model_load", p.ctypes.data_as(_abi.ctypes.POINTER(_abi.ctypes.c_float)), p.size)
    X = rng.uniform(0, 1, (50, learn.D)).astype(np.float32)
    got = learn.host_predict(X)
    want, _, _ = M.forward(p.astype(np.float64), X.astype(np.float64), learn.D, learn.H)
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-5)


def test_model_load_checks_the_size():
    p = np.zeros(10, dtype=np.float32)
    with pytest.raises(_abi.CootError):
        _abi.call("coot_model_load", p.ctypes.data_as(_abi.ctypes.POINTER(_abi.ctypes.c_float)), p.size)


def test_features_by_hand():
    tree = serialize(synth.MAT_EXPR)   # 6 operators (%, *, +, abs, +, /), no transcendental, 4 inputs
    f = learn.features(tree, learn.KIND_MAP, [0, 0, 0, 0], 0, 0, 8192, 8192, True, 256, 4, 4, 0)
    n = 8192.0 * 8192.0
    want = np.zeros(21)
    want[0] = 1
    want[5] = math.log2(1 + n) / 32
    want[6] = want[7] = math.log2(1 + 8192) / 16
    want[8] = 1.0
    want[9] = 6 / 16
    want[10] = 0.0
    want[11] = 4 / 8
    want[12] = 4 / 8
    want[13] = 0
    want[14] = 1
    want[15] = 0
    want[16] = math.log2(256) / 10
    want[17] = 4 / 8
    want[18] = math.log2(4) / 4
    want[19] = 0
    want[20] = math.log2(1 + n / (256 * 4 * 4)) / 32
    np.testing.assert_allclose(f, want, rtol=1e-6, atol=1e-7)
    g = learn.features(serialize(synth.MAT_CHAIN), learn.KIND_ROWSUM, [1, 1, 1, 1], -1, 0, 100, 7, False, 512, 8,
                       16, 32)
    assert g[4] == 1 and g[10] == pytest.approx(2 / 8) and g[11] == pytest.approx(2 / 8) and g[12] == 0
    assert g[14] == 0 and g[19] == pytest.approx(math.log2(33) / 8)
    h = learn.features(serialize(synth.LEAF0), learn.KIND_REDUCE, [0], -1, 1 | 4, 10, 1, True, 128, 4, 1, 0)
    assert h[2] == 1 and h[13] == pytest.approx(2 / 8) and h[9] == 0


def test_candidates_cover_every_kind():
    for kind in learn.KINDS:
        c = learn.candidates(kind)
        assert len(c) >= 10
        assert all(b % 64 == 0 and 1 <= u <= 16 for b, v, u, s in c)
    assert learn.candidates(4) == []


def test_learned_policy_needs_a_model():
    # a model is loaded by the earlier test in this module's process only if it ran first;
    # the policy switch itself must refuse an unknown policy
    with pytest.raises(_abi.CootError):
        _abi.call("coot_set_policy", 7)


def test_merged_sample_sets_keep_trees_whole():
    """Two timing sets (the second from calls of another size band, its
    trees numbered from 0 again) merge into distinct trees, and the
    held-out split never puts calls of one tree on both sides."""
    from paper_2308_03120_gb300 import learn
    first = [{"tree": t, "call": c} for t in range(10) for c in range(8)]
    second = [{"tree": t, "call": c, "large": True} for t in range(4) for c in range(8)]
    merged = learn.merge_sample_sets(first, second, 10)
    assert len({s["tree"] for s in merged}) == 14
    assert {s["tree"] for s in merged if s.get("large")} == set(range(10, 14))
    train, held = learn.split_by_tree(merged)
    assert {s["tree"] for s in train}.isdisjoint({s["tree"] for s in held})
    assert len(train) + len(held) == len(merged)
