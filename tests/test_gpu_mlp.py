"""The cost model's GPU kernels (forward, loss and gradient, Adam) against
the FP64 oracle, GPU training, and the learned policy in a call."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2308_03120_gb300 as coot
import synth
from oracle import mlp_oracle as M
from paper_2308_03120_gb300 import _abi, learn
from paper_2308_03120_gb300.expr import serialize

pytestmark = pytest.mark.gpu
D, H = learn.D, learn.H


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    yield
    learn.use_builtin()
    torch.cuda.synchronize()


def _problem(B, seed):
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(learn.n_params()) * 0.3).astype(np.float32)
    X = rng.uniform(-1, 1, (B, D)).astype(np.float32)
    t = rng.standard_normal(B).astype(np.float32)
    return p, X, t


@pytest.mark.parametrize("B", [1, 37, 1000])
def test_forward_matches_oracle(B):
    p, X, _ = _problem(B, B)
    m = learn.CostModel(p)
    got = m.predict(X)
    want, _, _ = M.forward(p.astype(np.float64), X.astype(np.float64), D, H)
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("B", [5, 300])
def test_loss_and_gradient_match_oracle(B):
    p, X, t = _problem(B, 100 + B)
    m = learn.CostModel(p)
    Xd = torch.as_tensor(X).cuda()
    td = torch.as_tensor(t).cuda()
    y, act = m.forward(Xd)
    grad = torch.zeros(p.size, device="cuda")
    loss = torch.zeros(1, device="cuda")
    work = torch.empty(B * (2 * H + 1), device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _abi.call("coot_mlp_loss_grad", m.p.data_ptr(), D, H, Xd.data_ptr(), td.data_ptr(), B, y.data_ptr(),
              act.data_ptr(), grad.data_ptr(), loss.data_ptr(), work.data_ptr(), st)
    L, g = M.loss_and_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64), D, H)
    assert loss.item() == pytest.approx(L, rel=1e-5)
    gg = grad.cpu().numpy()
    scale = np.max(np.abs(g))
    np.testing.assert_allclose(gg, g, rtol=1e-4, atol=1e-5 * scale)


def test_adam_matches_oracle():
    rng = np.random.default_rng(9)
    n = 1000
    p = rng.standard_normal(n).astype(np.float32)
    gs = [rng.standard_normal(n).astype(np.float32) for _ in range(3)]
    pd, md, vd = (torch.as_tensor(a).cuda() for a in (p, np.zeros(n, np.float32), np.zeros(n, np.float32)))
    po, mo, vo = p.astype(np.float64), np.zeros(n), np.zeros(n)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for k, g in enumerate(gs, start=1):
        gd = torch.as_tensor(g).cuda()
        _abi.call("coot_mlp_adam", pd.data_ptr(), gd.data_ptr(), md.data_ptr(), vd.data_ptr(), n, k,
                  ctypes.c_float(1e-2), ctypes.c_float(0.9), ctypes.c_float(0.999), ctypes.c_float(1e-8), st)
        po, mo, vo = M.adam(po, g.astype(np.float64), mo, vo, k, 1e-2)
    np.testing.assert_allclose(pd.cpu().numpy(), po, rtol=1e-5, atol=1e-6)


def test_gpu_training_fits_a_smooth_target_and_is_reproducible():
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, (2000, D)).astype(np.float32)
    t = (np.sin(3 * X[:, 5]) + X[:, 16] * X[:, 18] - 0.5 * X[:, 9]).astype(np.float32)
    a = learn.CostModel(seed=4)
    b = learn.CostModel(seed=4)
    ha = a.fit(X, t, steps=600, lr=3e-3)
    hb = b.fit(X, t, steps=600, lr=3e-3)
    assert ha[-1][1] < 0.05 * ha[0][1]
    assert np.array_equal(a.params(), b.params())     # fixed-order sums: bit for bit


def test_learned_policy_follows_the_model():
    """A hand-made model whose prediction grows with log2(block): the
    policy must pick the smallest candidate block for every kind."""
    p = np.zeros(learn.n_params(), dtype=np.float32)
    # one hidden unit copies feature 16 (log2 block / 10) through both layers
    p[16 * H + 0] = 1.0                       # W1[16, 0]
    off_W2 = D * H + H
    p[off_W2 + 0 * H + 0] = 1.0               # W2[0, 0]
    off_w3 = off_W2 + H * H + H
    p[off_w3 + 0] = 1.0                       # w3[0]
    _abi.call("coot_model_load", p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size)
    _abi.call("coot_set_policy", _abi.POLICY_LEARNED)
    try:
        r, c = 300, 40
        x = torch.rand(r * c, device="cuda")
        X = coot.Mat(x, r, c, r)
        tree = serialize(synth.LEAF0)
        out = torch.empty(r * c, device="cuda")
        coot.coot_expr_eval(tree, [X], coot.Mat(out, r, c, r))
        assert coot.coot_last_launch()["block"] == min(b for b, *_ in learn.candidates(0))
        col = torch.empty(c, device="cuda")
        coot.coot_sum_dim(tree, [X], 0, coot.Mat(col, 1, c, 1))
        assert coot.coot_last_launch()["block"] == min(b for b, *_ in learn.candidates(2))
        row = torch.empty(r, device="cuda")
        coot.coot_sum_dim(tree, [X], 1, coot.Mat(row, r, 1, r))
        assert coot.coot_last_launch()["block"] == min(b for b, *_ in learn.candidates(3))
        torch.cuda.synchronize()
        assert torch.equal(out, x)
        np.testing.assert_allclose(col.cpu().numpy(), x.view(c, r).sum(1).cpu().numpy(), rtol=1e-5)
    finally:
        learn.use_builtin()
