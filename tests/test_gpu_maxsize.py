"""Sizes past 2^31 elements, where every index has to be 64-bit end to end:
a vector of 2^31 + 77 elements and a 46341 x 46341 matrix (2,147,488,281
elements).  The inputs are built so that closed forms pin every result (no
oracle pass over 8.6 GB): ones for the vector, and the column number
j + 1 in every element of column j for the matrix, so that

    sum(A, 0)_j = R (j + 1),   sum(A, 1)_i = C (C + 1) / 2,
    accu(A) = R C (C + 1) / 2,
    row i's values are 1..C: mean (C + 1) / 2, sample variance C (C + 1) / 12,
    column j's values are all j + 1: variance 0.

Sum of 1..n and the variance of 1..n are textbook closed forms; the
reductions' definitions are those of Table 6 (sum along a dimension, accu)
and Table 5 (dot, norm)."""
import math

import numpy as np
import pytest
import torch

import paper_2308_03120_gb300 as coot
import synth
from paper_2308_03120_gb300.expr import serialize

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24  # FP32 unit roundoff


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    yield
    torch.cuda.synchronize()


def test_vector_past_2_31_elements():
    n = (1 << 31) + 77
    x = torch.ones(n, dtype=torch.float32, device="cuda")
    X = coot.Mat(x, n, 1, n)
    ws = coot.Workspace(1)
    heads = coot.HEAD_SUM | coot.HEAD_NORM2 | coot.HEAD_MIN | coot.HEAD_MAX
    r = coot.coot_expr_reduce(serialize(synth.LEAF0), [X], heads, ws=ws).tolist()
    d = coot.coot_dot(X, X, ws=ws).item()
    torch.cuda.synchronize()
    # every term is 1: each thread's sum is exact, and so is the combine
    assert r[0] == float(n)
    assert abs(r[1] - math.sqrt(n)) <= 1e-12 * math.sqrt(n)
    assert r[2] == 1.0 and r[3] == 1.0
    assert d == float(n)
    # y = 2x + 3z with z = x: 5 everywhere, the elements past 2^31 included
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    coot.coot_expr_eval(serialize(synth.AXPY_2X_3Z), [X, X], coot.Mat(y, n, 1, n))
    torch.cuda.synchronize()
    assert bool((y == 5.0).all())
    assert y[n - 1].item() == 5.0 and y[(1 << 31) + 3].item() == 5.0
    # sum along dim 0 of the n x 1 column, stored in FP64
    s = torch.empty(1, dtype=torch.float64, device="cuda")
    coot.coot_sum_dim(serialize(synth.LEAF0), [X], 0, coot.Mat(s, 1, 1, 1), ws=ws)
    torch.cuda.synchronize()
    assert s.item() == float(n)


@pytest.fixture(scope="module")
def column_number_matrix():
    R = C = 46341  # R * C > 2^31
    a = torch.empty((C, R), dtype=torch.float32, device="cuda")  # row-major C x R = column-major R x C
    a.copy_(torch.arange(1, C + 1, dtype=torch.float32, device="cuda")[:, None].expand(C, R))
    return R, C, a


def test_matrix_past_2_31_elements_sums(column_number_matrix):
    R, C, a = column_number_matrix
    A = coot.Mat(a.view(-1), R, C, R)
    ws = coot.Workspace(R)
    leaf = serialize(synth.LEAF0)
    col = torch.empty(C, dtype=torch.float64, device="cuda")
    row = torch.empty(R, dtype=torch.float64, device="cuda")
    coot.coot_sum_dim(leaf, [A], 0, coot.Mat(col, 1, C, 1), ws=ws)
    coot.coot_sum_dim(leaf, [A], 1, coot.Mat(row, R, 1, R), ws=ws)
    acc = coot.coot_accu(leaf, [A], ws=ws).item()
    mm = coot.coot_minmax(leaf, [A], ws=ws).tolist()
    torch.cuda.synchronize()
    # integers below 2^31 summed with TwoSum per element: exact
    want_col = R * np.arange(1, C + 1, dtype=np.float64)
    assert np.array_equal(col.cpu().numpy(), want_col)
    assert bool((row == C * (C + 1) / 2).all())
    exact = R * (C * (C + 1) // 2)  # 4.976e13, below 2^53
    assert abs(acc - exact) <= 1e-12 * exact
    assert mm == [1.0, float(C)]


def test_matrix_past_2_31_elements_stats(column_number_matrix):
    R, C, a = column_number_matrix
    A = coot.Mat(a.view(-1), R, C, R)
    ws = coot.Workspace(R)
    leaf = serialize(synth.LEAF0)
    stats = coot.STAT_MEAN | coot.STAT_VAR | coot.STAT_MIN | coot.STAT_MAX
    cols = [torch.empty(C, dtype=torch.float64, device="cuda") for _ in range(4)]
    rows = [torch.empty(R, dtype=torch.float64, device="cuda") for _ in range(4)]
    coot.coot_stats_dim(leaf, [A], 0, stats, [coot.Mat(t, 1, C, 1) for t in cols], ws=ws)
    coot.coot_stats_dim(leaf, [A], 1, stats, [coot.Mat(t, R, 1, R) for t in rows], ws=ws)
    torch.cuda.synchronize()
    j1 = np.arange(1, C + 1, dtype=np.float64)
    mean_c, var_c, min_c, max_c = (t.cpu().numpy() for t in cols)
    assert np.array_equal(mean_c, j1) and np.array_equal(min_c, j1) and np.array_equal(max_c, j1)
    assert np.array_equal(var_c, np.zeros(C))  # every value equals the shift
    mean_r, var_r, min_r, max_r = (t.cpu().numpy() for t in rows)
    assert np.array_equal(mean_r, np.full(R, (C + 1) / 2))
    assert np.array_equal(min_r, np.ones(R)) and np.array_equal(max_r, np.full(R, float(C)))
    # the shifted one-pass variance: within 12 u sum (y - K)^2 / (N - 1) of
    # C (C + 1) / 12, with K = 1 the row's first value
    var_exact = C * (C + 1) / 12
    bound = 12 * U32 * sum(float(k) ** 2 for k in range(C)) / (C - 1)
    assert np.abs(var_r - var_exact).max() <= bound
