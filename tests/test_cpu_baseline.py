"""The all-cores FP32 CPU evaluator of the benchmark's CPU baseline
(oracle/cpu_fp32.c) computes the workload step: its FP32 values, heads and
sums agree with the FP64 oracle within FP32 rounding, for one thread and
for every thread (the thread count changes only the FP64 summation order).
CPU only."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import coot_oracle as O
from oracle import cpu_build


@pytest.fixture(scope="module")
def lib():
    return cpu_build.load()


def _run(lib, sexpr, ins, r, c, threads):
    tree = O.encode(sexpr)
    ptrs = (ctypes.c_void_p * 4)(*([a.ctypes.data for a in ins] + [None] * (4 - len(ins))))
    out = np.empty(r * c, np.float32)
    heads = np.zeros(4)
    col = np.empty(c, np.float32)
    row = np.empty(r, np.float32)
    rc = lib.cpu_fp32_eval(tree, len(tree), ptrs, len(ins), r, c, r, out.ctypes.data, r, heads.ctypes.data,
                           col.ctypes.data, row.ctypes.data, threads)
    assert rc == 0
    return out.reshape(c, r).T, heads, col, row


@pytest.mark.parametrize("threads", [1, 0])
@pytest.mark.parametrize("sexpr", [synth.MAT_EXPR, synth.MAT_CHAIN, synth.AXPY_2X_3Z])
def test_step_matches_the_oracle(lib, sexpr, threads):
    r, c = 1000, 37
    n_in = synth.tree_inputs(sexpr)
    ins = [synth.uniform_f32(91 + k, r * c, 0.0 if k == 3 else -1.0, 2.0 if k == 3 else 1.0) for k in range(n_in)]
    hs = [synth.as_mat(a, "f32", r, c) for a in ins]
    tree = O.encode(sexpr)
    out, heads, col, row = _run(lib, sexpr, ins, r, c, threads)
    v, bound, unsafe = O.error_bound(tree, hs)
    assert not unsafe.any()
    assert np.all(np.abs(out - v) <= 1e-6 * np.abs(v) + 2.0 * bound)
    s_abs = float(np.sum(np.abs(v)))
    assert abs(heads[0] - O.accu(tree, hs)) <= 1e-6 * s_abs
    assert abs(heads[1] - O.norm(tree, hs, "fro") ** 2) <= 1e-5 * heads[1]
    assert (heads[2], heads[3]) == O.minmax(tree, hs) or np.allclose((heads[2], heads[3]), O.minmax(tree, hs),
                                                                     rtol=1e-6, atol=1e-6)
    assert np.allclose(col, O.sum_dim(tree, hs, 0), rtol=1e-5, atol=1e-4 * np.max(np.abs(v)))
    assert np.allclose(row, O.sum_dim(tree, hs, 1), rtol=1e-5, atol=1e-4 * np.max(np.abs(v)))


def test_bad_tree_is_an_error(lib):
    x = np.zeros(4, np.float32)
    ptrs = (ctypes.c_void_p * 4)(x.ctypes.data, None, None, None)
    assert lib.cpu_fp32_eval(b"NOPE" + bytes(12), 16, ptrs, 1, 4, 1, 4, None, 4, None, None, None, 1) < 0
