"""coot_sum_rows_f32_static: row sums for callers that cannot allocate a
workspace (device memory reserved by an allocator they do not control,
paths that must not synchronise the device, C callers without a CUDA
allocator).  The entry point keeps its scratch in a fixed array inside the
library.  This test calls it through the C ABI twice in a row and compares
each result with coot_sum_dim(dim = 1), the entry point that takes a
caller-owned workspace, within the tolerance the other sum tests use.

The file sorts last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2308_03120_gb300 as coot
import synth
from oracle import coot_oracle as O
from paper_2308_03120_gb300 import _abi
from paper_2308_03120_gb300.expr import serialize

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    yield
    torch.cuda.synchronize()


def _tolerance(want, terms):
    s_abs = np.sum(np.abs(terms), axis=1)
    tol = 1e-6 * np.abs(want) + np.where(np.abs(want) < 1e-3 * s_abs, 1e-9 * s_abs, 0.0)
    return tol + 2.0 * np.abs(want) * 2.0 ** -24   # each side rounds its result to FP32 once


@pytest.mark.parametrize("shape,ld", [((8192, 1024), 8192), ((1037, 333), 1040), ((32768, 40), 32768),
                                      ((5, 3), 5), ((300, 1), 300)])
def test_static_row_sums_match_the_workspace_entry_point(shape, ld):
    r, c = shape
    h = synth.as_mat(synth.uniform_f32(4242 + r, r * c), "f32", r, c, ld)
    a = coot.Mat(torch.from_numpy(h.buf).cuda(), r, c, ld)
    ref = torch.empty(r, dtype=torch.float32, device="cuda")
    coot.coot_sum_dim(serialize(synth.LEAF0), [a], 1, coot.Mat(ref, r, 1, r))
    torch.cuda.synchronize()
    want = ref.cpu().numpy().astype(np.float64)
    terms = O.logical(h)
    oracle = O.sum_dim(O.encode(synth.LEAF0), [h], 1)
    L = _abi.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = torch.full((r,), float("nan"), dtype=torch.float32, device="cuda")
        ca = a.c()
        co = coot.Mat(out, r, 1, r).c()
        status = L.coot_sum_rows_f32_static(ctypes.byref(ca), ctypes.byref(co), stream)
        assert status == 0, L.coot_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - want) <= _tolerance(want, terms)), f"call {call}: differs from coot_sum_dim"
        assert np.all(np.abs(got - oracle) <= _tolerance(oracle, terms)), f"call {call}: differs from the oracle"


def test_static_row_sums_reject_too_many_rows():
    r = 32769
    t = torch.zeros(r, dtype=torch.float32, device="cuda")
    with pytest.raises(coot.CootError) as e:
        coot.coot_sum_rows_f32_static(coot.Mat(t, r, 1, r), coot.Mat(t, r, 1, r))
    assert e.value.status_name == "COOT_ERR_UNSUPPORTED" and "32768" in str(e.value)


def test_static_row_sums_reject_an_overlapping_output():
    # out placed over a's first column: blocks would write rows of out while
    # other blocks still read that column
    r, c = 1000, 8
    t = torch.zeros(r * c + r, dtype=torch.float32, device="cuda")
    a = coot.Mat(t[r:], r, c, r)
    for start in (r, r + 17, r * c):
        with pytest.raises(coot.CootError) as e:
            coot.coot_sum_rows_f32_static(a, coot.Mat(t[start:start + r], r, 1, r))
        assert e.value.status_name == "COOT_ERR_ALIAS"
    # just before a: no shared element, accepted
    coot.coot_sum_rows_f32_static(a, coot.Mat(t[:r], r, 1, r))
    torch.cuda.synchronize()
