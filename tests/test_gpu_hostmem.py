"""Operands in pinned host memory, reached by the kernels through their
device mappings (coot_host_device_pointer; over NVLink-C2C on GB300): the
results equal those of the same calls on device copies bit for bit, and
match the oracle; memory that is not pinned host memory is refused."""
import numpy as np
import pytest
import torch

import paper_2308_03120_gb300 as coot
import synth
from oracle import coot_oracle as O
from paper_2308_03120_gb300.expr import serialize
from tests.gpu_util import assert_sum_close, check_elementwise, host_mats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    yield
    torch.cuda.synchronize()


def _pinned(h):
    return torch.from_numpy(np.ascontiguousarray(h.buf)).pin_memory()


def test_only_pinned_host_memory_maps():
    """Pageable host memory and device memory have no host mapping: the
    call refuses them (nothing is guessed); pinned memory maps, also from
    inside the allocation."""
    with pytest.raises(coot.CootError) as e:
        coot.Mat(torch.zeros(1000), 1000, 1, 1000).mapped()
    assert e.value.status_name == "COOT_ERR_INVALID_ARG"
    with pytest.raises(coot.CootError) as e:
        coot.Mat(torch.zeros(1000, device="cuda"), 1000, 1, 1000).mapped()
    assert e.value.status_name == "COOT_ERR_INVALID_ARG"
    p = torch.zeros(1000).pin_memory()
    m = coot.Mat(p, 1000, 1, 1000).mapped()
    assert m.base != 0
    inner = coot.Mat(p[100:], 900, 1, 900).mapped()
    assert inner.base == m.base + 100 * 4


def test_one_launch_step_on_host_buffers_equals_device_run():
    """The matrix step in one launch (both trees stored, heads, sums along
    both dims) with inputs and outputs in pinned host memory: bit for bit
    the device-resident run, and within the oracle's tolerances."""
    r, c = 1037, 605
    specs = [("f32", r, c, None, -1.0, 1.0)] * 3 + [("f32", r, c, None, 0.0, 2.0)]
    ins = host_mats(specs, 2024)
    t_expr, t_chain = serialize(synth.MAT_EXPR), serialize(synth.MAT_CHAIN)
    heads = coot.HEAD_SUM | coot.HEAD_NORM2 | coot.HEAD_MIN | coot.HEAD_MAX
    dh = [heads | coot.HEAD_COLSUM | coot.HEAD_ROWSUM, 0]
    pin = [_pinned(h) for h in ins]
    dev_in = [coot.Mat(p.cuda(), r, c, r) for p in pin]
    host_in = [coot.Mat(p, r, c, r).mapped() for p in pin]

    def run(mats, where):
        mk = (lambda n: torch.empty(n).pin_memory()) if where == "host" else (lambda n: torch.empty(n, device="cuda"))
        o1, o2, cs, rs = mk(r * c), mk(r * c), mk(c), mk(r)
        wrap = (lambda m: m.mapped()) if where == "host" else (lambda m: m)
        res = coot.coot_expr_multi_dims([t_expr, t_chain], mats,
                                        [wrap(coot.Mat(o1, r, c, r)), wrap(coot.Mat(o2, r, c, r))], dh,
                                        [wrap(coot.Mat(cs, 1, c, 1)), None], [wrap(coot.Mat(rs, r, 1, r)), None])
        torch.cuda.synchronize()
        return [t.cpu() for t in (o1, o2, cs, rs, res)]

    a = run(dev_in, "device")
    b = run(host_in, "host")
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    o1, o2, cs, rs, res = b
    check_elementwise(t_expr, ins, synth.as_mat(o1.numpy(), "f32", r, c))
    check_elementwise(t_chain, ins, synth.as_mat(o2.numpy(), "f32", r, c))
    v, bound, _ = O.error_bound(t_expr, ins)
    t, e = v.ravel(order="F"), bound.ravel(order="F")
    assert_sum_close(res[0].item(), O.accu(t_expr, ins), t, e, "accu")


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_reduction_and_eval_read_host_inputs(dt):
    """A full reduction and an element-wise evaluation whose inputs are
    pinned host vectors (a ragged length), outputs on the device."""
    n = 3_000_017
    ins = host_mats([(dt, n, 1, None, -1.0, 1.0)] * 2, 2025)
    pin = [_pinned(h) if dt == "f32" else torch.from_numpy(h.buf.view(np.int16).copy()).view(torch.bfloat16).pin_memory()
           for h in ins]
    mh = [coot.Mat(p, n, 1, n).mapped() for p in pin]
    md = [coot.Mat(p.cuda(), n, 1, n) for p in pin]
    tree = serialize(synth.SCHUR_XZ)
    got_h = coot.coot_expr_reduce(tree, mh, coot.HEAD_SUM | coot.HEAD_NORM2).cpu()
    got_d = coot.coot_expr_reduce(tree, md, coot.HEAD_SUM | coot.HEAD_NORM2).cpu()
    assert torch.equal(got_h, got_d)
    v, bound, _ = O.error_bound(tree, ins)
    assert_sum_close(got_h[0].item(), O.accu(tree, ins), v.ravel(), bound.ravel(), "accu")
    axpy = serialize(synth.AXPY_2X_3Z)
    out = torch.empty(n, device="cuda")
    coot.coot_expr_eval(axpy, mh, coot.Mat(out, n, 1, n))
    torch.cuda.synchronize()
    check_elementwise(axpy, ins, synth.as_mat(out.cpu().numpy(), "f32", n, 1))
