"""Benchmark of the fused expression + reduction path.

Default workload (one step = one pass of the whole hot path over one batch):
FP32 column-major 8192 x 8192 matrices A, B, C ~ U[-1, 1], D ~ U[0, 2]
(seeded), and the calls a user makes for

    out   = (A % B + 2 C) / (1 + abs(D))      with accu, norm2, min, max
                                               of out in the same pass
    chain = exp(-abs(A % B + 2 C)) / sqrt(1 + abs(D))
    sum(out, 0), sum(out, 1)

i.e. coot_expr_reduce (5 matrix streams), coot_expr_eval (5), and two
coot_sum_dim over the stored out (1 each): 12 matrix streams of 268 MB =
3.22 GB of algorithmic traffic per step.  `value` is that traffic over the
device time of the step (GB/s), the step captured once as a CUDA graph and
replayed; the inputs (1.07 GB) are larger than L2, so no flush is needed
between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl coot|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the reference arm: a deliberately slow
program; parity and the roofline fraction are the headline).
Under torchrun every rank runs its own instance (weak scaling, no
collective); rank 0 prints the one JSON line.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

N = 8192
ELEM = 4
MAT_BYTES = N * N * ELEM
STREAMS = {"expr_reduce": 5, "expr_eval": 5, "sum_dim0": 1, "sum_dim1": 1}
STEP_BYTES = sum(STREAMS.values()) * MAT_BYTES
METRIC = "fused expr+reduction HBM GB/s (% of GB300 peak) vs unfused same GPU; batch evals/s"
WORKLOAD = "matrices 8192x8192 fp32: (A%B+2C)/(1+|D|) with accu/norm2/min/max, exp/sqrt chain, sum dim 0 and 1"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = ("jit_rt.cuh", "jit_map.cuh", "jit_colsum.cuh", "jit_rowsum.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "matrices_8192_traffic.md")


def kernel_source_hash():
    """sha256 over the device code of the matrix workload's kernels (the
    runtime and the element-wise, column-sum and row-sum kernels)."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2308_03120_gb300", "csrc", name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def shape_text(last):
    return "block {block} vec {vec} unroll {unroll} grid {grid} split {split}".format(**last)


def committed_traffic(call, shape):
    """DRAM bytes (read + write) of one launch of `call` at 8192 x 8192 from
    the committed ncu summary, or (None, why) when there is none, or the
    device code or the launch shape changed since it was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            text = f.read()
    except OSError:
        return None, "no committed ncu traffic summary"
    digest = None
    for line in text.splitlines():
        if line.startswith("kernel-source: sha256 "):
            digest = line.split()[-1]
    if digest != kernel_source_hash():
        return None, "kernel sources changed since the ncu traffic capture"
    header = None
    for line in text.splitlines():
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if cells and cells[0] == "call":
            header = cells
        elif header and len(cells) == len(header) and cells[0] == call:
            row = dict(zip(header, cells))
            if row["launch"] != shape:
                return None, f"launch shape changed since the ncu traffic capture ({row['launch']} -> {shape})"
            return int(row["traffic (B)"]), "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch at 8192 x 8192"
    return None, f"no traffic row for {call}"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def inputs_host(seed):
    A = synth.uniform_f32(seed + 0, N * N)
    B = synth.uniform_f32(seed + 1, N * N)
    C = synth.uniform_f32(seed + 2, N * N)
    D = synth.uniform_f32(seed + 3, N * N, 0.0, 2.0)
    return [A, B, C, D]


class Clocks:
    """SM clock and clock-event reasons sampled DURING the timed region by a
    host thread polling NVML (read-only queries, libnvidia-ml from the
    driver) about every millisecond, so that even a short timed region gets
    samples; falls back to `nvidia-smi -lms 200` when NVML cannot be
    loaded."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_index, pci_bus_id=None):
        self.gpu = gpu_index
        self.pci = pci_bus_id
        self.samples = []
        self.max_mhz = None
        self._stop = None
        self._thread = None
        self.proc = None

    def _nvml(self):
        import ctypes
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = ctypes.c_void_p()
        ok = False
        if self.pci:
            ok = nv.nvmlDeviceGetHandleByPciBusId_v2(self.pci.encode(), ctypes.byref(h)) == 0
        if not ok and nv.nvmlDeviceGetHandleByIndex_v2(self.gpu, ctypes.byref(h)) != 0:
            raise RuntimeError("no NVML handle")
        return nv, h

    def start(self):
        import ctypes
        import threading
        try:
            nv, h = self._nvml()
        except Exception:
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                     "--format=csv,noheader,nounits", "-lms", "200"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except Exception:
                self.proc = None
            return
        mx = ctypes.c_uint()
        if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
            self.max_mhz = float(mx.value)
        get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
        self._stop = threading.Event()

        def poll():
            mhz = ctypes.c_uint()
            rs = ctypes.c_ulonglong()
            while not self._stop.is_set():
                if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) == 0 and get_reasons(h, ctypes.byref(rs)) == 0:
                    self.samples.append((float(mhz.value), int(rs.value)))
                time.sleep(0.001)
        self._thread = threading.Thread(target=poll, daemon=True)
        self._thread.start()

    def stop(self):
        if self._thread is not None:
            self._stop.set()
            self._thread.join(timeout=2)
            sm = [s[0] for s in self.samples]
            reasons = sorted({name for _, r in self.samples for bit, name in self.REASONS.items() if r & bit})
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
                    "reasons": reasons, "samples": len(sm), "source": "nvml"}
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 3]
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            try:
                bits = int(r[2].strip(), 16)
            except ValueError:
                continue
            reasons |= {name for bit, name in self.REASONS.items() if bits & bit}
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "source": "nvidia-smi"}


# ---------------------------------------------------------------- oracle (CPU) legs

def sample_inputs(seed, cols):
    """The first `cols` columns of the matrix workload's A, B, C, D (host)."""
    return [synth.uniform_f32(seed + k, N * cols, 0.0 if k == 3 else -1.0, 2.0 if k == 3 else 1.0) for k in range(4)]


def oracle_sample(seed, cols, time_budget=None):
    """Run the oracle over the first `cols` columns of the workload; returns
    (seconds, algorithmic bytes of the sample, the oracle's results)."""
    from oracle import coot_oracle as O
    A = [synth.as_mat(a, "f32", N, cols) for a in sample_inputs(seed, cols)]
    t_expr = O.encode(synth.MAT_EXPR)
    t_chain = O.encode(synth.MAT_CHAIN)
    t0 = time.perf_counter()
    out = O.evaluate(t_expr, A)
    accu = O.accu(t_expr, A)
    norm2 = O.norm(t_expr, A, "fro")
    lo, hi = O.minmax(t_expr, A)
    chain = O.evaluate(t_chain, A)
    om = synth.as_mat(out.astype(np.float32).ravel(order="F"), "f32", N, cols)
    leaf = O.encode(synth.LEAF0)
    col = O.sum_dim(leaf, [om], 0)
    row = O.sum_dim(leaf, [om], 1)
    dt = time.perf_counter() - t0
    res = {"out": out, "accu": accu, "norm2": norm2, "min": lo, "max": hi, "chain": chain, "col": col, "row": row}
    return dt, sum(STREAMS.values()) * N * cols * ELEM, res


def cpu_fp32_sample(seed, cols, reps=3):
    """The step on the first `cols` columns by the all-cores FP32 CPU
    evaluator (oracle/cpu_fp32.c, OpenMP): the matrix tree stored with its
    accu, sum of squares, min, max and column and row sums in one pass, then
    the chain tree stored.  Returns (best seconds of `reps`, algorithmic
    bytes of the sample, threads)."""
    import ctypes
    from oracle import cpu_build
    lib = cpu_build.load()
    ins = sample_inputs(seed, cols)
    ptrs = (ctypes.c_void_p * 4)(*[a.ctypes.data for a in ins])
    t_expr = bytes(coot_tree_bytes(synth.MAT_EXPR))
    t_chain = bytes(coot_tree_bytes(synth.MAT_CHAIN))
    out1 = np.empty(N * cols, np.float32)
    out2 = np.empty(N * cols, np.float32)
    heads = np.zeros(4)
    col = np.empty(cols, np.float32)
    row = np.empty(N, np.float32)
    best = math.inf
    for _ in range(reps):
        t0 = time.perf_counter()
        rc = lib.cpu_fp32_eval(t_expr, len(t_expr), ptrs, 4, N, cols, N, out1.ctypes.data, N, heads.ctypes.data,
                               col.ctypes.data, row.ctypes.data, 0)
        rc |= lib.cpu_fp32_eval(t_chain, len(t_chain), ptrs, 4, N, cols, N, out2.ctypes.data, N, None, None, None, 0)
        best = min(best, time.perf_counter() - t0)
        if rc != 0:
            raise RuntimeError(f"cpu_fp32_eval failed ({rc})")
    return best, sum(STREAMS.values()) * N * cols * ELEM, lib.cpu_fp32_threads()


def coot_tree_bytes(sexpr):
    """The serialised tree of a workload expression (the oracle's encoder:
    the CPU legs do not load the CUDA library)."""
    from oracle import coot_oracle as O
    return O.encode(sexpr)


def matrix_errors(coot, torch, dev, cols):
    """The step's results on the first `cols` columns of the device inputs,
    by the four calls of the timed step and by the one-launch call, against
    the FP64 oracle on the same columns: relative errors of accu and norm2,
    absolute errors of min / max, the largest relative error of each sum
    along a dimension, and for the stored trees the largest relative error
    and the largest error over the element-wise tolerance 1e-5 |o| + 2 E
    (E the oracle's first-order FP32 error bound of that element)."""
    from oracle import coot_oracle as O
    seed = synth.BASE_SEED + 1
    _, _, want = oracle_sample(seed, cols)
    host = [synth.as_mat(a, "f32", N, cols) for a in sample_inputs(seed, cols)]
    mats = [coot.Mat(t, N, cols, N) for t in dev]
    t_expr, t_chain = coot.serialize(synth.MAT_EXPR), coot.serialize(synth.MAT_CHAIN)
    leaf = coot.serialize(synth.LEAF0)
    heads = coot.HEAD_SUM | coot.HEAD_NORM2 | coot.HEAD_MIN | coot.HEAD_MAX
    ws = coot.Workspace(N)
    bounds = {}
    for name, tree in (("expr", t_expr), ("chain", t_chain)):
        _, e, unsafe = O.error_bound(O.decode(tree), host)
        bounds[name] = (e, int(unsafe.sum()))

    def elementwise(got, name, ref):
        g = got.view(cols, N).T.cpu().numpy().astype(np.float64)
        err = np.abs(g - ref)
        e, skipped = bounds[name]
        tol = 1e-5 * np.abs(ref) + 2.0 * e
        return {"max_rel": float(f"{np.max(err / np.maximum(np.abs(ref), 1e-300)):.3e}"),
                "max_err_over_tol": float(f"{np.max(err / tol):.3e}"), "unsafe_skipped": skipped}

    def sums(col, row):
        c = col.cpu().numpy().astype(np.float64)
        r = row.cpu().numpy().astype(np.float64)
        return ({"max_rel": float(f"{np.max(np.abs(c - want['col']) / np.abs(want['col'])):.3e}")},
                {"max_rel": float(f"{np.max(np.abs(r - want['row']) / np.abs(want['row'])):.3e}")})

    def heads_err(res):
        a, n2, lo, hi = res.cpu().tolist()
        return {"accu": _rel(a, want["accu"]), "norm2": _rel(n2, want["norm2"]),
                "min_abs": float(f"{abs(lo - want['min']):.3e}"), "max_abs": float(f"{abs(hi - want['max']):.3e}")}

    def summation_only(res, stored, col, row):
        """The sums against the correctly rounded sums (math.fsum) of the very
        FP32 values the GPU stored: the summation's own error, without the
        values' FP32 rounding that the oracle comparison includes."""
        v = stored.view(cols, N).T.cpu().numpy().astype(np.float64)
        c = col.cpu().numpy().astype(np.float64)
        r = row.cpu().numpy().astype(np.float64)
        fc = np.array([math.fsum(v[:, k]) for k in range(cols)])
        fr = np.array([math.fsum(v[i, :]) for i in range(N)])
        rel = lambda g, w: float(f"{np.max(np.abs(g - w) / np.maximum(np.abs(w), 1e-300)):.3e}")  # noqa: E731
        return {"accu": _rel(res.cpu().tolist()[0], math.fsum(v.ravel())), "sum_dim0_max_rel": rel(c, fc),
                "sum_dim1_max_rel": rel(r, fr)}

    o1 = torch.empty(N * cols, device="cuda")
    o2 = torch.empty(N * cols, device="cuda")
    col = torch.empty(cols, device="cuda")
    row = torch.empty(N, device="cuda")
    O1 = coot.Mat(o1, N, cols, N)
    res = coot.coot_expr_reduce(t_expr, mats, heads, out=O1, ws=ws)
    coot.coot_expr_eval(t_chain, mats, coot.Mat(o2, N, cols, N), ws=ws)
    coot.coot_sum_dim(leaf, [O1], 0, coot.Mat(col, 1, cols, 1), ws=ws)
    coot.coot_sum_dim(leaf, [O1], 1, coot.Mat(row, N, 1, N), ws=ws)
    torch.cuda.synchronize()
    four = dict(heads_err(res), expr_eval=elementwise(o1, "expr", want["out"]),
                chain=elementwise(o2, "chain", want["chain"]))
    four["sum_dim0"], four["sum_dim1"] = sums(col, row)
    four["summation_only"] = summation_only(res, o1, col, row)
    o1.fill_(float("nan"))
    o2.fill_(float("nan"))
    res = coot.coot_expr_multi_dims([t_expr, t_chain], mats, [O1, coot.Mat(o2, N, cols, N)],
                                    [heads | coot.HEAD_COLSUM | coot.HEAD_ROWSUM, 0],
                                    [coot.Mat(col, 1, cols, 1), None], [coot.Mat(row, N, 1, N), None], ws=ws)
    torch.cuda.synchronize()
    one = dict(heads_err(res), expr_eval=elementwise(o1, "expr", want["out"]),
               chain=elementwise(o2, "chain", want["chain"]))
    one["sum_dim0"], one["sum_dim1"] = sums(col, row)
    one["summation_only"] = summation_only(res, o1, col, row)
    return {"vs": "FP64 oracle", "sample": f"the step's calls on the first {cols} of {N} columns",
            "four_calls": four, "one_launch": one}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cols = args.ref_cols
    seed = synth.BASE_SEED + 1
    oracle_sample(seed, 8)  # warm caches / imports
    times = []
    for _ in range(args.warmup):
        oracle_sample(seed, cols)
    for _ in range(args.steps):
        dt, nbytes, _ = oracle_sample(seed, cols)
        times.append(dt)
    ms = 1e3 * statistics.mean(times)
    gbs = nbytes / (statistics.mean(times) * 1e9)
    line = {"metric": METRIC, "value": round(gbs, 4), "unit": "GB/s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + f" (oracle sample: first {cols} of 8192 columns)",
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": f"8192 x {cols} column block of every matrix, whole step"},
            "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU leg

def run_coot(args):
    import torch
    import torch.distributed as dist

    import paper_2308_03120_gb300 as coot
    from paper_2308_03120_gb300 import build as _build

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    coot.coot_init(local)
    stream = torch.cuda.current_stream()
    seed = synth.BASE_SEED + 1 + 1000 * rank
    host = inputs_host(seed)
    dev = [torch.from_numpy(h).cuda() for h in host]
    mats = [coot.Mat(t, N, N, N) for t in dev]
    out1 = torch.empty(N * N, dtype=torch.float32, device="cuda")
    out2 = torch.empty(N * N, dtype=torch.float32, device="cuda")
    col = torch.empty(N, dtype=torch.float32, device="cuda")
    row = torch.empty(N, dtype=torch.float32, device="cuda")
    res = torch.empty(4, dtype=torch.float64, device="cuda")
    ws = coot.Workspace(N)
    t_expr = coot.serialize(synth.MAT_EXPR)
    t_chain = coot.serialize(synth.MAT_CHAIN)
    leaf = coot.serialize(synth.LEAF0)
    heads = coot.HEAD_SUM | coot.HEAD_NORM2 | coot.HEAD_MIN | coot.HEAD_MAX
    O1 = coot.Mat(out1, N, N, N)
    O2 = coot.Mat(out2, N, N, N)
    COL = coot.Mat(col, 1, N, 1)
    ROW = coot.Mat(row, N, 1, N)
    names = list(STREAMS)

    def step(ev=None, s=None):
        if ev is not None:
            ev[0].record(stream)
        coot.coot_expr_reduce(t_expr, mats, heads, out=O1, out_dev=res, ws=ws, stream=s)
        if ev is not None:
            ev[1].record(stream)
        coot.coot_expr_eval(t_chain, mats, O2, ws=ws, stream=s)
        if ev is not None:
            ev[2].record(stream)
        coot.coot_sum_dim(leaf, [O1], 0, COL, ws=ws, stream=s)
        if ev is not None:
            ev[3].record(stream)
        coot.coot_sum_dim(leaf, [O1], 1, ROW, ws=ws, stream=s)
        if ev is not None:
            ev[4].record(stream)

    launches_per_step = 4

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        step()
    barrier()
    # launch shape of each call (untimed)
    shapes = {}
    for i, n in enumerate(names):
        [lambda: coot.coot_expr_reduce(t_expr, mats, heads, out=O1, out_dev=res, ws=ws),
         lambda: coot.coot_expr_eval(t_chain, mats, O2, ws=ws),
         lambda: coot.coot_sum_dim(leaf, [O1], 0, COL, ws=ws),
         lambda: coot.coot_sum_dim(leaf, [O1], 1, ROW, ws=ws)][i]()
        shapes[n] = shape_text(coot.coot_last_launch())
    barrier()
    props = torch.cuda.get_device_properties(local)
    pci = None
    if hasattr(props, "pci_bus_id"):
        pci = f"{getattr(props, 'pci_domain_id', 0):08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
    # The timed steps: the step's four calls captured once as a CUDA graph
    # and replayed (their launches queue without host work in between), K
    # replays between barriers.
    g_step = _graph(torch, lambda s=None: step(None, s))
    for _ in range(max(args.warmup, 3)):
        g_step.replay()
    clocks = Clocks(local, pci)
    clocks.start()
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        g_step.replay()
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    ms_step = t_start.elapsed_time(t_end) / args.steps
    # Per-call device times (calls, roofline): K more steps issued call by
    # call with an event between calls, timed the same way.  The events
    # cost the step about 2%, so they stay out of the steps above.
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        step(evs[k])
    barrier()
    per_call = {n: [] for n in names}
    for k in range(args.steps):
        for i, n in enumerate(names):
            per_call[n].append(evs[k][i].elapsed_time(evs[k][i + 1]))
    if world > 1:
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = world * STEP_BYTES / (ms_step * 1e-3) / 1e9

    # the same results with the two trees in one coot_expr_multi call (the
    # four inputs read once) and the two sums: supplementary, `value` is the
    # four-call step above
    def step_one_pass(s=None):
        coot.coot_expr_multi([t_expr, t_chain], mats, [O1, O2], [heads, 0], out_dev=res, ws=ws, stream=s)
        coot.coot_sum_dim(leaf, [O1], 0, COL, ws=ws, stream=s)
        coot.coot_sum_dim(leaf, [O1], 1, ROW, ws=ws, stream=s)

    g_one = _graph(torch, step_one_pass)
    ms_one = _timed(torch, stream, g_one.replay, args.steps, args.warmup)
    one_bytes = (4 + 2 + 1 + 1) * MAT_BYTES

    # every result of the step in ONE launch: both trees stored, the heads,
    # and the column and row sums of `out` formed as it is computed
    # (coot_expr_multi_dims): the inputs read once, nothing read back
    dims_heads = [heads | coot.HEAD_COLSUM | coot.HEAD_ROWSUM, 0]

    def step_one_launch(s=None):
        coot.coot_expr_multi_dims([t_expr, t_chain], mats, [O1, O2], dims_heads, [COL, None], [ROW, None],
                                  out_dev=res, ws=ws, stream=s)

    g_launch = _graph(torch, step_one_launch)
    ms_launch = _timed(torch, stream, g_launch.replay, args.steps, args.warmup)
    coot.coot_expr_multi_dims([t_expr, t_chain], mats, [O1, O2], dims_heads, [COL, None], [ROW, None],
                              out_dev=res, ws=ws)
    launch_shape = shape_text(coot.coot_last_launch())
    launch_bytes = (4 + 2) * MAT_BYTES + 2 * N * ELEM

    # unfused baseline of the same step: one kernel per node, temporaries in HBM
    ms_unfused = None
    if not args.no_unfused:
        tmp = torch.empty(8 * N * N * 4, dtype=torch.uint8, device="cuda")

        def step_unfused():
            coot.coot_unfused_eval(t_expr, mats, O1, tmp=tmp)
            coot.coot_accu(leaf, [O1], out_dev=res[0:1], ws=ws)
            coot.coot_norm(leaf, [O1], "fro", out_dev=res[1:2], ws=ws)
            coot.coot_minmax(leaf, [O1], out_dev=res[2:4], ws=ws)
            coot.coot_unfused_eval(t_chain, mats, O2, tmp=tmp)
            coot.coot_sum_dim(leaf, [O1], 0, COL, ws=ws)
            coot.coot_sum_dim(leaf, [O1], 1, ROW, ws=ws)

        for _ in range(3):
            step_unfused()
        torch.cuda.synchronize()
        u0 = torch.cuda.Event(enable_timing=True)
        u1 = torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        for _ in range(args.steps):
            step_unfused()
        u1.record(stream)
        torch.cuda.synchronize()
        ms_unfused = u0.elapsed_time(u1) / args.steps
        del tmp

    # end to end through the API from pinned host buffers: inputs in, both
    # stored results and every reduction out, every step
    e2e = None
    if not args.no_e2e:
        pinned_in = [torch.from_numpy(h).pin_memory() for h in host]
        pin_out1 = torch.empty(N * N, dtype=torch.float32).pin_memory()
        pin_out2 = torch.empty(N * N, dtype=torch.float32).pin_memory()
        pin_col = torch.empty(N, dtype=torch.float32).pin_memory()
        pin_row = torch.empty(N, dtype=torch.float32).pin_memory()
        pin_res = torch.empty(4, dtype=torch.float64).pin_memory()

        def step_e2e():
            for d, h in zip(dev, pinned_in):
                d.copy_(h, non_blocking=True)
            step()
            pin_out1.copy_(out1, non_blocking=True)
            pin_out2.copy_(out2, non_blocking=True)
            pin_col.copy_(col, non_blocking=True)
            pin_row.copy_(row, non_blocking=True)
            pin_res.copy_(res, non_blocking=True)

        step_e2e()
        torch.cuda.synchronize()
        e_steps = max(2, min(args.steps, 5))

        def timed_e2e(fn, side_streams=()):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            barrier()
            e0.record(stream)
            for st in side_streams:
                st.wait_event(e0)  # nothing of the timed steps starts before e0
            for _ in range(e_steps):
                fn()
            e1.record(stream)  # fn leaves the compute stream waiting for every copy
            barrier()
            return e0.elapsed_time(e1) / e_steps

        ms_serial = timed_e2e(step_e2e)

        # The same step pipelined over K column blocks on three streams: the
        # inputs of block k come in on s_in while block k - 1 is computed on
        # the compute stream and the outputs of block k - 2 go out on s_out
        # (a copy stream per operand measured no faster: the host link is
        # the limit).  Every block's calls are the public ones on column
        # views; the row sums of each block land in FP64 and one more
        # sum(., 1) over the N x K partials gives sum(out, 1); the heads come
        # back per block and are combined on the host (accu: sum, norm2: root
        # of the summed squares, min / max).
        K = 8 if N % 8 == 0 else 1
        Q = N // K
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        rowp = torch.empty(N * K, dtype=torch.float64, device="cuda")
        res_k = torch.empty(4 * K, dtype=torch.float64, device="cuda")
        pin_res_k = torch.empty(4 * K, dtype=torch.float64).pin_memory()
        ROWP = coot.Mat(rowp, N, K, N)
        leaf64 = coot.serialize(synth.LEAF0, compute="f64")
        ev_in = [torch.cuda.Event() for _ in range(K)]
        ev_cmp = [torch.cuda.Event() for _ in range(K)]
        ev_out = [torch.cuda.Event() for _ in range(K)]
        ev_done = torch.cuda.Event()
        ev_tail = torch.cuda.Event()
        first = [True]

        def step_e2e_pipelined():
            for k in range(K):
                a, b = k * Q * N, (k + 1) * Q * N
                with torch.cuda.stream(s_in):
                    if not first[0]:
                        s_in.wait_event(ev_cmp[k])  # the previous step is done reading block k
                    for d, h in zip(dev, pinned_in):
                        d[a:b].copy_(h[a:b], non_blocking=True)
                    ev_in[k].record(s_in)
                stream.wait_event(ev_in[k])
                if not first[0]:
                    # the previous step's block k, and for block 0 its
                    # sums and heads, have gone out
                    stream.wait_event(ev_tail if k == 0 else ev_out[k])
                mk = [coot.Mat(t, N, Q, N, a) for t in dev]
                o1 = coot.Mat(out1, N, Q, N, a)
                coot.coot_expr_reduce(t_expr, mk, heads, out=o1, out_dev=res_k[4 * k:4 * k + 4], ws=ws)
                coot.coot_expr_eval(t_chain, mk, coot.Mat(out2, N, Q, N, a), ws=ws)
                coot.coot_sum_dim(leaf, [o1], 0, coot.Mat(col, 1, Q, 1, k * Q), ws=ws)
                coot.coot_sum_dim(leaf, [o1], 1, coot.Mat(rowp, N, 1, N, k * N), ws=ws)
                ev_cmp[k].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_cmp[k])
                    pin_out1[a:b].copy_(out1[a:b], non_blocking=True)
                    pin_out2[a:b].copy_(out2[a:b], non_blocking=True)
                    ev_out[k].record(s_out)
            coot.coot_sum_dim(leaf64, [ROWP], 1, ROW, ws=ws)
            ev_done.record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done)
                pin_col.copy_(col, non_blocking=True)
                pin_row.copy_(row, non_blocking=True)
                pin_res_k.copy_(res_k, non_blocking=True)
                ev_tail.record(s_out)
            first[0] = False

        # the pipelined step gives the serial step's results (the host
        # combine of the heads and the two-level row sums round differently)
        step_e2e()
        torch.cuda.synchronize()
        ref = [pin_out1.clone(), pin_out2.clone(), pin_col.clone(), pin_row.clone(), pin_res.clone()]
        step_e2e_pipelined()
        torch.cuda.synchronize()
        rk = pin_res_k.view(K, 4).double()
        heads_p = torch.stack([rk[:, 0].sum(), rk[:, 1].square().sum().sqrt(), rk[:, 2].min(), rk[:, 3].max()])
        assert torch.equal(pin_out1, ref[0]) and torch.equal(pin_out2, ref[1]), "pipelined outputs differ"
        assert torch.allclose(pin_col, ref[2], rtol=1e-6, atol=1e-5), "pipelined column sums differ"
        assert torch.allclose(pin_row, ref[3], rtol=1e-6, atol=1e-5), "pipelined row sums differ"
        assert torch.allclose(heads_p, ref[4], rtol=1e-9, atol=1e-6), "pipelined heads differ"

        def step_e2e_pipelined_joined():
            step_e2e_pipelined()
            stream.wait_stream(s_out)  # the step ends when its last copy has landed

        ms_pipe = timed_e2e(step_e2e_pipelined_joined, (s_in, s_out))

        # The step in ONE launch that reads its inputs from, and stores its
        # results into, the pinned host buffers themselves (their device
        # mappings, coot_host_device_pointer): the GPU reaches the Grace
        # CPU's memory coherently over NVLink-C2C, so the kernel streams the
        # inputs in and the results out while it computes, using both
        # directions of the link at once, with no copy and no staging buffer
        # on the device.  Only the four heads come back by copy.
        MH = [coot.Mat(h, N, N, N).mapped() for h in pinned_in]
        OH = [coot.Mat(pin_out1, N, N, N).mapped(), coot.Mat(pin_out2, N, N, N).mapped()]
        CH, RH = coot.Mat(pin_col, 1, N, 1).mapped(), coot.Mat(pin_row, N, 1, N).mapped()

        def step_e2e_host():
            coot.coot_expr_multi_dims([t_expr, t_chain], MH, OH, dims_heads, [CH, None], [RH, None],
                                      out_dev=res, ws=ws)
            pin_res.copy_(res, non_blocking=True)

        # the same results as the one-launch step on device buffers, bit for bit
        step_one_launch()
        torch.cuda.synchronize()
        ref = [t.cpu() for t in (out1, out2, col, row, res)]
        step_e2e_host()
        torch.cuda.synchronize()
        same = all(torch.equal(a, b) for a, b in zip(ref, (pin_out1, pin_out2, pin_col, pin_row, pin_res)))
        if not same:
            print("warning: the host-resident step differs from the device-resident one", file=sys.stderr)
        ms_host = timed_e2e(step_e2e_host)
        e2e = {"value": round(world * STEP_BYTES / (ms_host * 1e-3) / 1e9, 2), "unit": "GB/s",
               "ms_per_step": round(ms_host, 3), "h2d_bytes_per_step": 4 * MAT_BYTES,
               "d2h_bytes_per_step": 2 * MAT_BYTES + 2 * N * 4 + 4 * 8,
               "mode": "one launch (coot_expr_multi_dims) on the pinned host buffers through their device "
                       "mappings: inputs read and results written over NVLink-C2C during the kernel",
               "bitwise_equal_to_device_run": same,
               "copy_in_step_copy_out": {"value": round(world * STEP_BYTES / (ms_serial * 1e-3) / 1e9, 2),
                                         "ms_per_step": round(ms_serial, 3),
                                         "mode": "copy in, four-call step, copy out on one stream"},
               "pipelined": {"value": round(world * STEP_BYTES / (ms_pipe * 1e-3) / 1e9, 2),
                             "ms_per_step": round(ms_pipe, 3),
                             "d2h_bytes_per_step": 2 * MAT_BYTES + 2 * N * 4 + 4 * 8 * K,
                             "mode": f"{K} column blocks pipelined on three streams (copy in, compute, copy out)"}}

    peak, peak_kind = peaks()
    dom = max(names, key=lambda n: statistics.mean(per_call[n]))
    traffic, traffic_note = (committed_traffic(dom, shapes[dom]) if N == 8192
                             else (None, "traffic is captured at 8192 x 8192"))
    dom_ms = statistics.mean(per_call[dom])
    achieved = STREAMS[dom] * MAT_BYTES / (dom_ms * 1e-3) / 1e9
    calls = {n: {"ms": round(statistics.mean(per_call[n]), 4),
                 "gbs": round(STREAMS[n] * MAT_BYTES / (statistics.mean(per_call[n]) * 1e-3) / 1e9, 1),
                 "launch": shapes[n]}
             for n in names}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, nbytes, _ = oracle_sample(seed, args.cpu_cols)
        cpu = {"value": round(nbytes / dt / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"{N} x {args.cpu_cols} column block of every matrix, whole step, {dt:.1f} s"}
        dt_all, nbytes_all, threads = cpu_fp32_sample(seed, args.cpu_cols)
        cpu["all_cores"] = {"value": round(nbytes_all / dt_all / 1e9, 3), "unit": "GB/s", "cores": threads,
                            "os_cpu_count": os.cpu_count(), "kind": "fp32 OpenMP evaluator (oracle/cpu_fp32.c)",
                            "sample": f"{N} x {args.cpu_cols} column block of every matrix, whole step, best of 3, "
                                      f"{dt_all * 1e3:.1f} ms"}
    errors = None
    if rank == 0 and not args.no_errors:
        errors = matrix_errors(coot, torch, dev, args.err_cols)
    workloads = None
    if rank == 0 and world == 1 and not args.no_workloads:
        # the other workloads, each with its own timing and clock record
        # (supplementary: `value` is the matrix step above)
        workloads = {"vectors": vectors_result(args),
                     "precision_bf16": precision_result(args, "bf16", error_elems=1 << 24),
                     "precision_f16": precision_result(args, "f16", error_elems=1 << 24),
                     "batched": batched_result(args)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if N == 8192 else WORKLOAD.replace("8192x8192", f"{N}x{N}"),
                       "n_rows": N, "n_cols": N, "step_bytes": STEP_BYTES,
                       "l2": f"inputs larger than L2 ({4 * MAT_BYTES / 1e9:.2f} GB of inputs per step), no flush",
                       "timing": "the step's four calls captured once as a CUDA graph and replayed K times; "
                                 "per-call times from K more steps issued call by call with events",
                       "parallelism": f"replicas x{world}"},
            "frac_of_hbm_peak": round(value / world / peak, 4),
            "unfused": None if ms_unfused is None else {
                "ms_per_step": round(ms_unfused, 4),
                "value": round(world * STEP_BYTES / (ms_unfused * 1e-3) / 1e9, 1),
                "fused_speedup": round(ms_unfused / ms_step, 3)},
            "calls": calls,
            "one_pass": {"ms_per_step": round(ms_one, 4), "step_speedup": round(ms_step / ms_one, 3),
                         "gbs": round(world * one_bytes / (ms_one * 1e-3) / 1e9, 1),
                         "algorithmic_bytes": one_bytes,
                         "calls": "coot_expr_multi (both trees, inputs read once) + two coot_sum_dim"},
            "one_launch": {"ms_per_step": round(ms_launch, 4), "step_speedup": round(ms_step / ms_launch, 3),
                           "gbs": round(world * launch_bytes / (ms_launch * 1e-3) / 1e9, 1),
                           "frac": round(launch_bytes / (ms_launch * 1e-3) / 1e9 / peak, 4),
                           "algorithmic_bytes": launch_bytes, "launch": launch_shape,
                           "calls": "coot_expr_multi_dims: both trees stored, accu/norm2/min/max, sum dim 0 "
                                    "and dim 1 of out, one kernel"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": traffic, "traffic_note": traffic_note, "launch": shapes[dom],
                         "algorithmic_bytes": STREAMS[dom] * MAT_BYTES},
            "cpu_baseline": cpu,
            "errors": errors,
            "workloads": workloads,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- other workloads (one JSON line each)

def _rel(got, want):
    """|got - want| / |want| in three significant digits (the absolute
    difference when want is 0)."""
    d = abs(got - want) / abs(want) if want != 0 else abs(got - want)
    return float(f"{d:.3e}")


def _timed(torch, stream, fn, steps, warmup):
    """Device time of `fn` per call (CUDA events on `stream`)."""
    for _ in range(max(warmup, 3)):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _graph(torch, fn):
    """`fn` captured once as a CUDA graph (compiled kernels are warmed first)."""
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            fn(s)
    torch.cuda.synchronize()
    return g


def vectors_result(args):
    """FP32 vectors n = 1,000,000: y = 2x + 3z, accu(x % z), norm2(x).  The
    step is latency-bound (24 MB fits in L2): reported as microseconds per
    step, eager calls and as one CUDA graph; plus the errors of accu(x % z)
    and norm2(x) against the FP64 oracle."""
    import torch
    import paper_2308_03120_gb300 as coot
    from paper_2308_03120_gb300 import build as _build
    from oracle import coot_oracle as O
    _build.build()
    coot.coot_init(0)
    n = 1_000_000
    seed = synth.BASE_SEED
    hx, hz = synth.uniform_f32(seed, n), synth.uniform_f32(seed + 1, n)
    x = torch.from_numpy(hx).cuda()
    z = torch.from_numpy(hz).cuda()
    y = torch.empty(n, device="cuda")
    X, Z, Y = coot.Mat(x, n, 1, n), coot.Mat(z, n, 1, n), coot.Mat(y, n, 1, n)
    res = torch.empty(2, dtype=torch.float64, device="cuda")
    ws = coot.Workspace(1)
    t_axpy = coot.serialize(synth.AXPY_2X_3Z)
    t_schur = coot.serialize(synth.SCHUR_XZ)
    leaf = coot.serialize(synth.LEAF0)

    def step(s=None):
        coot.coot_expr_eval(t_axpy, [X, Z], Y, stream=s)
        coot.coot_accu(t_schur, [X, Z], out_dev=res[0:1], ws=ws, stream=s)
        coot.coot_norm(leaf, [X], 2, out_dev=res[1:2], ws=ws, stream=s)

    # the same three results from one coot_expr_multi call: x and z read once
    trees = [t_axpy, t_schur, leaf]
    heads = [0, coot.HEAD_SUM, coot.HEAD_NORM2]

    def step_multi(s=None):
        coot.coot_expr_multi(trees, [X, Z], [Y, None, None], heads, out_dev=res, ws=ws, stream=s)

    stream = torch.cuda.current_stream()
    g = _graph(torch, step)
    gm = _graph(torch, step_multi)
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    ms = _timed(torch, stream, step, args.steps, args.warmup)
    ms_g = _timed(torch, stream, g.replay, args.steps, args.warmup)
    ms_m = _timed(torch, stream, step_multi, args.steps, args.warmup)
    ms_mg = _timed(torch, stream, gm.replay, args.steps, args.warmup)
    clk = clocks.stop()
    step()
    torch.cuda.synchronize()
    got = res.cpu().tolist()
    hs = [synth.as_mat(hx, "f32", n, 1), synth.as_mat(hz, "f32", n, 1)]
    want = [O.accu(t_schur, hs), O.norm(leaf, hs[:1], 2)]
    yw, yb, y_unsafe = (a.ravel() for a in O.error_bound(O.decode(t_axpy), hs))
    yg = y.cpu().numpy().astype(np.float64)
    # the element-wise tolerance: 1e-5 of the value plus twice the oracle's
    # bound on the FP32 evaluation's own error, which dominates where 2x and
    # 3z nearly cancel (there the relative error alone is large)
    y_tol = 1e-5 * np.abs(yw) + 2.0 * yb
    nbytes = (3 + 2 + 1) * n * 4
    return {"metric": "fused vector step latency", "workload": "vectors n=1e6 fp32: 2x+3z, accu(x%z), norm2(x)",
            "us_per_step": round(ms * 1e3, 2), "us_per_step_graph": round(ms_g * 1e3, 2),
            "gbs_graph": round(nbytes / (ms_g * 1e-3) / 1e9, 1), "bytes_per_step": nbytes,
            "launches_per_step": 3,
            "one_pass": {"us_per_step": round(ms_m * 1e3, 2), "us_per_step_graph": round(ms_mg * 1e3, 2),
                         "launches_per_step": 1, "bytes_per_step": 3 * n * 4,
                         "call": "coot_expr_multi: 2x+3z stored, accu(x%z), norm2(x)"},
            "errors": {"vs": "FP64 oracle", "accu(x%z)": _rel(got[0], want[0]), "norm2(x)": _rel(got[1], want[1]),
                       "2x+3z max_rel": float(f"{np.max(np.abs(yg - yw) / np.maximum(np.abs(yw), 1e-300)):.3e}"),
                       "2x+3z max_err_over_tol": float(f"{np.max(np.abs(yg - yw) / y_tol):.3e}"),
                       "2x+3z unsafe_skipped": int(y_unsafe.sum())},
            "note": "24 MB per step is L2-resident: latency, not HBM, bound", "clocks": clk}


def run_vectors(args):
    print(json.dumps(vectors_result(args)), flush=True)


def precision_errors(dt, hx, hz, y_bits, got, n):
    """Errors of the precision workload's results over the first n elements
    against the FP64 oracle: relative errors of accu(x), norm2(x) and
    dot(x, z) (exact oracle sums), and for y = 2x + 3z stored in dt the
    largest distance in storage ulps from the oracle value rounded to dt and
    the fraction of elements equal to it."""
    from oracle import coot_oracle as O
    step = 1 << 24
    chunks = range(0, n, step)
    vx = lambda i: O.decode_storage(hx[i:min(i + step, n)], dt)  # noqa: E731
    vz = lambda i: O.decode_storage(hz[i:min(i + step, n)], dt)  # noqa: E731
    acc = O._fsum(vx(i) for i in chunks)
    nrm = math.sqrt(O._fsum(vx(i) ** 2 for i in chunks))
    dot = O._fsum(vx(i) * vz(i) for i in chunks)
    tree = O.encode(synth.AXPY_2X_3Z)
    p, emin, _ = O.FORMATS[dt]
    worst, exact = 0.0, 0
    for i in chunks:
        m = min(i + step, n) - i
        ins = [synth.as_mat(hx[i:i + m], dt, m, 1), synth.as_mat(hz[i:i + m], dt, m, 1)]
        ref = O.round_to_format(O.evaluate(tree, ins).ravel(), dt)
        g = O.decode_storage(y_bits[i:i + m], dt)
        fin = np.isfinite(ref)
        a = np.abs(ref[fin])
        _, ex = np.frexp(np.where(a > 0, a, 1.0))
        ulp = np.ldexp(1.0, np.maximum(ex - 1, emin) - (p - 1))
        d = np.abs(g[fin] - ref[fin]) / ulp
        worst = max(worst, float(d.max()) if d.size else 0.0)
        exact += int(np.sum(d == 0)) + int(np.sum(~fin & (g == ref)))
    return {"vs": "FP64 oracle", "elements": n, "accu(x)": _rel(got[0], acc), "norm2(x)": _rel(got[1], nrm),
            "dot(x,z)": _rel(got[2], dot),
            f"2x+3z max {dt} ulps": worst, "2x+3z exact_frac": round(exact / n, 6)}


def precision_result(args, dt, error_elems=None):
    """n = 2^28 stored as BF16 or FP16 (signed lognormal, sigma 2): y = 2x + 3z
    stored in the same type, accu(x) and norm2(x) in one pass, dot(x, z);
    the errors of every result against the FP64 oracle over all 2^28
    elements, or, with error_elems, over the calls' results on the first
    error_elems elements."""
    import torch
    import paper_2308_03120_gb300 as coot
    from paper_2308_03120_gb300 import build as _build
    _build.build()
    coot.coot_init(0)
    n = 1 << 28
    seed = synth.BASE_SEED + 2
    tdt = torch.bfloat16 if dt == "bf16" else torch.float16
    hx, rx = synth.lognormal_signed(seed, n, dt)
    hz, rz = synth.lognormal_signed(seed + 1, n, dt)

    def dev(h):
        t = torch.from_numpy(h.view(np.int16)).view(tdt) if dt == "bf16" else torch.from_numpy(h)
        return t.cuda()
    x, z = dev(hx), dev(hz)
    y = torch.empty(n, dtype=tdt, device="cuda")
    X, Z, Y = coot.Mat(x, n, 1, n), coot.Mat(z, n, 1, n), coot.Mat(y, n, 1, n)
    res = torch.empty(3, dtype=torch.float64, device="cuda")
    ws = coot.Workspace(1)
    t_axpy = coot.serialize(synth.AXPY_2X_3Z)
    leaf = coot.serialize(synth.LEAF0)
    stream = torch.cuda.current_stream()
    calls = {
        "expr_eval 2x+3z": (lambda: coot.coot_expr_eval(t_axpy, [X, Z], Y), 3 * n * 2),
        "expr_reduce accu+norm2(x)": (lambda: coot.coot_expr_reduce(leaf, [X], coot.HEAD_SUM | coot.HEAD_NORM2,
                                                                    out_dev=res[0:2], ws=ws), n * 2),
        "dot(x, z)": (lambda: coot.coot_dot(X, Z, out_dev=res[2:3], ws=ws), 2 * n * 2),
    }
    peak, kind = peaks()
    out = {}
    total_ms = 0.0
    total_b = 0
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    for name, (fn, nbytes) in calls.items():
        ms = _timed(torch, stream, fn, args.steps, args.warmup)
        out[name] = {"ms": round(ms, 4), "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                     "frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4),
                     "launch": shape_text(coot.coot_last_launch())}
        total_ms += ms
        total_b += nbytes
    clk = clocks.stop()
    # the errors: the same calls over all n elements, or over a prefix
    m = n if error_elems is None else min(n, error_elems)
    Xm, Zm, Ym = coot.Mat(x, m, 1, m), coot.Mat(z, m, 1, m), coot.Mat(y, m, 1, m)
    coot.coot_expr_eval(t_axpy, [Xm, Zm], Ym)
    coot.coot_expr_reduce(leaf, [Xm], coot.HEAD_SUM | coot.HEAD_NORM2, out_dev=res[0:2], ws=ws)
    coot.coot_dot(Xm, Zm, out_dev=res[2:3], ws=ws)
    torch.cuda.synchronize()
    got = res.cpu().tolist()
    yh = y[:m].cpu()
    y_bits = yh.view(torch.int16).numpy().view(np.uint16) if dt == "bf16" else yh.numpy()
    errors = precision_errors(dt, hx, hz, y_bits, got, m)
    if error_elems is not None:
        errors["sample"] = f"the three calls on the first {m} of {n} elements"
    return {"metric": "fused low-precision step HBM GB/s", "workload": f"vectors n=2^28 {dt}",
            "value": round(total_b / (total_ms * 1e-3) / 1e9, 1), "unit": "GB/s",
            "frac_of_hbm_peak": round(total_b / (total_ms * 1e-3) / 1e9 / peak, 4), "peak_kind": kind,
            "calls": out, "errors": errors, "fp16_redraws": rx + rz if dt == "f16" else 0, "clocks": clk}


def run_precision(args, dt):
    print(json.dumps(precision_result(args, dt)), flush=True)


def batched_result(args):
    """4096 FP32 matrices, rows and cols log-uniform in [1, 512]:
    out = exp(-abs(A)) % B + 0.5 C and sum(out, 0) per matrix, in one
    persistent launch captured as a CUDA graph, against one launch per
    matrix (eager, and the same launches captured as one graph)."""
    import torch
    import paper_2308_03120_gb300 as coot
    from paper_2308_03120_gb300 import build as _build
    _build.build()
    coot.coot_init(0)
    nmat = 4096
    rows = synth.loguniform_int(synth.BASE_SEED + 3, nmat, 1, 512)
    cols = synth.loguniform_int(synth.BASE_SEED + 4, nmat, 1, 512)
    sizes = (rows * cols).astype(np.int64)
    # every operand of every matrix packed in one buffer per operand, each
    # matrix starting on a 16-byte boundary
    offs = np.zeros(nmat + 1, dtype=np.int64)
    offs[1:] = np.cumsum((sizes + 3) // 4 * 4)
    coff = np.zeros(nmat + 1, dtype=np.int64)
    coff[1:] = np.cumsum((cols + 3) // 4 * 4)
    total = int(offs[-1])
    bufs = [torch.from_numpy(synth.uniform_f32(synth.BASE_SEED + 10 + k, total)).cuda() for k in range(3)]
    out = torch.empty(total, device="cuda")
    csum = torch.empty(int(coff[-1]), device="cuda")
    tree = coot.serialize(synth.BATCH_EXPR)
    items, per = [], []
    for m in range(nmat):
        r, c, o = int(rows[m]), int(cols[m]), int(offs[m])
        ins = [coot.Mat(b, r, c, r, o) for b in bufs]
        om = coot.Mat(out, r, c, r, o)
        cm = coot.Mat(csum, 1, c, 1, int(coff[m]))
        items.append(coot.batch_item(ins, om, cm))
        per.append((ins, om, cm))
    plan, n_items, n_work = coot.coot_batch_plan(items, 3)
    stream = torch.cuda.current_stream()

    def batched(s=None):
        coot.coot_expr_eval_batched(tree, [0, 0, 0], 0, 0, plan, n_items, n_work, stream=s)

    g = _graph(torch, batched)
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    ms_graph = _timed(torch, stream, g.replay, args.steps, args.warmup)
    ms_eager = _timed(torch, stream, batched, args.steps, args.warmup)
    clk = clocks.stop()
    ws = coot.Workspace(1)

    def per_matrix(s=None):
        for ins, om, cm in per:
            coot.coot_expr_eval(tree, ins, om, stream=s)
            coot.coot_sum_dim(tree, ins, 0, cm, ws=ws, stream=s)

    if args.no_per_matrix:
        ms_per = ms_per_graph = float("nan")
    else:
        ms_per = _timed(torch, stream, per_matrix, max(2, args.steps // 10), 1)
        gp = _graph(torch, per_matrix)
        ms_per_graph = _timed(torch, stream, gp.replay, max(2, args.steps // 10), 1)
    elems = int(sizes.sum())
    nbytes = elems * 4 * 4 + int(cols.sum()) * 4
    peak, kind = peaks()
    return {
        "metric": "batch evals/s", "workload": "4096 fp32 matrices, rows/cols log-uniform [1,512]: "
        "exp(-abs(A))%B+0.5C and column sums", "unit": "matrices/s",
        "value": round(nmat / (ms_graph * 1e-3), 1), "batches_per_s": round(1.0 / (ms_graph * 1e-3), 1),
        "ms_per_batch_graph": round(ms_graph, 4), "ms_per_batch_eager": round(ms_eager, 4),
        "gbs": round(nbytes / (ms_graph * 1e-3) / 1e9, 1), "frac_of_hbm_peak": round(nbytes / (ms_graph * 1e-3) / 1e9 / peak, 4),
        "peak_kind": kind, "elements": elems, "work_units": n_work,
        "per_matrix_launches": {"ms_eager": round(ms_per, 3), "ms_graph": round(ms_per_graph, 3), "launches": 2 * nmat},
        "speedup_vs_per_matrix_eager": round(ms_per / ms_graph, 1),
        "speedup_vs_per_matrix_graph": round(ms_per_graph / ms_graph, 1), "clocks": clk}


def run_batched(args):
    print(json.dumps(batched_result(args)), flush=True)


def run_stats(args):
    """All six statistics (sum, mean, var, stddev, min, max) of every column
    and of every row of an 8192 x 8192 FP32 matrix in one pass per
    dimension: of the stored matrix A (one input) and of the tree
    (A%B+2C)/(1+|D|) (four inputs).  Algorithmic bytes: the inputs read once
    plus 6 x 8192 FP32 results per call."""
    import torch
    import paper_2308_03120_gb300 as coot
    from paper_2308_03120_gb300 import build as _build
    _build.build()
    coot.coot_init(0)
    seed = synth.BASE_SEED + 1
    dev = [torch.from_numpy(h).cuda() for h in inputs_host(seed)]
    mats = [coot.Mat(t, N, N, N) for t in dev]
    ws = coot.Workspace(N)
    outs = {d: [torch.empty(N, device="cuda") for _ in range(6)] for d in (0, 1)}
    omats = {0: [coot.Mat(t, 1, N, 1) for t in outs[0]], 1: [coot.Mat(t, N, 1, N) for t in outs[1]]}
    stream = torch.cuda.current_stream()
    peak, peak_kind = peaks()
    calls = {}
    for name, sexpr, ins in (("leaf", synth.LEAF0, mats[:1]), ("tree", synth.MAT_EXPR, mats)):
        tree = coot.serialize(sexpr)
        for dim in (0, 1):
            def fn(tree=tree, ins=ins, dim=dim):
                coot.coot_stats_dim(tree, ins, dim, 0x3F, omats[dim], ws=ws)
            ms = _timed(torch, stream, fn, args.steps, args.warmup)
            nbytes = len(ins) * MAT_BYTES + 6 * N * 4
            gbs = nbytes / (ms * 1e-3) / 1e9
            calls[f"{name}_dim{dim}"] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                                         "launch": shape_text(coot.coot_last_launch())}
    total_ms = sum(c["ms"] for c in calls.values())
    total_bytes = sum((1 if k.startswith("leaf") else 4) * MAT_BYTES + 6 * N * 4 for k in calls)
    dom = max(calls, key=lambda k: calls[k]["ms"])
    print(json.dumps({"metric": "fused per-dim statistics HBM GB/s", "workload": f"matrices {N}x{N} fp32: "
                      "sum/mean/var/stddev/min/max of every column and row, of A and of (A%B+2C)/(1+|D|)",
                      "value": round(total_bytes / (total_ms * 1e-3) / 1e9, 1), "unit": "GB/s",
                      "frac_of_hbm_peak": round(total_bytes / (total_ms * 1e-3) / 1e9 / peak, 4),
                      "peak": peak, "peak_kind": peak_kind, "calls": calls,
                      "roofline": {"bound": "hbm", "kernel": dom, "achieved": calls[dom]["gbs"], "peak": peak,
                                   "unit": "GB/s", "frac": calls[dom]["frac"]},
                      "l2": "inputs larger than L2, no flush"}), flush=True)


def run_convert(args):
    """Fused type conversion (Section 7: an integer matrix converted and
    used in one float expression): B = 2 A + 1 with A an 8192 x 8192 int32
    matrix and B FP32, in one kernel (read 4 B, write 4 B per element),
    against converting first into an FP32 temporary and then evaluating the
    expression (read 4, write 4, read 4, write 4)."""
    import torch
    import paper_2308_03120_gb300 as coot
    from paper_2308_03120_gb300 import build as _build
    _build.build()
    coot.coot_init(0)
    u = synth.uniform01(synth.BASE_SEED + 5, N * N)
    a = torch.from_numpy(np.floor(-1e6 + u * 2e6).astype(np.int32)).cuda()
    tmp = torch.empty(N * N, device="cuda")
    out = torch.empty(N * N, device="cuda")
    A, T, B = (coot.Mat(t, N, N, N) for t in (a, tmp, out))
    expr = coot.serialize(("add", ("mul", synth.C(2.0), synth.X(0)), synth.C(1.0)))
    leaf = coot.serialize(synth.LEAF0)
    stream = torch.cuda.current_stream()

    def fused():
        coot.coot_expr_eval(expr, [A], B)

    def two_step():
        coot.coot_expr_eval(leaf, [A], T)
        coot.coot_expr_eval(expr, [T], B)

    ms_f = _timed(torch, stream, fused, args.steps, args.warmup)
    ms_u = _timed(torch, stream, two_step, args.steps, args.warmup)
    peak, peak_kind = peaks()
    fused_bytes = 8 * N * N
    print(json.dumps({"metric": "fused int32->fp32 conversion + expression", "workload":
                      f"B = 2 A + 1, A {N}x{N} int32, B fp32", "unit": "ms",
                      "fused_ms": round(ms_f, 4), "two_step_ms": round(ms_u, 4),
                      "fusion_speedup": round(ms_u / ms_f, 3),
                      "fused_gbs": round(fused_bytes / (ms_f * 1e-3) / 1e9, 1),
                      "frac_of_hbm_peak": round(fused_bytes / (ms_f * 1e-3) / 1e9 / peak, 4), "peak_kind": peak_kind,
                      "two_step_gbs": round(2 * fused_bytes / (ms_u * 1e-3) / 1e9, 1),
                      "l2": "inputs larger than L2, no flush"}), flush=True)


def run_canonical(args):
    """Canonical forms at run time: dot(x, x) over 2^28 FP32 values issues
    one load per element instead of two, and a tree written with redundancy
    (-(-(A % 1)) + 2 % (4 % (B - 0)) + (2 + 3) % C) needs fewer nodes (the
    unfused baseline launches one kernel per node)."""
    import torch
    import paper_2308_03120_gb300 as coot
    from paper_2308_03120_gb300 import build as _build
    _build.build()
    coot.coot_init(0)
    stream = torch.cuda.current_stream()
    n = 1 << 28
    x = torch.from_numpy(synth.uniform_f32(synth.BASE_SEED + 6, n)).cuda()
    X = coot.Mat(x, n, 1, n)
    res = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = coot.Workspace(1)
    out = {}
    for on in (True, False):
        coot.coot_set_canonical(on)
        out[on] = _timed(torch, stream, lambda: coot.coot_dot(X, X, out_dev=res, ws=ws), args.steps, args.warmup)
    coot.coot_set_canonical(True)
    C_, X_ = synth.C, synth.X
    e = ("add", ("add", ("neg", ("neg", ("mul", X_(0), C_(1.0)))),
                 ("mul", C_(2.0), ("mul", C_(4.0), ("sub", X_(1), C_(0.0))))),
         ("mul", ("add", C_(2.0), C_(3.0)), X_(2)))
    tree = coot.serialize(e)
    nodes_before = len(tree) // 16 - 1
    nodes_after = len(coot.coot_tree_canonical(tree)) // 16 - 1
    m = 8192
    mats = [coot.Mat(torch.from_numpy(synth.uniform_f32(synth.BASE_SEED + 7 + k, m * m)).cuda(), m, m, m)
            for k in range(3)]
    o = coot.Mat(torch.empty(m * m, device="cuda"), m, m, m)
    tmp = torch.empty(coot.coot_unfused_tmp_count(tree) * m * m * 4, dtype=torch.uint8, device="cuda")
    t_unf = {}
    t_fused = {}
    for on in (True, False):
        coot.coot_set_canonical(on)
        t_unf[on] = _timed(torch, stream, lambda: coot.coot_unfused_eval(tree, mats, o, tmp=tmp), args.steps,
                           args.warmup)
        t_fused[on] = _timed(torch, stream, lambda: coot.coot_expr_eval(tree, mats, o), args.steps, args.warmup)
    coot.coot_set_canonical(True)
    ops = lambda raw: sum(1 for k in range(len(raw) // 16 - 1) if raw[16 + 16 * k] > 1)  # noqa: E731
    print(json.dumps({"metric": "run-time canonical forms", "unit": "ms",
                      "dot_x_x_2^28_fp32": {"canonical_ms": round(out[True], 4), "original_ms": round(out[False], 4),
                                            "speedup": round(out[False] / out[True], 3),
                                            "loads_canonical": n, "loads_original": 2 * n,
                                            "note": "DRAM bytes are equal: the second read of the same address "
                                                    "hits L2, so only the issued loads halve"},
                      "redundant_tree_8192^2": {"nodes_before": nodes_before, "nodes_after": nodes_after,
                                                "unfused_kernels_before": ops(tree),
                                                "unfused_kernels_after": ops(coot.coot_tree_canonical(tree)),
                                                "unfused_ms_canonical": round(t_unf[True], 4),
                                                "unfused_ms_original": round(t_unf[False], 4),
                                                "fused_ms_canonical": round(t_fused[True], 4),
                                                "fused_ms_original": round(t_fused[False], 4)}}), flush=True)


def run_views(args):
    """Submatrix views (ld = 8192 > rows): the matrix tree over the 6144 x
    6144 window starting at (1024, 1024) of the 8192 x 8192 inputs, stored
    into the same window of the output, and the column / row sums of the
    stored window.  Algorithmic bytes: the window's elements only."""
    import torch
    import paper_2308_03120_gb300 as coot
    from paper_2308_03120_gb300 import build as _build
    _build.build()
    coot.coot_init(0)
    seed = synth.BASE_SEED + 1
    dev = [torch.from_numpy(h).cuda() for h in inputs_host(seed)]
    full = [coot.Mat(t, N, N, N) for t in dev]
    w0, w1 = N // 8, N - N // 8 - 1
    mats = [m.submat(w0, w0, w1, w1) for m in full]
    O1 = coot.Mat(torch.empty(N * N, device="cuda"), N, N, N).submat(w0, w0, w1, w1)
    n = w1 - w0 + 1
    col = coot.Mat(torch.empty(n, device="cuda"), 1, n, 1)
    row = coot.Mat(torch.empty(n, device="cuda"), n, 1, n)
    ws = coot.Workspace(n)
    t_expr = coot.serialize(synth.MAT_EXPR)
    leaf = coot.serialize(synth.LEAF0)
    stream = torch.cuda.current_stream()
    peak, peak_kind = peaks()
    calls = {}
    for name, fn, streams in (("expr_eval", lambda: coot.coot_expr_eval(t_expr, mats, O1), 5),
                              ("sum_dim0", lambda: coot.coot_sum_dim(leaf, [O1], 0, col, ws=ws), 1),
                              ("sum_dim1", lambda: coot.coot_sum_dim(leaf, [O1], 1, row, ws=ws), 1)):
        ms = _timed(torch, stream, fn, args.steps, args.warmup)
        gbs = streams * n * n * 4 / (ms * 1e-3) / 1e9
        calls[name] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                       "launch": shape_text(coot.coot_last_launch())}
    print(json.dumps({"metric": "fused evaluation and sums over submatrix views HBM GB/s", "workload":
                      f"{n}x{n} window at ({w0}, {w0}) of {N}x{N} fp32 matrices (ld {N})", "unit": "GB/s",
                      "calls": calls,
                      "peak": peak, "peak_kind": peak_kind,
                      "l2": "inputs larger than L2, no flush"}), flush=True)


def run_learned(args):
    """Learned launch shapes on random trees the model never saw (fresh
    seeds): regret against the exhaustive tuner, model and built-in, over
    the training range of sizes (2^10 to 2^26 elements) and over larger
    calls (2^26 to 2^30 elements, never in training)."""
    import paper_2308_03120_gb300 as coot
    from paper_2308_03120_gb300 import build as _build, learn
    _build.build()
    coot.coot_init(0)
    t0 = time.time()
    learn.load_policy()   # loads the model for host_predict
    learn.use_builtin()
    bands = {}
    for name, n_trees, seed, lo, hi in (("2^10..2^26", args.learned_trees, 4242, 10, 26),
                                        ("2^26..2^30", args.learned_large_trees, 4343, 26, 30)):
        if n_trees <= 0:
            continue
        samples = learn.generate(n_trees, seed=seed, min_log2=lo, max_log2=hi, log=lambda *a: None)
        r = learn.regret(samples, learn.host_predict)
        bands[name] = {"model_geomean": round(r["model_geomean"], 4), "builtin_geomean": round(r["builtin_geomean"], 4),
                       "model_within_5pct": round(r["model_within_5pct"], 3),
                       "builtin_within_5pct": round(r["builtin_within_5pct"], 3),
                       "model_worst": round(r["model_worst"], 3), "samples": r["samples"], "unseen_trees": n_trees,
                       "seed": seed}
    first = next(iter(bands.values()))
    print(json.dumps({"metric": "learned launch-shape regret vs exhaustive tuner (geomean, lower is better)",
                      "value": first["model_geomean"], "unit": "ratio", "higher_is_better": False,
                      "builtin": first["builtin_geomean"], "target": 1.05, "by_size": bands,
                      "seconds": round(time.time() - t0, 1)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="coot", choices=["coot", "reference"])
    ap.add_argument("--ref-cols", type=int, default=256, help="columns in each reference-arm step's sample")
    ap.add_argument("--cpu-cols", type=int, default=4096, help="columns in the cpu_baseline sample")
    ap.add_argument("--kernel-source-hash", action="store_true",
                    help="print the digest of the kernel sources that committed traffic figures are tied to")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=8192, help="matrix order (8192 is the workload; smaller for profiling)")
    ap.add_argument("--no-unfused", action="store_true", help="skip the unfused-baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--no-per-matrix", action="store_true", help="batched: skip the one-launch-per-matrix leg")
    ap.add_argument("--no-errors", action="store_true", help="skip the errors against the oracle")
    ap.add_argument("--err-cols", type=int, default=512, help="columns in the errors' sample")
    ap.add_argument("--no-workloads", action="store_true",
                    help="matrices: skip the vectors, precision and batched workloads in the same line")
    ap.add_argument("--learned-trees", type=int, default=40, help="learned: unseen random trees to evaluate")
    ap.add_argument("--learned-large-trees", type=int, default=12,
                    help="learned: unseen random trees on 2^26..2^30-element calls")
    ap.add_argument("--workload", default="matrices",
                    choices=["matrices", "vectors", "precision-bf16", "precision-f16", "batched", "learned", "stats", "convert", "canonical", "views"],
                    help="matrices is the headline line; the others print their own line")
    args = ap.parse_args()
    if args.kernel_source_hash:
        print(kernel_source_hash())
        return
    global N, MAT_BYTES, STEP_BYTES
    N = args.n
    MAT_BYTES = N * N * ELEM
    STEP_BYTES = sum(STREAMS.values()) * MAT_BYTES
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "vectors":
        run_vectors(args)
    elif args.workload in ("precision-bf16", "precision-f16"):
        run_precision(args, args.workload.split("-")[1])
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "stats":
        run_stats(args)
    elif args.workload == "convert":
        run_convert(args)
    elif args.workload == "canonical":
        run_canonical(args)
    elif args.workload == "views":
        run_views(args)
    else:
        run_coot(args)


if __name__ == "__main__":
    main()
