"""Learned launch shapes: timing data, training on the GPU, evaluation.

The cost model (a 2-layer, width-64 MLP; coot.h "Learned launch shapes")
predicts log(kernel time in microseconds) from the features of a call and
of one candidate launch shape.  The data are the library's own timings:
random expression trees (synth.random_tree, 2-12 operators over 1-4
inputs) on random shapes (element count log-uniform), FP32 or BF16, for
the four kernel kinds, each timed under every candidate shape of its kind
and under the built-in choice.  The model trains on the GPU through the
library's own kernels (coot_mlp_forward, coot_mlp_loss_grad,
coot_mlp_adam).  Held-out trees (never seen in training) measure the
regret t(chosen shape) / t(fastest shape measured) of the model and of
the built-in choice.

    python -m paper_2308_03120_gb300.learn --trees 400 --out report.json
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import pickle
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import _abi

KIND_MAP, KIND_REDUCE, KIND_COLSUM, KIND_ROWSUM = 0, 1, 2, 3
KINDS = (KIND_MAP, KIND_REDUCE, KIND_COLSUM, KIND_ROWSUM)
D = _abi.MODEL_FEATURES
H = _abi.MODEL_HIDDEN
MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "launch_cost_model.json")
DTYPES = {"f32": 0, "bf16": 1}
REDUCE_HEADS = 1 | 4      # sum and norm2


def n_params(d: int = D, h: int = H) -> int:
    return d * h + h * h + 3 * h + 1     # W1, W2, and b1, b2, w3, b3


def candidates(kind: int):
    n = ctypes.c_int()
    _abi.call("coot_launch_candidates", kind, None, 0, ctypes.byref(n))
    buf = (ctypes.c_int32 * (4 * n.value))()
    _abi.call("coot_launch_candidates", kind, buf, n.value, ctypes.byref(n))
    return [tuple(buf[4 * i:4 * i + 4]) for i in range(n.value)]


def features(tree: bytes, kind: int, dtypes, out_dtype: int, heads: int, n_rows: int, n_cols: int, dense: bool,
             block: int, vec: int, unroll: int, split: int) -> np.ndarray:
    f = (ctypes.c_float * D)()
    dts = (ctypes.c_int32 * 4)(*(list(dtypes) + [0] * (4 - len(dtypes))))
    _abi.call("coot_call_features", tree, len(tree), kind, dts, out_dtype, heads, n_rows, n_cols, int(dense), block,
              vec, unroll, split, f)
    return np.frombuffer(f, dtype=np.float32).copy()


# ---------------------------------------------------------------- the model on the GPU

class CostModel:
    """The 2-layer MLP, parameters in one FP32 device array."""

    def __init__(self, params=None, seed: int = 0):
        import torch
        if params is None:
            rng = np.random.default_rng(seed)
            p = np.zeros(n_params(), dtype=np.float32)
            o = 0
            p[o:o + D * H] = rng.standard_normal(D * H) * math.sqrt(2.0 / D); o += D * H + H
            p[o:o + H * H] = rng.standard_normal(H * H) * math.sqrt(2.0 / H); o += H * H + H
            p[o:o + H] = rng.standard_normal(H) * math.sqrt(1.0 / H); o += H
            params = p
        self.p = torch.as_tensor(np.asarray(params, dtype=np.float32)).cuda()

    def _stream(self):
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def forward(self, X):
        """Predictions for the rows of X (device tensor B x D) and the
        activations (device)."""
        import torch
        B = X.shape[0]
        y = torch.empty(B, dtype=torch.float32, device="cuda")
        act = torch.empty(2 * B * H, dtype=torch.float32, device="cuda")
        _abi.call("coot_mlp_forward", self.p.data_ptr(), D, H, X.data_ptr(), B, y.data_ptr(), act.data_ptr(),
                  self._stream())
        return y, act

    def predict(self, X: np.ndarray) -> np.ndarray:
        import torch
        Xd = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        y, _ = self.forward(Xd)
        return y.cpu().numpy()

    def fit(self, X: np.ndarray, t: np.ndarray, steps: int = 3000, lr: float = 3e-3, decay_at=(0.6, 0.85)):
        """Full-batch Adam on mean squared error, on the GPU; returns the
        loss every 100 steps."""
        import torch
        Xd = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        td = torch.as_tensor(np.ascontiguousarray(t, dtype=np.float32)).cuda()
        B = Xd.shape[0]
        n = self.p.numel()
        grad = torch.zeros(n, dtype=torch.float32, device="cuda")
        m = torch.zeros(n, dtype=torch.float32, device="cuda")
        v = torch.zeros(n, dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        work = torch.empty(B * (2 * H + 1), dtype=torch.float32, device="cuda")
        st = self._stream()
        hist = []
        for k in range(1, steps + 1):
            rate = lr * (0.3 if k > decay_at[0] * steps else 1.0) * (0.3 if k > decay_at[1] * steps else 1.0)
            y, act = self.forward(Xd)
            _abi.call("coot_mlp_loss_grad", self.p.data_ptr(), D, H, Xd.data_ptr(), td.data_ptr(), B, y.data_ptr(),
                      act.data_ptr(), grad.data_ptr(), loss.data_ptr(), work.data_ptr(), st)
            _abi.call("coot_mlp_adam", self.p.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), n, k,
                      ctypes.c_float(rate), ctypes.c_float(0.9), ctypes.c_float(0.999), ctypes.c_float(1e-8), st)
            if k % 100 == 0 or k == 1:
                hist.append((k, float(loss.item())))
        return hist

    def params(self) -> np.ndarray:
        return self.p.cpu().numpy()

    def save(self, path: str, meta: dict | None = None):
        with open(path, "w") as f:
            json.dump({"d": D, "h": H, "params": [float(x) for x in self.params()], "meta": meta or {}}, f)


def load_params(path: str = MODEL_PATH) -> np.ndarray:
    with open(path) as f:
        doc = json.load(f)
    assert doc["d"] == D and doc["h"] == H
    return np.asarray(doc["params"], dtype=np.float32)


def load_policy(path: str = MODEL_PATH) -> None:
    """Load the cost model into the library and switch to the learned
    policy."""
    p = load_params(path)
    _abi.call("coot_model_load", p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size)
    _abi.call("coot_set_policy", _abi.POLICY_LEARNED)


def use_builtin() -> None:
    _abi.call("coot_set_policy", _abi.POLICY_BUILTIN)


def host_predict(X: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    out = np.zeros(X.shape[0], dtype=np.float32)
    _abi.call("coot_model_predict", X.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), X.shape[0],
              out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return out


# ---------------------------------------------------------------- timing data

class _Call:
    """One call (tree, kind, shape, dtype) with its device buffers and
    prebuilt ctypes arguments, so that timing sees little host overhead."""

    def __init__(self, tree_sexpr, n_inputs, kind, dtype, n_rows, n_cols, seed):
        import torch

        import paper_2308_03120_gb300 as coot
        self.tree = coot.serialize(tree_sexpr, n_inputs=n_inputs)
        self.kind, self.dtype, self.n_rows, self.n_cols = kind, dtype, n_rows, n_cols
        self.n_in = n_inputs
        tdt = torch.float32 if dtype == "f32" else torch.bfloat16
        g = torch.Generator(device="cuda").manual_seed(seed)
        n = n_rows * n_cols
        self.bufs = [(0.5 + torch.rand(n, generator=g, device="cuda")).to(tdt) for _ in range(n_inputs)]
        self.mats = (_abi.coot_mat * n_inputs)(*[coot.Mat(b, n_rows, n_cols, n_rows).c() for b in self.bufs])
        self.code = DTYPES[dtype]
        self.dts = (ctypes.c_int32 * 4)(*([self.code] * n_inputs + [0] * (4 - n_inputs)))
        self.heads = 0
        self.out_dtype = -1
        if kind == KIND_MAP:
            self.out = torch.empty(n, dtype=tdt, device="cuda")
            self.out_mat = coot.Mat(self.out, n_rows, n_cols, n_rows).c()
            self.out_dtype = self.code
        elif kind == KIND_REDUCE:
            self.heads = REDUCE_HEADS
            self.res = torch.empty(2, dtype=torch.float64, device="cuda")
        elif kind == KIND_COLSUM:
            self.out = torch.empty(n_cols, dtype=torch.float32, device="cuda")
            self.out_mat = coot.Mat(self.out, 1, n_cols, 1).c()
        else:
            self.out = torch.empty(n_rows, dtype=torch.float32, device="cuda")
            self.out_mat = coot.Mat(self.out, n_rows, 1, n_rows).c()
        self.ws = coot.Workspace(n_rows if kind == KIND_ROWSUM else 1)
        self.stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        self.L = _abi.lib()

    def __call__(self):
        L, t = self.L, self.tree
        if self.kind == KIND_MAP:
            st = L.coot_expr_eval(t, len(t), self.mats, self.n_in, ctypes.byref(self.out_mat), None, 0, self.stream)
        elif self.kind == KIND_REDUCE:
            st = L.coot_expr_reduce(t, len(t), self.mats, self.n_in, self.heads, None,
                                    ctypes.c_void_p(self.res.data_ptr()), self.ws.ptr, self.ws.bytes, self.stream)
        else:
            st = L.coot_sum_dim(t, len(t), self.mats, self.n_in, 0 if self.kind == KIND_COLSUM else 1,
                                ctypes.byref(self.out_mat), self.ws.ptr, self.ws.bytes, self.stream)
        if st != 0:
            raise _abi.CootError("timed call", st, L.coot_last_error().decode())

    def features(self, block, vec, unroll, split):
        return features(self.tree, self.kind, [self.code] * self.n_in, self.out_dtype, self.heads, self.n_rows,
                        self.n_cols, True, block, vec, unroll, split)


def _time(fn, budget_us: float = 400.0) -> float:
    """Mean device time of fn in microseconds: one warm call, a two-call
    estimate, then enough calls for about budget_us of work (3..40)."""
    import torch
    fn()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    fn()
    e1.record()
    e1.synchronize()
    est = e0.elapsed_time(e1) * 1e3 / 2
    reps = int(min(40, max(3, budget_us / max(est, 1.0))))
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) * 1e3 / reps


def _shape(rng, max_log2: int, min_log2: int = 10):
    n = int(2 ** rng.uniform(min_log2, max_log2))
    r = int(2 ** (rng.uniform(0, 1) * math.log2(n)))
    if r >= 8:
        r -= r % 8  # full-width vector accesses along columns
    r = max(1, min(r, 1 << 16))
    c = max(1, n // r)
    return r, c


def generate(n_trees: int, seed: int, max_log2: int = 26, kinds_per_tree: int = 2,
             shapes_per_kind: int = 4, threads: int = 16, log=print, min_log2: int = 10):
    """Timing samples for n_trees random trees with element counts
    2^U[min_log2, max_log2]; every sample holds the per-candidate times
    (microseconds), features and the built-in time."""
    import torch

    import paper_2308_03120_gb300 as coot
    import synth
    rng = np.random.default_rng(seed)
    plans = []
    for t in range(n_trees):
        n_in = int(rng.integers(1, 5))
        n_ops = int(rng.integers(2, 13))
        sexpr = synth.random_tree(seed * 100003 + t, n_ops, n_in)
        dtype = "f32" if rng.random() < 0.6 else "bf16"
        kinds = rng.choice(KINDS, size=kinds_per_tree, replace=False)
        for k in kinds:
            for s in range(shapes_per_kind):
                plans.append((t, sexpr, n_in, int(k), dtype, _shape(rng, max_log2, min_log2)))
    # compile every (tree, kind, dtype, candidate) in parallel threads
    t0 = time.time()
    jobs = set()
    for t, sexpr, n_in, k, dtype, _ in plans:
        code = DTYPES[dtype]
        vec = 4 if dtype == "f32" else 8
        for block, _, unroll, _ in candidates(k):
            jobs.add((t, k, dtype, block, vec, unroll))
    trees = {t: (coot.serialize(sexpr, n_inputs=n_in), n_in) for t, sexpr, n_in, *_ in plans}

    def prep(job):
        t, k, dtype, block, vec, unroll = job
        tree, n_in = trees[t]
        code = DTYPES[dtype]
        dts = (ctypes.c_int32 * 4)(*([code] * n_in + [0] * (4 - n_in)))
        out_dtype = code if k == KIND_MAP else -1
        heads = REDUCE_HEADS if k == KIND_REDUCE else 0
        _abi.lib().coot_prepare(tree, len(tree), k, dts, out_dtype, heads, block, vec, unroll)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(prep, sorted(jobs)))
    log(f"compiled {len(jobs)} kernels in {time.time() - t0:.1f} s")
    t0 = time.time()
    samples = []
    for i, (t, sexpr, n_in, k, dtype, (r, c)) in enumerate(plans):
        call = _Call(sexpr, n_in, k, dtype, r, c, seed * 7919 + i)
        cands = candidates(k)
        rec = {"tree": t, "kind": k, "dtype": dtype, "n_rows": r, "n_cols": c, "n_inputs": n_in,
               "cand": cands, "us_a": [0.0] * len(cands), "us_b": [0.0] * len(cands), "X": [None] * len(cands)}
        # two independent passes (the second in reverse order): the tuner
        # picks on pass a, every choice is scored on pass b
        for pass_name, order in (("a", range(len(cands))), ("b", reversed(range(len(cands))))):
            for j in order:
                block, vec, unroll, split = cands[j]
                coot.coot_set_launch_config(k, block, vec, unroll, 0, split)
                rec["us_" + pass_name][j] = _time(call)
                if rec["X"][j] is None:
                    last = coot.coot_last_launch()
                    rec["X"][j] = call.features(last["block"], last["vec"], last["unroll"], split)
            coot.coot_set_launch_config(k, 0)
            rec["builtin_" + pass_name] = _time(call)
        rec["us"] = [(a + b) / 2 for a, b in zip(rec["us_a"], rec["us_b"])]
        rec["builtin_us"] = (rec["builtin_a"] + rec["builtin_b"]) / 2
        samples.append(rec)
        del call
        if (i + 1) % 200 == 0:
            torch.cuda.synchronize()
            log(f"timed {i + 1}/{len(plans)} samples ({time.time() - t0:.1f} s)")
    return samples


def merge_sample_sets(first, second, n_first: int):
    """The samples of two generate() calls as one set: the second call's
    tree ids are shifted past the first call's n_first trees, so that
    split_by_tree keeps every tree whole on one side."""
    for smp in second:
        smp["tree"] += n_first
    return first + second


def split_by_tree(samples, held_out_frac: float = 0.2, seed: int = 0):
    trees = sorted({s["tree"] for s in samples})
    rng = np.random.default_rng(seed)
    held = set(rng.choice(trees, size=max(1, int(len(trees) * held_out_frac)), replace=False).tolist())
    return [s for s in samples if s["tree"] not in held], [s for s in samples if s["tree"] in held]


def design(samples):
    """Rows (features, target): the target is log(t / t_builtin) of the same
    call, so the model learns how each shape compares within a call (what
    choosing needs) rather than absolute times spanning decades."""
    X = np.concatenate([np.stack(s["X"]) for s in samples]).astype(np.float32)
    y = np.concatenate([np.log(np.maximum(np.asarray(s["us"]), 1e-3) / max(s["builtin_us"], 1e-3))
                        for s in samples]).astype(np.float32)
    return X, y


def regret(samples, predict) -> dict:
    """Regret against the exhaustive tuner: the tuner takes the fastest
    candidate of pass a; the model's choice, the built-in shape and the
    tuner's choice are all scored on pass b (independent timings, so the
    tuner's pick is not flattered by its own noise).  Geometric means."""
    rm, rb = [], []
    for s in samples:
        a, b = np.asarray(s["us_a"]), np.asarray(s["us_b"])
        tuner = b[int(np.argmin(a))]
        pred = predict(np.stack(s["X"]))
        rm.append(b[int(np.argmin(pred))] / tuner)
        rb.append(s["builtin_b"] / tuner)
    rm, rb = np.asarray(rm), np.asarray(rb)
    return {"samples": len(samples), "model_geomean": float(np.exp(np.mean(np.log(rm)))),
            "builtin_geomean": float(np.exp(np.mean(np.log(rb)))), "model_within_5pct": float(np.mean(rm <= 1.05)),
            "builtin_within_5pct": float(np.mean(rb <= 1.05)), "model_worst": float(rm.max()),
            "builtin_worst": float(rb.max())}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--trees", type=int, default=400)
    ap.add_argument("--seed", type=int, default=20230806)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--max-log2", type=int, default=26)
    ap.add_argument("--large-trees", type=int, default=0,
                    help="further trees timed on calls of 2^26 to 2^30 elements")
    ap.add_argument("--large-seed", type=int, default=20231127)
    ap.add_argument("--out", default=None, help="report JSON path")
    ap.add_argument("--model", default=MODEL_PATH)
    ap.add_argument("--data", default=None, help="save the timing samples here (pickle)")
    ap.add_argument("--from-data", default=None, help="train on saved samples instead of measuring")
    args = ap.parse_args(argv)
    import torch

    import paper_2308_03120_gb300 as coot
    from paper_2308_03120_gb300 import build
    build.build()
    coot.coot_init(0)
    t0 = time.time()
    if args.from_data:
        with open(args.from_data, "rb") as f:
            samples = pickle.load(f)
    else:
        samples = generate(args.trees, args.seed, max_log2=args.max_log2)
        if args.large_trees > 0:
            large = generate(args.large_trees, args.large_seed, min_log2=26, max_log2=30)
            samples = merge_sample_sets(samples, large, args.trees)
    if args.data:
        with open(args.data, "wb") as f:
            pickle.dump(samples, f)
    train, held = split_by_tree(samples)
    X, y = design(train)
    model = CostModel(seed=1)
    hist = model.fit(X, y, steps=args.steps)
    train_rmse = float(np.sqrt(np.mean((model.predict(X) - y) ** 2)))
    Xh, yh = design(held)
    held_rmse = float(np.sqrt(np.mean((model.predict(Xh) - yh) ** 2)))
    model.save(args.model, meta={"trees": args.trees, "large_trees": args.large_trees,
                                 "train_rows": int(X.shape[0]), "held_rows": int(Xh.shape[0]),
                                 "seed": args.seed, "train_rmse_log": train_rmse, "held_rmse_log": held_rmse})
    _abi.call("coot_model_load", model.params().ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n_params())
    report = {"trees": args.trees, "samples": len(samples), "train_rows": int(X.shape[0]),
              "held_rows": int(Xh.shape[0]), "loss_history": hist, "train_rmse_log": train_rmse,
              "held_rmse_log": held_rmse, "held_out": regret(held, host_predict), "train": regret(train, host_predict),
              "seconds": round(time.time() - t0, 1)}
    print(json.dumps({k: v for k, v in report.items() if k != "loss_history"}))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(report, f)
    torch.cuda.synchronize()
    return report


if __name__ == "__main__":
    main()
