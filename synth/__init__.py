"""Seeded synthetic inputs shared by the oracle-side tests and the GPU path.

This module holds no arithmetic of the method: it draws random numbers,
stores them in the storage types the expressions read (FP32, BF16 bits,
FP16), lays them out column-major, and describes the expression trees of
the workloads as plain nested tuples.  Both the FP64 oracle and the CUDA
path receive exactly the bits produced here.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated as a counter-based
generator: output i of stream s is mix(s + (i + 1) * golden_gamma).  Because
the value of element i does not depend on how many elements were drawn
before it, generation can be chunked without changing the data, and the
result is identical on every platform.

Workloads (the paper's Task 1 and Task 2 draw `randu` vectors of swept size;
Section 5):
  * vectors: FP32, n = 1,000,000, uniform [-1, 1];
  * matrices: FP32 column-major 8192 x 8192, A, B, C uniform [-1, 1],
    D uniform [0, 2];
  * precision: n = 2^28 stored as BF16 and FP16, magnitudes lognormal
    (mu = 0, sigma = 2) with random signs, FP16 draws that do not round to
    a finite FP16 are redrawn;
  * batching: 4096 matrices with rows and cols floor(exp(U[0, ln 513)))
    clamped to [1, 512];
  * launch-config learning: random expression DAGs of 2-12 operators over
    1-4 inputs on shapes whose element count is log-uniform.

Expression trees are nested tuples ("sexpr"):
  ("x", k)            input slot k (0..3)
  ("c", value)        scalar constant (Python float)
  (op, a)             op in {"neg", "abs", "exp", "log", "sqrt", "square"}
  (op, a, b)          op in {"add", "sub", "mul", "div"}; "mul" is the
                      element-wise (Schur) product written A % B in the
                      paper's Table 2.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

BASE_SEED = 20230806

UNARY_OPS = ("neg", "abs", "exp", "log", "sqrt", "square")
BINARY_OPS = ("add", "sub", "mul", "div")


def stream_seed(seed: int, stream: int) -> int:
    """Seed of an independent sub-stream (SplitMix64 of the pair)."""
    z = (seed * 0x9E3779B97F4A7C15 + stream * 0xD1B54A32D192ED03 + 0x632BE59BD9B4E019) & ((1 << 64) - 1)
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & ((1 << 64) - 1)
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & ((1 << 64) - 1)
    return z ^ (z >> 31)


def splitmix64(seed: int, start: int, n: int) -> np.ndarray:
    """Outputs start .. start+n-1 of the SplitMix64 stream `seed` (uint64)."""
    i = np.arange(start, start + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (i + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _chunked(n: int, fill) -> None:
    """Run fill(start, count) over chunks of [0, n), in threads (numpy
    releases the GIL).  Element values depend only on their index, so the
    split does not change the result."""
    starts = list(range(0, n, _CHUNK))
    if len(starts) <= 1:
        for s in starts:
            fill(s, min(_CHUNK, n - s))
        return
    workers = max(1, min(16, os.cpu_count() or 1, len(starts)))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(lambda s: fill(s, min(_CHUNK, n - s)), starts))


def uniform01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """FP64 uniforms in [0, 1) with 53 random bits."""
    out = np.empty(n, dtype=np.float64)

    def fill(s, m):
        z = splitmix64(seed, start + s, m)
        out[s:s + m] = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    _chunked(n, fill)
    return out


def uniform_f32(seed: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """FP32 values lo + (hi - lo) * U, rounded to nearest FP32."""
    out = np.empty(n, dtype=np.float32)

    def fill(s, m):
        z = splitmix64(seed, s, m)
        u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        out[s:s + m] = (lo + (hi - lo) * u).astype(np.float32)
    _chunked(n, fill)
    return out


def normal_f64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller from two independent uniform streams.

    Uses libm log/cos, so the last bits may differ between platforms; no
    stored expected value depends on these draws.
    """
    z1 = splitmix64(stream_seed(seed, 1), start, n)
    z2 = splitmix64(stream_seed(seed, 2), start, n)
    u1 = (z1 >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def _f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round FP32 to BF16 (nearest, ties to even) and return the uint16 bits."""
    b = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = (b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)
    return r.astype(np.uint16)


def lognormal_signed(seed: int, n: int, storage: str, sigma: float = 2.0) -> tuple[np.ndarray, int]:
    """Signed lognormal(0, sigma) draws in a storage type.

    storage: "bf16" -> uint16 BF16 bit patterns; "f16" -> np.float16;
    "f32" -> np.float32.  Returns (array, number of FP16 redraws).
    """
    out = np.empty(n, dtype={"bf16": np.uint16, "f16": np.float16, "f32": np.float32}[storage])
    redraws = []
    sign_seed = stream_seed(seed, 3)

    def fill(s, m):
        mag = np.exp(sigma * normal_f64(seed, m, start=s))
        sgn = np.where((splitmix64(sign_seed, s, m) >> np.uint64(63)) == 1, -1.0, 1.0)
        v = sgn * mag
        if storage == "f16":
            with np.errstate(over="ignore"):
                bad = ~np.isfinite(v.astype(np.float16))
            attempt = 0
            while bad.any():
                attempt += 1
                idx = np.nonzero(bad)[0]
                redraws.append(idx.size)
                rs = stream_seed(seed, 100 + attempt)
                z = normal_f64(rs, m, start=s)[idx]
                v[idx] = sgn[idx] * np.exp(sigma * z)
                with np.errstate(over="ignore"):
                    bad = ~np.isfinite(v.astype(np.float16))
            out[s:s + m] = v.astype(np.float16)
        elif storage == "bf16":
            out[s:s + m] = _f32_to_bf16_bits(v.astype(np.float32))
        else:
            out[s:s + m] = v.astype(np.float32)
    _chunked(n, fill)
    return out, int(sum(redraws))


def loguniform_int(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """floor(exp(U[ln lo, ln(hi + 1)))) clamped to [lo, hi] (int64)."""
    u = uniform01(seed, n)
    v = np.floor(np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))).astype(np.int64)
    return np.clip(v, lo, hi)


# ----------------------------------------------------------------------------
# Column-major matrices
# ----------------------------------------------------------------------------

@dataclass
class HostMat:
    """A column-major matrix as the C ABI sees it: element (i, j) is
    buf[i + j * ld]; `dtype` is one of "f32", "bf16" (uint16 bits), "f16",
    "f64"."""
    buf: np.ndarray
    dtype: str
    n_rows: int
    n_cols: int
    ld: int

    @property
    def n_elem(self) -> int:
        return self.n_rows * self.n_cols


def as_mat(flat: np.ndarray, dtype: str, n_rows: int, n_cols: int, ld: int | None = None,
           pad_value=None) -> HostMat:
    """Lay a flat column-major array out with leading dimension ld >= n_rows.
    Padding rows (ld > n_rows) hold `pad_value` (NaN by default for float
    types) so that any read of them shows up in a result."""
    ld = max(n_rows, 1) if ld is None else ld
    assert ld >= max(n_rows, 1)
    if ld == n_rows or (n_cols <= 1 and n_rows > 0):
        return HostMat(np.ascontiguousarray(flat), dtype, n_rows, n_cols, ld)
    buf = np.empty(max(ld * n_cols, 0), dtype=flat.dtype)
    if pad_value is None:
        pad_value = 0x7FC0 if dtype == "bf16" else np.nan
    buf[:] = pad_value
    for j in range(n_cols):
        buf[j * ld:j * ld + n_rows] = flat[j * n_rows:(j + 1) * n_rows]
    return HostMat(buf, dtype, n_rows, n_cols, ld)


# ----------------------------------------------------------------------------
# Workload trees (nested tuples)
# ----------------------------------------------------------------------------

def X(k: int):
    return ("x", k)


def C(v: float):
    return ("c", float(v))


# Task 2 axpy shape generalised: y = 2x + 3z
AXPY_2X_3Z = ("add", ("mul", C(2.0), X(0)), ("mul", C(3.0), X(1)))
# Schur product feeding accu / dot
SCHUR_XZ = ("mul", X(0), X(1))
LEAF0 = X(0)
# Matrix workload: out = (A % B + 2*C) / (1 + abs(D))
_ABC = ("add", ("mul", X(0), X(1)), ("mul", C(2.0), X(2)))
_DEN = ("add", C(1.0), ("abs", X(3)))
MAT_EXPR = ("div", _ABC, _DEN)
# exp/sqrt chain variant: exp(-abs(A % B + 2*C)) / sqrt(1 + abs(D))
MAT_CHAIN = ("div", ("exp", ("neg", ("abs", _ABC))), ("sqrt", _DEN))
# Batched workload: exp(-abs(A)) % B + 0.5*C
BATCH_EXPR = ("add", ("mul", ("exp", ("neg", ("abs", X(0)))), X(1)), ("mul", C(0.5), X(2)))


def tree_inputs(t) -> int:
    """Number of input slots a tree refers to (max slot + 1)."""
    if t[0] == "x":
        return t[1] + 1
    if t[0] == "c":
        return 0
    return max(tree_inputs(c) for c in t[1:])


def tree_ops(t) -> int:
    if t[0] in ("x", "c"):
        return 0
    return 1 + sum(tree_ops(c) for c in t[1:])


# ----------------------------------------------------------------------------
# Random expression DAGs
# ----------------------------------------------------------------------------

_RAND_OPS = ("add", "sub", "mul", "div", "scal", "exp", "log", "sqrt", "abs")


def random_tree(seed: int, n_ops: int, n_inputs: int):
    """A random expression DAG over input slots 0..n_inputs-1 built from
    n_ops operators drawn from {+, -, %, /, scalar*, exp, log, sqrt, abs};
    if more than one subtree is left at the end they are joined with "+"
    (so the operator count can exceed n_ops by n_inputs - 1).  An operand
    stays available after use with probability 1/8, which makes shared
    subtrees (a DAG rather than a tree)."""
    u = iter(uniform01(seed, 16 * n_ops + 16 * n_inputs + 64).tolist())
    live = [X(k) for k in range(n_inputs)]

    def take():
        i = int(next(u) * len(live))
        node = live[i]
        if len(live) > 1 and next(u) >= 0.125:
            live.pop(i)
        return node

    for _ in range(n_ops):
        op = _RAND_OPS[int(next(u) * len(_RAND_OPS))]
        if op == "scal":
            k = round(-3.0 + 6.0 * next(u), 2)
            node = ("mul", C(k if k != 0.0 else 0.5), take())
        elif op == "exp":
            # a bounded argument keeps most values inside the FP32 range
            node = ("exp", ("mul", C(0.25), take()))
        elif op in ("log", "sqrt", "abs"):
            node = (op, take())
        else:
            a = take()
            b = take()
            node = (op, a, b)
        live.append(node)
    while len(live) > 1:
        b = live.pop()
        a = live.pop()
        live.append(("add", a, b))
    return live[0]


def random_shape(seed: int, max_elems: int = 32768 * 32768) -> tuple[int, int]:
    """(n_rows, n_cols) with element count log-uniform in [1, max_elems] and
    aspect ratio log-uniform."""
    u = uniform01(seed, 2)
    n = int(math.exp(u[0] * math.log(max_elems)))
    n = max(1, min(n, max_elems))
    log_r = u[1] * math.log(n) if n > 1 else 0.0
    r = max(1, int(round(math.exp(log_r))))
    r = min(r, 32768)
    c = max(1, min(32768, n // r))
    return r, c
