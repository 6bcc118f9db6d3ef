"""Builds oracle/libcpu_fp32.so, the all-cores FP32 CPU evaluator of the
benchmark's CPU baseline (cpu_fp32.c), with gcc and OpenMP; and loads it.
Test and benchmark infrastructure only, like the rest of this directory."""
from __future__ import annotations

import ctypes
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_fp32.c")
LIB = os.path.join(HERE, "libcpu_fp32.so")


def build() -> str:
    """Compile the evaluator if its source is newer than the library (with
    OpenMP; without it, on one core, where the compiler has no OpenMP
    runtime -- cpu_fp32_threads() then reports 1)."""
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp"
    base = ["gcc", "-std=c11", "-O3", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:4] + ["-fopenmp"] + base[4:], stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        subprocess.run(base, check=True, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    os.replace(tmp, LIB)
    return LIB


def load() -> ctypes.CDLL:
    lib = ctypes.CDLL(build())
    f = lib.cpu_fp32_eval
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int64,
                  ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_int]
    lib.cpu_fp32_threads.restype = ctypes.c_int
    return lib
