"""Builds libcoot.so in the package directory.

The library holds the host code of the C ABI (include/coot.h), the device
runtime of the fused kernels as an embedded string (compiled per tree at
run time by NVRTC for the device, sm_103a on GB300), and the ahead-of-time
kernels compiled here with nvcc for sm_103a.  Translation units are compiled
in parallel; only the CUDA toolkit, g++ and the Python standard library are
needed.

    python -m paper_2308_03120_gb300.build          # or build() from Python
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libcoot.so")

ARCH = "-gencode=arch=compute_103a,code=sm_103a"
HOST_SOURCES = ["coot_api.cpp", "coot_tree.cpp", "coot_jit.cpp", "coot_policy.cpp", "coot_canon.cpp"]
CUDA_SOURCES = ["coot_aot.cu", "coot_static.cu", "coot_mlp.cu"]


def cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if cand and os.path.isdir(cand):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    raise RuntimeError("CUDA toolkit not found (set CUDA_HOME)")


JIT_SOURCES = ["jit_rt.cuh", "jit_map.cuh", "jit_colsum.cuh", "jit_rowsum.cuh", "jit_batched.cuh", "jit_stats.cuh",
               "jit_multi.cuh", "jit_dims.cuh"]


def _embed_runtime() -> str:
    """The device runtime (jit_rt.cuh and the per-kernel files, in order) as
    one C string in a generated translation unit."""
    src = "".join(open(os.path.join(CSRC, f), encoding="utf-8").read() + "\n" for f in JIT_SOURCES)
    out = os.path.join(BUILD, "jit_rt_embed.cpp")
    body = ['// generated from jit_rt.cuh by build.py\nextern "C" const char* coot_jit_rt_source =\n']
    # raw string pieces well below compiler limits on literal length
    step = 8000
    for i in range(0, len(src), step):
        body.append('R"COOTRT(' + src[i:i + step] + ')COOTRT"\n')
    body.append(";\n")
    text = "".join(body)
    if not os.path.exists(out) or open(out).read() != text:
        with open(out, "w") as f:
            f.write(text)
    return out


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + p.stdout)
    return p.stdout


def _stamp(paths, extra: str) -> str:
    h = hashlib.sha256(extra.encode())
    for p in sorted(paths):
        with open(p, "rb") as f:
            h.update(p.encode())
            h.update(f.read())
    return h.hexdigest()


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile libcoot.so if any source changed; returns its path."""
    cuda = cuda_home()
    os.makedirs(BUILD, exist_ok=True)
    embed = _embed_runtime()
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "coot.h"), __file__]
    stamp = _stamp([d for d in deps if os.path.isfile(d)], cuda + sys.platform + os.uname().machine)
    stamp_file = os.path.join(BUILD, "stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file) and open(stamp_file).read() == stamp:
        return LIB
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = ["-I" + INCLUDE, "-I" + CSRC, "-I" + os.path.join(cuda, "include")]
    jobs = []
    for f in HOST_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append((["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-Wall", "-Wno-unused-function", *inc, "-c",
                      os.path.join(CSRC, f), "-o", obj], obj))
    obj = os.path.join(BUILD, "jit_rt_embed.o")
    jobs.append((["g++", "-std=c++17", "-O0", "-fPIC", "-c", embed, "-o", obj], obj))
    for f in CUDA_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append(([nvcc, ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
                      *inc, "-c", os.path.join(CSRC, f), "-o", obj], obj))
    logs = []
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        for out in ex.map(lambda j: _run(j[0]), jobs):
            logs.append(out)
    objs = [j[1] for j in jobs]
    tmp = LIB + ".tmp"
    _run([nvcc, ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static",
          "-L" + os.path.join(cuda, "lib64"), "-lnvrtc", "-ldl", "-lpthread", "-lrt",
          "-Xlinker", "-rpath=" + os.path.join(cuda, "lib64")])
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        f.write("\n".join(logs))
    if verbose:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
