"""Builds the in-tree shared library libras.so for sm_103a.

Two translation units: csrc/ras_kernels.cu (nvcc, -gencode compute_103a /
sm_103a) and csrc/ras_api.cpp (the host compiler, -ffp-contract=off so the
partitioner's floating-point expressions round identically on every host),
compiled in parallel and linked by nvcc into _build/libras.so.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libras.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _sources():
    srcs = [os.path.join(CSRC, f) for f in ("ras_kernels.cu", "ras_api.cpp", "ras_noalloc.cu")]
    deps = srcs + [os.path.join(CSRC, f) for f in ("ras_internal.h", "ras_launch.h", "ras_convert.h")]
    deps.append(os.path.join(ROOT, "include", "ras.h"))
    return srcs, deps


def is_stale() -> bool:
    _, deps = _sources()
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not is_stale():
        return LIB
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(OUT, exist_ok=True)
    srcs, _ = _sources()
    tag = f".{os.getpid()}"
    obj_cu = os.path.join(OUT, f"ras_kernels{tag}.o")
    obj_cpp = os.path.join(OUT, f"ras_api{tag}.o")
    obj_na = os.path.join(OUT, f"ras_noalloc{tag}.o")
    cmds = [
        [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c", srcs[0],
         "-o", obj_cu],
        ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-pthread",
         f"-I{os.path.join(cuda, 'include')}", "-c", srcs[1], "-o", obj_cpp],
        [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c", srcs[2],
         "-o", obj_na],
    ]

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r

    with ThreadPoolExecutor(3) as ex:
        list(ex.map(run, cmds))
    tmp = os.path.join(OUT, f"libras{tag}.so")
    run([nvcc, *ARCH, "-shared", "-o", tmp, obj_cu, obj_cpp, obj_na, "-lpthread"])
    os.replace(tmp, LIB)
    for o in (obj_cu, obj_cpp, obj_na):
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
