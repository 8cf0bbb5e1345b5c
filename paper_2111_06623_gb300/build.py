"""In-tree build of libll.so for sm_103a: three translation units compiled in parallel with
nvcc, then linked into one shared library (CUDA runtime linked statically)."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB_PATH = os.path.join(HERE, "libll.so")
UNITS = ("ll_api", "ll_f64", "ll_f32", "ll_server")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def build_library(force: bool = False, extra_flags: list[str] | None = None) -> str:
    srcs = [os.path.join(SRC, u + ".cu") for u in UNITS]
    deps = srcs + [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".cuh")] + \
        [os.path.join(ROOT, "include", "ll.h")]
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(p) for p in deps)):
        return LIB_PATH
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    flags = FLAGS + (extra_flags or [])

    def compile_one(u):
        obj = os.path.join(BUILD, u + ".o")
        cmd = [nvcc, *ARCH, *flags, "-c", os.path.join(SRC, u + ".cu"), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {u}:\n{r.stderr[-4000:]}")
        return obj

    with ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH
