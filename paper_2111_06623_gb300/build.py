"""In-tree build of libll.so for sm_103a: three translation units compiled in parallel with
nvcc, then linked into one shared library (CUDA runtime linked statically)."""
from __future__ import annotations

import hashlib
import os
import platform
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB_PATH = os.path.join(HERE, "libll.so")
# the bounds-checked variant (-DLL_CHECK): every table-driven index tested before its access
CHECK_LIB_PATH = os.path.join(HERE, "libll_check.so")
UNITS = ("ll_api", "ll_f64", "ll_f32", "ll_server")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def source_hash(extra_flags: list[str] | None = None) -> str:
    """sha256 over every source the library is built from, the flags and the nvcc version."""
    h = hashlib.sha256()
    files = sorted(f for f in os.listdir(SRC) if f.endswith((".cu", ".cuh")))
    for p in [os.path.join(SRC, f) for f in files] + [os.path.join(ROOT, "include", "ll.h")]:
        h.update(os.path.basename(p).encode() + b"\0")
        with open(p, "rb") as fh:
            h.update(fh.read())
    h.update("\0".join(ARCH + FLAGS + list(extra_flags or []) + [platform.machine()]).encode())
    r = subprocess.run([_nvcc(), "--version"], capture_output=True, text=True)
    h.update(r.stdout.encode())
    return h.hexdigest()


def build_library(force: bool = False, extra_flags: list[str] | None = None, check: bool = False) -> str:
    """Build libll.so unless the one in the tree was built from exactly these sources, flags
    and compiler (a content hash kept beside it, not file times); force=True always builds.
    check=True: the bounds-checked variant libll_check.so (-DLL_CHECK), objects apart."""
    extra_flags = list(extra_flags or []) + (["-DLL_CHECK"] if check else [])
    lib_path = CHECK_LIB_PATH if check else LIB_PATH
    build_dir = os.path.join(BUILD, "check") if check else BUILD
    digest = source_hash(extra_flags)
    stamp = lib_path + ".sha256"
    if not force and os.path.exists(lib_path) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return lib_path
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    flags = FLAGS + extra_flags

    def compile_one(u):
        obj = os.path.join(build_dir, u + ".o")
        cmd = [nvcc, *ARCH, *flags, "-c", os.path.join(SRC, u + ".cu"), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {u}:\n{r.stderr[-4000:]}")
        return obj

    with ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = lib_path + f".{os.getpid()}.tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, lib_path)
    with open(stamp + f".{os.getpid()}.tmp", "w") as fh:
        fh.write(digest + "\n")
    os.replace(stamp + f".{os.getpid()}.tmp", stamp)
    return lib_path
