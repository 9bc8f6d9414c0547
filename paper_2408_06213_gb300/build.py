"""Build libbrr (the CUDA library) for sm_103a, in-tree.

Each .cu translation unit is compiled by its own nvcc process (in parallel),
then linked into ``_build/libbrr.so`` with the CUDA runtime linked
statically.  Also builds the small C helper of the input generators.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libbrr.so")
INPUTS_SRC = os.path.join(HERE, "inputs_group.c")
INPUTS_LIB = os.path.join(OUT, "libbrr_inputs.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]
SOURCES = ["api.cu", "dice.cu", "shuffle.cu", "batched.cu", "chains.cu", "windows.cu", "noalloc.cu", "calib.cu"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the brr CUDA library cannot be built")
    return p


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _deps() -> list[str]:
    ds = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    ds.append(os.path.join(ROOT, "include", "brr.h"))
    return ds


def build_inputs_helper(force: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    if force or _stale(INPUTS_LIB, [INPUTS_SRC]):
        tmp = INPUTS_LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", INPUTS_SRC, "-o", tmp], check=True)
        os.replace(tmp, INPUTS_LIB)
    return INPUTS_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit for sm_103a and link libbrr.so."""
    os.makedirs(OUT, exist_ok=True)
    build_inputs_helper(force)
    deps = _deps()
    if not force and not _stale(LIB, deps):
        return LIB
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if verbose else []

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
