"""Build ``libcho.so`` in-tree with nvcc for sm_103a.

Every translation unit under ``csrc/`` is compiled in parallel into
``_build/obj`` and linked into ``_build/libcho.so``.  ``-Xptxas -v`` output
(registers, spills, shared memory per kernel) is kept in ``_build/ptxas.log``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libcho.so")
ROOT = os.path.dirname(HERE)

SOURCES = [
    "api.cpp",
    "linalg.cpp",
    "serve.cpp",
    "tune.cpp",
    "rk4_small.cu",
    "rk4_chain.cu",
    "rk4_chain_ext.cu",
    "rk4_dense.cu",
    "rk4_dense_tc.cu",
    "energy.cu",
    "plain.cu",
    "plain_noalloc.cu",
    "serve_kernels.cu",
    "peaks.cu",
    "packed.cu",
]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(src: str) -> list[str]:
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if src.endswith(".cu"):
        return ARCH + ["-lineinfo", "--expt-relaxed-constexpr", "-Xptxas", "-v"] + common
    return common + ["-x", "c++"]


def _deps_mtime() -> float:
    m = 0.0
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            m = max(m, os.path.getmtime(os.path.join(d, f)))
    return max(m, os.path.getmtime(__file__))


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile and link the library; returns the path of ``libcho.so``."""
    os.makedirs(os.path.join(OUT, "obj"), exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(OUT, "obj", src + ".o")
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(src)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(compile_one, SOURCES))
    with open(os.path.join(OUT, "ptxas.log"), "w") as f:
        for (obj, log), src in zip(results, SOURCES):
            f.write(f"==== {src}\n{log}\n")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", "-o", tmp] + [o for o, _ in results] + ARCH + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
