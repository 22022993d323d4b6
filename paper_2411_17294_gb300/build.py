"""Build libtfs.so (the C-ABI library) for sm_103a with nvcc.

Each translation unit under csrc/ is compiled in parallel to an object file
and the objects are linked into ``_build/libtfs.so`` next to this file.  The
CUDA runtime is linked statically, so the library depends only on the driver.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libtfs.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["tfs_api.cu", "tfs_forward.cu", "tfs_adjoint.cu", "tfs_util.cu", "tfs_static.cu", "tfs_implicit.cu",
           "tfs_start.cu", "tfs_selftest.cu", "tfs_adjoint_paper.cu", "tfs_ns.cu"]


def nvcc() -> str:
    path = shutil.which("nvcc")
    if path:
        return path
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtfs.so")


def _flags(verbose: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                "-I", os.path.join(HERE, "..", "include")]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "tfs.h"))
    objs, todo = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(o)
        if force or verbose or _stale(o, [s] + headers):
            todo.append((s, o))
    exe = nvcc()

    def compile_one(item):
        s, o = item
        cmd = [exe] + _flags(verbose) + ["-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(s)}:\n{r.stderr}")
        return r.stderr

    logs = []
    if todo:
        with concurrent.futures.ThreadPoolExecutor(max_workers=jobs or len(todo)) as ex:
            logs = list(ex.map(compile_one, todo))
    if verbose:
        for lg in logs:
            sys.stderr.write(lg)
    if force or todo or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [exe] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":   # pragma: no cover
    v = "-v" in sys.argv
    print(build(force="-f" in sys.argv or v, verbose=v))
