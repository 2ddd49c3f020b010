"""Build libbeamtrack.so (the CUDA kernels and the C ABI) in-tree for sm_103a.

`python -m paper_2208_02382_b300.build` or build().  Needs nvcc only (no GPU).
Each translation unit is compiled to an object file in parallel (under
`_build/`, rebuilt only when it or a header changed), then linked.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libbeamtrack.so")
OBJ_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
          "-diag-suppress", "177"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def _headers():
    return glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + \
        [os.path.join(ROOT, "include", "beamtrack.h")]


def _obj(src: str) -> str:
    return os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + ".o")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(nvcc: str, src: str, verbose: bool) -> str:
    out = _obj(src)
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc, *CFLAGS, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", tmp]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    srcs = sources()
    hdrs = _headers()
    objs = [_obj(s) for s in srcs]
    if not force and not _stale(LIB, srcs + hdrs):
        return LIB
    os.makedirs(OBJ_DIR, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")
    todo = [s for s in srcs if force or _stale(_obj(s), [s] + hdrs)]
    if todo:
        workers = max(1, min(len(todo), os.cpu_count() or 1))
        with cf.ThreadPoolExecutor(workers) as ex:
            for f in [ex.submit(_compile, nvcc, s, verbose) for s in todo]:
                f.result()
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "--shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
