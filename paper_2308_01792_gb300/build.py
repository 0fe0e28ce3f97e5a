"""Build the C-ABI shared library ``lib/libhytet.so`` for sm_103a.

Every ``csrc/*.cu`` and ``csrc/*.cpp`` is compiled by nvcc in parallel
(``-gencode arch=compute_103a,code=sm_103a``) and linked into one shared
library that exports the functions declared in ``include/hytet.h``.
Objects are rebuilt when a source or header is newer than its object.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "lib")
INC = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(OUT, "libhytet.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError(f"nvcc not found (looked at {cand})")
    return cand


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
                   "-I" + INC, "-I" + SRC, *extra]


def build(verbose: bool = False, extra_flags=()) -> str:
    nvcc = _nvcc()
    os.makedirs(os.path.join(OUT, "obj"), exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(SRC, "*.cu")) + glob.glob(os.path.join(SRC, "*.cpp")))
    headers = glob.glob(os.path.join(SRC, "*.h")) + glob.glob(os.path.join(SRC, "*.cuh")) + \
        glob.glob(os.path.join(INC, "*.h"))
    newest_hdr = max((os.path.getmtime(h) for h in headers), default=0.0)

    def compile_one(src):
        obj = os.path.join(OUT, "obj", os.path.basename(src) + ".o")
        if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), newest_hdr) \
                and not extra_flags:
            return obj, None
        cmd = [nvcc, *_flags(extra_flags), "-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd.insert(1, "-x")
            cmd.insert(2, "c++")
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            return obj, f"{' '.join(cmd)}\n{p.stdout}\n{p.stderr}"
        if verbose and p.stderr.strip():
            print(p.stderr, file=sys.stderr)
        return obj, None

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, srcs))
    errs = [e for _, e in results if e]
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    objs = [o for o, _ in results]
    cmd = [nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *objs, "-lcudart"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
