"""Build the in-tree shared library libt2s2.so for sm_103a.

Compiles every translation unit of csrc/ in parallel with nvcc (one
-gencode, -lineinfo), the host C++ part with g++, and links with nvcc.
Run as ``python -m paper_2506_04732_gb300.build`` or through
``__graft_entry__.build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libt2s2.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _stale(obj, src_paths):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in src_paths)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    cu, cpp = _sources()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "t2s2.h"))
    jobs = []
    for f in cu:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", "-c", src, "-o", obj]
        jobs.append((obj, [src] + headers, cmd))
    for f in cpp:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        cmd = ["g++", "-O2", "-fPIC", "-std=c++17", "-c", src, "-o", obj]
        jobs.append((obj, [src] + headers, cmd))
    todo = [j for j in jobs if force or _stale(j[0], j[1])]

    def run(job):
        obj, _, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return obj, r

    errors = []
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 4))) as ex:
        for obj, r in ex.map(run, todo):
            if r.returncode != 0:
                errors.append(f"{obj}:\n{r.stderr}")
            elif verbose and r.stderr.strip():
                print(r.stderr, file=sys.stderr)
    if errors:
        raise RuntimeError("build failed:\n" + "\n".join(errors))
    objs = [j[0] for j in jobs]
    if force or todo or not os.path.exists(LIB) or _stale(LIB, objs):
        cmd = [nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
