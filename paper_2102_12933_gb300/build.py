"""Build libfdu.so in-tree: host preprocessing (g++) + sm_103a kernels (nvcc).

Usage: ``python -m paper_2102_12933_gb300.build [--force] [--verbose]``.
The translation units compile in parallel; the result is
``paper_2102_12933_gb300/_build/libfdu.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libfdu.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

HOST_SRC = ["fdu_host.cpp"]
CUDA_SRC = ["fdu_kernels.cu", "fdu_api.cu", "fdu_adjoint.cu", "fdu_dw.cu", "fdu_adjoint_dw.cu"]
HEADERS = ["fdu_internal.h", "fdu_kernels.cuh", "fdu_device.cuh", "fdu_adjoint.cuh", "fdu_dw.cuh", "fdu_dw_euler.cuh", "fdu_dw_edge.cuh"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in HOST_SRC + CUDA_SRC + HEADERS] + [os.path.join(INCLUDE, "fdu.h")]
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    inc = [f"-I{INCLUDE}", f"-I{CSRC}"]
    jobs = []
    objs = []
    for f in HOST_SRC:
        o = os.path.join(OUT_DIR, f + ".o")
        objs.append(o)
        jobs.append(["g++", "-std=c++17", "-O3", "-ffp-contract=off", "-fPIC", "-pthread", *inc, "-c",
                     os.path.join(CSRC, f), "-o", o])
    for f in CUDA_SRC:
        o = os.path.join(OUT_DIR, f + ".o")
        objs.append(o)
        cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *inc, "-c",
               os.path.join(CSRC, f), "-o", o]
        if verbose:
            cmd.insert(2, "-Xptxas=-v")
        jobs.append(cmd)
    procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for j in jobs]
    failed = []
    for j, p in zip(jobs, procs):
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out)
        if p.returncode != 0:
            failed.append((j, out))
    if failed:
        msg = "\n".join(" ".join(j) + "\n" + out for j, out in failed)
        raise RuntimeError("libfdu build failed:\n" + msg)
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("libfdu link failed:\n" + " ".join(link) + "\n" + r.stdout)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
