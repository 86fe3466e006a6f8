"""Builds the CUDA library (libkp.so) in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked with the static
CUDA runtime into paper_0910_2004_gb300/_build/libkp.so.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libkp.so")
SOURCES = ["capi.cu", "coarsen.cu", "match.cu", "contract.cu", "tail.cu", "evaluate.cu", "server.cu", "tune.cu", "refine.cu", "hierarchy_io.cu"]
HEADERS = [os.path.join(CSRC, h) for h in ("kp_internal.cuh", "engine.cuh", "match.cuh", "gpa.cuh", "contract.cuh")] + [os.path.join(INCLUDE, "kp.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The persistent tail kernel reads data written earlier in the same launch by
# other blocks: its unit serves every global load from L2 (coherent); it also
# keeps the 128-bit rating compare only (see cmp_frac).
PER_FILE = {"tail.cu": ["-Xptxas", "-dlcm=cg", "-DKP_COHERENT_LOADS", "-DKP_FRAC_WIDE_ONLY"]}
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _nvcc() -> str:
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(cuda, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + HEADERS):
            jobs.append([nvcc] + FLAGS + PER_FILE.get(src, []) + list(extra_flags) + ["-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
