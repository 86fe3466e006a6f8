"""Builds the CUDA libraries in-tree for sm_103a with nvcc.

The same sources are built twice: libkp.so with 32-bit entry offsets and
libkp64.so with 64-bit ones (KP_WIDE_OFFSETS, for graphs of 2^31 entries or
more).  Every translation unit of both is compiled in parallel, then each
set is linked with the static CUDA runtime into
paper_0910_2004_gb300/_build/.
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
LIB64 = os.path.join(OUT, "libkp64.so")
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


def build(force: bool = False, verbose: bool = False, extra_flags=(), widths=(32, 64)) -> str:
    """Builds the libraries of the given offset widths; returns libkp.so's
    path (or libkp64.so's when only 64 is asked for)."""
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    objs = {w: [] for w in widths}
    jobs = []
    for w in widths:
        for src in SOURCES:
            s = os.path.join(CSRC, src)
            o = os.path.join(OUT, src.replace(".cu", ".o" if w == 32 else ".w64.o"))
            objs[w].append(o)
            if force or _stale(o, [s] + HEADERS):
                wide = ["-DKP_WIDE_OFFSETS"] if w == 64 else []
                jobs.append([nvcc] + FLAGS + wide + PER_FILE.get(src, []) + list(extra_flags) + ["-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), max(os.cpu_count() or 1, 1))) as ex:
            list(ex.map(run, jobs))
    for w in widths:
        lib = LIB if w == 32 else LIB64
        if force or jobs or _stale(lib, objs[w]):
            tmp = lib + f".tmp{os.getpid()}"
            run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs[w] + ["-lpthread"])
            os.replace(tmp, lib)
    return LIB if 32 in widths else LIB64


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
