"""No entry offset is narrowed to 32 bits in the device code.

The library's device and host sources are compiled by the host compiler
(g++, syntax only, with stand-ins for the CUDA builtins in
hostcc/cuda_stubs.h and kernel launches reduced to calls) with
-Wconversion, in both offset widths: in the 64-bit build (KP_WIDE_OFFSETS)
every implicit conversion from a 64-bit integer to a 32-bit one is a place
where a row offset or entry index above 2^31 could be truncated.  Both
widths must compile without one.  CPU only."""
import os
import re
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0910_2004_gb300", "csrc")
STUBS = os.path.join(ROOT, "tests", "hostcc", "cuda_stubs.h")
NARROW = re.compile(r"conversion from .(long int|long long int|int64_t|kp::eoff|kp_eoff|long unsigned int|"
                    r"long long unsigned int|uint64_t). .*to .(int|int32_t|unsigned int|uint32_t)\b")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.mark.parametrize("wide", [False, True])
def test_no_offset_narrowing(tmp_path, wide):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "csrc"
    src.mkdir()
    for f in os.listdir(CSRC):
        t = open(os.path.join(CSRC, f)).read()
        t = re.sub(r"<<<[^;]*?>>>", "", t, flags=re.S)               # launches become calls
        t = t.replace("(const void *)k_", "(const void *)(void *)&k_")
        t = t.replace("cudaFuncSetAttribute(k_", "cudaFuncSetAttribute((const void *)(void *)&k_")
        (src / f).write_text(t)
    flags = ["g++", "-std=c++17", "-fsyntax-only", "-Wconversion", "-Wno-sign-conversion", "-Wno-attributes",
             "-include", STUBS, "-I", os.path.join(ROOT, "include"), "-I", inc, "-D__CUDA_ARCH__=1030"]
    if wide:
        flags.append("-DKP_WIDE_OFFSETS")
    units = sorted(f for f in os.listdir(src) if f.endswith(".cu"))

    def run(f):
        extra = ["-DKP_COHERENT_LOADS"] if f == "tail.cu" else []
        r = subprocess.run(flags + extra + ["-x", "c++", str(src / f)], capture_output=True, text=True)
        return f, r.returncode, r.stderr

    with ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(run, units))
    errors = [(f, err[-2000:]) for f, rc, err in results if rc != 0]
    assert not errors, errors[0]
    found = sorted({l.split(str(src) + "/")[-1][:200] for f, rc, err in results for l in err.splitlines()
                    if "warning:" in l and NARROW.search(l)})
    assert not found, "\n".join(found)
