"""include/kp.h is a C ABI: a translation unit that names every entry point
it declares compiles as strict C99 and as C++ (-pedantic -Wall -Wextra
-Werror) in both offset widths, without any CUDA header, and links against
the library of its width with every symbol resolved.  CPU only."""
import os
import shutil
import subprocess

import pytest

from tests.test_abi import _declared

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BUILD = os.path.join(ROOT, "paper_0910_2004_gb300", "_build")


def _source():
    names = [n for n in _declared() if n != "kp_initial_partition_fn"]
    table = ",\n    ".join(f"(entry){n}" for n in names)
    return f"""#include "kp.h"
typedef void (*entry)(void);
static const entry entries[] = {{
    {table}
}};
int main(void) {{
    kp_graph g = {{0, 0, 0, 0, 0, 0}};
    kp_eoff nnz = g.nnz;
    return (int)(sizeof entries / sizeof entries[0]) + (int)nnz - {len(names)} + (KP_OFFSET_BITS == 32 || KP_OFFSET_BITS == 64 ? 0 : 1);
}}
"""


@pytest.fixture(scope="module")
def libs():
    import __graft_entry__
    __graft_entry__.build()
    return {32: "kp", 64: "kp64"}


@pytest.mark.parametrize("wide", [False, True])
@pytest.mark.parametrize("lang", ["c99", "c++11"])
def test_header_compiles_and_links(libs, tmp_path, wide, lang):
    cc = "gcc" if lang == "c99" else "g++"
    if shutil.which(cc) is None:
        pytest.skip(f"needs {cc}")
    src = tmp_path / ("entries.c" if lang == "c99" else "entries.cpp")
    src.write_text(_source())
    exe = str(tmp_path / "entries")
    cmd = [cc, f"-std={lang}", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include")]
    if wide:
        cmd.append("-DKP_WIDE_OFFSETS")
    cmd += [str(src), "-L", BUILD, f"-l{libs[64 if wide else 32]}", "-Wl,--unresolved-symbols=ignore-in-shared-libs",
            "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    # every entry point resolves in the library of this width (symbols only: nothing runs)
    nm = subprocess.run(["nm", "-D", "--defined-only", os.path.join(BUILD, f"lib{libs[64 if wide else 32]}.so")],
                        capture_output=True, text=True)
    defined = {line.split()[-1] for line in nm.stdout.splitlines() if line.strip()}
    missing = [n for n in _declared() if n != "kp_initial_partition_fn" and n not in defined]
    assert not missing, missing
