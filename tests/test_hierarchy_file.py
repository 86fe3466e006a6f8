"""kp_hierarchy_load checks a file on the host before anything reaches the
device: maps that would send the projection outside a level, or outside a
graph of a batch, are refused with KP_ERR_INVALID.  CPU only: every file here
is rejected before the first CUDA call; the valid ones pass the checks and then
either load (with a GPU) or stop at the first CUDA call (without one)."""
import ctypes
import os
import struct

import numpy as np
import pytest

MAGIC = b"KPHIER01"


def write(path, levels, maps, goffs=None, glevels=None, gid0=None, version=1):
    """levels: [(xadj, adjncy, ewgt, vwgt)], maps: one per level but the last.
    version 1: 32-bit row offsets; version 2: 64-bit (i32 n, i32 0, i64 nnz,
    int64 xadj)."""
    G = 0 if goffs is None else len(goffs[0]) - 1
    out = bytearray(MAGIC + struct.pack("<4i", version, len(levels), G, 0))
    for l, (xadj, adj, ew, vw) in enumerate(levels):
        n, nnz = len(xadj) - 1, len(adj)
        if version == 1:
            out += struct.pack("<2i", n, nnz) + np.asarray(xadj, dtype="<i4").tobytes()
        else:
            out += struct.pack("<2iq", n, 0, nnz) + np.asarray(xadj, dtype="<i8").tobytes()
        for a in (adj, ew, vw):
            out += np.asarray(a, dtype="<i4").tobytes()
        if l < len(levels) - 1:
            out += np.asarray(maps[l], dtype="<i4").tobytes()
        if G:
            out += np.asarray(goffs[l], dtype="<i4").tobytes()
    if G:
        out += np.asarray(glevels, dtype="<i4").tobytes() + np.asarray(gid0, dtype="<i4").tobytes()
    open(path, "wb").write(bytes(out))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_2004_gb300 import binding
    return binding.load()


def load_status(lib, path):
    h = ctypes.c_void_p()
    st = lib.kp_hierarchy_load(os.fsencode(str(path)), None, ctypes.byref(h))
    if st == 0:
        lib.kp_hierarchy_free(h)
    return st


# a path 0-1-2-3 contracted to the edge {0,1}: level 1 has 2 nodes
PATH = ([0, 1, 3, 5, 6], [1, 0, 2, 1, 3, 2], [1] * 6, [1] * 4)
EDGE = ([0, 1, 2], [1, 0], [1, 1], [2, 2])
SINGLE_NODE = ([0, 0], [], [], [2])


def union(*gs):
    xadj, adj, ew, vw, base = [0], [], [], [], 0
    for x, a, e, v in gs:
        start = xadj[-1]
        xadj += [start + int(d) for d in x[1:]]
        adj += [u + base for u in a]
        ew += list(e)
        vw += list(v)
        base += len(x) - 1
    return xadj, adj, ew, vw


@pytest.mark.parametrize("version", [1, 2])
def test_single_graph_maps_must_stay_in_the_next_level(lib, tmp_path, version):
    from paper_0910_2004_gb300 import binding as B
    good = tmp_path / "good.kph"
    write(good, [PATH, EDGE], [[0, 0, 1, 1]], version=version)
    assert load_status(lib, good) in (B.KP_OK, B.KP_ERR_CUDA)
    for bad_map in ([0, 0, 1, 2], [0, 0, 1, -1], [-1, 0, 1, 1]):
        p = tmp_path / "bad.kph"
        write(p, [PATH, EDGE], [bad_map], version=version)
        assert load_status(lib, p) == B.KP_ERR_INVALID, bad_map
    # row offsets that decrease, or end elsewhere than nnz
    for bad_x in ([0, 1, 3, 2, 6], [0, 1, 3, 5, 5]):
        p = tmp_path / "badx.kph"
        write(p, [(bad_x,) + PATH[1:], EDGE], [[0, 0, 1, 1]], version=version)
        assert load_status(lib, p) == B.KP_ERR_INVALID, bad_x


def test_64_bit_offsets_beyond_the_32_bit_range_are_refused(lib, tmp_path):
    """A version-2 level of 2^31 entries does not fit 32-bit offsets: the
    32-bit library answers KP_ERR_OVERFLOW right after the level's sizes."""
    from paper_0910_2004_gb300 import binding as B
    p = tmp_path / "big.kph"
    open(p, "wb").write(MAGIC + struct.pack("<4i", 2, 1, 0, 0) + struct.pack("<2iq", 5, 0, 1 << 31))
    assert load_status(lib, p) == B.KP_ERR_OVERFLOW
    open(p, "wb").write(MAGIC + struct.pack("<4i", 3, 1, 0, 0))
    assert load_status(lib, p) == B.KP_ERR_UNSUPPORTED


_CAPPED_LOAD = """
import ctypes, os, resource, sys
resource.setrlimit(resource.RLIMIT_AS, (3 << 30, 3 << 30))
lib = ctypes.CDLL(sys.argv[1])
lib.kp_last_error.restype = ctypes.c_char_p
h = ctypes.c_void_p()
st = lib.kp_hierarchy_load(os.fsencode(sys.argv[2]), None, ctypes.byref(h))
print(st, lib.kp_last_error().decode())
"""


@pytest.mark.parametrize("version", [1, 2])
@pytest.mark.parametrize("libname", ["libkp.so", "libkp64.so"])
def test_sizes_beyond_the_file_are_refused_before_any_buffer(lib, tmp_path, version, libname):
    """A header that claims 2^31-2 nodes in a file of a few bytes: the loader
    compares each array with what is left of the file before it sizes a
    buffer, so the answer is KP_ERR_INVALID (truncated), not an allocation of
    8-16 GB.  Run in a child whose address space is capped at 3 GB, where
    allocating first fails with KP_ERR_OOM instead."""
    import subprocess
    import sys
    from paper_0910_2004_gb300 import binding as B
    path = os.path.join(os.path.dirname(B.LIB_PATH), libname)
    n = (1 << 31) - 2
    p = tmp_path / "claims_too_much.kph"
    sizes = struct.pack("<2i", n, 0) if version == 1 else struct.pack("<2iq", n, 0, 0)
    open(p, "wb").write(MAGIC + struct.pack("<4i", version, 1, 0, 0) + sizes + bytes(64))
    r = subprocess.run([sys.executable, "-c", _CAPPED_LOAD, path, str(p)], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    st, msg = r.stdout.strip().split(" ", 1)
    assert int(st) == B.KP_ERR_INVALID and "truncated" in msg, r.stdout


def test_batch_maps_stay_inside_their_graph(lib, tmp_path):
    from paper_0910_2004_gb300 import binding as B
    # graph 0: the path (two levels); graph 1: one edge contracted to a node
    lv0 = union(PATH, EDGE)
    lv1 = union(EDGE, SINGLE_NODE)
    goffs = [[0, 4, 6], [0, 2, 3]]
    good_map = [0, 0, 1, 1, 2, 2]
    good = tmp_path / "good.kph"
    write(good, [lv0, lv1], [good_map], goffs, [2, 2], [0, 0, 0, 0, 1, 1])
    assert load_status(lib, good) in (B.KP_OK, B.KP_ERR_CUDA)
    cases = {
        "into the other graph": ([0, 0, 1, 1, 1, 2], [2, 2], [0, 0, 0, 0, 1, 1]),
        "carried node not carried": ([0, 0, 1, -1, 2, 2], [2, 2], [0, 0, 0, 0, 1, 1]),
        "graph id disagrees with the offsets": (good_map, [2, 2], [0, 0, 0, 1, 1, 1]),
    }
    for what, (m, gl, gid) in cases.items():
        p = tmp_path / "bad.kph"
        write(p, [lv0, lv1], [m], goffs, gl, gid)
        assert load_status(lib, p) == B.KP_ERR_INVALID, what


def test_batch_graph_that_stopped_maps_nowhere(lib, tmp_path):
    from paper_0910_2004_gb300 import binding as B
    # graph 1 stops at the input (one level): its nodes map to -1
    lv0 = union(PATH, EDGE)
    lv1 = EDGE
    goffs = [[0, 4, 6], [0, 2, 2]]
    good = tmp_path / "good.kph"
    write(good, [lv0, lv1], [[0, 0, 1, 1, -1, -1]], goffs, [2, 1], [0, 0, 0, 0, 1, 1])
    assert load_status(lib, good) in (B.KP_OK, B.KP_ERR_CUDA)
    p = tmp_path / "bad.kph"
    write(p, [lv0, lv1], [[0, 0, 1, 1, 0, -1]], goffs, [2, 1], [0, 0, 0, 0, 1, 1])
    assert load_status(lib, p) == B.KP_ERR_INVALID
