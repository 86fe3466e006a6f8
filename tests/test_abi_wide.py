"""The 64-bit offset build (libkp64.so, KP_WIDE_OFFSETS): it loads, exports
every entry point include/kp.h declares, reports its width, lays kp_graph
out with an int64 nnz and int64 row offsets, refuses nnz >= 2^32 on the host
(the weight range: nnz = 2|E| with omega >= 1 and the sum of omega below
2^31), and reads a hierarchy file of either offset width.  CPU only: each
check runs in a child process whose binding selects the wide library, and
no call here reaches the GPU."""
import os
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_wide(code: str):
    env = dict(os.environ, KP_OFFSET_BITS="64")
    r = subprocess.run([sys.executable, "-c", textwrap.dedent(code)], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


def test_wide_library_loads_and_exports_every_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from tests.test_abi import _declared
    names = [n for n in _declared() if n != "kp_initial_partition_fn"]
    out = run_wide(f"""
        import ctypes
        from paper_0910_2004_gb300 import binding as B
        L = B.load()
        assert B.OFFSET_BITS == 64 and B.LIB_PATH.endswith("libkp64.so")
        assert L.kp_offset_bits() == 64
        for name in {names!r}:
            assert hasattr(L, name), name
        assert "64-bit offsets" in B.kp_version()
        # int32 n, padding, int64 nnz, four pointers
        assert ctypes.sizeof(B.kp_graph) == 48 and B.kp_graph.nnz.offset == 8
        # offsets of 2^31 and more pass the binding in this width
        B.check_offset_width(1 << 31, "t")
        x = B.host_offsets([0, 1 << 31, (1 << 32) - 1], "t")
        assert x.dtype.itemsize == 8 and int(x[-1]) == (1 << 32) - 1
        print("ok")
    """)
    assert out.strip().endswith("ok")


def test_wide_library_refuses_nnz_beyond_the_weight_range():
    out = run_wide("""
        import ctypes
        from paper_0910_2004_gb300 import binding as B
        L = B.load()
        h = ctypes.c_void_p()
        o = B.kp_options_default()
        # the pointers are never read: the size check comes first
        g = B.kp_graph(1, 1 << 32, 16, 16, 16, 16)
        assert L.kp_coarsen(ctypes.byref(g), ctypes.byref(o), None, ctypes.byref(h)) == B.KP_ERR_OVERFLOW
        assert "2^32" in B.kp_last_error()
        g = B.kp_graph(1, -1, 16, 16, 16, 16)
        assert L.kp_coarsen(ctypes.byref(g), ctypes.byref(o), None, ctypes.byref(h)) == B.KP_ERR_INVALID
        out = B.kp_cut_gain_out()
        out.gain, out.target, out.block_w = 16, 16, 16
        g = B.kp_graph(1, 1 << 32, 16, 16, 16, 16)
        for fn in (L.kp_cut_gain, L.kp_cut_gain_noalloc):
            assert fn(ctypes.byref(g), ctypes.c_void_p(16), 2, 0.03, ctypes.byref(out), None) == B.KP_ERR_OVERFLOW
        q_nnz = ctypes.c_int64()
        assert L.kp_quotient_graph(ctypes.byref(g), ctypes.c_void_p(16), 2, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                   ctypes.c_void_p(16), 4, ctypes.byref(q_nnz), None) == B.KP_ERR_OVERFLOW
        assert L.kp_boundary_band(ctypes.byref(g), ctypes.c_void_p(16), 2, 1, -1, -1, ctypes.c_void_p(16),
                                  None) == B.KP_ERR_OVERFLOW
        print("ok")
    """)
    assert out.strip().endswith("ok")


def test_wide_library_reads_both_file_versions(tmp_path):
    out = run_wide(f"""
        import ctypes, os, struct
        from paper_0910_2004_gb300 import binding as B
        from tests.test_hierarchy_file import write, PATH, EDGE, MAGIC
        L = B.load()
        def status(p):
            h = ctypes.c_void_p()
            st = L.kp_hierarchy_load(os.fsencode(p), None, ctypes.byref(h))
            if st == 0:
                L.kp_hierarchy_free(h)
            return st
        for version in (1, 2):
            p = os.path.join({str(tmp_path)!r}, f"v{{version}}.kph")
            write(p, [PATH, EDGE], [[0, 0, 1, 1]], version=version)
            assert status(p) in (B.KP_OK, B.KP_ERR_CUDA), version
            write(p, [PATH, EDGE], [[0, 0, 1, 2]], version=version)
            assert status(p) == B.KP_ERR_INVALID, version
        # 2^31 entries fit 64-bit offsets: this file fails only for its
        # missing arrays; 2^32 does not fit the weight range
        p = os.path.join({str(tmp_path)!r}, "big.kph")
        open(p, "wb").write(MAGIC + struct.pack("<4i", 2, 1, 0, 0) + struct.pack("<2iq", 5, 0, 1 << 31))
        assert status(p) == B.KP_ERR_INVALID and "truncated" in B.kp_last_error()
        open(p, "wb").write(MAGIC + struct.pack("<4i", 2, 1, 0, 0) + struct.pack("<2iq", 5, 0, 1 << 32))
        assert status(p) == B.KP_ERR_OVERFLOW
        print("ok")
    """)
    assert out.strip().endswith("ok")
