"""The C-ABI library loads and exports every entry point include/kp.h
declares (CPU only: no call here reaches the GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_2004_gb300 import binding
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "kp_coarsen" in names and "kp_project" in names and "kp_cut_gain" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_0910_2004_gb300 import binding
    assert sorted(binding.EXPORTED) == sorted(n for n in _declared() if n != "kp_initial_partition_fn")


def test_options_defaults_and_version(lib):
    from paper_0910_2004_gb300 import binding as B
    o = B.kp_options_default()
    assert (o.rating, o.seed, o.stop_size, o.max_levels, o.min_shrink_permille, o.validate) == (0, 1, 40, 64, 50, 1)
    assert o.spin_limit == 1 << 22
    assert "sm_103a" in B.kp_version()


def test_host_side_argument_errors(lib):
    """Argument checks that return before any CUDA call."""
    from paper_0910_2004_gb300 import binding as B
    h = ctypes.c_void_p()
    assert lib.kp_coarsen(None, None, None, ctypes.byref(h)) == B.KP_ERR_INVALID
    assert "null" in B.kp_last_error()
    n = ctypes.c_int32()
    assert lib.kp_hierarchy_num_levels(None, ctypes.byref(n)) == B.KP_ERR_INVALID
    g = B.kp_graph(0, 0, None, None, None, None)
    out = B.kp_cut_gain_out()
    assert lib.kp_cut_gain(ctypes.byref(g), None, 0, 0.03, ctypes.byref(out), None) == B.KP_ERR_INVALID
    assert "k must be" in B.kp_last_error()
    assert lib.kp_cut_gain(ctypes.byref(g), None, 2, -1.0, ctypes.byref(out), None) == B.KP_ERR_INVALID
    o = B.kp_options_default()
    o.max_levels = 500
    assert lib.kp_coarsen(ctypes.byref(g), ctypes.byref(o), None, ctypes.byref(h)) == B.KP_ERR_UNSUPPORTED


def test_product_path_has_no_oracle_import():
    """The package never imports the oracle (the oracle is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_0910_2004_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_binding_refuses_sizes_beyond_the_32_bit_offsets(lib):
    """The 32-bit library holds nnz and the row offsets in int32: the binding
    refuses larger values before numpy or ctypes would wrap them (a graph of
    2^32 + 5 entries would otherwise reach the library as a consistent graph of
    5)."""
    import numpy as np
    from paper_0910_2004_gb300 import binding as B
    assert B.OFFSET_BITS == 32
    B.check_offset_width((1 << 31) - 1, "t")
    with pytest.raises(B.KpError) as e:
        B.check_offset_width(1 << 31, "t")
    assert e.value.status == B.KP_ERR_OVERFLOW
    x = B.host_offsets(np.array([0, 3, 5], np.int64), "t")
    assert x.dtype == np.int32 and x.flags.c_contiguous and list(x) == [0, 3, 5]
    for bad in ([0, 1 << 31], np.array([0, 1 << 32], np.int64), [0, -(1 << 31) - 1]):
        with pytest.raises(B.KpError) as e:
            B.host_offsets(bad, "t")
        assert e.value.status == B.KP_ERR_OVERFLOW
    never = lambda *a: pytest.fail("the initial partitioner must not run")
    with pytest.raises(B.KpError) as e:                  # offsets beyond int32, few entries
        B.pipeline_host([0, 1 << 31], [0], [1], [1], 2, 0.03, never)
    assert e.value.status == B.KP_ERR_OVERFLOW
    huge = np.broadcast_to(np.int32(0), ((1 << 32) + 5,))  # 2^32 + 5 entries, no memory behind them
    with pytest.raises(B.KpError) as e:
        B.pipeline_host([0, 0], huge, huge, [1], 2, 0.03, never)
    assert e.value.status == B.KP_ERR_OVERFLOW


def test_cut_gain_refuses_bad_sizes_and_null_arrays_on_the_host(lib):
    """kp_cut_gain and kp_cut_gain_noalloc check the graph's sizes and arrays
    before any CUDA call, as kp_coarsen does (the pointers here are never
    read)."""
    from paper_0910_2004_gb300 import binding as B
    out = B.kp_cut_gain_out()
    out.gain, out.target, out.block_w = 16, 16, 16
    for fn in (lib.kp_cut_gain, lib.kp_cut_gain_noalloc):
        g = B.kp_graph(2, -1, 16, 16, 16, 16)
        assert fn(ctypes.byref(g), ctypes.c_void_p(16), 2, 0.03, ctypes.byref(out), None) == B.KP_ERR_INVALID
        assert "negative" in B.kp_last_error()
        g = B.kp_graph(2, 2, 16, None, 16, 16)      # entries without adjncy
        assert fn(ctypes.byref(g), ctypes.c_void_p(16), 2, 0.03, ctypes.byref(out), None) == B.KP_ERR_INVALID
        assert "null" in B.kp_last_error()
        g = B.kp_graph(2, 2, 16, 16, None, 16)      # entries without ewgt
        assert fn(ctypes.byref(g), ctypes.c_void_p(16), 2, 0.03, ctypes.byref(out), None) == B.KP_ERR_INVALID
