"""The C-ABI library builds, loads without a GPU and exports what gribov.h declares."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gribov.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(gc_[a-z0-9_]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("gc_create_orbit", "gc_enumerate_copies", "gc_fetch_copies", "gc_fetch_starts",
                 "gc_orbit_stats", "gc_destroy_orbit", "gc_last_error", "gc_options_default",
                 "gc_set_allocator", "gc_version"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    import paper_1403_0555_b300 as gb
    lib = gb.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    # the binding wraps every exported entry point under the same name
    for name in gb.EXPORTED:
        assert callable(getattr(gb, name)), name


def test_host_only_entry_points_without_gpu():
    import paper_1403_0555_b300 as gb
    opt = gb.gc_options_default()
    assert opt.precision == gb.GC_FP64 and opt.check_every == 1 and opt.max_sweeps == 100000
    assert opt.eps32 == 1e-10 and opt.dedup_delta == 1e-6 and opt.fp_tau == 1e-9
    assert gb.gc_version().startswith("gribov-b300")
    phi = np.zeros((16, 2))
    with pytest.raises(gb.GribovError) as e:
        gb.gc_create_orbit(5, 2, np.zeros((32, 5)))
    assert e.value.code == gb.GC_EINVAL
    with pytest.raises(gb.GribovError) as e:
        gb.gc_create_orbit(2, 1, np.zeros((1, 2)))
    assert e.value.code == gb.GC_EINVAL
    bad = phi.copy()
    bad[3, 1] = np.nan
    with pytest.raises(gb.GribovError) as e:
        gb.gc_create_orbit(2, 4, bad)
    assert e.value.code == gb.GC_EINVAL
    assert "not finite" in gb.gc_last_error()


def test_options_struct_matches_header_layout():
    import paper_1403_0555_b300 as gb
    # gc_options_default writes the whole struct; a size mismatch would corrupt
    # the guard bytes that follow it
    buf = (ctypes.c_ubyte * (ctypes.sizeof(gb.gc_options) + 64))()
    for i in range(len(buf)):
        buf[i] = 0xAB
    gb.load().gc_options_default(ctypes.cast(buf, ctypes.POINTER(gb.gc_options)))
    assert all(b == 0xAB for b in bytes(buf)[ctypes.sizeof(gb.gc_options):])
