"""The C-ABI library builds, loads without a GPU, and exports every entry
point include/gbmc.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gbmc_\w+)\s*\(", src, re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    from paper_2403_12345_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("gbmc_init_materials", "gbmc_load_xs_tables", "gbmc_run_batch",
                     "gbmc_read_tallies"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export(built):
    from paper_2403_12345_gb300 import gbmc
    assert sorted(gbmc.EXPORTS) == declared_entry_points()
    gbmc.lib()


def test_default_options_without_gpu(built):
    from paper_2403_12345_gb300 import gbmc
    opt = gbmc.Options()
    assert gbmc.lib().gbmc_default_options(ctypes.byref(opt)) == 0
    assert opt.precision == gbmc.FP64 and opt.sort == 1 and opt.blocks_per_sm == 8
    assert opt.max_iterations == 4 * gbmc.MAX_FLIGHTS
    assert opt.sort_min == 4096 and opt.warp_lookup_max == 4096 and opt.tail_max == 4096
    assert opt.group_lookup_max == 160000 and opt.search == 1 and opt.sparse_windows == 0
    # the same sizes are static_asserts of the C side
    assert ctypes.sizeof(gbmc.Options) == 72
    assert ctypes.sizeof(gbmc.Geometry) == 104 and ctypes.sizeof(gbmc.Problem) == 136
    assert ctypes.sizeof(gbmc.HostResults) == 11 * 8   # gbmc_host_results: 11 pointers


def test_create_without_gpu_fails_cleanly(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2403_12345_gb300 import gbmc
    with pytest.raises(gbmc.GbmcError) as e:
        gbmc.Context(0)
    assert e.value.code == gbmc.ERR_CUDA


def test_host_alloc_argument_checks_without_gpu(built):
    # gbmc_host_alloc checks its arguments before any CUDA call; freeing NULL
    # is a no-op (no compute call is made)
    from paper_2403_12345_gb300 import gbmc
    L = gbmc.lib()
    p = ctypes.c_void_p(1234)
    assert L.gbmc_host_alloc(ctypes.c_size_t(0), ctypes.byref(p)) == gbmc.ERR_INVALID_ARG
    assert L.gbmc_host_alloc(ctypes.c_size_t(64), None) == gbmc.ERR_INVALID_ARG
    assert L.gbmc_host_free(None) == 0
