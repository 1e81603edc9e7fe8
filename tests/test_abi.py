"""The C-ABI library loads and exports every function include/gals.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_0905_3409_gb300 import gals

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(gals_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as ge
    ge.build()
    return gals.lib()


def test_checked_library_builds_and_exports_the_same_symbols():
    """The checked build (-DGALS_CHECKED) compiles for sm_103a and exports the same ABI."""
    from paper_0905_3409_gb300 import build
    L = ctypes.CDLL(build.build_checked())
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_library_exports_all_declared_symbols(built):
    decl = _declared()
    assert decl, "no declarations found"
    missing = [n for n in sorted(decl) if not hasattr(built, n)]
    assert not missing, missing
    assert set(decl) == set(gals.EXPORTS) | (set(decl) - set(gals.EXPORTS))
    for n in gals.EXPORTS:
        assert n in decl, n


def test_version_and_argument_errors_without_gpu(built):
    assert "sm_103a" in gals.version()
    # argument validation happens before any CUDA call
    d = gals.GridDesc()
    d.dim = 4
    h = ctypes.c_void_p()
    assert built.gals_create_grid(ctypes.byref(d), ctypes.byref(h)) == gals.ERR_ARG
    assert b"dim" in built.gals_last_error(None)
    d.dim = 2
    d.n[0], d.n[1] = 3, 10
    d.hi[0] = d.hi[1] = 1.0
    assert built.gals_create_grid(ctypes.byref(d), ctypes.byref(h)) == gals.ERR_ARG
    assert built.gals_create_grid(None, ctypes.byref(h)) == gals.ERR_ARG
    # size limits of the kernels' 32-bit plane offsets and launch grids (no allocation)
    d.n[0], d.n[1] = 46344, 46341            # pitch 46344 x 46341 rows > 2^31 - 1
    assert built.gals_create_grid(ctypes.byref(d), ctypes.byref(h)) == gals.ERR_ARG
    assert b"2^31" in built.gals_last_error(None)
    d.n[0], d.n[1] = 4, 917491               # more than 65535 blocks of 14 rows
    assert built.gals_create_grid(ctypes.byref(d), ctypes.byref(h)) == gals.ERR_ARG
    d.dim = 3
    d.n[0], d.n[1], d.n[2] = 8, 8, 262141    # more than 65535 blocks of 4 z-slices
    d.hi[2] = 1.0
    assert built.gals_create_grid(ctypes.byref(d), ctypes.byref(h)) == gals.ERR_ARG
    assert b"n[2]" in built.gals_last_error(None)
    d.dim = 2
    assert built.gals_step(None, None, 0.1, 1) == gals.ERR_ARG
    assert built.gals_destroy_grid(None) == gals.OK


def test_struct_layouts_match_header():
    # sizes of the public structs as laid out by the C compiler (x86-64 / aarch64 LP64)
    assert ctypes.sizeof(gals.GridDesc) == 4 + 12 + 24 + 24 + 4 + 4 + 8  # layout, cross_scheme: 80
    assert gals.GridDesc.cross_scheme.offset == 68 and gals.GridDesc.cuda_stream.offset == 72
    assert ctypes.sizeof(gals.DiagOut) == 11 * 8


def test_wait_test_hook_only_in_checked_build(built):
    """gals_checked_wait_test changes nothing in the normal build (UNSUPPORTED); the checked
    build validates its argument (no CUDA call either way)."""
    from paper_0905_3409_gb300 import build
    assert built.gals_checked_wait_test(ctypes.c_uint32(2048), 1) == gals.ERR_UNSUPPORTED
    L = ctypes.CDLL(build.build_checked())
    L.gals_checked_wait_test.argtypes = [ctypes.c_uint32, ctypes.c_int]
    assert L.gals_checked_wait_test(0, 1) == gals.ERR_ARG
    assert L.gals_checked_wait_test(1 << 24, 0) == gals.OK
