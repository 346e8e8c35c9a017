"""The C-ABI library builds, loads and exports every function include/hamr.h
declares (no compute calls: these run without a GPU)."""
import ctypes
import os

import pytest

from paper_1912_10192_gb300 import _build, hamr


@pytest.fixture(scope="module")
def libpath():
    return _build.build()


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    names = hamr.header_functions()
    assert {"hamr_grid_create", "hamr_block_step", "hamr_con2prim", "hamr_batch_step"} <= set(names)
    for n in names:
        assert hasattr(L, n), n


def test_last_error_is_empty_string_initially(libpath):
    L = hamr.lib()
    assert L.hamr_last_error() == b""


def test_invalid_descriptors_rejected_without_gpu_work(libpath):
    """Descriptor validation happens before any device call."""
    L = hamr.lib()
    h = ctypes.c_void_p()
    assert L.hamr_grid_create(None, ctypes.byref(h)) == hamr.EINVAL
    b = hamr.block(2, 8, 8, 0.0, 0.0, 0.0, 0.1, 0.1, 0.1, (0, 0, 0, 0, 1, 1))
    d = hamr.GridDesc()
    d.metric, d.a, d.gam, d.cour = 0, 0.5, 13 / 9, 0.8
    d.nblocks = 1
    arr = (hamr.BlockDesc * 1)(b)
    d.blocks = arr
    assert L.hamr_grid_create(ctypes.byref(d), ctypes.byref(h)) == hamr.EINVAL
    assert b"n must be >= 4" in L.hamr_last_error()
    arr[0].n1 = 8
    arr[0].bc[2] = hamr.BC_POLAR
    arr[0].n3 = 7
    assert L.hamr_grid_create(ctypes.byref(d), ctypes.byref(h)) == hamr.EINVAL
    d2 = hamr.C2PDesc()
    d2.metric, d2.a, d2.gam, d2.flags = 0, 0.5, 13 / 9, 0x10
    assert L.hamr_con2prim(ctypes.byref(d2), 5, 1, 1, 1, 1, 1, 1, None, None) == hamr.EINVAL
    assert L.hamr_con2prim(ctypes.byref(d2), 0, None, None, None, None, None, None, None, None) == hamr.OK
