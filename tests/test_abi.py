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
    d2.metric, d2.a, d2.gam, d2.flags = 0, 0.5, 13 / 9, 0x20
    assert L.hamr_con2prim(ctypes.byref(d2), 5, 1, 1, 1, 1, 1, 1, None, None) == hamr.EINVAL
    assert L.hamr_con2prim(ctypes.byref(d2), 0, None, None, None, None, None, None, None, None) == hamr.OK


def _desc(blocks, **kw):
    arr = (hamr.BlockDesc * len(blocks))(*blocks)
    d = hamr.GridDesc()
    d.metric, d.a, d.gam, d.cour = kw.pop("metric", 0), 0.5, 13 / 9, 0.8
    d.nblocks = len(blocks)
    d.blocks = arr
    for k, v in kw.items():
        setattr(d, k, v)
    return d, arr


def test_option_fields_are_validated_before_any_device_call(libpath):
    """Each option of the step refuses an unknown value with HAMR_EINVAL and a message, on CPU."""
    L = hamr.lib()
    h = ctypes.c_void_p()
    polar = hamr.block(16, 16, 16, 0.0, 0.0, 0.0, 0.1, 0.1, 0.1, (3, 3, 2, 2, 1, 1))
    for field, bad, msg in (("emf", 2, b"unknown emf"), ("flatten", 3, b"flatten must be 0 or 1"),
                            ("inversion", 5, b"unknown inversion"), ("floor_frame", 2, b"unknown floor_frame"),
                            ("smr", 5, b"smr must be in 0..4"), ("metric", 3, b"unknown metric")):
        d, arr = _desc([polar], **{field: bad})
        assert L.hamr_grid_create(ctypes.byref(d), ctypes.byref(h)) == hamr.EINVAL, field
        assert msg in L.hamr_last_error(), (field, L.hamr_last_error())
    # internal SMR: single blocks with a polar face and n3 divisible by 2^(smr+1)
    flat = hamr.block(16, 16, 16, 0.0, 0.0, 0.0, 0.1, 0.1, 0.1, (1, 1, 1, 1, 1, 1))
    d, arr = _desc([flat], smr=1)
    assert L.hamr_grid_create(ctypes.byref(d), ctypes.byref(h)) == hamr.EINVAL
    assert b"polar" in L.hamr_last_error()
    odd = hamr.block(16, 16, 12, 0.0, 0.0, 0.0, 0.1, 0.1, 0.1, (3, 3, 2, 2, 1, 1))
    d, arr = _desc([odd], smr=3)
    assert L.hamr_grid_create(ctypes.byref(d), ctypes.byref(h)) == hamr.EINVAL
    assert b"multiple of 16" in L.hamr_last_error()
    # in a block tree every polar block's widths are a power of 2 finer than the coarsest polar block's
    base = hamr.block(16, 16, 16, 0.0, 0.0, 0.0, 0.1, 0.1, 0.1, (3, 4, 2, 2, 1, 1))
    third = hamr.block(16, 16, 16, 1.6, 0.0, 0.0, 0.1, 0.1, 0.1 / 3.0, (4, 3, 2, 2, 1, 1))
    d, arr = _desc([base, third], smr=1)
    assert L.hamr_grid_create(ctypes.byref(d), ctypes.byref(h)) == hamr.EINVAL
    assert b"block 1: internal SMR needs" in L.hamr_last_error(), L.hamr_last_error()
    # polar boundaries need spherical coordinates: refused in flat Cartesian space
    d, arr = _desc([polar], metric=1)
    assert L.hamr_grid_create(ctypes.byref(d), ctypes.byref(h)) == hamr.EINVAL
    assert b"spherical" in L.hamr_last_error()


def test_tree_and_regrid_arguments_checked_on_cpu(libpath):
    L = hamr.lib()
    assert L.hamr_grid_regrid(None, 2, None, None) == hamr.EINVAL
    assert L.hamr_grid_block_max(None, 0, None, None) == hamr.EINVAL
    assert L.hamr_grid_set_fine_dt(None, 0.1) == hamr.EINVAL
    assert L.hamr_grid_set_ghost_maps(None, 1, None) == hamr.EINVAL
    n = ctypes.c_int()
    assert L.hamr_tree_adapt(None, 0, None, None, None, None, None, 0, ctypes.byref(n)) == hamr.EINVAL


def test_noalloc_step_validates_like_grid_create(libpath):
    """hamr_block_step_noalloc refuses every descriptor hamr_grid_create refuses, before touching the
    device or the (here never dereferenced) state pointers, plus its own limits."""
    L = hamr.lib()
    ok_block = hamr.block(8, 8, 8, 0.0, 0.0, 0.0, 0.1, 0.1, 0.1, (0, 0, 1, 1, 1, 1))
    fake = ctypes.c_void_p(256)
    cases = []
    cases.append((*_desc([ok_block], a=1.5), b"spin"))
    bad_dx = hamr.block(8, 8, 8, 0.0, 0.0, 0.0, 0.0, 0.1, 0.1, (0, 0, 1, 1, 1, 1))
    cases.append((*_desc([bad_dx]), b"dx must be > 0"))
    polar_x1 = hamr.block(8, 8, 8, 0.0, 0.0, 0.0, 0.1, 0.1, 0.1, (2, 2, 1, 1, 1, 1))
    cases.append((*_desc([polar_x1]), b"polar bc only on x2"))
    half_periodic = hamr.block(8, 8, 8, 0.0, 0.0, 0.0, 0.1, 0.1, 0.1, (0, 0, 1, 0, 1, 1))
    cases.append((*_desc([half_periodic]), b"periodic bc must be on both sides"))
    cases.append((*_desc([ok_block], gam=3.0), b"gam"))
    cases.append((*_desc([ok_block], cour=0.0), b"cour"))
    cases.append((*_desc([ok_block], recon=7), b"unknown recon"))
    cases.append((*_desc([ok_block], riemann=4), b"unknown riemann"))
    cases.append((*_desc([ok_block], precision=1), b"FP64 only"))
    cases.append((*_desc([ok_block], smr=1), b"polar"))
    big = hamr.block(20, 20, 20, 0.0, 0.0, 0.0, 0.1, 0.1, 0.1, (0, 0, 1, 1, 1, 1))
    cases.append((*_desc([big]), b"too large for the no-allocation step"))
    cases.append((*_desc([ok_block, ok_block]), b"one block"))
    for d, arr, msg in cases:
        assert L.hamr_block_step_noalloc(ctypes.byref(d), fake, fake, -1.0, None) == hamr.EINVAL, msg
        assert msg in L.hamr_last_error(), (msg, L.hamr_last_error())
