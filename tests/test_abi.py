"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/vr.h declares; host-only calls behave (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1001_2049_b300 import _lib, build

HEADER = os.path.join(build.ROOT, "include", "vr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(vr_\w+)\s*\(", text, re.M)))


def test_header_declares_the_north_star_calls():
    names = declared_functions()
    for n in ("vr_volume_create", "vr_set_transfer", "vr_render", "vr_volume_bytes",
              "vr_volume_destroy", "vr_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(_lib.SIGNATURES), "binding lacks a signature"


def test_library_is_built_for_sm_103a():
    src = open(build.__file__).read()
    assert "arch=compute_103a,code=sm_103a" in src
    assert os.path.exists(build.build())


def test_version_and_volume_bytes_host_only():
    lib = _lib.load()
    assert lib.vr_version() == 2
    out = ctypes.c_size_t(0)
    dims = (ctypes.c_int64 * 3)(64, 64, 128)
    assert lib.vr_volume_bytes(dims, _lib.VR_F32, ctypes.byref(out)) == 0
    assert out.value == 2 * 2 * 4 * 32768 * 4
    assert lib.vr_volume_bytes(dims, _lib.VR_F16, ctypes.byref(out)) == 0
    assert out.value == 2 * 2 * 4 * 32768 * 2
    # int8: codes + two 256-byte aligned per-plane tables
    assert lib.vr_volume_bytes(dims, _lib.VR_I8, ctypes.byref(out)) == 0
    assert out.value == 2 * 2 * 4 * 32768 + 2 * 512
    # ragged dims round up to whole bricks
    dims = (ctypes.c_int64 * 3)(33, 2, 65)
    assert lib.vr_volume_bytes(dims, _lib.VR_F32, ctypes.byref(out)) == 0
    assert out.value == 2 * 1 * 3 * 32768 * 4


@pytest.mark.parametrize("dims", [(1, 4, 4), (4, 0, 4), (4, 4, (1 << 20) + 1)])
def test_volume_bytes_rejects_bad_dims(dims):
    lib = _lib.load()
    out = ctypes.c_size_t(0)
    rc = lib.vr_volume_bytes((ctypes.c_int64 * 3)(*dims), _lib.VR_F32, ctypes.byref(out))
    assert rc == _lib.VR_ERR_ARG
    assert b"outside" in lib.vr_last_error()


def test_null_arguments_are_rejected_synchronously():
    lib = _lib.load()
    assert lib.vr_volume_bytes(None, 0, None) == _lib.VR_ERR_ARG
    assert lib.vr_set_transfer(None, None, 2, 0, 1, 0, 1) == _lib.VR_ERR_ARG
    assert lib.vr_render(None, None, 1, 1, 1, 0, 0.5, None, None) == _lib.VR_ERR_ARG
    assert lib.vr_volume_upload(None, 0, 1, None, 1, None) == _lib.VR_ERR_ARG
    h = ctypes.c_void_p(0)
    dims = (ctypes.c_int64 * 3)(8, 8, 8)
    assert lib.vr_volume_create(dims, 7, None, 1, None, 0, None, ctypes.byref(h)) == _lib.VR_ERR_ARG
    assert b"dtype" in lib.vr_last_error()


def test_batch_shapes_and_config_host_only():
    lib = _lib.load()
    n = lib.vr_batch_tune_count()
    assert n >= 4
    seen = set()
    for c in range(n):
        v = [ctypes.c_int(0) for _ in range(4)]
        assert lib.vr_batch_tune_describe(c, *[ctypes.byref(x) for x in v]) == 0
        tx, ty, px, py = (x.value for x in v)
        assert tx * ty == 256 and px * py == 32 and tx % px == 0 and ty % py == 0
        seen.add((tx, ty, px, py))
    assert len(seen) == n                      # no shape listed twice
    assert lib.vr_batch_tune_describe(n, None, None, None, None) != 0
    assert lib.vr_batch_tune_describe(-1, None, None, None, None) != 0
    saved = lib.vr_get_batch_config()
    try:
        assert lib.vr_set_batch_config(n - 1) == 0 and lib.vr_get_batch_config() == n - 1
        assert lib.vr_set_batch_config(n) != 0 and lib.vr_get_batch_config() == n - 1
    finally:
        lib.vr_set_batch_config(saved)


def test_library_storage_byte_queries_host_only():
    # what the library would allocate for texture storage and MIP bounds:
    # one texel per voxel of every slice (planes plus the two repeated edge
    # planes; pair texels one per cell plane), int8 decode records, 8-bit
    # bound code pairs (2 bytes per cell slice texel) plus the 32-byte scale
    # record
    from paper_1001_2049_b300 import mip_bounds_bytes, texture_bytes
    nx, ny, nz = 40, 36, 50
    assert texture_bytes((nx, ny, nz), "f32") == nx * ny * (nz + 2) * 4
    assert texture_bytes((nx, ny, nz), "f16") == nx * ny * (nz + 2) * 2
    assert texture_bytes((nx, ny, nz), "i8") == nx * ny * (nz + 2) + (nz + 2) * 8
    assert texture_bytes((nx, ny, nz), "f16", pair=True) == nx * ny * (nz + 1) * 4
    assert texture_bytes((nx, ny, nz), "i8", pair=True) == nx * ny * (nz + 1) * 2 + (nz + 1) * 16
    assert mip_bounds_bytes((nx, ny, nz)) == nx * ny * (nz + 1) * 2 + 32
    # deep cubes stack slices into at most 2048 layers (a power of two per
    # layer), each slice with a copy of its first and last rows: 4002 slices
    # -> 2 per layer, 4098 -> 4 per layer
    assert texture_bytes((64, 32, 4000), "f16") == 64 * (2 * (32 + 2)) * 2001 * 2
    assert texture_bytes((64, 32, 4096), "f16") == 64 * (4 * (32 + 2)) * 1025 * 2
    from paper_1001_2049_b300 import VRError
    with pytest.raises(VRError):
        texture_bytes((nx, ny, 50), "f32", pair=True)


def test_checked_build_exports_its_status_and_the_regular_one_refuses():
    import subprocess
    lib = _lib.load()
    flags = ctypes.c_uint(7)
    assert lib.vr_debug_status(ctypes.byref(flags), 0) == _lib.VR_ERR_UNSUPPORTED
    assert flags.value == 0
    path = build.build(debug=True)
    dbg = ctypes.CDLL(path)
    names = declared_functions()
    for n in names:
        assert hasattr(dbg, n), n
    # the regular library's kernels carry no checks: its objects were built
    # without VR_DEBUG (the checked library is a separate file)
    assert os.path.basename(path) == "libvr_debug.so" and path != build.LIB
