"""ctypes declarations of libvr's C ABI (include/vr.h).  Argument marshalling
only: every step of the render path runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

VR_OK = 0
VR_ERR_ARG, VR_ERR_OOM, VR_ERR_CUDA, VR_ERR_TIMEOUT, VR_ERR_UNSUPPORTED = -1, -2, -3, -4, -5
VR_F32, VR_F16, VR_I8 = 0, 1, 2
VR_MIP, VR_COMPOSITE, VR_SUM = 0, 1, 2
VR_ORTHO, VR_PERSP = 0, 1
VR_MAX_LUT = 256

c_void_p, c_int, c_int64, c_size_t, c_float = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                              ctypes.c_size_t, ctypes.c_float)

#: Exported symbols and their (restype, argtypes); must match include/vr.h.
SIGNATURES = {
    "vr_version": (c_int, []),
    "vr_last_error": (ctypes.c_char_p, []),
    "vr_volume_bytes": (c_int, [ctypes.POINTER(c_int64), c_int, ctypes.POINTER(c_size_t)]),
    "vr_texture_bytes": (c_int, [ctypes.POINTER(c_int64), c_int, c_int,
                                 ctypes.POINTER(c_size_t)]),
    "vr_mip_bounds_bytes": (c_int, [ctypes.POINTER(c_int64), ctypes.POINTER(c_size_t)]),
    "vr_volume_device_bytes": (c_int, [c_void_p, ctypes.POINTER(c_size_t),
                                       ctypes.POINTER(c_size_t)]),
    "vr_volume_create": (c_int, [ctypes.POINTER(c_int64), c_int, c_void_p, c_int, c_void_p,
                                 c_size_t, c_void_p, ctypes.POINTER(c_void_p)]),
    "vr_volume_upload": (c_int, [c_void_p, c_int64, c_int64, c_void_p, c_int, c_void_p]),
    "vr_set_transfer": (c_int, [c_void_p, c_void_p, c_int, c_float, c_float, c_float, c_float]),
    "vr_render": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_float, c_void_p,
                          c_void_p]),
    "vr_render_counted": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_float,
                                  c_void_p, c_void_p, c_void_p]),
    "vr_render_object_order": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int,
                                       c_float, c_void_p, c_void_p, c_void_p]),
    "vr_volume_destroy": (c_int, [c_void_p]),
    "vr_volume_attach_texture": (c_int, [c_void_p, c_void_p]),
    "vr_volume_mask_bytes": (c_int, [c_void_p, ctypes.POINTER(c_size_t)]),
    "vr_volume_attach_masks": (c_int, [c_void_p, c_void_p, c_size_t]),
    "vr_volume_attach_pair_texture": (c_int, [c_void_p, c_void_p]),
    "vr_volume_detach_texture": (c_int, [c_void_p]),
    "vr_volume_attach_mip_bounds": (c_int, [c_void_p, c_void_p]),
    "vr_volume_build_masks": (c_int, [c_void_p, c_void_p]),
    "vr_volume_detach_mip_bounds": (c_int, [c_void_p]),
    "vr_volume_drop_bricks": (c_int, [c_void_p]),
    "vr_render_init": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p]),
    "vr_integrate_partials": (c_int, [c_void_p, c_int, c_void_p, c_int, c_int, c_int, c_int,
                                      c_void_p, c_void_p]),
    "vr_render_part": (c_int, [c_void_p, ctypes.POINTER(c_int64), c_int64, c_int64, c_int64,
                               c_void_p, c_int, c_int, c_int, c_int, c_float, c_int, c_void_p,
                               c_void_p, c_void_p]),
    "vr_volume_info": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int),
                               ctypes.POINTER(c_void_p)]),
    "vr_batch_workspace_bytes": (c_size_t, []),
    "vr_render_batch": (c_int, [c_void_p, c_int, c_void_p, c_size_t, c_void_p]),
    "vr_render_batch_noalloc": (c_int, [c_void_p, c_int, c_void_p]),
    "vr_batch_tune_count": (c_int, []),
    "vr_batch_tune_describe": (c_int, [c_int] + [ctypes.POINTER(c_int)] * 4),
    "vr_set_batch_config": (c_int, [c_int]),
    "vr_get_batch_config": (c_int, []),
    "vr_batch_autotune": (c_int, [c_void_p, c_int, c_void_p, c_size_t, c_void_p,
                                  ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_float)]),
    "vr_tune_count": (c_int, []),
    "vr_tune_describe": (c_int, [c_int] + [ctypes.POINTER(c_int)] * 5),
    "vr_autotune": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_float, c_void_p,
                            c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_float)]),
    "vr_set_launch_config": (c_int, [c_void_p, c_int, c_int]),
    "vr_debug_status": (c_int, [ctypes.POINTER(ctypes.c_uint), c_int]),
}


class VRError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libvr error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load() -> ctypes.CDLL:
    """Load libvr.so (building it first when it is missing or older than its
    sources; with VR_DEBUG=1 in the environment, the checked libvr_debug.so).
    Raises if it cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is None:
        debug = os.environ.get("VR_DEBUG") == "1"
        path = _build.DEBUG_LIB if debug else _build.LIB
        if _build.stale(path):
            path = _build.build(debug=debug)
        if not os.path.exists(path):
            raise ImportError("libvr.so is missing and could not be built")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(rc: int) -> None:
    if rc != VR_OK:
        raise VRError(rc, load().vr_last_error().decode(errors="replace"))
