"""Python front end of libvr: torch supplies device memory and streams, the
library does all the work.  Every call here marshals arguments to one C-ABI
entry point (include/vr.h) and returns torch tensors."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import VR_COMPOSITE, VR_F16, VR_F32, VR_I8, VR_MIP, VR_SUM, check, load

DTYPES = {"f32": VR_F32, "f16": VR_F16, "i8": VR_I8}
MODES = {"mip": VR_MIP, "composite": VR_COMPOSITE, "sum": VR_SUM}

#: One camera record (64 bytes), identical to ``vr_camera``.
CAMERA_DTYPE = np.dtype([
    ("proj", "<i4"), ("eye", "<f4", 3), ("fwd", "<f4", 3),
    ("du", "<f4", 3), ("dv", "<f4", 3), ("pad", "<f4", 3)])


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dims_arr(dims):
    return (ctypes.c_int64 * 3)(*[int(d) for d in dims])


class _Camera(ctypes.Structure):
    _fields_ = [("proj", ctypes.c_int32), ("eye", ctypes.c_float * 3), ("fwd", ctypes.c_float * 3),
                ("du", ctypes.c_float * 3), ("dv", ctypes.c_float * 3),
                ("reserved", ctypes.c_float * 3)]


class _Transfer(ctypes.Structure):
    _fields_ = [("rgba_lut", ctypes.c_void_p), ("n", ctypes.c_int32), ("v_lo", ctypes.c_float),
                ("v_hi", ctypes.c_float), ("clip", ctypes.c_float),
                ("term_alpha", ctypes.c_float)]


class _Request(ctypes.Structure):
    _fields_ = [("vol", ctypes.c_void_p), ("cam", _Camera), ("w", ctypes.c_int32),
                ("h", ctypes.c_int32), ("mode", ctypes.c_int32), ("step", ctypes.c_float),
                ("out", ctypes.c_void_p), ("tf", ctypes.c_void_p),
                ("samples", ctypes.c_void_p), ("done", ctypes.c_void_p),
                ("done_value", ctypes.c_uint32), ("row0", ctypes.c_int32),
                ("rows", ctypes.c_int32)]


assert ctypes.sizeof(_Camera) == 64 and ctypes.sizeof(_Request) == 136


@dataclass
class Request:
    """One view of one volume for ``render_batch``.  ``tf`` = (lut, v_lo,
    v_hi, clip, term_alpha) overrides the volume's transfer function;
    ``done`` = (int32 tensor, index) gets ``done_value`` when the image is
    complete (a pinned host tensor lets the host watch it).  ``band`` =
    (row0, rows) renders only those rows of the w x h image, into an ``out``
    of rows x w pixels (the same rays as the whole image's)."""
    volume: "Volume"
    cam: np.void
    w: int
    h: int
    mode: str = "composite"
    step: float = 0.5
    out: torch.Tensor | None = None
    tf: tuple | None = None
    samples: torch.Tensor | None = None
    done: tuple | None = None
    done_value: int = 1
    band: tuple | None = None


def render_init(out: torch.Tensor, mode: str, stream=None) -> torch.Tensor:
    """Fill images (views, h, w[, 4]) with the empty state of ``mode`` (0, or
    -inf for MIP) before rendering a cube part by part."""
    m = MODES[mode]
    if out.dtype != torch.float32 or not out.is_contiguous() or not out.is_cuda:
        raise ValueError("out must be a contiguous float32 CUDA tensor")
    views, h, w = out.shape[:3]
    check(load().vr_render_init(out.data_ptr(), views, w, h, m, _stream_ptr(stream)))
    return out


def integrate_partials(partials: torch.Tensor, cams: np.ndarray, mode: str,
                       out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Scene integration: ``partials`` (parts, views, h, w[, 4]), the
    sub-cubes' partial images in ascending z, combined per pixel in the
    order its ray meets them ("over" for composite, max for MIP, sum for
    SUM) into ``out`` (views, h, w[, 4])."""
    cams = np.ascontiguousarray(cams)
    m = MODES[mode]
    if partials.dtype != torch.float32 or not partials.is_contiguous() or not partials.is_cuda:
        raise ValueError("partials must be a contiguous float32 CUDA tensor")
    shape = tuple(partials.shape[1:])
    if len(shape) != (4 if m == VR_COMPOSITE else 3) or shape[0] != len(cams):
        raise ValueError("partials must be (parts, views, h, w%s)" % (", 4" if m == VR_COMPOSITE
                                                                      else ""))
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=partials.device)
    elif tuple(out.shape) != shape or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 tensor of shape %s" % (shape,))
    views, h, w = shape[:3]
    check(load().vr_integrate_partials(partials.data_ptr(), partials.shape[0], cams.ctypes.data,
                                       views, w, h, m, out.data_ptr(), _stream_ptr(stream)))
    return out


def batch_workspace(device=None) -> torch.Tensor:
    n = load().vr_batch_workspace_bytes()
    return torch.empty(n, dtype=torch.uint8, device=device or torch.device("cuda"))


def _batch_args(requests):
    """The vr_request array of ``requests`` (outputs allocated where a
    request has none), the objects it points into, and the outputs."""
    n = len(requests)
    arr = (_Request * max(n, 1))()
    keep, outs = [], []
    for i, rq in enumerate(requests):
        m = MODES[rq.mode]
        rows = rq.band[1] if rq.band is not None else rq.h
        shape = (rows, rq.w, 4) if m == VR_COMPOSITE else (rows, rq.w)
        out = rq.out
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=rq.volume.device)
        elif tuple(out.shape[-len(shape):]) != shape or out.numel() != int(np.prod(shape)):
            raise ValueError("request %d: out must hold %s floats" % (i, shape))
        outs.append(out)
        r = arr[i]
        r.vol = rq.volume.handle.value
        cam = np.ascontiguousarray(np.asarray(rq.cam).reshape(1))
        ctypes.memmove(ctypes.addressof(r.cam), cam.ctypes.data, 64)
        r.w, r.h, r.mode, r.step = rq.w, rq.h, m, float(rq.step)
        r.out = out.data_ptr()
        if rq.tf is not None:
            lut, v_lo, v_hi, clip, ta = rq.tf
            lut = np.ascontiguousarray(np.asarray(lut, dtype=np.float32))
            t = _Transfer(lut.ctypes.data, lut.shape[0], v_lo, v_hi, clip, ta)
            keep += [lut, t]
            r.tf = ctypes.addressof(t)
        if rq.samples is not None:
            r.samples = rq.samples.data_ptr()
        if rq.done is not None:
            flags, idx = rq.done
            r.done = flags.data_ptr() + 4 * int(idx)
            r.done_value = int(rq.done_value)
        if rq.band is not None:
            r.row0, r.rows = int(rq.band[0]), int(rq.band[1])
    return arr, keep, outs


def render_batch(requests, workspace: torch.Tensor | None = None, stream=None):
    """Render every request with the batched persistent kernel; returns the
    output tensors (allocated here when a request has none)."""
    arr, keep, outs = _batch_args(requests)
    if workspace is None:
        workspace = batch_workspace(outs[0].device if outs else None)
    check(load().vr_render_batch(arr, len(requests), workspace.data_ptr(), workspace.numel(),
                                 _stream_ptr(stream)))
    del keep
    return outs


def batch_shapes():
    """The batched launch's tile and ray-packet shapes: (tile_x, tile_y,
    packet_x, packet_y) per configuration index."""
    lib = load()
    out = []
    for c in range(lib.vr_batch_tune_count()):
        v = [ctypes.c_int(0) for _ in range(4)]
        check(lib.vr_batch_tune_describe(c, *[ctypes.byref(x) for x in v]))
        out.append(tuple(x.value for x in v))
    return out


def set_batch_config(cfg: int):
    """Use batch shape ``cfg`` for every later batched render of the process."""
    check(load().vr_set_batch_config(int(cfg)))


def get_batch_config() -> int:
    return int(load().vr_get_batch_config())


def batch_autotune(requests, workspace: torch.Tensor | None = None, stream=None):
    """Time every batch shape on these requests (their images are written)
    and keep the fastest for the process; returns (config, ms)."""
    arr, keep, outs = _batch_args(requests)
    if workspace is None:
        workspace = batch_workspace(outs[0].device if outs else None)
    best, ms = ctypes.c_int(0), ctypes.c_float(0.0)
    check(load().vr_batch_autotune(arr, len(requests), workspace.data_ptr(), workspace.numel(),
                                   _stream_ptr(stream), ctypes.byref(best), ctypes.byref(ms)))
    del keep
    return int(best.value), float(ms.value)


def launch_shapes():
    """The texture kernel's launch shapes: (block_x, block_y, packet_x,
    packet_y, min_blocks) per configuration index."""
    lib = load()
    out = []
    for c in range(lib.vr_tune_count()):
        v = [ctypes.c_int(0) for _ in range(5)]
        check(lib.vr_tune_describe(c, *[ctypes.byref(x) for x in v]))
        out.append(tuple(x.value for x in v))
    return out


def volume_bytes(dims, dtype="f32") -> int:
    out = ctypes.c_size_t(0)
    check(load().vr_volume_bytes(_dims_arr(dims), DTYPES[dtype], ctypes.byref(out)))
    return out.value


def texture_bytes(dims, dtype="f32", pair=False) -> int:
    """Device bytes of the texture storage the library allocates on
    attach_texture (pair=True: attach_pair_texture) for such a cube."""
    out = ctypes.c_size_t(0)
    check(load().vr_texture_bytes(_dims_arr(dims), DTYPES[dtype], int(bool(pair)),
                                  ctypes.byref(out)))
    return out.value


def mip_bounds_bytes(dims) -> int:
    """Device bytes of the MIP bounds the library allocates on
    attach_mip_bounds for an FP32 cube of these dims."""
    out = ctypes.c_size_t(0)
    check(load().vr_mip_bounds_bytes(_dims_arr(dims), ctypes.byref(out)))
    return out.value


class Volume:
    """A spectral cube resident on the GPU in the library's brick layout.

    ``cube`` is a float32 tensor of shape (nz, ny, nx) (x = RA fastest, z =
    frequency slowest) on the current CUDA device or in pinned host memory;
    ``dtype`` is the storage type ("f32", "f16" or "i8").  The brick buffer
    is a torch allocation owned by this object, or ``buffer`` (a uint8
    device tensor of at least volume_bytes(dims, dtype)).  Volumes may share
    one buffer, as the part volumes of stream.PartStream do: an upload
    repacks the buffer and refreshes only its own volume's texture, so such
    volumes render from their textures and must not upload concurrently.
    """

    def __init__(self, cube: torch.Tensor | None = None, dtype: str = "f32", dims=None,
                 stream=None, device=None, buffer: torch.Tensor | None = None):
        lib = load()
        if cube is not None:
            if cube.dtype != torch.float32 or cube.dim() != 3:
                raise ValueError("cube must be a 3-D float32 tensor (nz, ny, nx)")
            cube = cube.contiguous()
            nz, ny, nx = cube.shape
            dims = (nx, ny, nz)
        if dims is None:
            raise ValueError("need a cube or dims")
        self.dims = tuple(int(d) for d in dims)
        self.dtype = dtype
        self.nbytes = volume_bytes(self.dims, dtype)
        if buffer is not None:
            if buffer.dtype != torch.uint8 or not buffer.is_cuda or buffer.numel() < self.nbytes:
                raise ValueError("buffer must be a uint8 CUDA tensor of at least %d bytes"
                                 % self.nbytes)
            dev = buffer.device
        else:
            dev = device if device is not None else (
                cube.device if cube is not None and cube.is_cuda else torch.device("cuda"))
        self.device = torch.device(dev)
        self.buffer = buffer if buffer is not None else torch.empty(self.nbytes, dtype=torch.uint8,
                                                                    device=dev)
        handle = ctypes.c_void_p(0)
        src, on_dev = None, 1
        if cube is not None:
            src, on_dev = cube.data_ptr(), int(cube.is_cuda)
        check(lib.vr_volume_create(_dims_arr(self.dims), DTYPES[dtype], src, on_dev,
                                   self.buffer.data_ptr(), self.nbytes, _stream_ptr(stream),
                                   ctypes.byref(handle)))
        self._h = handle
        self._keep = cube   # the source must live until the stream passes the pack

    @property
    def handle(self):
        return self._h

    def upload(self, z0: int, planes: torch.Tensor, stream=None):
        """Pack planes [z0, z0 + planes.shape[0]) from a float32 (n, ny, nx)
        tensor (device or pinned host)."""
        planes = planes.contiguous()
        check(load().vr_volume_upload(self._h, int(z0), int(planes.shape[0]), planes.data_ptr(),
                                      int(planes.is_cuda), _stream_ptr(stream)))
        self._keep = planes

    def attach_texture(self, stream=None):
        """Also hold the cube as layered textures (library-owned device memory
        of the cube's size); renders then use the texture-gather kernel."""
        check(load().vr_volume_attach_texture(self._h, _stream_ptr(stream)))

    def attach_pair_texture(self, stream=None):
        """FP16 / int8 volumes: texture storage whose texels pack a voxel with
        its neighbour in the next plane, so one gather yields a whole cell
        (twice the bytes of attach_texture)."""
        check(load().vr_volume_attach_pair_texture(self._h, _stream_ptr(stream)))

    def detach_texture(self):
        check(load().vr_volume_detach_texture(self._h))

    def attach_mip_bounds(self, stream=None):
        """FP32 volumes with texture storage: 8-bit upper-bound codes of the
        voxels on one scale for the whole cube, two planes per texel
        (library-owned, about 2 bytes per voxel); MIP renders then read the
        FP32 texels only where a sample could raise the maximum, with
        identical images.  An upload of every plane derives the scale again;
        a partial upload with values outside the cube's range turns the
        skipping off (still identical images) until the bounds are attached
        again."""
        check(load().vr_volume_attach_mip_bounds(self._h, _stream_ptr(stream)))

    def detach_mip_bounds(self):
        check(load().vr_volume_detach_mip_bounds(self._h))

    def drop_bricks(self, stream=None):
        """Keep only the texture storage and free the brick buffer (after the
        work queued on ``stream`` has finished); the volume becomes
        read-only."""
        check(load().vr_volume_drop_bricks(self._h))
        (stream or torch.cuda.current_stream(self.device)).synchronize()
        self.buffer = None
        self._keep = None

    def device_bytes(self):
        """(library-owned, caller-owned) device bytes this volume holds now:
        texture storage and MIP bounds; the brick buffer and the masks."""
        lib_b, caller_b = ctypes.c_size_t(0), ctypes.c_size_t(0)
        check(load().vr_volume_device_bytes(self._h, ctypes.byref(lib_b), ctypes.byref(caller_b)))
        return int(lib_b.value), int(caller_b.value)

    def mask_bytes(self) -> int:
        n = ctypes.c_size_t(0)
        check(load().vr_volume_mask_bytes(self._h, ctypes.byref(n)))
        return int(n.value)

    def attach_masks(self):
        """Empty-space masks (8 bytes per 4^3-cell macrocell, in a torch-owned
        device buffer kept by this object): composite renders then skip the
        samples the clip makes transparent, with identical results."""
        buf = torch.empty(max(1, self.mask_bytes() // 8), dtype=torch.int64,
                          device=self.device)
        check(load().vr_volume_attach_masks(self._h, buf.data_ptr(), buf.numel() * 8))
        self._masks = buf
        return buf

    def detach_masks(self):
        check(load().vr_volume_attach_masks(self._h, None, 0))
        self._masks = None

    def build_masks(self, stream=None):
        """Build the attached masks now, for the current clip, on ``stream``
        (for volumes whose brick buffer will soon hold other data)."""
        check(load().vr_volume_build_masks(self._h, _stream_ptr(stream)))

    def set_transfer(self, lut, v_lo: float, v_hi: float, clip: float, term_alpha: float = 1.0):
        """RGBA table (n, 4) with alpha per unit voxel length over [v_lo, v_hi];
        samples below ``clip`` are transparent; rays stop at ``term_alpha``."""
        lut = np.ascontiguousarray(np.asarray(lut, dtype=np.float32))
        if lut.ndim != 2 or lut.shape[1] != 4:
            raise ValueError("lut must have shape (n, 4)")
        check(load().vr_set_transfer(self._h, lut.ctypes.data, lut.shape[0], float(v_lo),
                                     float(v_hi), float(clip), float(term_alpha)))

    def render(self, cams: np.ndarray, w: int, h: int, mode: str = "composite",
               step: float = 0.5, out: torch.Tensor | None = None, stream=None,
               count: torch.Tensor | None = None) -> torch.Tensor:
        """Render len(cams) views.  Returns (views, h, w) for "mip"/"sum" and
        (views, h, w, 4) premultiplied RGBA for "composite".  ``count``, a
        one-element int64 CUDA tensor, receives the evaluated-sample count
        (added to its value)."""
        cams = np.ascontiguousarray(cams)
        if cams.dtype.itemsize != 64:
            raise ValueError("cams must be an array of 64-byte camera records")
        m = MODES[mode]
        shape = (len(cams), h, w, 4) if m == VR_COMPOSITE else (len(cams), h, w)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=self.device)
        elif tuple(out.shape) != shape or out.dtype != torch.float32 or not out.is_contiguous():
            raise ValueError("out must be a contiguous float32 tensor of shape %s" % (shape,))
        lib = load()
        if count is None:
            check(lib.vr_render(self._h, cams.ctypes.data, len(cams), w, h, m, float(step),
                                out.data_ptr(), _stream_ptr(stream)))
        else:
            if count.dtype != torch.int64 or not count.is_cuda:
                raise ValueError("count must be an int64 CUDA tensor")
            check(lib.vr_render_counted(self._h, cams.ctypes.data, len(cams), w, h, m,
                                        float(step), out.data_ptr(), count.data_ptr(),
                                        _stream_ptr(stream)))
        return out

    def render_object_order(self, cams: np.ndarray, w: int, h: int, mode: str = "mip",
                            step: float = 0.5, out: torch.Tensor | None = None, stream=None,
                            count: torch.Tensor | None = None) -> torch.Tensor:
        """MIP of len(cams) views in object order (vr_render_object_order):
        sub-cubes of 32^3 cells staged in shared memory once for all views,
        the same images and counts as ``render(..., "mip")``.  Returns
        (views, h, w); ``count`` as in render."""
        cams = np.ascontiguousarray(cams)
        if cams.dtype.itemsize != 64:
            raise ValueError("cams must be an array of 64-byte camera records")
        m = MODES[mode]
        shape = (len(cams), h, w)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=self.device)
        elif tuple(out.shape) != shape or out.dtype != torch.float32 or not out.is_contiguous():
            raise ValueError("out must be a contiguous float32 tensor of shape %s" % (shape,))
        if count is not None and (count.dtype != torch.int64 or not count.is_cuda):
            raise ValueError("count must be an int64 CUDA tensor")
        check(load().vr_render_object_order(self._h, cams.ctypes.data, len(cams), w, h, m,
                                            float(step), out.data_ptr(),
                                            count.data_ptr() if count is not None else None,
                                            _stream_ptr(stream)))
        return out

    def render_part(self, full_dims, z_first: int, cell_lo: int, cell_hi: int, cams: np.ndarray,
                    w: int, h: int, mode: str, step: float, sweep: int, out: torch.Tensor,
                    count: torch.Tensor | None = None, stream=None):
        """This volume holds planes [z_first, z_first + nz) of a cube of
        ``full_dims``: continue ``out`` (from render_init or earlier parts)
        with the samples of cells [cell_lo, cell_hi) of the rays going up
        (sweep +1), down (sweep -1) or both (0: a partial image for
        integrate_partials)."""
        cams = np.ascontiguousarray(cams)
        m = MODES[mode]
        shape = (len(cams), h, w, 4) if m == VR_COMPOSITE else (len(cams), h, w)
        if tuple(out.shape) != shape or out.dtype != torch.float32 or not out.is_contiguous():
            raise ValueError("out must be a contiguous float32 tensor of shape %s" % (shape,))
        if count is not None and (count.dtype != torch.int64 or not count.is_cuda):
            raise ValueError("count must be an int64 CUDA tensor")
        check(load().vr_render_part(self._h, _dims_arr(full_dims), int(z_first), int(cell_lo),
                                    int(cell_hi), cams.ctypes.data, len(cams), w, h, m,
                                    float(step), int(sweep), out.data_ptr(),
                                    count.data_ptr() if count is not None else None,
                                    _stream_ptr(stream)))
        return out

    def autotune(self, cams: np.ndarray, w: int, h: int, mode: str = "composite",
                 step: float = 0.5, out: torch.Tensor | None = None, stream=None):
        """Time the texture kernel's launch shapes on this render and keep the
        fastest for ``mode``; returns (configuration, ms).  Synchronises."""
        cams = np.ascontiguousarray(cams)
        m = MODES[mode]
        shape = (len(cams), h, w, 4) if m == VR_COMPOSITE else (len(cams), h, w)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=self.device)
        best, ms = ctypes.c_int(0), ctypes.c_float(0)
        check(load().vr_autotune(self._h, cams.ctypes.data, len(cams), w, h, m, float(step),
                                 out.data_ptr(), _stream_ptr(stream), ctypes.byref(best),
                                 ctypes.byref(ms)))
        return best.value, ms.value

    def set_launch_config(self, mode: str, cfg: int):
        check(load().vr_set_launch_config(self._h, MODES[mode], int(cfg)))

    def close(self):
        if getattr(self, "_h", None):
            load().vr_volume_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
