"""FP64 CPU oracle for the spectral-cube ray caster.

TEST INFRASTRUCTURE.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
package.  It shares no code with the CUDA path (``paper_1001_2049_b300``):
the C source ``vr_oracle.c`` is compiled here with gcc and called through
ctypes; quantisation for the reduced-precision storage formats lives in
``quantize.py``; ``brute.py`` is an exact rational re-derivation used to pin
this oracle on tiny inputs.

Every function follows the rendering definition stated at the top of
``vr_oracle.c`` (paper §3.1, process item 3, with the readings this project
fixes for the steps the paper leaves open).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vr_oracle.c")
_LIB = os.path.join(_HERE, "libvr_oracle.so")

MIP, COMPOSITE, SUM = 0, 1, 2
F32, F16, I8 = 0, 1, 2

CAMERA_DTYPE = np.dtype([
    ("proj", "<i4"), ("eye", "<f4", 3), ("fwd", "<f4", 3),
    ("du", "<f4", 3), ("dv", "<f4", 3), ("pad", "<f4", 3)])


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) if it is missing or stale."""
    if (force or not os.path.exists(_LIB)
            or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Volume(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64 * 3), ("dtype", ctypes.c_int32),
                ("data", ctypes.c_void_p), ("scale", ctypes.c_void_p),
                ("offset", ctypes.c_void_p)]


class _TF(ctypes.Structure):
    _fields_ = [("lut", ctypes.c_void_p), ("n_lut", ctypes.c_int32),
                ("v_lo", ctypes.c_double), ("v_hi", ctypes.c_double),
                ("clip", ctypes.c_double), ("term_alpha", ctypes.c_double)]


class _Bands(ctypes.Structure):
    _fields_ = [("band_k", ctypes.c_double), ("band_pos", ctypes.c_double),
                ("band_clip", ctypes.c_double), ("band_a", ctypes.c_double),
                ("band_t", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.vro_render.restype = ctypes.c_int
        _lib.vro_render.argtypes = [
            ctypes.POINTER(_Volume), ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
            ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_TF),
            ctypes.POINTER(_Bands), ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int]
        _lib.vro_render_subcubes.restype = ctypes.c_int
        _lib.vro_render_subcubes.argtypes = [
            ctypes.POINTER(_Volume), ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
            ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_TF),
            ctypes.POINTER(_Bands), ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        _lib.vro_render_partial.restype = ctypes.c_int
        _lib.vro_render_partial.argtypes = [
            ctypes.POINTER(_Volume), ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
            ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_TF),
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_int]
        _lib.vro_maxalt.restype = ctypes.c_int
        _lib.vro_num_threads.restype = ctypes.c_int
        _lib.vro_sample_at.restype = ctypes.c_double
        _lib.vro_sample_at.argtypes = [ctypes.POINTER(_Volume), ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double]
        _lib.vro_classify.restype = None
        _lib.vro_classify.argtypes = [ctypes.POINTER(_TF), ctypes.c_double,
                                      ctypes.c_double, ctypes.c_void_p]
        _lib.vro_half_to_double.restype = ctypes.c_double
        _lib.vro_half_to_double.argtypes = [ctypes.c_uint16]
    return _lib


def maxalt() -> int:
    return lib().vro_maxalt()


def num_threads() -> int:
    return lib().vro_num_threads()


@dataclass
class Volume:
    """A cube in plain linear layout, shape (nz, ny, nx), for the oracle.

    ``data`` is float32 values, float16 values (their bits are decoded by the
    oracle) or int8 codes with per-plane ``scale``/``offset`` float32 arrays.
    """
    data: np.ndarray
    scale: np.ndarray | None = None
    offset: np.ndarray | None = None

    def _c(self):
        d = np.ascontiguousarray(self.data)
        if d.dtype == np.float32:
            dt = F32
        elif d.dtype == np.float16:
            dt = F16
        elif d.dtype == np.int8:
            dt = I8
        else:
            raise TypeError("oracle volume must be float32, float16 or int8")
        nz, ny, nx = d.shape
        v = _Volume()
        v.n[0], v.n[1], v.n[2] = nx, ny, nz
        v.dtype = dt
        v.data = d.ctypes.data
        keep = [d]
        if dt == I8:
            sc = np.ascontiguousarray(self.scale, dtype=np.float32)
            of = np.ascontiguousarray(self.offset, dtype=np.float32)
            assert sc.shape == (nz,) and of.shape == (nz,)
            v.scale, v.offset = sc.ctypes.data, of.ctypes.data
            keep += [sc, of]
        return v, keep


@dataclass
class TF:
    """Raw RGBA table (n, 4) float32 with alpha per unit voxel length, the
    value domain [v_lo, v_hi], the clip level and the termination alpha."""
    lut: np.ndarray
    v_lo: float
    v_hi: float
    clip: float
    term_alpha: float = 1.0

    def _c(self):
        lut = np.ascontiguousarray(self.lut, dtype=np.float32)
        assert lut.ndim == 2 and lut.shape[1] == 4
        t = _TF()
        t.lut = lut.ctypes.data
        t.n_lut = lut.shape[0]
        t.v_lo, t.v_hi = float(self.v_lo), float(self.v_hi)
        t.clip, t.term_alpha = float(self.clip), float(self.term_alpha)
        return t, [lut]


@dataclass
class Bands:
    """Widths of the tie bands around the three discontinuities (see the
    header of ``vr_oracle.c``): ``band_k`` an absolute floor of the K band,
    ``band_pos`` the absolute error of a ray origin, ``band_clip`` the
    relative error of an interpolated value (per unit of its largest
    |corner|), ``band_a`` the termination band in alpha, ``band_t`` the
    relative error of a ray parameter t (0: the K band is band_k alone)."""
    band_k: float = 2e-3
    band_pos: float = 1e-5
    band_clip: float = 1e-4
    band_a: float = 1e-4
    band_t: float = 0.0

    def _c(self):
        return _Bands(self.band_k, self.band_pos, self.band_clip, self.band_a, self.band_t)


#: Units of 2^-24 (half an ulp at 1) of the rounding a single-precision
#: evaluation of the definition makes, as the bands model it:
#:  * a ray parameter t = (plane - o_a) / d_a: the division (1), the
#:    direction component d_a from fwd + u du + v dv in two fused steps and
#:    the normalisation (about 3 of |d| = 1, which the oracle divides by the
#:    deciding |d_a|), the subtraction t_exit - t_entry (1), one of slack: 6;
#:  * an orthographic origin eye + u du + v dv in two fused steps: 2 of the
#:    largest term, doubled: 4;
#:  * an interpolated value: three levels of lerps fma(f, b - a, a), each
#:    rounding b - a and the fused step (3 of the largest |corner| per
#:    level, 9 in all), the int8 decode of each plane's value (2 more),
#:    rounded up: 16.
FP32_T_UNITS = 6.0
FP32_ORIGIN_UNITS = 4.0
FP32_VALUE_UNITS = 16.0


def fp32_bands(dims, cams, step, w=None, h=None, band_a=1e-4) -> "Bands":
    """Tie bands for a single-precision evaluation of these views (see the
    header of ``vr_oracle.c`` for how each band enters the decisions).

    ``band_a`` is the termination band in alpha: a result whose alpha is
    within the image tolerance of the oracle's can take the other
    termination decision only where the oracle's alpha is within that
    tolerance of the threshold, so the tests pass their tolerance (1e-4)."""
    u = 2.0 ** -24
    half = max(w or 0, h or 0) / 2.0 if (w or h) else 2.0 * max(dims)
    scale = 1.0            # a perspective origin is the eye itself, exactly
    for c in np.asarray(cams):
        if int(c["proj"]) == 0:   # orthographic: eye + u du + v dv, rounded
            scale = max(scale, float(np.abs(c["eye"]).max()) + 1.0
                        + half * (float(np.abs(c["du"]).max()) + float(np.abs(c["dv"]).max())))
    origin = FP32_ORIGIN_UNITS * u * scale
    return Bands(band_k=2.0 ** -20, band_pos=origin, band_clip=FP32_VALUE_UNITS * u,
                 band_a=band_a, band_t=FP32_T_UNITS * u)


@dataclass
class Result:
    values: np.ndarray    # (npix, MAXALT, 4) float64; [:, 0] is primary
    nalt: np.ndarray      # (npix,) int32
    flags: np.ndarray     # (npix,) int32
    nsamples: np.ndarray  # (npix,) int64

    @property
    def primary(self):
        return self.values[:, 0, :]


def render(volume: Volume, cams: np.ndarray, w: int, h: int, mode: int,
           step: float, tf: TF, pixels: np.ndarray | None = None,
           bands: Bands | None = None, nthreads: int = 0) -> Result:
    """Render the given pixels ((view, px, py) int rows) or every pixel of
    every view (view-major, then row, then column) when ``pixels`` is None."""
    cams = np.ascontiguousarray(cams)
    assert cams.dtype.itemsize == 64
    n_views = cams.shape[0]
    if pixels is None:
        v, py, px = np.meshgrid(np.arange(n_views), np.arange(h), np.arange(w),
                                indexing="ij")
        pixels = np.stack([v.ravel(), px.ravel(), py.ravel()], axis=1)
    pixels = np.ascontiguousarray(pixels, dtype=np.int32)
    npix = pixels.shape[0]
    bands = bands or Bands()
    m = maxalt()
    out = np.zeros((npix, m, 4), dtype=np.float64)
    nalt = np.zeros(npix, dtype=np.int32)
    flags = np.zeros(npix, dtype=np.int32)
    nsam = np.zeros(npix, dtype=np.int64)
    cv, keep_v = volume._c()
    ct, keep_t = tf._c()
    cb = bands._c()
    rc = lib().vro_render(ctypes.byref(cv), cams.ctypes.data, n_views, w, h, mode,
                          float(step), ctypes.byref(ct), ctypes.byref(cb),
                          pixels.ctypes.data, npix, out.ctypes.data,
                          nalt.ctypes.data, flags.ctypes.data, nsam.ctypes.data,
                          int(nthreads))
    del keep_v, keep_t
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return Result(out, nalt, flags, nsam)


def render_subcubes(volume: Volume, cams: np.ndarray, w: int, h: int, mode: int,
                    step: float, tf: TF, cell_lo, pixels: np.ndarray | None = None,
                    bands: Bands | None = None, nthreads: int = 0) -> Result:
    """The pixels rendered as sub-cubes (sub-cube i owns the cells
    [cell_lo[i], cell_lo[i+1]) along z; cell_lo[0] = 0), each into its own
    partial result from an empty start, combined in the order each ray meets
    them ("over" for composite, max for MIP, sum for SUM): the paper's
    sub-cube pipeline (§3.1 items 1, 4, 5).  Returns a Result as ``render``
    (``nsamples`` zero): the primary FP64 result and the alternatives of the
    tie bands; flags bit 0 K tie, 1 clip tie, 2 termination tie, 3 list
    truncated, 4 a sample on a sub-cube boundary plane up to rounding."""
    cams = np.ascontiguousarray(cams)
    assert cams.dtype.itemsize == 64
    n_views = cams.shape[0]
    if pixels is None:
        v, py, px = np.meshgrid(np.arange(n_views), np.arange(h), np.arange(w),
                                indexing="ij")
        pixels = np.stack([v.ravel(), px.ravel(), py.ravel()], axis=1)
    pixels = np.ascontiguousarray(pixels, dtype=np.int32)
    npix = pixels.shape[0]
    lo = np.ascontiguousarray(cell_lo, dtype=np.int64)
    bands = bands or Bands()
    m = maxalt()
    out = np.zeros((npix, m, 4), dtype=np.float64)
    nalt = np.zeros(npix, dtype=np.int32)
    flags = np.zeros(npix, dtype=np.int32)
    cv, keep_v = volume._c()
    ct, keep_t = tf._c()
    cb = bands._c()
    rc = lib().vro_render_subcubes(ctypes.byref(cv), cams.ctypes.data, n_views, w, h, mode,
                                   float(step), ctypes.byref(ct), ctypes.byref(cb),
                                   lo.ctypes.data, int(lo.size), pixels.ctypes.data, npix,
                                   out.ctypes.data, nalt.ctypes.data, flags.ctypes.data,
                                   int(nthreads))
    del keep_v, keep_t
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return Result(out, nalt, flags, np.zeros(npix, dtype=np.int64))


def render_partial(volume: Volume, cams: np.ndarray, w: int, h: int, mode: int,
                   step: float, tf: TF, cell_lo, part: int,
                   pixels: np.ndarray | None = None, nthreads: int = 0) -> np.ndarray:
    """Sub-cube ``part`` of the split ``cell_lo`` rendered alone into its
    partial result (the primary FP64 values, (npix, 4): composite (C, A);
    MIP / SUM in channel 0), from an empty start, stopping at its own
    opacity -- what one node renders before scene integration (§3.1 item
    4)."""
    cams = np.ascontiguousarray(cams)
    assert cams.dtype.itemsize == 64
    n_views = cams.shape[0]
    if pixels is None:
        v, py, px = np.meshgrid(np.arange(n_views), np.arange(h), np.arange(w),
                                indexing="ij")
        pixels = np.stack([v.ravel(), px.ravel(), py.ravel()], axis=1)
    pixels = np.ascontiguousarray(pixels, dtype=np.int32)
    npix = pixels.shape[0]
    lo = np.ascontiguousarray(cell_lo, dtype=np.int64)
    out = np.zeros((npix, 4), dtype=np.float64)
    cv, keep_v = volume._c()
    ct, keep_t = tf._c()
    rc = lib().vro_render_partial(ctypes.byref(cv), cams.ctypes.data, n_views, w, h, mode,
                                  float(step), ctypes.byref(ct), lo.ctypes.data, int(lo.size),
                                  int(part), pixels.ctypes.data, npix, out.ctypes.data,
                                  int(nthreads))
    del keep_v, keep_t
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return out


def sample_at(volume: Volume, x: float, y: float, z: float) -> float:
    """One trilinear sample at a point (clamped to the box)."""
    cv, keep = volume._c()
    r = lib().vro_sample_at(ctypes.byref(cv), x, y, z)
    del keep
    return r


def classify(tf: TF, step: float, s: float) -> np.ndarray:
    """RGBA of one value through the opacity-corrected table."""
    ct, keep = tf._c()
    out = np.zeros(4, dtype=np.float64)
    lib().vro_classify(ctypes.byref(ct), float(step), float(s), out.ctypes.data)
    del keep
    return out


def half_to_double(bits: int) -> float:
    return lib().vro_half_to_double(bits)


def match(result: Result, got: np.ndarray, tol: float, channels: int,
          scale: float = 1.0):
    """Compare a device result with the oracle's acceptance sets.

    ``got`` is (npix, channels).  A pixel passes when, for some acceptable
    result a, max_c |got - value_a| / scale <= tol (``scale`` a number, or an
    (npix, 1, 1) array of per-pixel scales); for MIP a -infinity
    primary (a miss) must be matched exactly.  When the alternative list was
    truncated (flag 8) the pixel also passes if every channel lies within the
    per-channel range spanned by the listed alternatives (widened by tol),
    since accumulated colour and alpha never decrease along the ray.
    Returns (ok mask, per-pixel best error).
    """
    got = np.asarray(got, dtype=np.float64).reshape(-1, channels)
    vals = result.values[:, :, :channels]
    npix, m, _ = vals.shape
    valid = np.arange(m)[None, :] < result.nalt[:, None]
    with np.errstate(invalid="ignore"):
        diff = np.abs(got[:, None, :] - vals)
        same_inf = np.isinf(got[:, None, :]) & (got[:, None, :] == vals)
        diff = np.where(same_inf, 0.0, diff)
        diff = np.where(np.isnan(diff), np.inf, diff) / scale
    err = np.where(valid, diff.max(axis=2), np.inf).min(axis=1)
    ok = err <= tol
    trunc = (result.flags & 8) != 0
    if trunc.any():
        sc = np.asarray(scale, dtype=np.float64).reshape(-1, 1) if np.ndim(scale) else scale
        lo = np.where(valid[:, :, None], vals, np.inf).min(axis=1) - tol * sc
        hi = np.where(valid[:, :, None], vals, -np.inf).max(axis=1) + tol * sc
        inside = ((got >= lo) & (got <= hi)).all(axis=1)
        ok = ok | (trunc & inside)
    return ok, err
