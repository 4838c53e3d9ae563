"""Helpers shared by the parity tests (no rendering arithmetic here)."""
from __future__ import annotations

import math

import numpy as np

import oracle

#: Tolerances (max abs per channel) of device images against the oracle.
#: FP32 arithmetic on FP32, or on decoded FP16/int8, voxels: 1e-4 (composite
#: RGBA in [0, 1]; MIP divided by the cube's max - min; SUM divided by the
#: larger of the image's largest |value| and, per pixel, 1 + M where
#: M = sum_k |s_k| step: the additive mode accumulates every sample's FP32
#: rounding -- of the sum itself and of the sample position, which grows with
#: the camera's distance -- so its error follows M, not the (possibly
#: cancelled) result).  Reduced-precision storage against the FP32 source
#: cube: 2e-3 (FP16) and 1e-2 (int8).
TOL_FP32 = 1e-4
TOL_PREC = {"f16": 2e-3, "i8": 1e-2}


def bands_for(dims, cams, step):
    """Tie bands for single-precision arithmetic on this geometry.

    The sample count K = floor((t_exit - t_entry)/step) + 1 moves when the
    quotient is within the rounding error of t_entry/t_exit (a few ulps of the
    largest distance involved) of an integer; positions of rays parallel to a
    face carry a few ulps of the camera coordinates.
    """
    eye = np.abs(np.asarray(cams["eye"], dtype=np.float64)).max()
    diag = math.sqrt(sum((d - 1.0) ** 2 for d in dims))
    t_scale = eye + diag + max(dims)
    ulp = 2.0 ** -23
    return oracle.Bands(band_k=2e-3 + 64 * ulp * t_scale / step,
                        band_pos=16 * ulp * max(1.0, t_scale),
                        band_clip=1e-4, band_a=1e-4)


def sum_scale(abs_volume: oracle.Volume, cams, w, h, step, image, pixels=None):
    """Per-pixel SUM scale: max(max |image|, 1 + M), M the oracle's SUM over
    |voxel values| (an upper bound of sum_k |s_k| step)."""
    flat = oracle.Volume(np.abs(abs_volume.data).astype(np.float32))
    tf = oracle.TF(np.array([[0, 0, 0, 0], [1, 1, 1, 1]], np.float32), 0, 1, 0)
    m = oracle.render(flat, cams, w, h, oracle.SUM, step, tf, pixels=pixels).primary[:, 0]
    fin = np.abs(image[np.isfinite(image)])
    img = max(1.0, float(fin.max()) if fin.size else 1.0)
    return np.maximum(img, 1.0 + m)


def compare(res: oracle.Result, got: np.ndarray, mode: int, tol: float, scale=1.0,
            what: str = ""):
    """Assert every pixel matches one member of its acceptance set; return a
    short report (max error, pixels flagged as ties).  ``scale`` is a number
    or one value per pixel."""
    ch = 4 if mode == oracle.COMPOSITE else 1
    got = np.asarray(got, dtype=np.float64).reshape(-1, ch)
    if np.ndim(scale):
        scale = np.asarray(scale, dtype=np.float64).reshape(-1, 1, 1)
    ok, err = oracle.match(res, got, tol, ch, scale)
    bad = np.flatnonzero(~ok)
    ties = int(np.count_nonzero(res.flags))
    if bad.size:
        i = bad[np.argmax(np.where(np.isfinite(err[bad]), err[bad], 1e30))]
        raise AssertionError(
            "%s: %d of %d pixels outside tol %g (worst pixel %d err %g, got %s, oracle %s, "
            "flags %d)" % (what, bad.size, got.shape[0], tol, i, err[i], got[i],
                           res.values[i, :max(1, res.nalt[i]), :ch], res.flags[i]))
    fin = err[np.isfinite(err)]
    return {"max_err": float(fin.max()) if fin.size else 0.0, "ties": ties,
            "pixels": int(got.shape[0])}
