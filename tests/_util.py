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


def bands_for(dims, cams, step, w=None, h=None):
    """Tie bands for single-precision arithmetic on this geometry
    (``oracle.fp32_bands``): per ray, the sample count K may differ where
    (t_exit - t_entry)/step lies within the rounding of t_entry and t_exit
    (6 units of 2^-24 of |t| divided by the deciding direction component,
    plus the origin's error) of an integer; per sample, the clip decision
    where the value lies within its own rounding plus the position's
    rounding times the local gradient of the clip; the termination decision
    where alpha lies within the image tolerance of the threshold."""
    return oracle.fp32_bands(dims, cams, step, w, h, band_a=TOL_FP32)


def tie_counts(res: oracle.Result) -> dict:
    """Pixels flagged per tie kind (K, clip, termination, truncated list,
    sub-cube boundary) and their fraction of all pixels."""
    f = np.asarray(res.flags)
    n = max(1, f.size)
    out = {name: int(np.count_nonzero(f & bit))
           for name, bit in (("k", 1), ("clip", 2), ("term", 4), ("trunc", 8),
                             ("boundary", 16))}
    out["any"] = int(np.count_nonzero(f))
    out["frac"] = out["any"] / n
    return out


def assert_ties(res: oracle.Result, what="", k=0.01, clip=0.0, term=0.02, trunc=0.0):
    """Bound the fraction of pixels whose acceptance set holds alternatives,
    per kind: the bands are derived from the arithmetic, so a test whose
    pixels are mostly ties checks little."""
    t = tie_counts(res)
    n = max(1, len(res.flags))
    for name, bound in (("k", k), ("clip", clip), ("term", term), ("trunc", trunc)):
        assert t[name] <= bound * n, "%s: %d of %d pixels are %s ties (bound %g)" % (
            what, t[name], n, name, bound)
    return t


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
