"""Reduced-precision storage encodings, computed on the host for the oracle.

TEST INFRASTRUCTURE (see the package docstring).  These encoders define what
the device-side packer must produce, code for code:

* FP16: IEEE binary16 with round-to-nearest-even (numpy's float16 cast).
* int8 with a scale and an offset per frequency plane z (the frequency axis is
  the one along which radio cubes change their noise level and bandpass):
      lo_z = min of plane z,  hi_z = max of plane z
      scale_z  = (hi_z - lo_z) / 254          (float32 arithmetic)
      offset_z = (hi_z + lo_z) * 0.5          (float32 arithmetic)
      q = clamp(rint_even((v - offset_z) / scale_z), -127, 127)
  and when hi_z == lo_z: scale_z = 1, q = 0 (so the plane decodes to lo_z).
  Decoding is v' = q * scale_z + offset_z.  The encoding decision (which code
  an input gets) is taken in float32, the precision the device packer uses,
  so both sides reach the same integer codes.
"""
from __future__ import annotations

import numpy as np


def to_f16(cube: np.ndarray) -> np.ndarray:
    """float32 (nz, ny, nx) -> float16 with round-to-nearest-even."""
    return np.asarray(cube, dtype=np.float32).astype(np.float16)


def quantize_i8(cube: np.ndarray):
    """float32 (nz, ny, nx) -> (int8 codes, float32 scale[nz], float32 offset[nz])."""
    cube = np.asarray(cube, dtype=np.float32)
    nz = cube.shape[0]
    flat = cube.reshape(nz, -1)
    lo = flat.min(axis=1)
    hi = flat.max(axis=1)
    scale = ((hi - lo) / np.float32(254.0)).astype(np.float32)
    offset = ((hi + lo) * np.float32(0.5)).astype(np.float32)
    flat_plane = hi == lo
    scale = np.where(flat_plane, np.float32(1.0), scale).astype(np.float32)
    r = (cube - offset[:, None, None]) / scale[:, None, None]
    assert r.dtype == np.float32
    q = np.clip(np.rint(r), -127, 127).astype(np.int8)
    q[flat_plane] = 0
    return q, scale, offset


def dequantize_i8(q: np.ndarray, scale: np.ndarray, offset: np.ndarray) -> np.ndarray:
    """Decoded values in float64: q * scale_z + offset_z."""
    return (q.astype(np.float64) * scale.astype(np.float64)[:, None, None]
            + offset.astype(np.float64)[:, None, None])
