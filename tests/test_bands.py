"""Pins for the oracle's tie bands (CPU).

The bands claim: wherever a single-precision evaluation of the definition
can take a different discrete decision than the FP64 oracle (the sample
count K, a sample's clip test), the oracle flags the pixel and lists the
alternative.  These tests check that claim against an independent
single-precision evaluation written here with numpy float32 arithmetic
(fused multiply-adds emulated by an exact product in float64 rounded once),
on the geometries the GPU tests use, and bound how many pixels the bands
flag.  They share nothing with the CUDA path.
"""
import numpy as np

import oracle
from paper_1001_2049_b300 import synth

from _util import bands_for, tie_counts

F = np.float32


def fma32(a, b, c):
    """round_f32(a * b + c) for float32 inputs (the product is exact in
    float64; the sum rounds once there, then to float32)."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64)
            + np.asarray(c, np.float64)).astype(F)


def ray32(cam, w, h, px, py, dims):
    """Camera -> ray -> box in single precision: (o, d, t_entry, K) per pixel."""
    u = (px.astype(F) + F(0.5)) - F(0.5) * F(w)
    v = (py.astype(F) + F(0.5)) - F(0.5) * F(h)
    eye, fwd, du, dv = (np.asarray(cam[k], F) for k in ("eye", "fwd", "du", "dv"))
    if int(cam["proj"]) == 0:
        o = [fma32(v, dv[a], fma32(u, du[a], np.full(u.shape, eye[a], F))) for a in range(3)]
        d = [np.full(u.shape, fwd[a], F) for a in range(3)]
    else:
        o = [np.full(u.shape, eye[a], F) for a in range(3)]
        d = [fma32(v, dv[a], fma32(u, du[a], np.full(u.shape, fwd[a], F))) for a in range(3)]
    nrm = np.sqrt(fma32(d[0], d[0], fma32(d[1], d[1], d[2] * d[2]))).astype(F)
    d = [(x / nrm).astype(F) for x in d]
    tn = np.full(u.shape, -np.inf, F)
    tf = np.full(u.shape, np.inf, F)
    inside = np.ones(u.shape, bool)
    for a in range(3):
        hi = F(dims[a] - 1)
        par = d[a] == 0
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = ((F(0) - o[a]) / d[a]).astype(F)
            tb = ((hi - o[a]) / d[a]).astype(F)
        tn = np.where(par, tn, np.maximum(tn, np.minimum(ta, tb)))
        tf = np.where(par, tf, np.minimum(tf, np.maximum(ta, tb)))
        inside &= ~par | ((o[a] >= 0) & (o[a] <= hi))
    te = np.maximum(tn, F(0))
    hit = inside & (tf >= te)
    return o, d, te, tf, hit


def k32(cam, w, h, px, py, dims, step):
    o, d, te, tf, hit = ray32(cam, w, h, px, py, dims)
    with np.errstate(invalid="ignore"):
        q = ((tf - te).astype(F) / F(step)).astype(F)
    return np.where(hit, np.floor(np.where(hit, q, 0)).astype(np.int64) + 1, 0)


def _pixels(n_views, w, h, n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, n_views, n), rng.integers(0, w, n),
                     rng.integers(0, h, n)], axis=1).astype(np.int32)


def _check_k(dims, cams, w, h, step, pix):
    # a zero cube of the right shape: only the geometry matters for K (the
    # pages of np.zeros are never written, so even 1024^3 costs nothing)
    vol = oracle.Volume(np.zeros(tuple(reversed(dims)), np.float32))
    tf = oracle.TF(synth.default_lut(8), 0.0, 1.0, 0.0)
    res = oracle.render(vol, cams, w, h, oracle.MIP, step, tf, pixels=pix,
                        bands=bands_for(dims, cams, step, w, h))
    K = np.zeros(len(pix), np.int64)
    for v in np.unique(pix[:, 0]):
        sel = pix[:, 0] == v
        K[sel] = k32(cams[v], w, h, pix[sel, 1], pix[sel, 2], dims, step)
    differ = K != res.nsamples
    unflagged = np.flatnonzero(differ & ((res.flags & 1) == 0))
    assert unflagged.size == 0, (dims, unflagged[:5], K[unflagged[:5]],
                                 res.nsamples[unflagged[:5]])
    return res, int(differ.sum())


def test_k_band_covers_single_precision_counts_at_full_size():
    # the 1024^3 workload's 32 orbiting 1080p views (rays up to ~3000 voxels
    # long): every pixel whose single-precision K differs is flagged, and
    # the K band flags at most 1 % of the pixels
    dims, w, h, step = synth.LARGE.dims, 1920, 1080, synth.LARGE.step
    cams = synth.large_cameras()
    pix = _pixels(len(cams), w, h, 200000, 3)
    res, differ = _check_k(dims, cams, w, h, step, pix)
    t = tie_counts(res)
    assert t["k"] <= 0.01 * len(pix), t
    assert differ >= 1          # the check is not empty: some counts do differ


def test_k_band_covers_single_precision_counts_on_test_geometries():
    cases = [((64, 64, 128), synth.small_camera(), 256, 256, 0.5),
             ((37, 45, 70), synth.random_sphere_cameras((37, 45, 70), 6, 23, 17, 5, 70.0),
              23, 17, 0.37),
             ((96, 80, 120), synth.orbit_cameras((96, 80, 120), 8, 64, 48), 64, 48, 0.5),
             ((9, 12, 7), synth.cameras([synth.axis_camera((9, 12, 7), 16, 16, axis=a, sign=s)
                                         for a in range(3) for s in (1, -1)]), 16, 16, 0.5)]
    for dims, cams, w, h, step in cases:
        v, py, px = np.meshgrid(np.arange(len(cams)), np.arange(h), np.arange(w), indexing="ij")
        pix = np.stack([v.ravel(), px.ravel(), py.ravel()], axis=1).astype(np.int32)
        _check_k(dims, cams, w, h, step, pix)


def lerp32(a, b, f):
    return fma32(f, (b - a).astype(F), a)


def ray64(cam, w, h, px, py, dims):
    """The same ray in double precision (the definition's arithmetic)."""
    u = px + 0.5 - w / 2.0
    v = py + 0.5 - h / 2.0
    eye, fwd, du, dv = (np.asarray(cam[k], np.float64) for k in ("eye", "fwd", "du", "dv"))
    if int(cam["proj"]) == 0:
        o = [eye[a] + u * du[a] + v * dv[a] for a in range(3)]
        d = [np.full(u.shape, fwd[a]) for a in range(3)]
    else:
        o = [np.full(u.shape, eye[a]) for a in range(3)]
        d = [fwd[a] + u * du[a] + v * dv[a] for a in range(3)]
    nrm = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    d = [x / nrm for x in d]
    tn = np.full(u.shape, -np.inf)
    for a in range(3):
        with np.errstate(divide="ignore"):
            ta, tb = (0.0 - o[a]) / d[a], (dims[a] - 1.0 - o[a]) / d[a]
        tn = np.maximum(tn, np.minimum(ta, tb))
    return o, d, np.maximum(tn, 0.0)


def test_clip_band_covers_single_precision_clip_decisions():
    # every sample near the clip of every ray of orbit views of a noise cube,
    # evaluated in single precision (position from the integer index,
    # trilinear in x, then y, then z) and in FP64 through the oracle's own
    # sample function at the FP64 position: where the two clip decisions
    # differ, the oracle flags a clip tie on that pixel
    dims = (48, 40, 60)
    cube = synth.make_cube(dims, 2, ("uniform", 3.0, 6.0), 12).numpy()
    cams = synth.orbit_cameras(dims, 3, 40, 30, radius=150.0)
    w, h, step, clip = 40, 30, 0.5, 0.8
    tf = oracle.TF(synth.default_lut(32), 0.0, 6.0, clip, 2.0)
    vol = oracle.Volume(cube)
    res = oracle.render(vol, cams, w, h, oracle.COMPOSITE, step, tf,
                        bands=bands_for(dims, cams, step, w, h))
    nx, ny, nz = dims
    flips, near_total = 0, 0
    for vi in range(len(cams)):
        py, px = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
        px, py = px.ravel(), py.ravel()
        o, d, te, _, hit = ray32(cams[vi], w, h, px, py, dims)
        o64, d64, te64 = ray64(cams[vi], w, h, px.astype(np.float64), py.astype(np.float64),
                               dims)
        K = np.minimum(k32(cams[vi], w, h, px, py, dims, step), res.nsamples[
            vi * w * h:(vi + 1) * w * h])
        base = vi * w * h
        for r in np.flatnonzero(hit & (K > 0)):
            k = np.arange(K[r], dtype=F)
            t = fma32(k, F(step), te[r])
            p = [fma32(t, d[a][r], o[a][r]) for a in range(3)]
            i0 = [np.clip(np.floor(p[a]).astype(np.int64), 0, dims[a] - 2) for a in range(3)]
            f = [(p[a] - i0[a].astype(F)).astype(F) for a in range(3)]

            def c(a, b, e):
                return cube[np.clip(i0[2] + e, 0, nz - 1), np.clip(i0[1] + b, 0, ny - 1),
                            np.clip(i0[0] + a, 0, nx - 1)]
            y0z0 = lerp32(c(0, 0, 0), c(1, 0, 0), f[0])
            y1z0 = lerp32(c(0, 1, 0), c(1, 1, 0), f[0])
            y0z1 = lerp32(c(0, 0, 1), c(1, 0, 1), f[0])
            y1z1 = lerp32(c(0, 1, 1), c(1, 1, 1), f[0])
            s32 = lerp32(lerp32(y0z0, y1z0, f[1]), lerp32(y0z1, y1z1, f[1]), f[2])
            near = np.flatnonzero(np.abs(s32 - clip) < 1e-2)
            near_total += near.size
            for j in near:
                tk = te64[r] + float(j) * step
                q = [min(max(o64[a][r] + tk * d64[a][r], 0.0), dims[a] - 1.0) for a in range(3)]
                s64 = oracle.sample_at(vol, *q)
                if (s32[j] < clip) != (s64 < clip):
                    flips += 1
                    assert res.flags[base + r] & 2, ("unflagged clip flip", vi, r, j,
                                                     float(s32[j]), s64)
    assert near_total > 100          # many samples come near the clip
    t = tie_counts(res)
    assert 0 < t["clip"] <= 0.1 * len(res.flags), t


def test_one_subcube_gives_the_one_pass_acceptance_set():
    dims = (48, 40, 60)
    cube = synth.make_cube(dims, 2, ("uniform", 3.0, 6.0), 12).numpy()
    cams = synth.orbit_cameras(dims, 3, 40, 30, radius=150.0)
    vol = oracle.Volume(cube)
    tf = oracle.TF(synth.default_lut(32, alpha_max=0.3), 0.0, 6.0, 0.8, 0.6)
    b = bands_for(dims, cams, 0.5, 40, 30)
    for mode in (oracle.COMPOSITE, oracle.MIP):
        one = oracle.render(vol, cams, 40, 30, mode, 0.5, tf, bands=b)
        sub = oracle.render_subcubes(vol, cams, 40, 30, mode, 0.5, tf, [0], bands=b)
        # the same primary result and K ties; every alternative of the
        # sub-cube set (one decision changed) is one of the one-pass set's
        assert np.array_equal(one.primary, sub.primary)
        assert np.array_equal(one.flags & 1, sub.flags & 1)
        for i in range(len(one.flags)):
            a = {tuple(np.round(x, 12)) for x in one.values[i, :one.nalt[i]]}
            s = {tuple(np.round(x, 12)) for x in sub.values[i, :sub.nalt[i]]}
            if not one.flags[i] & 8:
                assert s <= a, (mode, i, s - a)
        if mode == oracle.COMPOSITE:
            assert (sub.nalt > 1).sum() >= 5
