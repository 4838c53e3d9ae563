"""Pins for the FP64 oracle: closed forms, library routines, invariants,
hand-enumerated cases and an exact brute force on tiny cubes.

None of these re-types the oracle's own formulas: each checks it against a
relation the rendering definition implies (paper §3.1 process item 3 with this
project's readings of the steps the paper leaves open).
"""
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from oracle import brute, quantize

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cam(proj, eye, fwd, du, dv):
    c = np.zeros(1, dtype=oracle.CAMERA_DTYPE)
    c[0]["proj"], c[0]["eye"], c[0]["fwd"], c[0]["du"], c[0]["dv"] = proj, eye, fwd, du, dv
    return c


def cams(records):
    return np.concatenate([cam(*r) for r in records])


NO_TIES = oracle.Bands(band_k=0.0, band_pos=0.0, band_clip=0.0, band_a=0.0)


def flat_tf():
    return oracle.TF(np.array([[1, 1, 1, 0], [1, 1, 1, 0]], np.float32), 0, 1, 0)


# ---------------------------------------------------------------------------
# storage decoding
# ---------------------------------------------------------------------------
def test_half_decode_matches_numpy_for_every_bit_pattern():
    bits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    ref = bits.view(np.float16).astype(np.float64)
    got = np.array([oracle.half_to_double(int(b)) for b in bits])
    finite = np.isfinite(ref)
    assert np.array_equal(got[finite], ref[finite])
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.array_equal(got[np.isinf(ref)], ref[np.isinf(ref)])


def test_int8_quantizer_definition_brute_force():
    rng = np.random.default_rng(3)
    cube = (rng.standard_normal((5, 3, 4)) * 3).astype(np.float32)
    cube[2] = 1.25                          # a constant plane
    q, scale, offset = quantize.quantize_i8(cube)
    for z in range(5):
        plane = cube[z]
        lo, hi = float(plane.min()), float(plane.max())
        if lo == hi:
            assert scale[z] == 1.0 and offset[z] == np.float32(lo)
            assert (q[z] == 0).all()
            continue
        assert q[z].min() == -127 and q[z].max() == 127
        for idx in np.ndindex(plane.shape):
            v = float(plane[idx])
            dec = [c * float(scale[z]) + float(offset[z]) for c in range(-127, 128)]
            best = min(range(-127, 128), key=lambda c: abs(v - dec[c + 127]))
            # nearest code (up to the float32 rounding of the decision)
            assert abs(abs(v - dec[int(q[z][idx]) + 127]) - abs(v - dec[best + 127])) \
                <= 1e-6 * max(1.0, abs(v))
            assert abs(v - dec[int(q[z][idx]) + 127]) <= 0.5 * float(scale[z]) * (1 + 1e-5)


def test_int8_volume_decodes_per_plane():
    q = np.arange(-4, 4, dtype=np.int8).reshape(2, 2, 2)
    scale = np.array([0.5, 2.0], np.float32)
    offset = np.array([1.0, -3.0], np.float32)
    vol = oracle.Volume(q, scale, offset)
    for z in range(2):
        for y in range(2):
            for x in range(2):
                want = float(q[z, y, x]) * scale[z] + offset[z]
                assert oracle.sample_at(vol, x, y, z) == want


# ---------------------------------------------------------------------------
# trilinear interpolation
# ---------------------------------------------------------------------------
def test_trilinear_hits_voxel_values_at_centres():
    rng = np.random.default_rng(0)
    cube = rng.standard_normal((4, 5, 6)).astype(np.float32)
    vol = oracle.Volume(cube)
    for z in range(4):
        for y in range(5):
            for x in range(6):
                assert oracle.sample_at(vol, x, y, z) == float(cube[z, y, x])


def test_trilinear_reproduces_separable_multilinear_field():
    # trilinear interpolation is exact for (a + b x)(c + d y)(e + f z); an
    # asymmetric choice catches transposed axes or swapped corners
    nz, ny, nx = 5, 4, 6
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = lambda x, y, z: (1 + 0.5 * x) * (3 - 0.25 * y) * (2 + 0.125 * z)
    cube = f(x, y, z).astype(np.float32)
    assert np.array_equal(cube.astype(np.float64), f(x, y, z))
    vol = oracle.Volume(cube)
    rng = np.random.default_rng(1)
    for _ in range(200):
        p = rng.uniform(0, 1, 3) * [nx - 1, ny - 1, nz - 1]
        assert abs(oracle.sample_at(vol, *p) - f(*p)) < 1e-12


def test_trilinear_clamps_outside_points():
    cube = np.arange(8, dtype=np.float32).reshape(2, 2, 2)
    vol = oracle.Volume(cube)
    assert oracle.sample_at(vol, -5, -5, -5) == 0.0
    assert oracle.sample_at(vol, 9, 9, 9) == 7.0


# ---------------------------------------------------------------------------
# transfer function
# ---------------------------------------------------------------------------
def test_classify_nodes_and_opacity_correction_closed_form():
    lut = np.array([[0, 0, 0, 0], [1, 0.5, 0, 0.75], [0, 1, 1, 0.5]], np.float32)
    tf = oracle.TF(lut, v_lo=2.0, v_hi=6.0, clip=2.0)
    for step in (1.0, 0.5, 0.25, 2.0):
        r = oracle.classify(tf, step, 4.0)             # node 1 exactly
        assert np.allclose(r[:3], [1, 0.5, 0])
        assert abs(r[3] - (1 - 0.25 ** step)) < 1e-15
        # halfway between nodes 1 and 2: linear in the corrected alphas
        r = oracle.classify(tf, step, 5.0)
        a1, a2 = 1 - 0.25 ** step, 1 - 0.5 ** step
        assert abs(r[3] - 0.5 * (a1 + a2)) < 1e-15
        assert np.allclose(r[:3], [0.5, 0.75, 0.5])
    # values beyond the domain clamp to the end nodes
    assert np.allclose(oracle.classify(tf, 1.0, 100.0), [0, 1, 1, 0.5])
    assert np.allclose(oracle.classify(tf, 1.0, -100.0), [0, 0, 0, 0])


# ---------------------------------------------------------------------------
# closed forms of whole rays
# ---------------------------------------------------------------------------
def test_constant_cube_alpha_closed_form():
    n = (6, 7, 9)
    c = 3.0
    cube = np.full((n[2], n[1], n[0]), c, np.float32)
    vol = oracle.Volume(cube)
    # c sits exactly on node 2 of a 5-entry table over [1, 5]
    lut = np.array([[0.2, 0.4, 0.6, 0.1 * i] for i in range(5)], np.float32)
    tf = oracle.TF(lut, 1.0, 5.0, clip=0.5)
    step = 0.5
    cams_ = cam(0, [2.5, 3.0, -2.0], [0, 0, 1], [1, 0, 0], [0, 1, 0])
    res = oracle.render(vol, cams_, 1, 1, oracle.COMPOSITE, step, tf, bands=NO_TIES)
    K = math.floor((n[2] - 1) / step) + 1                         # 17
    a = 1 - (1 - np.float64(np.float32(0.2))) ** step
    A = 1 - (1 - a) ** K
    rgb = np.float32([0.2, 0.4, 0.6]).astype(np.float64)
    assert np.allclose(res.primary[0], list(rgb * A) + [A], rtol=0, atol=1e-14)
    assert res.nsamples[0] == K


def test_constant_cube_early_termination_closed_form():
    cube = np.full((40, 4, 4), 2.0, np.float32)
    vol = oracle.Volume(cube)
    lut = np.array([[1, 0, 0, 0.3], [1, 0, 0, 0.3]], np.float32)
    for ta in (0.5, 0.9, 0.99):
        tf = oracle.TF(lut, 0.0, 4.0, clip=1.0, term_alpha=ta)
        step = 0.5
        res = oracle.render(vol, cam(0, [1.5, 1.5, -1], [0, 0, 1], [1, 0, 0], [0, 1, 0]),
                            1, 1, oracle.COMPOSITE, step, tf, bands=NO_TIES)
        a = 1 - (1 - np.float64(np.float32(0.3))) ** step
        nstar = math.ceil(math.log(1 - ta) / math.log(1 - a))
        if 1 - (1 - a) ** (nstar - 1) >= ta:   # guard the ceil at exact ties
            nstar -= 1
        A = 1 - (1 - a) ** nstar
        assert abs(res.primary[0][3] - A) < 1e-14
        assert abs(res.primary[0][0] - A) < 1e-14
        assert res.nsamples[0] == nstar


def test_single_bright_voxel_mip_closed_form():
    n = 8
    i, j, k = 3, 5, 4
    V = 7.0
    cube = np.zeros((n, n, n), np.float32)
    cube[k, j, i] = V
    vol = oracle.Volume(cube)
    w = h = 16
    sp = 7.0 / 16.0
    c = cam(0, [3.5, 3.5, -1.0], [0, 0, 1], [sp, 0, 0], [0, sp, 0])
    res = oracle.render(vol, c, w, h, oracle.MIP, 0.5, flat_tf(), bands=NO_TIES)
    py, px = np.mgrid[0:h, 0:w]
    x = 3.5 + (px + 0.5 - w / 2) * sp
    y = 3.5 + (py + 0.5 - h / 2) * sp
    want = V * np.maximum(0, 1 - np.abs(x - i)) * np.maximum(0, 1 - np.abs(y - j))
    assert np.allclose(res.primary[:, 0], want.ravel(), rtol=0, atol=1e-13)
    # any camera: MIP never exceeds the voxel value
    c2 = cam(1, [20.0, -9.0, 13.0], [-16.5, 12.5, -9.5], [0.01, 0.013, 0], [0, 0.004, 0.012])
    r2 = oracle.render(vol, c2, 12, 12, oracle.MIP, 0.25, flat_tf(), bands=NO_TIES)
    assert np.nanmax(np.where(np.isinf(r2.primary[:, 0]), np.nan, r2.primary[:, 0])) <= V


def _axis_camera(dims, axis):
    nx, ny, nz = dims
    c = [(nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2]
    a, b = [t for t in range(3) if t != axis]
    eye = list(c)
    eye[axis] = -1.0
    fwd = [0, 0, 0]
    fwd[axis] = 1
    du = [0, 0, 0]
    du[a] = 1
    dv = [0, 0, 0]
    dv[b] = 1
    return cam(0, eye, fwd, du, dv), dims[a], dims[b]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_axis_sums_equal_array_sums(axis):
    rng = np.random.default_rng(10 + axis)
    dims = (5, 6, 7)
    cube = rng.integers(-20, 20, size=(dims[2], dims[1], dims[0])).astype(np.float32)
    vol = oracle.Volume(cube)
    c, w, h = _axis_camera(dims, axis)
    np_axis = 2 - axis                      # (z, y, x) storage order
    S = cube.astype(np.float64).sum(axis=np_axis)
    # image pixel (px, py) walks the two remaining axes in increasing order
    # the image axes are the two remaining axes in increasing order, which is
    # also the order numpy keeps them in after the reduction: image[py, px]
    first = np.take(cube, 0, axis=np_axis).astype(np.float64)
    last = np.take(cube, dims[axis] - 1, axis=np_axis).astype(np.float64)
    res = oracle.render(vol, c, w, h, oracle.SUM, 1.0, flat_tf(), bands=NO_TIES)
    got = res.primary[:, 0].reshape(h, w)
    assert got.shape == S.shape
    assert np.allclose(got, S, rtol=0, atol=1e-12)
    # step 1/2: samples at every voxel and every midpoint
    res = oracle.render(vol, c, w, h, oracle.SUM, 0.5, flat_tf(), bands=NO_TIES)
    got = res.primary[:, 0].reshape(h, w)
    assert np.allclose(got, S - (first + last) / 4.0, atol=1e-12)


@pytest.mark.parametrize("eye", [(-6.0, 15.0, 4.0), (4.0, 3.5, 5.0)])
def test_linear_field_perspective_closed_form(eye):
    # for V = a + b.x the samples are a + b.(o + t_k d); MIP is attained at an
    # end sample and SUM is an arithmetic series in t_k.  The ray segment is
    # found here by bisection on the inside-the-box predicate, independently
    # of the slab test.
    dims = np.array([9, 7, 11])
    a0, b = 1.5, np.array([0.5, -0.75, 0.25])
    z, y, x = np.meshgrid(*(np.arange(n) for n in dims[::-1]), indexing="ij")
    cube = (a0 + b[0] * x + b[1] * y + b[2] * z).astype(np.float32)
    vol = oracle.Volume(cube)
    eye = np.array(eye)            # outside the box, and inside it
    fwd = np.array([10.0, -11.0, 1.5])
    du = np.array([0.05, 0.04, 0.0])
    dv = np.array([0.0, 0.01, -0.06])
    c = cam(1, eye, fwd, du, dv)
    w, h, step = 9, 7, 0.37
    res = oracle.render(vol, c, w, h, oracle.SUM, step, flat_tf(), bands=NO_TIES)
    rmip = oracle.render(vol, c, w, h, oracle.MIP, step, flat_tf(), bands=NO_TIES)
    hi = dims - 1.0
    hits = 0
    for py in range(h):
        for px in range(w):
            e32 = c[0]
            dd = (e32["fwd"].astype(np.float64) + (px + 0.5 - w / 2) * e32["du"]
                  + (py + 0.5 - h / 2) * e32["dv"])
            dd /= np.linalg.norm(dd)
            o = e32["eye"].astype(np.float64)
            inside = lambda t: np.all(o + t * dd >= -1e-12) and np.all(o + t * dd <= hi + 1e-12)
            ts = np.linspace(0, 60, 600001)
            pts = o[None, :] + ts[:, None] * dd[None, :]
            ins = np.all((pts >= 0) & (pts <= hi), axis=1)
            i = px + py * w
            if not ins.any():
                assert res.primary[i, 0] == 0 and np.isneginf(rmip.primary[i, 0])
                continue
            hits += 1
            lo_i, hi_i = np.argmax(ins), len(ins) - 1 - np.argmax(ins[::-1])
            t0, t1 = ts[lo_i], ts[hi_i]
            # refine both ends by bisection
            def refine(tin, tout):
                for _ in range(80):
                    m = 0.5 * (tin + tout)
                    if inside(m):
                        tin = m
                    else:
                        tout = m
                return tin
            t0 = refine(t0, ts[lo_i - 1]) if lo_i > 0 else t0
            t1 = refine(t1, ts[min(hi_i + 1, len(ts) - 1)])
            q = (t1 - t0) / step
            K = math.floor(q) + 1
            if min(q - math.floor(q), math.ceil(q) - q) < 1e-6:
                continue                      # a K tie: covered elsewhere
            tk = t0 + step * np.arange(K)
            vals = a0 + (o[None, :] + tk[:, None] * dd[None, :]) @ b
            assert res.nsamples[i] == K
            assert abs(res.primary[i, 0] - step * vals.sum()) < 1e-6
            assert abs(rmip.primary[i, 0] - max(vals[0], vals[-1])) < 1e-6
    assert hits > 10


# ---------------------------------------------------------------------------
# hand-enumerated golden cases
# ---------------------------------------------------------------------------
def _golden(name):
    d = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (s.strip() for s in line.split("=", 1))
            d[k] = v
    return d


def _nums(s):
    return [float(t) for t in s.split()]


def test_golden_linear_column():
    g = _golden("column4_linear.txt")
    n = [int(t) for t in g["n"].split()]
    z, y, x = np.meshgrid(*(np.arange(k) for k in n[::-1]), indexing="ij")
    cube = (x + 2 * y + 4 * z).astype(np.float32)
    vol = oracle.Volume(cube)
    c = cam(0, _nums(g["eye"]), [0, 0, 1], [1, 0, 0], [0, 1, 0])
    step = float(g["step"])
    rm = oracle.render(vol, c, 1, 1, oracle.MIP, step, flat_tf())
    rs = oracle.render(vol, c, 1, 1, oracle.SUM, step, flat_tf())
    assert rm.primary[0, 0] == float(g["mip"]) and rs.primary[0, 0] == float(g["sum"])
    assert rm.nsamples[0] == int(g["K"])
    # the exact K tie is flagged and its alternative listed
    assert rm.flags[0] & 1 and rs.flags[0] & 1
    assert float(g["mip_alt"]) in rm.values[0, :rm.nalt[0], 0]
    assert float(g["sum_alt"]) in rs.values[0, :rs.nalt[0], 0]


def test_golden_composite_column():
    g = _golden("column4_composite.txt")
    cube = np.zeros((4, 4, 4), np.float32)
    cube[1, 1, 1] = 8
    cube[2, 1, 1] = 4
    vol = oracle.Volume(cube)
    c = cam(0, _nums(g["eye"]), [0, 0, 1], [1, 0, 0], [0, 1, 0])
    step = float(g["step"])
    lut = np.array([_nums(e) for e in g["lut"].split(";")], np.float32)
    tf = oracle.TF(lut, float(g["v_lo"]), float(g["v_hi"]), float(g["clip"]))
    assert oracle.render(vol, c, 1, 1, oracle.MIP, step, tf).primary[0, 0] == float(g["mip"])
    assert oracle.render(vol, c, 1, 1, oracle.SUM, step, tf).primary[0, 0] == float(g["sum"])
    r = oracle.render(vol, c, 1, 1, oracle.COMPOSITE, step, tf)
    assert np.allclose(r.primary[0], _nums(g["rgba_full"]), rtol=0, atol=1e-15)
    tf.term_alpha = float(g["term_alpha"])
    r = oracle.render(vol, c, 1, 1, oracle.COMPOSITE, step, tf)
    assert np.allclose(r.primary[0], _nums(g["rgba_term"]), rtol=0, atol=1e-15)
    assert r.nsamples[0] == int(g["term_samples"])


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
def test_composite_of_cube_below_clip_is_zero():
    rng = np.random.default_rng(4)
    cube = rng.uniform(-5, 1.99, (8, 9, 10)).astype(np.float32)
    vol = oracle.Volume(cube)
    lut = np.array([[1, 1, 1, 0.9]] * 4, np.float32)
    tf = oracle.TF(lut, -5, 5, clip=2.0)
    c = cam(1, [30, 4, 3], [-1, 0, 0], [0, 0.05, 0], [0, 0, 0.05])
    r = oracle.render(vol, c, 16, 16, oracle.COMPOSITE, 0.5, tf)
    assert (r.values == 0).all()


def test_alpha_bounded_and_monotone_in_ray_length():
    rng = np.random.default_rng(5)
    cube = rng.uniform(0, 10, (12, 6, 6)).astype(np.float32)
    vol = oracle.Volume(cube)
    lut = np.stack([np.linspace(0, 1, 16)] * 3 + [np.linspace(0, 0.8, 16)], 1).astype(np.float32)
    tf = oracle.TF(lut, 0, 10, clip=1.0)
    prev = None
    for zt in range(1, 12):
        sub = oracle.Volume(np.ascontiguousarray(cube[: zt + 1]))
        c = cam(0, [2.5, 2.5, -1], [0, 0, 1], [1, 0, 0], [0, 1, 0])
        A = oracle.render(sub, c, 4, 4, oracle.COMPOSITE, 0.5, tf).primary[:, 3]
        assert ((A >= 0) & (A <= 1)).all()
        if prev is not None:
            assert (A >= prev - 1e-15).all()
        prev = A


def test_rotating_cube_with_camera_gives_identical_ortho_image():
    rng = np.random.default_rng(6)
    cube = rng.standard_normal((6, 5, 7)).astype(np.float32)   # (z, y, x)
    lut = np.stack([np.linspace(0, 1, 8)] * 3 + [np.linspace(0, 0.6, 8)], 1).astype(np.float32)
    tf = oracle.TF(lut, -1, 2, clip=-0.5)
    vol = oracle.Volume(cube)
    # view along +z with du = +x, dv = +y
    c1 = cam(0, [3.0, 2.0, -1], [0, 0, 1], [0.5, 0, 0], [0, 0.5, 0])
    # rotate 90 degrees about z: np.rot90 over (y, x) gives
    # new[z, y', x'] = old[z, y = x', x = nx - 1 - y']
    rot = np.ascontiguousarray(np.rot90(cube, k=1, axes=(1, 2)))
    assert rot.shape == (6, 7, 5)
    # so an old point (x, y) sits at (x', y') = (y, nx - 1 - x): the eye
    # (3, 2) moves to (2, 3), du = +x becomes -y', dv = +y becomes +x'
    c2 = cam(0, [2.0, 3.0, -1], [0, 0, 1], [0, -0.5, 0], [0.5, 0, 0])
    for mode in (oracle.MIP, oracle.COMPOSITE, oracle.SUM):
        r1 = oracle.render(vol, c1, 9, 7, mode, 0.5, tf)
        r2 = oracle.render(oracle.Volume(rot), c2, 9, 7, mode, 0.5, tf)
        assert np.allclose(r1.primary, r2.primary, rtol=0, atol=1e-13)


def test_opacity_correction_makes_composite_step_convergent():
    z, y, x = np.meshgrid(np.arange(24), np.arange(6), np.arange(6), indexing="ij")
    cube = (2 + 3 * np.sin(z / 4.0) ** 2 + 0.1 * x).astype(np.float32)
    vol = oracle.Volume(cube)
    lut = np.stack([np.linspace(0, 1, 32), np.linspace(1, 0, 32), np.full(32, 0.5),
                    np.linspace(0, 0.2, 32)], 1).astype(np.float32)
    tf = oracle.TF(lut, 0, 6, clip=0)
    c = cam(0, [2.5, 2.5, -1], [0, 0, 1], [1, 0, 0], [0, 1, 0])
    prev, diffs = None, []
    for step in (0.5, 0.25, 0.125, 0.0625):
        r = oracle.render(vol, c, 2, 2, oracle.COMPOSITE, step, tf).primary
        if prev is not None:
            diffs.append(np.abs(r - prev).max())
        prev = r
    # first-order convergence: each halving roughly halves the change
    assert diffs[-1] < 0.6 * diffs[0] and diffs[-1] < 0.02
    # without the correction the opacity would grow ~2x per halving
    assert prev[:, 3].max() < 1.0


# ---------------------------------------------------------------------------
# exact brute force on tiny cubes
# ---------------------------------------------------------------------------
def _brute_case(seed, mode):
    rng = np.random.default_rng(seed)
    dims = tuple(int(v) for v in rng.integers(3, 6, 3))
    V = (rng.integers(-32, 160, size=(dims[2], dims[1], dims[0])) / 16.0).astype(np.float32)
    lut = np.stack([rng.integers(0, 9, 5) / 8.0 for _ in range(3)]
                   + [rng.integers(0, 8, 5) / 8.0], 1).astype(np.float32)
    step = [Fr(1), Fr(1, 2), Fr(3, 4)][seed % 3]
    tfp = dict(v_lo=-1.0, v_hi=9.0, clip=float(rng.integers(-1, 5)),
               term_alpha=[1.0, 0.75, 0.9][seed % 3])
    if seed % 2:
        # orthographic along a Pythagorean direction (exact unit vector)
        recs = [(0, [-2.0, 0.75, 0.5], [0.6, 0.0, 0.8], [0.0, 0.5, 0.0],
                 [-0.8 * 0.5, 0.0, 0.6 * 0.5])]
    else:
        recs = [(1, [dims[0] + 3.0, -2.5, dims[2] / 2.0], [-5.0, 3.0, -0.5],
                 [0.125, 0.25, 0.0], [0.0, 0.0, -0.25])]
    return dims, V, lut, step, tfp, recs


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("mode", [oracle.MIP, oracle.SUM, oracle.COMPOSITE])
def test_oracle_matches_exact_brute_force(seed, mode):
    dims, V, lut, step, tfp, recs = _brute_case(seed, mode)
    w = h = 5
    vol = oracle.Volume(V)
    tf = oracle.TF(lut, **tfp)
    res = oracle.render(vol, cams(recs), w, h, mode, float(step), tf,
                        bands=oracle.Bands(band_k=1e-9, band_pos=1e-12,
                                           band_clip=1e-12, band_a=1e-12))
    Vf = [[[Fr(float(v)) for v in row] for row in plane] for plane in V]
    # the exact caster sees the camera exactly as stored (float32 numbers)
    c32 = cams(recs)[0]
    rec = (int(c32["proj"]),) + tuple([float(t) for t in c32[k]]
                                      for k in ("eye", "fwd", "du", "dv"))
    hits = 0
    for py in range(h):
        for px in range(w):
            exact, count = brute.render_pixel(
                Vf, dims, rec, w, h, px, py, mode, step, lut=lut.tolist(), **tfp)
            i = py * w + px
            cand = res.values[i, :res.nalt[i]]
            if mode == oracle.MIP and exact is None:
                assert np.isneginf(res.primary[i, 0])
                continue
            hits += count > 0
            ex = np.array([float(e) for e in (exact if mode == oracle.COMPOSITE else [exact])])
            errs = np.abs(cand[:, :len(ex)] - ex[None, :]).max(axis=1)
            assert errs.min() < 1e-12, (px, py, ex, cand)
            if res.flags[i] == 0:
                assert errs[0] < 1e-12 and res.nsamples[i] == count
    assert hits > 0
