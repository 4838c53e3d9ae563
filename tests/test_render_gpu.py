"""Parity of the CUDA render path (through the C ABI) with the FP64 oracle.

Every image is compared pixel by pixel with the oracle's acceptance set
(primary double-precision result plus the alternatives at the three
discontinuities), within the tolerances stated in tests/_util.py.
"""
import functools
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import quantize
from paper_1001_2049_b300 import Request, Volume, VRError, render_batch, synth
from paper_1001_2049_b300.api import volume_bytes

from _util import TOL_FP32, TOL_PREC, assert_ties, bands_for, compare, sum_scale

pytestmark = pytest.mark.gpu

MODES = {"mip": oracle.MIP, "composite": oracle.COMPOSITE, "sum": oracle.SUM}


def oracle_volume(cube: np.ndarray, dtype: str) -> oracle.Volume:
    if dtype == "f32":
        return oracle.Volume(cube)
    if dtype == "f16":
        return oracle.Volume(quantize.to_f16(cube))
    q, s, o = quantize.quantize_i8(cube)
    return oracle.Volume(q, s, o)


def gpu_images(cube_t, dtype, cams, w, h, mode, step, lut, v_lo, v_hi, clip, ta, count=None,
               tex=False, masks=False, bounds=False):
    vol = Volume(cube_t.cuda(), dtype)
    if tex == "pair":
        vol.attach_pair_texture()
    elif tex:
        vol.attach_texture()
    if masks:
        vol.attach_masks()
    if bounds:
        vol.attach_mip_bounds()
    vol.set_transfer(lut, v_lo, v_hi, clip, ta)
    out = vol.render(cams, w, h, mode, step, count=count)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def scale_for(mode, cube, got):
    if mode == "mip":
        return float(cube.max() - cube.min())
    if mode == "sum":
        fin = np.abs(got[np.isfinite(got)])
        return max(1.0, float(fin.max()) if fin.size else 1.0)
    return 1.0


def run_parity(cube, dtype, cams, w, h, mode, step, lut, v_lo, v_hi, clip, ta, tol=TOL_FP32,
               reference="decoded", pixels=None, what="", tex=False, masks=False, bounds=False,
               ties=None):
    """Render on the GPU (bricks, or texture storage with tex=True, with the
    empty-space masks with masks=True, with MIP bounds with bounds=True) and
    compare with the oracle (on the decoded storage values, or on the float32
    source with reference="source").  ``ties``: bounds on the fraction of
    pixels per tie kind (assert_ties; default at most 1 % K ties and 2 %
    termination ties, no clip ties)."""
    got = gpu_images(torch.from_numpy(cube), dtype, cams, w, h, mode, step, lut, v_lo, v_hi,
                     clip, ta, tex=tex, masks=masks, bounds=bounds)
    ovol = oracle_volume(cube, dtype if reference == "decoded" else "f32")
    tf = oracle.TF(lut, v_lo, v_hi, clip, ta)
    nz, ny, nx = cube.shape
    res = oracle.render(ovol, cams, w, h, MODES[mode], step, tf, pixels=pixels,
                        bands=bands_for((nx, ny, nz), cams, step, w, h))
    assert_ties(res, what, **(ties or {}))
    ch = 4 if mode == "composite" else 1
    flat = got.reshape(len(cams), h, w, ch) if ch == 4 else got.reshape(len(cams), h, w, 1)
    if pixels is not None:
        flat = flat[pixels[:, 0], pixels[:, 2], pixels[:, 1]]
    scale = scale_for(mode, cube, got)
    if mode == "sum":
        scale = sum_scale(oracle.Volume(cube), cams, w, h, step, got, pixels)
    rep = compare(res, flat, MODES[mode], tol, scale, what=what)
    return got, res, rep


# ---------------------------------------------------------------------------
# the 64x64x128 workload: 256^2 orthographic view along the frequency axis
# ---------------------------------------------------------------------------
#: Tie bounds of axis-aligned orthographic views of small cubes: rays cross
#: a whole number of half-voxel steps and some lie in face planes, so K is a
#: structural tie on a large share of the pixels.
AXIS_TIES = {"k": 0.5}
#: Deep cubes seen along z without termination: as the axis views, plus
#: long rays whose alpha settles within the band of 1.
DEEP_TIES = {"k": 0.5, "term": 0.5, "trunc": 0.5}

#: Tie bounds of the 64x64x128 orthographic view: every ray crosses the
#: 127 voxels along z in exactly 254 steps of 1/2, so every pixel's K is a
#: structural tie (test_small_workload_sample_count checks that the device
#: takes the primary count, 255, on every ray); without termination
#: (alpha 1) the rays through opaque sources reach alpha within the band of
#: 1 and stay there, so up to 5 % of pixels carry termination alternatives.
SMALL_TIES = {"k": 1.0, "term": 0.05, "trunc": 0.05}


@pytest.fixture(scope="module")
def small():
    wl = synth.SMALL
    cube = wl.cube("cpu").numpy()
    lut = synth.default_lut()
    return wl, cube, lut, synth.small_camera()


@pytest.mark.parametrize("mode", ["mip", "composite", "sum"])
def test_small_workload_fp32_full_frame(small, mode):
    wl, cube, lut, cams = small
    _, res, rep = run_parity(cube, "f32", cams, 256, 256, mode, wl.step, lut, wl.clip, wl.v_hi,
                             wl.clip, wl.term_alpha, what="small fp32 " + mode,
                             ties=SMALL_TIES)
    # (t_exit - t_entry)/step = 127/0.5 is an integer for every ray of this
    # view, so every pixel carries the K and K - 1 alternatives
    assert (res.flags & 1).all()


@pytest.mark.parametrize("dtype", ["f16", "i8"])
@pytest.mark.parametrize("mode", ["mip", "composite"])
def test_small_workload_reduced_precision(small, dtype, mode):
    wl, cube, lut, cams = small
    # kernel parity: against the oracle on the decoded storage values
    run_parity(cube, dtype, cams, 256, 256, mode, wl.step, lut, wl.clip, wl.v_hi, wl.clip,
               wl.term_alpha, what="small %s %s decoded" % (dtype, mode),
               ties=SMALL_TIES)
    # stated precision cost: against the oracle on the float32 source
    run_parity(cube, dtype, cams, 256, 256, mode, wl.step, lut, wl.clip, wl.v_hi, wl.clip,
               wl.term_alpha, tol=TOL_PREC[dtype], reference="source",
               what="small %s %s vs fp32 source" % (dtype, mode),
               ties=SMALL_TIES)


@pytest.mark.parametrize("dtype", ["f16", "i8"])
@pytest.mark.parametrize("mode", ["mip", "composite"])
def test_small_workload_orbit_views_reduced_precision(small, dtype, mode):
    # the precision variants' 32 orbit views of the 64x64x128 cube at 256^2
    # (texture storage, as the benchmark renders them): kernel parity
    # against the oracle on the decoded storage, and the stated precision
    # cost against the oracle on the float32 source
    wl, cube, lut, _ = small
    cams = synth.orbit_cameras(wl.dims, 32, 256, 256)
    run_parity(cube, dtype, cams, 256, 256, mode, wl.step, lut, wl.clip, wl.v_hi, wl.clip,
               wl.term_alpha, what="small orbit %s %s decoded" % (dtype, mode), tex=True,
               ties={"term": 0.05, "trunc": 0.05})
    run_parity(cube, dtype, cams, 256, 256, mode, wl.step, lut, wl.clip, wl.v_hi, wl.clip,
               wl.term_alpha, tol=TOL_PREC[dtype], reference="source", tex=True,
               what="small orbit %s %s vs fp32 source" % (dtype, mode),
               ties={"term": 0.05, "trunc": 0.05})


def test_small_workload_sample_count(small):
    wl, cube, lut, cams = small
    for mode in ("mip", "composite"):
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        gpu_images(torch.from_numpy(cube), "f32", cams, 256, 256, mode, wl.step, lut, wl.clip,
                   wl.v_hi, wl.clip, wl.term_alpha, count=cnt)
        res = oracle.render(oracle.Volume(cube), cams, 256, 256, MODES[mode], wl.step,
                            oracle.TF(lut, wl.clip, wl.v_hi, wl.clip, wl.term_alpha),
                            bands=bands_for(wl.dims, cams, wl.step))
        want = int(res.nsamples.sum())
        slack = 8 * int(np.count_nonzero(res.flags))
        assert abs(int(cnt.item()) - want) <= slack
    # every ray of this view takes K = 255 samples
    assert int(res.nsamples.max()) == 255


# ---------------------------------------------------------------------------
# ragged cubes (several bricks plus partial ones), perspective cameras from
# many directions (one inside the cube), ragged image tiles
# ---------------------------------------------------------------------------
RAGGED = [((37, 45, 70), 0.5), ((2, 2, 2), 0.25), ((33, 31, 65), 0.37), ((64, 5, 40), 0.5)]


def ragged_case(dims, seed):
    cube = synth.make_cube(dims, 3, ("uniform", 3.0, 8.0), seed).numpy()
    cams = synth.random_sphere_cameras(dims, 3, 23, 17, seed, fov_deg=70.0)
    c = np.array([(d - 1) / 2.0 for d in dims])
    inside = synth.look_at_camera(c + 0.3, c + np.array([5.0, -3.0, 2.0]), 23, 17, 90.0)
    cams = np.concatenate([cams, synth.cameras([inside]).astype(cams.dtype)])
    lut = synth.default_lut(64)
    return cube, cams, lut


@pytest.mark.parametrize("dims,step", RAGGED)
@pytest.mark.parametrize("mode", ["mip", "composite", "sum"])
def test_ragged_cubes_perspective_fp32(dims, step, mode):
    cube, cams, lut = ragged_case(dims, 17 + dims[0])
    run_parity(cube, "f32", cams, 23, 17, mode, step, lut, 1.0, 8.0, 1.0, 0.95,
               what="ragged %s %s" % (dims, mode))


@pytest.mark.parametrize("dtype", ["f16", "i8"])
def test_ragged_cube_reduced_precision(dtype):
    cube, cams, lut = ragged_case((37, 45, 70), 3)
    for mode in ("mip", "composite"):
        run_parity(cube, dtype, cams, 23, 17, mode, 0.5, lut, 1.0, 8.0, 1.0, 0.95,
                   what="ragged %s %s" % (dtype, mode))


def test_orthographic_axis_views_and_misses():
    # views along each axis, wider than the cube (many rays miss) and with
    # rays lying exactly in the face planes
    rng = np.random.default_rng(5)
    dims = (9, 12, 7)
    cube = rng.standard_normal((7, 12, 9)).astype(np.float32)
    recs = [synth.axis_camera(dims, 16, 16, axis=a, sign=s) for a in range(3) for s in (1, -1)]
    cams = synth.cameras(recs)
    lut = synth.default_lut(16)
    for mode in ("mip", "composite", "sum"):
        run_parity(cube, "f32", cams, 16, 16, mode, 0.5, lut, -1.0, 2.0, -1.0, 1.0,
                   what="axis views " + mode,
                   ties=AXIS_TIES)


def test_many_views_span_several_launches():
    dims = (20, 18, 24)
    cube = synth.make_cube(dims, 2, ("uniform", 4.0, 6.0), 9).numpy()
    cams = synth.random_sphere_cameras(dims, 70, 8, 8, 21)
    run_parity(cube, "f32", cams, 8, 8, "composite", 0.5, synth.default_lut(), 1.0, 6.0, 1.0,
               0.99, what="70 views")


def test_all_samples_below_clip_give_zero():
    dims = (16, 16, 16)
    cube = synth.make_cube(dims, 0, ("uniform", 1, 2), 1).numpy()
    got = gpu_images(torch.from_numpy(cube), "f32", synth.random_sphere_cameras(dims, 2, 9, 9, 2),
                     9, 9, "composite", 0.5, synth.default_lut(), 100.0, 200.0, 100.0, 1.0)
    assert (got == 0).all()


# ---------------------------------------------------------------------------
# texture storage: the same parity through the texture-gather kernel
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["f32", "f16", "i8"])
@pytest.mark.parametrize("mode", ["mip", "composite", "sum"])
def test_texture_path_small_workload(small, dtype, mode):
    wl, cube, lut, cams = small
    run_parity(cube, dtype, cams, 256, 256, mode, wl.step, lut, wl.clip, wl.v_hi, wl.clip,
               wl.term_alpha, what="small tex %s %s" % (dtype, mode), tex=True,
               ties=SMALL_TIES)
    if dtype != "f32" and mode != "sum":
        run_parity(cube, dtype, cams, 256, 256, mode, wl.step, lut, wl.clip, wl.v_hi, wl.clip,
                   wl.term_alpha, tol=TOL_PREC[dtype], reference="source",
                   what="small tex %s %s vs source" % (dtype, mode), tex=True,
               ties=SMALL_TIES)


@pytest.mark.parametrize("dims,step", RAGGED)
@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_texture_path_ragged_cubes(dims, step, dtype):
    cube, cams, lut = ragged_case(dims, 17 + dims[0])
    for mode in ("mip", "composite", "sum"):
        run_parity(cube, dtype, cams, 23, 17, mode, step, lut, 1.0, 8.0, 1.0, 0.95,
                   what="tex ragged %s %s %s" % (dims, dtype, mode), tex=True)


def test_texture_path_axis_views_and_misses():
    rng = np.random.default_rng(5)
    dims = (9, 12, 7)
    cube = rng.standard_normal((7, 12, 9)).astype(np.float32)
    recs = [synth.axis_camera(dims, 16, 16, axis=a, sign=s) for a in range(3) for s in (1, -1)]
    cams = synth.cameras(recs)
    lut = synth.default_lut(16)
    for mode in ("mip", "composite", "sum"):
        run_parity(cube, "f32", cams, 16, 16, mode, 0.5, lut, -1.0, 2.0, -1.0, 1.0,
                   what="tex axis views " + mode, tex=True,
                   ties=AXIS_TIES)


def test_texture_path_stacks_planes_of_deep_cubes():
    # more planes than a layered texture has layers: 4 planes per layer
    dims = (6, 5, 4500)
    cube = synth.make_cube(dims, 20, ("uniform", 3.0, 8.0), 31).numpy()
    recs = [synth.axis_camera(dims, 8, 8, axis=2, spacing=(0.7, 0.6)),
            synth.axis_camera(dims, 8, 8, axis=2, sign=-1, spacing=(0.7, 0.6)),
            synth.look_at_camera((40.0, -30.0, 2047.3), (2.5, 2.0, 2047.0), 8, 8, 60.0),
            synth.look_at_camera((-20.0, 25.0, 4094.5), (2.5, 2.0, 4094.0), 8, 8, 60.0)]
    cams = synth.cameras(recs)
    for dtype in ("f32", "i8"):
        for mode in ("mip", "composite"):
            run_parity(cube, dtype, cams, 8, 8, mode, 0.5, synth.default_lut(), 1.0, 8.0, 1.0,
                       1.0, what="tex 4500 planes %s %s" % (dtype, mode), tex=True,
                       ties=DEEP_TIES)


@pytest.mark.parametrize("dtype", ["f16", "i8"])
@pytest.mark.parametrize("mode", ["mip", "composite", "sum"])
def test_pair_texture_small_workload(small, dtype, mode):
    wl, cube, lut, cams = small
    run_parity(cube, dtype, cams, 256, 256, mode, wl.step, lut, wl.clip, wl.v_hi, wl.clip,
               wl.term_alpha, what="small pair %s %s" % (dtype, mode), tex="pair",
               ties=SMALL_TIES)


@pytest.mark.parametrize("dims,step", RAGGED)
@pytest.mark.parametrize("dtype", ["f16", "i8"])
def test_pair_texture_ragged_cubes(dims, step, dtype):
    cube, cams, lut = ragged_case(dims, 17 + dims[0])
    for mode in ("mip", "composite"):
        run_parity(cube, dtype, cams, 23, 17, mode, step, lut, 1.0, 8.0, 1.0, 0.95,
                   what="pair ragged %s %s %s" % (dims, dtype, mode), tex="pair")


@pytest.mark.parametrize("dtype", ["f16", "i8"])
def test_pair_texels_give_the_plain_texels_images(dtype):
    # the packed pair texels travel through the march as raw bits and are
    # unpacked at interpolation: the images are those of one texel per voxel
    # bit for bit, also where halves of a texel are zero or tiny (bit
    # patterns that read as subnormal floats)
    dims = (29, 23, 41)
    cube = synth.make_cube(dims, 3, ("uniform", 3.0, 8.0), 66).numpy()
    rng = np.random.default_rng(8)
    m = rng.random(cube.shape)
    cube[m < 0.3] = 0.0
    cube[(m >= 0.3) & (m < 0.4)] = 1e-6
    cube[(m >= 0.4) & (m < 0.45)] *= -1.0
    cams = synth.random_sphere_cameras(dims, 3, 27, 21, 4)
    imgs = {}
    for pair in (False, True):
        vol = Volume(torch.from_numpy(cube).cuda(), dtype)
        vol.attach_pair_texture() if pair else vol.attach_texture()
        vol.set_transfer(synth.default_lut(32), -1.0, 8.0, -1.0, 0.97)
        imgs[pair] = {mode: vol.render(cams, 27, 21, mode, 0.37).cpu() for mode in MODES}
    for mode in MODES:
        assert torch.equal(imgs[False][mode], imgs[True][mode]), (dtype, mode)


def test_pair_texture_stacks_cell_planes_of_deep_cubes():
    dims = (6, 5, 4500)
    cube = synth.make_cube(dims, 20, ("uniform", 3.0, 8.0), 31).numpy()
    recs = [synth.axis_camera(dims, 8, 8, axis=2, spacing=(0.7, 0.6)),
            synth.axis_camera(dims, 8, 8, axis=2, sign=-1, spacing=(0.7, 0.6)),
            synth.look_at_camera((40.0, -30.0, 2048.3), (2.5, 2.0, 2048.0), 8, 8, 60.0),
            synth.look_at_camera((-20.0, 25.0, 4096.5), (2.5, 2.0, 4096.0), 8, 8, 60.0)]
    cams = synth.cameras(recs)
    for dtype in ("f16", "i8"):
        for mode in ("mip", "composite"):
            run_parity(cube, dtype, cams, 8, 8, mode, 0.5, synth.default_lut(), 1.0, 8.0, 1.0,
                       1.0, what="pair 4500 planes %s %s" % (dtype, mode), tex="pair",
                       ties=DEEP_TIES)


def test_pair_texture_is_refreshed_by_uploads_and_refused_for_f32():
    dims = (24, 20, 30)
    a = synth.make_cube(dims, 3, ("uniform", 3, 9), 40)
    b = synth.make_cube(dims, 3, ("uniform", 3, 9), 41)
    cams = synth.random_sphere_cameras(dims, 2, 16, 16, 3)
    vol = Volume(a.cuda(), "i8")
    vol.attach_pair_texture()
    vol.set_transfer(synth.default_lut(), 1.0, 9.0, 1.0, 1.0)
    vol.upload(5, b[5:20].cuda())
    mixed = a.clone()
    mixed[5:20] = b[5:20]
    ref = Volume(mixed.cuda(), "i8")
    ref.set_transfer(synth.default_lut(), 1.0, 9.0, 1.0, 1.0)
    got = vol.render(cams, 16, 16, "mip", 0.5)
    want = ref.render(cams, 16, 16, "mip", 0.5)
    torch.cuda.synchronize()
    assert torch.allclose(got, want, rtol=0, atol=1e-5)
    with pytest.raises(VRError):
        Volume(a.cuda(), "f32").attach_pair_texture()


def test_texture_is_refreshed_by_uploads():
    dims = (24, 20, 30)
    a = synth.make_cube(dims, 3, ("uniform", 3, 9), 40)
    b = synth.make_cube(dims, 3, ("uniform", 3, 9), 41)
    cams = synth.random_sphere_cameras(dims, 2, 16, 16, 3)
    vol = Volume(a.cuda(), "f32")
    vol.attach_texture()
    vol.set_transfer(synth.default_lut(), 1.0, 9.0, 1.0, 1.0)
    vol.upload(5, b[5:20].cuda())
    mixed = a.clone()
    mixed[5:20] = b[5:20]
    ref = Volume(mixed.cuda(), "f32")
    ref.set_transfer(synth.default_lut(), 1.0, 9.0, 1.0, 1.0)
    got = vol.render(cams, 16, 16, "mip", 0.5)
    want = ref.render(cams, 16, 16, "mip", 0.5)
    torch.cuda.synchronize()
    assert torch.allclose(got, want, rtol=0, atol=1e-5)
    vol.detach_texture()                      # back to the brick gather
    assert torch.allclose(vol.render(cams, 16, 16, "mip", 0.5), want, rtol=0, atol=1e-5)


def test_every_launch_shape_gives_identical_images():
    # the per-ray arithmetic does not depend on the block or packet shape
    from paper_1001_2049_b300.api import launch_shapes
    dims = (40, 33, 57)
    cube = synth.make_cube(dims, 4, ("uniform", 3, 9), 50).cuda()
    vol = Volume(cube, "f32")
    vol.attach_texture()
    vol.set_transfer(synth.default_lut(), 1.0, 9.0, 1.0, 0.97)
    cams = synth.random_sphere_cameras(dims, 3, 45, 29, 7)
    shapes = launch_shapes()
    assert len(shapes) >= 4
    refs = {}
    for case in ("composite", "mip", "mip bounds"):
        mode = case.split()[0]
        if case == "mip bounds":              # the same images as without bounds
            vol.attach_mip_bounds()
        ref = refs.get(mode)
        for cfg in range(len(shapes)):
            vol.set_launch_config(mode, cfg)
            img = vol.render(cams, 45, 29, mode, 0.5)
            if ref is None:
                ref = refs[mode] = img.clone()
            assert torch.equal(img, ref), (case, cfg, shapes[cfg])
        best, ms = vol.autotune(cams, 45, 29, mode, 0.5)
        assert 0 <= best < len(shapes) and ms > 0
        assert torch.equal(vol.render(cams, 45, 29, mode, 0.5), ref)


# ---------------------------------------------------------------------------
# packing: bit-exact brick contents, host and slab uploads
# ---------------------------------------------------------------------------
def unbrick(buf: torch.Tensor, dims, dtype):
    nx, ny, nz = dims
    nb = [math.ceil(d / 32) for d in dims]
    np_dt = {"f32": np.float32, "f16": np.float16, "i8": np.int8}[dtype]
    n = nb[0] * nb[1] * nb[2] * 32768
    raw = buf.cpu().numpy()
    vox = raw[: n * np.dtype(np_dt).itemsize].view(np_dt)
    a = vox.reshape(nb[2], nb[1], nb[0], 32, 32, 32).transpose(0, 3, 1, 4, 2, 5)
    lin = a.reshape(nb[2] * 32, nb[1] * 32, nb[0] * 32)
    tables = None
    if dtype == "i8":
        off = (n + 255) // 256 * 256
        tsz = (nz * 4 + 255) // 256 * 256
        scale = raw[off: off + nz * 4].view(np.float32)
        offset = raw[off + tsz: off + tsz + nz * 4].view(np.float32)
        tables = (scale, offset)
    return lin, tables


@pytest.mark.parametrize("dtype", ["f32", "f16", "i8"])
def test_pack_is_bit_exact(dtype):
    dims = (45, 33, 70)
    cube = synth.make_cube(dims, 4, ("uniform", 3, 30), 11).numpy()
    cube[5] = 2.5                                 # a constant plane
    vol = Volume(torch.from_numpy(cube).cuda(), dtype)
    torch.cuda.synchronize()
    lin, tables = unbrick(vol.buffer, dims, dtype)
    inner = lin[:70, :33, :45]
    if dtype == "f32":
        assert np.array_equal(inner, cube)
    elif dtype == "f16":
        assert np.array_equal(inner.view(np.uint16), quantize.to_f16(cube).view(np.uint16))
    else:
        q, s, o = quantize.quantize_i8(cube)
        assert np.array_equal(inner, q)
        assert np.array_equal(tables[0].view(np.uint32), s.view(np.uint32))
        assert np.array_equal(tables[1].view(np.uint32), o.view(np.uint32))
    # padding is zero
    pad = lin.copy()
    pad[:70, :33, :45] = 0
    assert not pad.astype(np.float64).any()


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_pinned_host_source_and_slab_uploads_match_device_source(dtype):
    dims = (40, 36, 50)
    cube_t = synth.make_cube(dims, 3, ("uniform", 3, 9), 12)
    ref = Volume(cube_t.cuda(), dtype)
    pinned = Volume(cube_t.pin_memory(), dtype)
    slabs = Volume(dims=dims, dtype=dtype)
    for z0, z1 in ((0, 7), (7, 33), (33, 50)):
        slabs.upload(z0, cube_t[z0:z1].cuda())
    torch.cuda.synchronize()
    # compare the defined bytes: voxels, and for int8 the nz table entries
    # (the tables' 256-byte alignment padding is never written)
    a, ta = unbrick(ref.buffer, dims, dtype)
    for other in (pinned, slabs):
        b, tb = unbrick(other.buffer, dims, dtype)
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
        if ta is not None:
            assert np.array_equal(ta[0].view(np.uint32), tb[0].view(np.uint32))
            assert np.array_equal(ta[1].view(np.uint32), tb[1].view(np.uint32))


# ---------------------------------------------------------------------------
# determinism and argument errors
# ---------------------------------------------------------------------------
def test_repeated_views_are_bit_identical():
    dims = (30, 30, 30)
    cube = synth.make_cube(dims, 3, ("uniform", 3, 9), 13).cuda()
    vol = Volume(cube, "f32")
    vol.set_transfer(synth.default_lut(), 1.0, 9.0, 1.0, 0.99)
    cams = synth.random_sphere_cameras(dims, 1, 33, 31, 4)
    out = vol.render(np.concatenate([cams, cams, cams]), 33, 31, "composite", 0.5)
    assert torch.equal(out[0], out[1]) and torch.equal(out[0], out[2])


def test_argument_errors_raise():
    dims = (16, 16, 16)
    vol = Volume(synth.make_cube(dims, 0, ("uniform", 1, 2), 1).cuda(), "f32")
    cams = synth.random_sphere_cameras(dims, 1, 8, 8, 1)
    base = torch.empty(1 * 8 * 8 * 4 + 1, device="cuda")
    with pytest.raises(VRError):
        vol.render(cams, 8, 8, "composite", 0.5, out=base[1:].view(1, 8, 8, 4))  # misaligned
    with pytest.raises(VRError):
        vol.render(cams, 8, 8, "composite", 0.0)
    with pytest.raises(VRError):
        vol.render(cams, 8, 8, "composite", 1e-7)           # 2^24 samples per ray
    bad = cams.copy()
    bad[0]["eye"][0] = np.nan
    with pytest.raises(VRError):
        vol.render(bad, 8, 8, "mip", 0.5)
    with pytest.raises(VRError):
        vol.set_transfer(np.ones((1, 4), np.float32), 0, 1, 0)
    with pytest.raises(VRError):
        vol.set_transfer(np.full((4, 4), 2.0, np.float32), 0, 1, 0)
    with pytest.raises(VRError):
        vol.set_transfer(synth.default_lut(), 1.0, 1.0, 0)
    with pytest.raises(ValueError):
        vol.render(cams, 8, 8, "mip", 0.5, out=torch.empty(2, 8, 8, device="cuda"))
    # an empty image set: no views, or images without pixels
    for n, w, h in ((0, 8, 8), (1, 0, 8), (1, 8, 0)):
        with pytest.raises(VRError):
            vol.render(cams[:n], w, h, "composite", 0.5)


def test_brick_buffer_too_small_is_rejected():
    from paper_1001_2049_b300 import _lib
    import ctypes
    lib = _lib.load()
    buf = torch.empty(1024, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p(0)
    dims = (ctypes.c_int64 * 3)(64, 64, 64)
    rc = lib.vr_volume_create(dims, 0, None, 1, buf.data_ptr(), 1024, None, ctypes.byref(h))
    assert rc == _lib.VR_ERR_OOM
    assert volume_bytes((64, 64, 64), "f32") == 8 * 32768 * 4


def test_texture_only_volume_after_dropping_bricks():
    dims = (40, 36, 50)
    cube = synth.make_cube(dims, 4, ("uniform", 3.0, 8.0), 71).numpy()
    cams = synth.random_sphere_cameras(dims, 3, 21, 17, 9)
    lut = synth.default_lut(32)
    for dtype, pair in (("f32", False), ("f16", False), ("i8", False), ("i8", True)):
        vol = Volume(torch.from_numpy(cube).cuda(), dtype)
        vol.attach_pair_texture() if pair else vol.attach_texture()
        # a mask-free twin: the images at a clip below the masks' level
        twin = Volume(torch.from_numpy(cube).cuda(), dtype)
        twin.attach_pair_texture() if pair else twin.attach_texture()
        twin.set_transfer(lut, 0.6, 8.0, 0.6, 0.95)
        low = twin.render(cams, 21, 17, "composite", 0.5).cpu()
        vol.attach_masks()
        vol.set_transfer(lut, 1.0, 8.0, 1.0, 0.95)
        before = {m: vol.render(cams, 21, 17, m, 0.5).cpu() for m in ("composite", "mip")}
        vol.drop_bricks()
        assert vol.buffer is None
        for m in ("composite", "mip"):
            assert torch.equal(vol.render(cams, 21, 17, m, 0.5).cpu(), before[m])
        # the masks built for clip 1 stay, frozen: a lower clip renders
        # without them (they would drop its samples between 0.6 and 1), a
        # batch too, and the clip they were built for uses them again
        vol.set_transfer(lut, 0.6, 8.0, 0.6, 0.95)
        assert torch.equal(vol.render(cams, 21, 17, "composite", 0.5).cpu(), low)
        got = render_batch([Request(vol, c, 21, 17, "composite", 0.5) for c in cams])
        assert all(torch.equal(g.cpu(), low[i]) for i, g in enumerate(got))
        vol.set_transfer(lut, 1.0, 8.0, 1.0, 0.95)
        assert torch.equal(vol.render(cams, 21, 17, "composite", 0.5).cpu(), before["composite"])
        got = render_batch([Request(vol, c, 21, 17, "composite", 0.5) for c in cams])
        assert all(torch.equal(g.cpu(), before["composite"][i]) for i, g in enumerate(got))
        twin.close()
        with pytest.raises(VRError):
            vol.upload(0, torch.from_numpy(cube[:2]).cuda())
        with pytest.raises(VRError):
            vol.detach_texture()
        with pytest.raises(VRError):
            vol.attach_masks()
        vol.close()
    v32 = Volume(torch.from_numpy(cube).cuda(), "f32")
    with pytest.raises(VRError):                 # nothing to keep
        v32.drop_bricks()


# ---------------------------------------------------------------------------
# empty-space masks: every cell whose bit is clear is below the clip, and
# composite renders with the masks are identical to renders without them
# ---------------------------------------------------------------------------
def _decoded(cube, dtype):
    """Storage values as the kernels decode them (float32)."""
    if dtype == "f32":
        return cube.astype(np.float32)
    if dtype == "f16":
        return quantize.to_f16(cube).astype(np.float32)
    q, sc, of = quantize.quantize_i8(cube)
    return (q.astype(np.float64) * sc.astype(np.float64)[:, None, None]
            + of.astype(np.float64)[:, None, None]).astype(np.float32)


MASK_DIMS = [(37, 45, 70), (2, 2, 2), (6, 5, 9), (64, 3, 33), (6, 5, 4500)]


@pytest.mark.parametrize("dims", MASK_DIMS)
@pytest.mark.parametrize("dtype", ["f32", "f16", "i8"])
def test_masks_mark_every_cell_that_can_reach_the_clip(dims, dtype):
    cube = synth.make_cube(dims, 3, ("uniform", 3.0, 8.0), 40 + dims[0]).numpy()
    vol = Volume(torch.from_numpy(cube).cuda(), dtype)
    vol.attach_texture()
    vol.attach_masks()
    nx, ny, nz = dims
    mnx, mny, mnz = (nx >> 2) + 1, (ny >> 2) + 1, (nz >> 2) + 1
    assert vol.mask_bytes() == 8 * mnx * mny * mnz
    dec = _decoded(cube, dtype).astype(np.float64)
    # bound of each cell's eight corners, for gather coordinates in [0, n]
    # on every axis (cells -1 .. n - 1, the outermost reading the edge cell)
    hi = np.full((nz - 1, ny - 1, nx - 1), -np.inf)
    mag = np.zeros_like(hi)
    for c in range(8):
        sl = dec[(c >> 2):nz - 1 + (c >> 2), ((c >> 1) & 1):ny - 1 + ((c >> 1) & 1),
                 (c & 1):nx - 1 + (c & 1)]
        hi = np.maximum(hi, sl)
        mag = np.maximum(mag, np.abs(sl))
    bound = hi + 2.0 ** -19 * mag
    if dtype == "i8":
        # int8 interpolates each plane's codes, then decodes: 2^-14 of the
        # larger scale of a cell's two planes covers that rounding
        sc = np.abs(quantize.quantize_i8(cube)[1].astype(np.float64))
        bound = bound + 2.0 ** -14 * np.maximum(sc[:-1], sc[1:])[:, None, None]
    gx = np.clip(np.arange(nx + 1) - 1, 0, nx - 2)
    gy = np.clip(np.arange(ny + 1) - 1, 0, ny - 2)
    gz = np.clip(np.arange(nz + 1) - 1, 0, nz - 2)
    bound = bound[gz][:, gy][:, :, gx]                   # (nz + 1, ny + 1, nx + 1)
    hi = hi[gz][:, gy][:, :, gx]
    cams = synth.random_sphere_cameras(dims, 1, 4, 4, 3)
    z, y, x = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1),
                          indexing="ij")
    bit = ((x & 3) | ((y & 3) << 2) | ((z & 3) << 4)).astype(np.uint64)
    def bits(clip):
        vol.set_transfer(synth.default_lut(16), clip, 9.0, clip, 1.0)
        vol.render(cams, 4, 4, "composite", 0.5)     # builds the masks when needed
        torch.cuda.synchronize()
        words = vol._masks.cpu().numpy().view(np.uint64)[:mnx * mny * mnz]
        words = words.reshape(mnz, mny, mnx)
        return ((words[z >> 2, y >> 2, x >> 2] >> bit) & np.uint64(1)).astype(bool)

    def check(got, clip):
        want = bound >= clip
        clear = np.abs(bound - clip) > 1e-5 * max(1.0, abs(clip))   # not a rounding tie
        assert (got == want)[clear].all(), (dtype, dims, clip)
        # a clear bit never hides a corner at or above the clip
        assert not (~got & (hi >= clip)).any()

    for clip in (2.0, 4.5):                 # fresh masks are exact for their clip
        vol.attach_masks()
        check(bits(clip), clip)
    low = bits(2.0)                         # lowering the clip rebuilds them
    check(low, 2.0)
    assert (bits(4.5) == low).all()         # raising it keeps them (conservative)
    check(bits(1.5), 1.5)


def _skip_cases(dims, seed):
    cube = synth.make_cube(dims, 3, ("uniform", 3.0, 8.0), seed).numpy()
    cams = synth.random_sphere_cameras(dims, 4, 29, 19, seed, fov_deg=70.0)
    c = np.array([(d - 1) / 2.0 for d in dims])
    recs = [synth.look_at_camera(c + 0.3, c + np.array([5.0, -3.0, 2.0]), 29, 19, 90.0)]
    recs += [synth.axis_camera(dims, 29, 19, axis=a, sign=sg) for a in range(3) for sg in (1, -1)]
    cams = np.concatenate([cams, synth.cameras(recs).astype(cams.dtype)])
    return cube, cams


@pytest.mark.parametrize("dims", MASK_DIMS)
@pytest.mark.parametrize("store", ["f32", "f16", "i8", "f16-pair", "i8-pair"])
def test_masks_leave_images_and_counts_unchanged(dims, store):
    dtype, _, pair = store.partition("-")
    cube, cams = _skip_cases(dims, 50 + dims[1])
    vol = Volume(torch.from_numpy(cube).cuda(), dtype)
    if pair:
        vol.attach_pair_texture()
    else:
        vol.attach_texture()
    lut = synth.default_lut(64)
    for clip in (-10.0, 1.0, 3.0, 100.0):       # nothing, some, most, everything skippable
        vol.set_transfer(lut, min(clip, 7.0), 8.0, clip, 0.95)
        outs = []
        for masks in (False, True):
            if masks:
                vol.attach_masks()
            n = torch.zeros(1, dtype=torch.int64, device="cuda")
            img = vol.render(cams, 29, 19, "composite", 0.37, count=n)
            torch.cuda.synchronize()
            outs.append((img.cpu(), int(n.item())))
            vol.detach_masks()
        assert torch.equal(outs[0][0], outs[1][0]), (store, dims, clip)
        assert outs[0][1] == outs[1][1], (store, dims, clip)


def test_masks_follow_clip_changes_and_uploads():
    dims = (40, 36, 50)
    cube = synth.make_cube(dims, 4, ("uniform", 3.0, 8.0), 61).numpy()
    cams = synth.random_sphere_cameras(dims, 3, 21, 21, 5)
    vol = Volume(torch.from_numpy(cube).cuda(), "f32")
    vol.attach_texture()
    ref = Volume(torch.from_numpy(cube).cuda(), "f32")
    ref.attach_texture()
    vol.attach_masks()
    lut = synth.default_lut(32)
    for clip in (3.0, 1.0, 3.0):
        for v in (vol, ref):
            v.set_transfer(lut, clip, 8.0, clip, 1.0)
        assert torch.equal(vol.render(cams, 21, 21, "composite", 0.5),
                           ref.render(cams, 21, 21, "composite", 0.5))
    # new planes: the masks are rebuilt for them
    cube2 = cube.copy()
    cube2[20:30] += 5.0
    for v in (vol, ref):
        v.upload(20, torch.from_numpy(cube2[20:30]).cuda())
    assert torch.equal(vol.render(cams, 21, 21, "composite", 0.5),
                       ref.render(cams, 21, 21, "composite", 0.5))


def test_masks_on_a_sparse_cube():
    # one bright voxel in an empty cube: every cell but the eight around it
    # is skipped
    dims = (40, 36, 50)
    cube = np.zeros((50, 36, 40), dtype=np.float32)
    cube[21, 17, 13] = 9.0
    cams = synth.random_sphere_cameras(dims, 6, 31, 31, 7, fov_deg=40.0)
    recs = [synth.axis_camera(dims, 40, 36, axis=2, sign=1)]
    cams = np.concatenate([cams, synth.cameras(recs).astype(cams.dtype)])
    # the axis view (one of seven) has structural K ties on its rays
    run_parity(cube, "f32", cams, 31, 31, "composite", 0.5, synth.default_lut(32), 0.5, 9.0,
               0.5, 1.0, what="sparse masks", tex=True, masks=True, ties={"k": 1.0 / 7 + 0.01})


@pytest.mark.parametrize("tex", [True, "pair"], ids=["texture", "pair"])
def test_masks_small_workload(small, tex):
    wl, cube, lut, cams = small
    dtype = "f32" if tex is True else "f16"
    run_parity(cube, dtype, cams, 256, 256, "composite", wl.step, lut, wl.clip, wl.v_hi, wl.clip,
               wl.term_alpha, what="small masks " + dtype, tex=tex, masks=True,
               ties=SMALL_TIES)


@pytest.mark.parametrize("dims,step", RAGGED)
@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_masks_ragged_cubes(dims, step, dtype):
    cube, cams, lut = ragged_case(dims, 17 + dims[0])
    # the clip (3) lies above the table's bottom (1): clip ties can occur
    run_parity(cube, dtype, cams, 23, 17, "composite", step, lut, 1.0, 8.0, 3.0, 0.95,
               what="masks ragged %s %s" % (dims, dtype), tex=True, masks=True,
               ties={"clip": 0.01})


# ---------------------------------------------------------------------------
# MIP bounds: 8-bit upper-bound codes decide which samples read the FP32 texels
# ---------------------------------------------------------------------------
def _mip_with_and_without_bounds(vol, cams, w, h, step):
    outs = []
    for bounds in (False, True):
        if bounds:
            vol.attach_mip_bounds()
        n = torch.zeros(1, dtype=torch.int64, device="cuda")
        img = vol.render(cams, w, h, "mip", step, count=n)
        torch.cuda.synchronize()
        outs.append((img.cpu(), int(n.item())))
        vol.detach_mip_bounds()
    return outs


@pytest.mark.parametrize("dims", MASK_DIMS)
def test_mip_bounds_leave_images_and_counts_unchanged(dims):
    cube, cams = _skip_cases(dims, 70 + dims[2])
    vol = Volume(torch.from_numpy(cube).cuda(), "f32")
    vol.attach_texture()
    (a, na), (b, nb) = _mip_with_and_without_bounds(vol, cams, 29, 19, 0.37)
    assert torch.equal(a, b), dims
    assert na == nb


def test_mip_bounds_with_extreme_values():
    # voxels beyond binary16's range, hugely negative, NaN and infinite
    # voxels, tiny and subnormal values: identical images
    dims = (23, 19, 31)
    cube, cams = _skip_cases(dims, 77)
    rng = np.random.default_rng(5)
    flat = cube.reshape(-1)
    idx = rng.choice(flat.size, 60, replace=False)
    flat[idx[:10]] = 7.0e4
    flat[idx[10:20]] = -3.0e6
    flat[idx[20:25]] = np.nan
    flat[idx[25:28]] = np.inf
    flat[idx[28:31]] = -np.inf
    flat[idx[31:45]] = 1.0e-30
    flat[idx[45:60]] = 3.0e-41
    vol = Volume(torch.from_numpy(cube).cuda(), "f32")
    vol.attach_texture()
    (a, na), (b, nb) = _mip_with_and_without_bounds(vol, cams, 29, 19, 0.5)
    assert torch.equal(a, b) or torch.equal(torch.nan_to_num(a), torch.nan_to_num(b))
    assert na == nb
    # a cube of subnormal values only: the margin covers their rounding
    tiny = (np.abs(cube) * 1e-40).astype(np.float32)
    vol = Volume(torch.from_numpy(np.nan_to_num(tiny, posinf=0.0)).cuda(), "f32")
    vol.attach_texture()
    (a, _), (b, _) = _mip_with_and_without_bounds(vol, cams, 29, 19, 0.5)
    assert torch.equal(a, b)
    # the largest finite floats beside ordinary noise (a range that overflows:
    # no code scale, every sample a candidate)
    big, _ = _skip_cases(dims, 78)
    fb = big.reshape(-1)
    fmax = np.finfo(np.float32).max
    fb[idx[:5]] = fmax
    fb[idx[5:10]] = -fmax
    vol = Volume(torch.from_numpy(big).cuda(), "f32")
    vol.attach_texture()
    (a, na), (b, nb) = _mip_with_and_without_bounds(vol, cams, 29, 19, 0.5)
    assert torch.equal(a, b) and na == nb


def test_mip_bounds_on_degenerate_ranges():
    # the code scale's edge cases: a constant cube (range 0: every sample a
    # candidate), a cube of NaN but one plane, a range far below one code
    # step of a normal scale (subnormal differences) and one that overflows
    # a float (no scale: skipping off); images and counts as without bounds
    dims = (21, 18, 26)
    _, cams = _skip_cases(dims, 80)
    rng = np.random.default_rng(9)
    cases = {
        "constant": np.full(dims[::-1], 2.5, np.float32),
        "nan": np.full(dims[::-1], np.nan, np.float32),
        "tiny range": (np.float32(1.0) + rng.integers(0, 3, dims[::-1]).astype(np.float32)
                       * np.float32(2.0 ** -23)),
        "overflowing range": np.clip(rng.standard_normal(dims[::-1]) * 1e38, -3e38,
                                     3e38).astype(np.float32),
    }
    cases["nan"][5] = rng.standard_normal(dims[1::-1]).astype(np.float32)
    for name, cube in cases.items():
        vol = Volume(torch.from_numpy(np.ascontiguousarray(cube)).cuda(), "f32")
        vol.attach_texture()
        (a, na), (b, nb) = _mip_with_and_without_bounds(vol, cams, 29, 19, 0.41)
        assert torch.equal(torch.nan_to_num(a), torch.nan_to_num(b)), name
        assert na == nb, name


def test_mip_bounds_on_negative_cubes():
    # every voxel negative, so every ray's maximum is negative (the limit of
    # the running maximum is then below the codes' origin until the maximum
    # passes it); values with low bits set in every magnitude
    dims = (29, 23, 37)
    cube, cams = _skip_cases(dims, 79)
    for shift, scale in ((-40.0, 1.0), (-1.0e-3, 1.0e-4), (-3.0e5, 7.0e3)):
        neg = (cube * np.float32(scale) + np.float32(shift)).astype(np.float32)
        neg = np.minimum(neg, np.float32(-1e-38))
        vol = Volume(torch.from_numpy(neg).cuda(), "f32")
        vol.attach_texture()
        (a, na), (b, nb) = _mip_with_and_without_bounds(vol, cams, 29, 19, 0.37)
        assert torch.equal(a, b), shift
        assert na == nb
        assert float(a.max()) < 0.0


def test_mip_bounds_small_workload_against_the_oracle(small):
    wl, cube, lut, cams = small
    run_parity(cube, "f32", cams, 256, 256, "mip", wl.step, lut, wl.clip, wl.v_hi, wl.clip,
               wl.term_alpha, what="small mip bounds", tex=True, bounds=True,
               ties=SMALL_TIES)


@pytest.mark.parametrize("dims,step", RAGGED)
def test_mip_bounds_ragged_cubes(dims, step):
    cube, cams, lut = ragged_case(dims, 29 + dims[0])
    run_parity(cube, "f32", cams, 23, 17, "mip", step, lut, 1.0, 8.0, 3.0, 0.95,
               what="mip bounds ragged %s" % (dims,), tex=True, bounds=True)


def test_mip_bounds_follow_uploads_and_survive_dropping_bricks():
    dims = (40, 36, 50)
    cube = synth.make_cube(dims, 4, ("uniform", 3.0, 8.0), 62).numpy()
    cams = synth.random_sphere_cameras(dims, 3, 21, 21, 6)
    vol = Volume(torch.from_numpy(cube).cuda(), "f32")
    vol.attach_texture()
    vol.attach_mip_bounds()
    ref = Volume(torch.from_numpy(cube).cuda(), "f32")
    ref.attach_texture()
    assert torch.equal(vol.render(cams, 21, 21, "mip", 0.5), ref.render(cams, 21, 21, "mip", 0.5))
    # new planes beyond the cube's range: skipping is turned off, images stay
    cube2 = cube.copy()
    cube2[20:30] = cube2[20:30] * 40.0 + 3.0
    for v in (vol, ref):
        v.upload(20, torch.from_numpy(cube2[20:30]).cuda())
    assert torch.equal(vol.render(cams, 21, 21, "mip", 0.5), ref.render(cams, 21, 21, "mip", 0.5))
    vol.drop_bricks()
    assert torch.equal(vol.render(cams, 21, 21, "mip", 0.5), ref.render(cams, 21, 21, "mip", 0.5))
    vol.detach_mip_bounds()
    with pytest.raises(VRError):                  # the bricks are gone: no new bounds
        vol.attach_mip_bounds()


def test_mip_bounds_are_refused_where_they_do_not_apply():
    cube = synth.make_cube((16, 16, 16), 2, ("uniform", 3.0, 8.0), 63)
    for dtype in ("f16", "i8"):
        v = Volume(cube.cuda(), dtype)
        v.attach_texture()
        with pytest.raises(VRError):
            v.attach_mip_bounds()
    v = Volume(cube.cuda(), "f32")
    with pytest.raises(VRError):                  # no texture storage
        v.attach_mip_bounds()
    v.attach_texture()
    v.attach_mip_bounds()
    v.attach_mip_bounds()                         # attaching twice is a no-op
    v.detach_texture()                            # releases the bounds too
    with pytest.raises(VRError):
        v.attach_mip_bounds()


# ---------------------------------------------------------------------------
# the 1024^3 workload at full size, in the benchmark's launch configuration
# (32 orbiting 1920x1080 views in one call), checked on sampled pixels
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def large():
    wl = synth.LARGE
    cube = wl.cube("cuda")
    host = cube.cpu().numpy()
    return wl, cube, host


def _sample_pixels(n_views, w, h, n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, n_views, n), rng.integers(0, w, n),
                     rng.integers(0, h, n)], axis=1).astype(np.int32)


@functools.lru_cache(maxsize=2)
def _hard_pixels_cached(n_views, w, h, dims, step, n, seed):
    return _hard_pixels(synth.large_cameras(n_views, w, h), w, h, dims, step, n, seed)


def _hard_pixels(cams, w, h, dims, step, n, seed):
    """Pixels where a single-precision render is most likely to part from
    the definition: rays that graze the box (at most 8 samples, or missing
    it by less than a voxel) and rays whose (t_exit - t_entry)/step is
    within 0.01 of an integer (the K decision).  The ray-box geometry is
    evaluated here in FP64 with numpy, only to choose the pixels."""
    rng = np.random.default_rng(seed)
    graze, ktie = [], []
    py, px = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64),
                         indexing="ij")
    u, v = px.ravel() + 0.5 - w / 2.0, py.ravel() + 0.5 - h / 2.0
    for vi, c in enumerate(cams):
        eye, fwd, du, dv = (np.asarray(c[k], np.float64) for k in ("eye", "fwd", "du", "dv"))
        d = fwd[:, None] + du[:, None] * u + dv[:, None] * v
        d /= np.linalg.norm(d, axis=0)
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (0.0 - eye[:, None]) / d
            tb = (np.asarray(dims, np.float64)[:, None] - 1.0 - eye[:, None]) / d
        te = np.maximum(np.minimum(ta, tb).max(axis=0), 0.0)
        tf = np.maximum(ta, tb).min(axis=0)
        q = (tf - te) / step
        g = np.flatnonzero((q > -2.0) & (q < 8.0))
        fr = q - np.floor(q)
        k = np.flatnonzero((q >= 0) & ((fr < 0.01) | (fr > 0.99)))
        graze += [(vi, i % w, i // w) for i in g]
        ktie += [(vi, i % w, i // w) for i in k]
    out = []
    for lst in (graze, ktie):
        a = np.asarray(lst, dtype=np.int32).reshape(-1, 3)
        if len(a) > n:
            a = a[rng.choice(len(a), n, replace=False)]
        out.append(a)
    return np.concatenate(out)


@pytest.mark.parametrize("tex", [True, False], ids=["texture", "bricks"])
@pytest.mark.parametrize("dtype", ["f32", "f16", "i8"])
def test_large_workload_sampled_pixels(large, dtype, tex):
    wl, cube, host = large
    cams = synth.large_cameras()
    w, h = 1920, 1080
    lut = synth.default_lut()
    vol = Volume(cube, dtype)
    if tex:
        vol.attach_texture()
    vol.set_transfer(lut, wl.clip, wl.v_hi, wl.clip, wl.term_alpha)
    # 60,000 random pixels (for the tie fractions) and 8,000 pixels of
    # grazing rays and near-integer sample counts
    n_rand = 60000
    pix = np.concatenate([_sample_pixels(len(cams), w, h, n_rand, 99),
                          _hard_pixels_cached(len(cams), w, h, wl.dims, wl.step, 4000, 98)])
    ovol = oracle_volume(host, dtype)
    src = oracle.Volume(host)
    tf = oracle.TF(lut, wl.clip, wl.v_hi, wl.clip, wl.term_alpha)
    bands = bands_for(wl.dims, cams, wl.step, w, h)
    reports = {}
    for mode in ("composite", "mip"):
        n0 = torch.zeros(1, dtype=torch.int64, device="cuda")
        img = vol.render(cams, w, h, mode, wl.step, count=n0)
        if tex and mode == "composite":
            # with the empty-space masks (the benchmark's configuration) the
            # images and the sample counts are the same, bit for bit
            vol.attach_masks()
            n1 = torch.zeros(1, dtype=torch.int64, device="cuda")
            img1 = vol.render(cams, w, h, mode, wl.step, count=n1)
            vol.detach_masks()
            torch.cuda.synchronize()
            assert torch.equal(img, img1), "large %s %s: masks change the image" % (dtype, mode)
            assert int(n0.item()) == int(n1.item())
            img = img1
        if tex and dtype == "f32" and mode == "mip":
            # with the MIP bounds (the benchmark's configuration) likewise
            vol.attach_mip_bounds()
            n1 = torch.zeros(1, dtype=torch.int64, device="cuda")
            img1 = vol.render(cams, w, h, mode, wl.step, count=n1)
            vol.detach_mip_bounds()
            torch.cuda.synchronize()
            assert torch.equal(img, img1), "large mip: bounds change the image"
            assert int(n0.item()) == int(n1.item())
            img = img1
        torch.cuda.synchronize()
        got = img.cpu().numpy()
        ch = 4 if mode == "composite" else 1
        flat = got.reshape(len(cams), h, w, ch)[pix[:, 0], pix[:, 2], pix[:, 1]]
        sc = scale_for(mode, host, got)
        res = oracle.render(ovol, cams, w, h, MODES[mode], wl.step, tf, pixels=pix, bands=bands)
        reports[mode] = compare(res, flat, MODES[mode], TOL_FP32, sc,
                                what="large %s %s" % (dtype, mode))
        # on the random pixels: at most 1 % K ties, 2 % termination ties
        rnd = oracle.Result(res.values[:n_rand], res.nalt[:n_rand], res.flags[:n_rand],
                            res.nsamples[:n_rand])
        reports[mode]["ties"] = assert_ties(rnd, "large %s %s" % (dtype, mode), k=0.01,
                                            term=0.02)
        if dtype != "f32":
            res = oracle.render(src, cams, w, h, MODES[mode], wl.step, tf, pixels=pix,
                                bands=bands)
            reports[mode + "_vs_source"] = compare(res, flat, MODES[mode], TOL_PREC[dtype], sc,
                                                   what="large %s %s vs source" % (dtype, mode))
    print("large", dtype, "texture" if tex else "bricks", reports)


def test_device_bytes_match_what_an_attach_takes():
    # the byte queries against the device's free memory around each attach
    # (the driver rounds allocations up to its 2 MiB pages and tile edges)
    from paper_1001_2049_b300 import mip_bounds_bytes, texture_bytes
    dims = (256, 256, 300)
    cube = synth.make_cube(dims, 2, ("uniform", 3.0, 6.0), 5).cuda()
    for dtype, pair in (("f32", False), ("f16", True), ("i8", False)):
        vol = Volume(cube, dtype)
        torch.cuda.synchronize()
        lib0, caller0 = vol.device_bytes()
        assert lib0 == 0 and caller0 == volume_bytes(dims, dtype)
        steps = [("texture", texture_bytes(dims, dtype, pair),
                  vol.attach_pair_texture if pair else vol.attach_texture)]
        if dtype == "f32":
            steps.append(("bounds", mip_bounds_bytes(dims), vol.attach_mip_bounds))
        held = 0
        for name, want, attach in steps:
            free0 = torch.cuda.mem_get_info()[0]
            attach()
            torch.cuda.synchronize()
            took = free0 - torch.cuda.mem_get_info()[0]
            assert abs(took - want) <= max(4 << 20, 0.03 * want), (dtype, name, took, want)
            held += want
            assert vol.device_bytes()[0] == held
        vol.attach_masks()
        assert vol.device_bytes()[1] == volume_bytes(dims, dtype) + vol.mask_bytes()
        vol.close()
