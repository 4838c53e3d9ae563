"""Object-order MIP (vr_render_object_order) on the GPU.

Sub-cubes of 32^3 cells are staged in shared memory once per launch and each
ray's samples are taken by the sub-cube whose k-interval holds them, so the
images and sample counts must be the texture march's MIP bit for bit (every
storage type, cubes smaller than one sub-cube and spanning several, ragged
edges, perspective and orthographic views, rays in face planes, a camera
inside the cube, more views than one launch takes, extreme voxel values),
and within the FP64 oracle's acceptance sets."""
import numpy as np
import pytest
import torch

import oracle
from oracle import quantize
from paper_1001_2049_b300 import Volume, VRError, synth

from _util import TOL_FP32, TOL_PREC, assert_ties, bands_for, compare

pytestmark = pytest.mark.gpu


def _cams(dims, w, h, seed, n_random=4):
    cams = synth.random_sphere_cameras(dims, n_random, w, h, seed, fov_deg=70.0)
    c = np.array([(d - 1) / 2.0 for d in dims])
    recs = [synth.look_at_camera(c + 0.3, c + np.array([5.0, -3.0, 2.0]), w, h, 90.0)]
    recs += [synth.axis_camera(dims, w, h, axis=a, sign=s) for a in range(3) for s in (1, -1)]
    return np.concatenate([cams, synth.cameras(recs).astype(cams.dtype)])


def _both(vol, cams, w, h, step):
    """(texture-march MIP, count), (object-order MIP, count)."""
    outs = []
    for obj in (False, True):
        n = torch.zeros(1, dtype=torch.int64, device="cuda")
        f = vol.render_object_order if obj else vol.render
        img = f(cams, w, h, "mip", step, count=n)
        torch.cuda.synchronize()
        outs.append((img.cpu(), int(n.item())))
    return outs


@pytest.mark.parametrize("dims", [(23, 19, 31), (33, 65, 34), (70, 45, 97), (96, 80, 67)])
@pytest.mark.parametrize("dtype", ["f32", "f16", "i8"])
def test_object_order_is_the_texture_march_bit_for_bit(dims, dtype):
    cube = synth.make_cube(dims, 3, ("uniform", 3.0, 8.0), 11 + dims[0]).numpy()
    cams = _cams(dims, 29, 19, 5 + dims[1])
    vol = Volume(torch.from_numpy(cube).cuda(), dtype)
    vol.attach_texture()
    (a, na), (b, nb) = _both(vol, cams, 29, 19, 0.37)
    assert torch.equal(a, b), (dims, dtype, int((a != b).sum()))
    assert na == nb and na > 0


def test_object_order_spans_launches_and_steps():
    # 70 views (two launches of at most 64), coarse and fine steps
    dims = (50, 41, 66)
    cube = synth.make_cube(dims, 4, ("uniform", 3.0, 8.0), 3).numpy()
    cams = synth.random_sphere_cameras(dims, 70, 12, 10, 21)
    vol = Volume(torch.from_numpy(cube).cuda(), "f32")
    vol.attach_texture()
    for step in (0.23, 0.5, 1.7):
        (a, na), (b, nb) = _both(vol, cams, 12, 10, step)
        assert torch.equal(a, b), step
        assert na == nb


def test_object_order_with_extreme_values():
    dims = (40, 35, 45)
    cube = synth.make_cube(dims, 3, ("uniform", 3.0, 8.0), 77).numpy()
    rng = np.random.default_rng(5)
    flat = cube.reshape(-1)
    idx = rng.choice(flat.size, 80, replace=False)
    flat[idx[:10]] = 7.0e4
    flat[idx[10:20]] = -3.0e6
    flat[idx[20:25]] = np.nan
    flat[idx[25:28]] = np.inf
    flat[idx[28:31]] = -np.inf
    flat[idx[31:45]] = 1.0e-30
    flat[idx[45:60]] = 3.0e-41
    flat[idx[60:70]] = np.finfo(np.float32).max
    cams = _cams(dims, 29, 19, 8)
    vol = Volume(torch.from_numpy(cube).cuda(), "f32")
    vol.attach_texture()
    (a, na), (b, nb) = _both(vol, cams, 29, 19, 0.5)
    assert torch.equal(torch.nan_to_num(a), torch.nan_to_num(b))
    assert torch.equal(torch.isnan(a), torch.isnan(b))
    assert na == nb
    neg = (synth.make_cube(dims, 3, ("uniform", 3.0, 8.0), 78).numpy() - 40.0).astype(np.float32)
    vol = Volume(torch.from_numpy(neg).cuda(), "f32")
    vol.attach_texture()
    (a, na), (b, nb) = _both(vol, cams, 29, 19, 0.5)
    assert torch.equal(a, b) and na == nb


def test_object_order_on_a_512_cube_at_the_workload_framing():
    # the 1024^3 workload's orbit framing and ray spacing, halved: several
    # hundred sub-cubes, long rays, 960 x 540 views
    edge = 512
    dims = (edge,) * 3
    cube = synth.make_cube(dims, 250, ("uniform", 3.0, 50.0), 4, device="cuda")
    cams = synth.orbit_cameras(dims, 4, 960, 540)
    vol = Volume(cube, "f32")
    vol.attach_texture()
    vol.attach_mip_bounds()
    (a, na), (b, nb) = _both(vol, cams, 960, 540, 0.5)
    assert torch.equal(a, b)
    assert na == nb and na > 10 ** 8


def _oracle_volume(cube, dtype):
    if dtype == "f32":
        return oracle.Volume(cube)
    if dtype == "f16":
        return oracle.Volume(quantize.to_f16(cube))
    q, s, o = quantize.quantize_i8(cube)
    return oracle.Volume(q, s, o)


@pytest.mark.parametrize("dtype", ["f32", "f16", "i8"])
def test_object_order_against_the_oracle(dtype):
    wl = synth.SMALL
    cube = wl.cube("cpu").numpy()
    nz, ny, nx = cube.shape
    lut = synth.default_lut()
    tf = oracle.TF(lut, wl.clip, wl.v_hi, wl.clip, wl.term_alpha)
    vol = Volume(torch.from_numpy(cube).cuda(), dtype)
    ovol = _oracle_volume(cube, dtype)
    for cams, w, h, ties in ((synth.small_camera(), 256, 256, {"k": 1.0}),
                             (synth.orbit_cameras((nx, ny, nz), 8, 64, 64), 64, 64, None)):
        got = vol.render_object_order(cams, w, h, "mip", wl.step).cpu().numpy()
        res = oracle.render(ovol, cams, w, h, oracle.MIP, wl.step, tf,
                            bands=bands_for((nx, ny, nz), cams, wl.step, w, h))
        assert_ties(res, "object order %s" % dtype, **(ties or {}))
        compare(res, got.reshape(-1, 1), oracle.MIP, TOL_FP32,
                float(cube.max() - cube.min()), what="object order %s" % dtype)
        if dtype != "f32":
            src = oracle.render(oracle.Volume(cube), cams, w, h, oracle.MIP, wl.step, tf,
                                bands=bands_for((nx, ny, nz), cams, wl.step, w, h))
            compare(src, got.reshape(-1, 1), oracle.MIP, TOL_PREC[dtype],
                    float(cube.max() - cube.min()), what="object order %s vs source" % dtype)


def test_object_order_without_texture_and_refusals():
    dims = (23, 19, 31)
    cube = synth.make_cube(dims, 3, ("uniform", 3.0, 8.0), 2).numpy()
    cams = _cams(dims, 16, 12, 3)
    vol = Volume(torch.from_numpy(cube).cuda(), "f32")
    plain = vol.render_object_order(cams, 16, 12, "mip", 0.5)    # bricks only
    vol.attach_texture()
    tex = vol.render(cams, 16, 12, "mip", 0.5)
    assert torch.equal(plain, tex)
    with pytest.raises(VRError):
        vol.render_object_order(cams, 16, 12, "composite", 0.5)
    with pytest.raises(ValueError):
        vol.render_object_order(cams, 16, 12, "mip", 0.5,
                                out=torch.empty((len(cams), 12, 16, 4), device="cuda"))
    vol.drop_bricks()
    with pytest.raises(VRError):
        vol.render_object_order(cams, 16, 12, "mip", 0.5)
