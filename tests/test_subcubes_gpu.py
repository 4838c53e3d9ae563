"""Sub-cubes rendered independently and integrated (the paper's pipeline:
§3.1 items 1, 4, 5): every part's partial image from vr_render_part with
sweep 0, combined by vr_integrate_partials in each ray's order, against the
oracle's sub-cube rendering (FP64, each sub-cube stopping at its own
opacity); without early termination, also against the one-pass images."""
import numpy as np
import pytest
import torch

import oracle
from oracle import quantize
from paper_1001_2049_b300 import Volume, VRError, integrate_partials, synth
from paper_1001_2049_b300.stream import PartStream

from _util import TOL_FP32, assert_ties, bands_for, compare, sum_scale

pytestmark = pytest.mark.gpu

OMODE = {"mip": oracle.MIP, "composite": oracle.COMPOSITE, "sum": oracle.SUM}


def _oracle_volume(cube, dtype):
    if dtype == "f32":
        return oracle.Volume(cube)
    if dtype == "f16":
        return oracle.Volume(quantize.to_f16(cube))
    q, s, o = quantize.quantize_i8(cube)
    return oracle.Volume(q, s, o)


def _case(dims, seed, w=23, h=17):
    cube = synth.make_cube(dims, 4, ("uniform", 3.0, 8.0), seed).numpy()
    cams = synth.random_sphere_cameras(dims, 4, w, h, seed, fov_deg=70.0)
    c = np.array([(d - 1) / 2.0 for d in dims])
    inside = synth.look_at_camera(c + 0.3, c + np.array([5.0, -3.0, 2.0]), w, h, 90.0)
    cams = np.concatenate([cams, synth.cameras([inside]).astype(cams.dtype)])
    return cube, cams


def _check(got, res, mode, tol, scale, what):
    """Every pixel against the oracle's acceptance set (the primary FP64
    sub-cube result and the alternatives of the tie bands, including
    samples within rounding of a sub-cube boundary plane), with the ties
    bounded."""
    ch = 4 if mode == "composite" else 1
    rep = compare(res, np.asarray(got, dtype=np.float64).reshape(-1, ch), OMODE[mode], tol,
                  scale, what=str(what))
    rep["ties"] = assert_ties(res, str(what), clip=0.0, term=0.05)
    return rep


@pytest.mark.parametrize("store", ["f32", "f16-pair", "i8"])
@pytest.mark.parametrize("dims,part_planes", [((37, 45, 70), 9), ((33, 31, 65), 24),
                                              ((20, 17, 9), 3)])
def test_integrated_subcubes_match_the_oracle(store, dims, part_planes):
    dtype, _, pair = store.partition("-")
    cube, cams = _case(dims, 200 + part_planes)
    w, h, step = 23, 17, 0.37
    lut = synth.default_lut(64, alpha_max=0.8)
    tf = (1.0, 8.0, 1.0, 0.9)                 # early termination inside sub-cubes
    dev = torch.from_numpy(cube).cuda()
    ps = PartStream(dims, dtype, lambda z0, n: dev[z0:z0 + n], part_planes, pair=bool(pair),
                    cache_parts=3)
    ps.set_transfer(lut, *tf)
    outs = [(m, torch.empty((len(cams), h, w, 4) if m == "composite" else (len(cams), h, w),
                            device="cuda")) for m in OMODE]
    ps.render_subcubes(cams, w, h, outs, step)
    torch.cuda.synchronize()
    cell_lo = [p.cell_lo for p in ps.parts]
    ovol = _oracle_volume(cube, dtype)
    otf = oracle.TF(lut, *tf)
    for mode, out in outs:
        res = oracle.render_subcubes(ovol, cams, w, h, OMODE[mode], step, otf, cell_lo,
                                     bands=bands_for(dims, cams, step, w, h))
        got = out.cpu().numpy()
        if mode == "mip":
            scale = np.full(got.size, float(cube.max() - cube.min()))
        elif mode == "sum":
            scale = sum_scale(oracle.Volume(cube), cams, w, h, step, got)
        else:
            scale = np.ones(got.shape[0] * h * w)
        _check(got, res, mode, TOL_FP32, scale, (store, dims, part_planes, mode))
    ps.close()


def test_integration_without_termination_is_the_one_pass_image():
    # the front-to-back operator is associative: with term_alpha > 1 the
    # integrated image is the one-pass render's up to FP32 rounding; MIP is
    # the one-pass image bit for bit (the maximum is exact)
    dims = (37, 45, 70)
    cube, cams = _case(dims, 7)
    w, h, step = 23, 17, 0.5
    lut = synth.default_lut(64, alpha_max=0.8)
    tf = (1.0, 8.0, 1.0, 2.0)
    vol = Volume(torch.from_numpy(cube).cuda(), "f32")
    vol.attach_texture()
    vol.set_transfer(lut, *tf)
    ref = {m: vol.render(cams, w, h, m, step) for m in ("composite", "mip")}
    dev = torch.from_numpy(cube).cuda()
    ps = PartStream(dims, "f32", lambda z0, n: dev[z0:z0 + n], 11, cache_parts=2)
    ps.set_transfer(lut, *tf)
    outs = [(m, torch.empty_like(ref[m])) for m in ("composite", "mip")]
    ps.render_subcubes(cams, w, h, outs, step)
    torch.cuda.synchronize()
    assert torch.equal(outs[1][1], ref["mip"])
    d = (outs[0][1] - ref["composite"]).abs().max().item()
    assert d < 1e-5, d
    assert (ref["composite"][..., 3] > 0.3).sum().item() > 20
    ps.close()


def test_integration_order_follows_each_ray():
    # two synthetic partial image sets, as seen by rays going up (the first
    # set in front) and down (the second in front): the composite of a
    # half-opaque red front over an opaque blue back
    w, h = 8, 6
    up = synth.cameras([synth.axis_camera((8, 6, 10), w, h, axis=2, sign=1)])
    down = synth.cameras([synth.axis_camera((8, 6, 10), w, h, axis=2, sign=-1)])
    red = torch.tensor([0.5, 0.0, 0.0, 0.5], device="cuda")
    blue = torch.tensor([0.0, 0.0, 1.0, 1.0], device="cuda")
    parts = torch.stack([red.expand(1, h, w, 4), blue.expand(1, h, w, 4)]).contiguous()
    a = integrate_partials(parts, up, "composite")
    b = integrate_partials(parts, down, "composite")
    torch.cuda.synchronize()
    assert torch.allclose(a, torch.tensor([0.5, 0.0, 0.5, 1.0], device="cuda").expand_as(a))
    assert torch.allclose(b, torch.tensor([0.0, 0.0, 1.0, 1.0], device="cuda").expand_as(b))
    m = torch.tensor([[3.0], [5.0]], device="cuda").reshape(2, 1, 1, 1).expand(2, 1, h, w)
    assert (integrate_partials(m.contiguous(), up, "mip") == 5.0).all()
    assert (integrate_partials(m.contiguous(), up, "sum") == 8.0).all()


def test_integration_arguments_are_checked():
    w, h = 8, 6
    cams = synth.cameras([synth.axis_camera((8, 6, 10), w, h, axis=2, sign=1)])
    parts = torch.zeros((2, 1, h, w, 4), device="cuda")
    with pytest.raises(VRError):                # the output overlaps the partials
        integrate_partials(parts, cams, "composite", out=parts[1])
    with pytest.raises(ValueError):             # shape
        integrate_partials(parts, cams, "mip")
    bad = cams.copy()
    bad[0]["fwd"][2] = np.nan
    with pytest.raises(VRError):
        integrate_partials(parts, bad, "composite")


def test_subcubes_with_masks_and_bounds_are_bit_identical():
    # empty-space masks (composite) and MIP bounds (FP32 MIP) change only the
    # work of the partial renders, so the integrated images are those of the
    # same pipeline without them, bit for bit
    dims = (33, 31, 65)
    cube, cams = _case(dims, 61)
    w, h, step = 23, 17, 0.5
    lut = synth.default_lut(64, alpha_max=0.8)
    tf = (2.0, 8.0, 2.0, 0.9)
    dev = torch.from_numpy(cube).cuda()
    imgs = []
    for extra in (False, True):
        ps = PartStream(dims, "f32", lambda z0, n: dev[z0:z0 + n], 17, cache_parts=2,
                        bounds=extra, masks=extra)
        ps.set_transfer(lut, *tf)
        outs = [(m, torch.empty((len(cams), h, w, 4) if m == "composite" else (len(cams), h, w),
                                device="cuda")) for m in ("composite", "mip")]
        ps.render_subcubes(cams, w, h, outs, step)
        ps.render_subcubes(cams, w, h, outs, step)          # with the cache warm
        torch.cuda.synchronize()
        imgs.append([o.clone() for _, o in outs])
        ps.close()
    for a, b in zip(*imgs):
        assert torch.equal(a, b)


def test_integration_spans_several_launches_of_views():
    # more views than one launch carries (64 cameras): each view's partials
    # hold values of its own, and every view comes out in its own order
    w, h, n = 5, 3, 70
    dims = (8, 6, 10)
    recs = [synth.axis_camera(dims, w, h, axis=2, sign=1 if v % 2 == 0 else -1)
            for v in range(n)]
    cams = synth.cameras(recs)
    view = torch.arange(n, dtype=torch.float32, device="cuda").reshape(n, 1, 1, 1)
    front = torch.zeros((n, h, w, 4), device="cuda")
    front[..., 3] = 0.5
    front[..., 0] = 0.5 * view[..., 0] / n          # premultiplied red, per view
    back = torch.zeros((n, h, w, 4), device="cuda")
    back[..., 3] = 1.0
    back[..., 2] = 1.0
    parts = torch.stack([front, back]).contiguous()
    out = integrate_partials(parts, cams, "composite")
    torch.cuda.synchronize()
    for v in range(n):
        if v % 2 == 0:                               # up: the first partial in front
            want = torch.tensor([0.5 * v / n, 0.0, 0.5, 1.0], device="cuda")
        else:                                        # down: the opaque one in front
            want = torch.tensor([0.0, 0.0, 1.0, 1.0], device="cuda")
        assert torch.allclose(out[v], want.expand_as(out[v]), atol=1e-6), v
    m = view.reshape(1, n, 1, 1).expand(2, n, h, w) * torch.tensor(
        [1.0, -1.0], device="cuda").reshape(2, 1, 1, 1)
    mip = integrate_partials(m.contiguous(), cams, "mip")
    assert torch.equal(mip, view.reshape(n, 1, 1).expand(n, h, w))
