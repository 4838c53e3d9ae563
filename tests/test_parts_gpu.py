"""Rendering a cube part by part (vr_render_part through stream.PartStream)
gives the one-pass images and sample counts bit for bit: every sample is
computed as the one-pass render computes it, in the same order along each
ray, the parts continuing the images the earlier parts left."""
import numpy as np
import pytest
import torch

from paper_1001_2049_b300 import Volume, VRError, render_init, synth
from paper_1001_2049_b300.stream import PartStream, sweeps

pytestmark = pytest.mark.gpu

MODES = ("composite", "mip", "sum")


def _case(dims, seed, w=29, h=19):
    cube = synth.make_cube(dims, 3, ("uniform", 3.0, 8.0), seed)
    cams = synth.random_sphere_cameras(dims, 4, w, h, seed, fov_deg=70.0)
    c = np.array([(d - 1) / 2.0 for d in dims])
    recs = [synth.look_at_camera(c + 0.3, c + np.array([5.0, -3.0, 2.0]), w, h, 90.0)]
    recs += [synth.axis_camera(dims, w, h, axis=a, sign=sg) for a in range(3) for sg in (1, -1)]
    cams = np.concatenate([cams, synth.cameras(recs).astype(cams.dtype)])
    return cube, cams


def _one_pass(cube, dtype, pair, cams, w, h, step, lut, tf):
    vol = Volume(cube.cuda(), dtype)
    vol.attach_pair_texture() if pair else vol.attach_texture()
    vol.set_transfer(lut, *tf)
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    imgs = {m: vol.render(cams, w, h, m, step, count=n) for m in MODES}
    torch.cuda.synchronize()
    return imgs, int(n.item())


@pytest.mark.parametrize("store", ["f32", "f16-pair", "i8", "i8-pair"])
@pytest.mark.parametrize("dims,part_planes", [((37, 45, 70), 2), ((37, 45, 70), 9),
                                              ((37, 45, 70), 16), ((20, 17, 9), 64),
                                              ((6, 5, 4500), 700)])
def test_parts_give_the_one_pass_images(store, dims, part_planes):
    dtype, _, pair = store.partition("-")
    cube, cams = _case(dims, 80 + part_planes)
    w, h, step = 29, 19, 0.37
    lut = synth.default_lut(64)
    tf = (1.0, 8.0, 1.0, 0.95)
    ref, n_ref = _one_pass(cube, dtype, bool(pair), cams, w, h, step, lut, tf)
    dev = cube.cuda()
    ps = PartStream(dims, dtype, lambda z0, n: dev[z0:z0 + n], part_planes, pair=bool(pair))
    ps.set_transfer(lut, *tf)
    outs = [(m, torch.empty(ref[m].shape, dtype=torch.float32, device="cuda")) for m in MODES]
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    ps.render(cams, w, h, outs, step, count=n)
    torch.cuda.synchronize()
    for m, out in outs:
        assert torch.equal(out, ref[m]), (store, dims, part_planes, m)
    assert int(n.item()) == n_ref
    ps.close()


@pytest.mark.parametrize("store", ["f32", "i8", "f16-pair"])
@pytest.mark.parametrize("cache", [3, 5, 12])
def test_part_cache_keeps_parts_resident_between_renders(store, cache):
    # the part volumes share one brick buffer; the least recently used one
    # takes the next part; the images stay those of one pass, render after
    # render, and a warm cache loads 2 (parts - cache) parts per render
    dtype, _, pair = store.partition("-")
    dims = (33, 29, 90)
    cube, cams = _case(dims, 97 + cache)
    w, h, step = 29, 19, 0.5
    lut = synth.default_lut(64)
    tf = (1.0, 8.0, 1.0, 0.95)
    ref, n_ref = _one_pass(cube, dtype, bool(pair), cams, w, h, step, lut, tf)
    host = cube.pin_memory()
    ps = PartStream(dims, dtype, lambda z0, n: host[z0:z0 + n], 12, pair=bool(pair),
                    cache_parts=cache)
    n_parts = len(ps.parts)
    assert len(ps.vols) == min(max(2, cache), n_parts)
    assert len(sweeps(cams, w, h, dims)) == 2
    ps.set_transfer(lut, *tf)
    outs = [(m, torch.empty(ref[m].shape, dtype=torch.float32, device="cuda")) for m in MODES]
    for r in range(3):
        before = ps.parts_loaded
        n = torch.zeros(1, dtype=torch.int64, device="cuda")
        ps.render(cams, w, h, outs, step, count=n)
        torch.cuda.synchronize()
        for m, out in outs:
            assert torch.equal(out, ref[m]), (store, cache, r, m)
        assert int(n.item()) == n_ref
        loads = ps.parts_loaded - before
        c = len(ps.vols)
        if r == 0:
            assert loads == 2 * n_parts - c
        else:
            assert loads == 2 * max(0, n_parts - c)
    ps.close()


@pytest.mark.parametrize("dims,part_planes,cache", [((33, 29, 90), 12, 3), ((37, 45, 70), 2, 2),
                                                    ((6, 5, 4500), 700, 4)])
def test_parts_with_mip_bounds_give_the_one_pass_images(dims, part_planes, cache):
    # FP32 part volumes with MIP bounds (filled from the shared bricks at each
    # part's upload): the one-pass images and counts, render after render
    cube, cams = _case(dims, 120 + part_planes)
    w, h, step = 29, 19, 0.37
    lut = synth.default_lut(64)
    tf = (1.0, 8.0, 1.0, 0.95)
    ref, n_ref = _one_pass(cube, "f32", False, cams, w, h, step, lut, tf)
    host = cube.pin_memory()
    dev = cube.cuda()
    for source in (lambda z0, n: host[z0:z0 + n], lambda z0, n: dev[z0:z0 + n]):
        ps = PartStream(dims, "f32", source, part_planes, cache_parts=cache, bounds=True)
        assert ps.bounds
        ps.set_transfer(lut, *tf)
        outs = [(m, torch.empty(ref[m].shape, dtype=torch.float32, device="cuda")) for m in MODES]
        for r in range(2):
            n = torch.zeros(1, dtype=torch.int64, device="cuda")
            ps.render(cams, w, h, outs, step, count=n)
            torch.cuda.synchronize()
            for m, out in outs:
                assert torch.equal(out, ref[m]), (dims, part_planes, r, m)
            assert int(n.item()) == n_ref
        ps.close()


@pytest.mark.parametrize("store", ["f32", "i8", "f16-pair"])
@pytest.mark.parametrize("dims,part_planes,cache", [((33, 29, 90), 12, 3), ((37, 45, 70), 2, 2),
                                                    ((6, 5, 4500), 700, 4)])
def test_parts_with_masks_give_the_one_pass_images(store, dims, part_planes, cache):
    # part volumes with empty-space masks built at each part's upload (and,
    # for FP32, MIP bounds): the one-pass images and counts at every clip,
    # a lower clip reloading the parts
    dtype, _, pair = store.partition("-")
    cube, cams = _case(dims, 140 + part_planes)
    w, h, step = 29, 19, 0.37
    lut = synth.default_lut(64)
    host = cube.pin_memory()
    ps = PartStream(dims, dtype, lambda z0, n: host[z0:z0 + n], part_planes, pair=bool(pair),
                    cache_parts=cache, masks=True, bounds=dtype == "f32")
    outs = [(m, torch.empty((len(cams), h, w, 4) if m == "composite" else (len(cams), h, w),
                            dtype=torch.float32, device="cuda")) for m in MODES]
    for clip in (1.0, 3.0, 0.5):
        tf = (min(clip, 1.0), 8.0, clip, 0.95)
        ref, n_ref = _one_pass(cube, dtype, bool(pair), cams, w, h, step, lut, tf)
        ps.set_transfer(lut, *tf)
        n = torch.zeros(1, dtype=torch.int64, device="cuda")
        ps.render(cams, w, h, outs, step, count=n)
        torch.cuda.synchronize()
        for m, out in outs:
            assert torch.equal(out, ref[m]), (store, dims, part_planes, clip, m)
        assert int(n.item()) == n_ref
    ps.close()


@pytest.mark.parametrize("cache,masks", [(3, False), (4, True), (2, False)])
def test_views_from_above_take_one_sweep_and_keep_the_first_parts(cache, masks):
    # orbit cameras above the cube: their ascending rays never enter it, so
    # one descending sweep serves them; the part volumes keep the parts a
    # sweep starts with, so repeated renders load fewer parts than the
    # least recently used choice would (all of them), with the images and
    # counts of one pass every time
    from paper_1001_2049_b300.stream import pick_volume
    dims = (31, 27, 96)
    cube = synth.make_cube(dims, 5, ("uniform", 3.0, 8.0), 140 + cache)
    w, h, step = 33, 21, 0.5
    cams = synth.orbit_cameras(dims, 6, w, h, elev_deg=20.0)
    assert sweeps(cams, w, h) == [1, -1] and sweeps(cams, w, h, dims) == [-1]
    lut = synth.default_lut(64)
    tf = (1.5, 8.0, 1.5, 0.95)
    ref, n_ref = _one_pass(cube, "f32", False, cams, w, h, step, lut, tf)
    host = cube.pin_memory()
    ps = PartStream(dims, "f32", lambda z0, n: host[z0:z0 + n], 13, cache_parts=cache,
                    bounds=True, masks=masks)
    ps.set_transfer(lut, *tf)
    n_parts, n_vols = len(ps.parts), len(ps.vols)
    # the host model of the volume choice over the same visits
    visits = [p.z_first for p in ps.parts[::-1]]
    holds, last, uses, expect = [None] * n_vols, [-1] * n_vols, 0, []
    for _ in range(4):
        loads = 0
        for k, z in enumerate(visits):
            if z in holds:
                i = holds.index(z)
            else:
                i = pick_volume(holds, last, visits, k)
                holds[i] = z
                loads += 1
            uses += 1
            last[i] = uses
        expect.append(loads)
    outs = [(m, torch.empty(ref[m].shape, dtype=torch.float32, device="cuda")) for m in MODES]
    got = []
    for r in range(4):
        before = ps.parts_loaded
        n = torch.zeros(1, dtype=torch.int64, device="cuda")
        ps.render(cams, w, h, outs, step, count=n)
        torch.cuda.synchronize()
        for m, out in outs:
            assert torch.equal(out, ref[m]), (cache, masks, r, m)
        assert int(n.item()) == n_ref
        got.append(ps.parts_loaded - before)
    assert got == expect
    assert got[0] == n_parts
    if n_vols > 2:
        assert max(got[1:]) < n_parts
    ps.close()


def test_parts_from_pinned_host_memory_and_one_way_views():
    dims = (48, 40, 96)
    cube = synth.make_cube(dims, 4, ("uniform", 3.0, 8.0), 91).pin_memory()
    w, h = 32, 24
    # orthographic views along -z and +z: one sweep each
    down = synth.cameras([synth.axis_camera(dims, w, h, axis=2, sign=-1)])
    up = synth.cameras([synth.axis_camera(dims, w, h, axis=2, sign=1)])
    assert sweeps(down, w, h, dims) == [-1] and sweeps(up, w, h, dims) == [1]
    lut = synth.default_lut(32)
    for cams in (down, up, np.concatenate([down, up])):
        ref, n_ref = _one_pass(cube, "f32", False, cams, w, h, 0.5, lut, (1.0, 8.0, 1.0, 0.9))
        ps = PartStream(dims, "f32", lambda z0, n: cube[z0:z0 + n], 17)
        ps.set_transfer(lut, 1.0, 8.0, 1.0, 0.9)
        out = torch.empty(ref["composite"].shape, dtype=torch.float32, device="cuda")
        n = torch.zeros(1, dtype=torch.int64, device="cuda")
        ps.render(cams, w, h, [("composite", out)], 0.5, count=n)
        torch.cuda.synchronize()
        assert torch.equal(out, ref["composite"])
        # each part is loaded once per sweep, except that the second sweep
        # starts with the parts the two part volumes still hold
        n_sweeps = len(sweeps(cams, w, h, dims))
        loads = len(ps.parts) * n_sweeps - (n_sweeps - 1) * min(len(ps.vols), len(ps.parts))
        assert ps.bytes_loaded == loads * 17 * 40 * 48 * 4
        ps.close()


def test_part_arguments_are_checked():
    dims = (16, 16, 40)
    cube = synth.make_cube(dims, 2, ("uniform", 3.0, 8.0), 5).cuda()
    part = Volume(cube[10:20].contiguous(), "f32")
    cams = synth.random_sphere_cameras(dims, 1, 8, 8, 1)
    out = render_init(torch.empty((1, 8, 8), device="cuda"), "mip")
    assert torch.isinf(out).all() and (out < 0).all()
    with pytest.raises(VRError):          # no texture storage
        part.render_part(dims, 10, 10, 19, cams, 8, 8, "mip", 0.5, 1, out)
    part.attach_texture()
    with pytest.raises(VRError):          # cells beyond the part's planes
        part.render_part(dims, 10, 10, 20, cams, 8, 8, "mip", 0.5, 1, out)
    with pytest.raises(VRError):          # planes beyond the cube
        part.render_part((16, 16, 15), 10, 10, 14, cams, 8, 8, "mip", 0.5, 1, out)
    with pytest.raises(VRError):
        part.render_part(dims, 10, 10, 19, cams, 8, 8, "mip", 0.5, 2, out)
    part.render_part(dims, 10, 10, 19, cams, 8, 8, "mip", 0.5, 1, out)
