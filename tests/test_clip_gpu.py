"""The noise clip on the GPU, where it changes the image.

The clip (samples below it are transparent; the abstract's emphasis on low
signal-to-noise data, §3.1 item 3's pre-selected transfer function) is only
a discontinuity where the table's opacity at the clip level is non-zero.
With the workloads' tables (the table starts at the clip with zero opacity)
skipping a sample below the clip and compositing it give the same image, so
those tests cannot tell whether a kernel honours the clip.  Here two kinds
of table make it matter:

* ``raised``: the table spans [0, v_hi] and the clip sits above its bottom
  (opacity at the clip about 0.05 per voxel length);
* ``opaque``: the table starts at the clip with non-zero opacity (0.1 at
  the bottom rising to 0.5).

on noise cubes (sigma = 1) with the clip at 1 sigma, where many samples
lie near the clip, so the oracle's clip-tie alternatives are reached.
Every render path is compared with the FP64 oracle's acceptance sets:
brick, texture and pair-texture storage in FP32 / FP16 / int8, with and
without empty-space masks, the batched launch, part-by-part rendering, the
sub-cube pipeline with scene integration and the served mix.  Each case
also asserts its sensitivity: at the checked pixels the oracle with the
clip differs from the oracle without it (clip at -infinity) by far more
than the tolerance, so a kernel that ignored the clip would fail.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import quantize
from paper_1001_2049_b300 import Request, Volume, render_batch, synth
from paper_1001_2049_b300.serve import RenderJob, Server
from paper_1001_2049_b300.stream import PartStream

from _util import TOL_FP32, assert_ties, bands_for, compare

pytestmark = pytest.mark.gpu

OMODE = {"composite": oracle.COMPOSITE, "mip": oracle.MIP}


def raised_table():
    lut = synth.default_lut()
    return lut, 0.0, 10.0, 1.0          # lut, v_lo, v_hi, clip


def opaque_table():
    lut = synth.default_lut().copy()
    lut[:, 3] = 0.1 + 0.4 * np.arange(lut.shape[0]) / (lut.shape[0] - 1)
    return lut, 1.0, 10.0, 1.0


TABLES = {"raised": raised_table, "opaque": opaque_table}


def oracle_volume(cube, dtype):
    if dtype == "f32":
        return oracle.Volume(cube)
    if dtype == "f16":
        return oracle.Volume(quantize.to_f16(cube))
    return oracle.Volume(*quantize.quantize_i8(cube))


def noisy_case(dims, seed, n_views=4, w=29, h=23):
    """A noise cube with a few faint sources, perspective views from random
    directions and one camera inside the cube."""
    cube = synth.make_cube(dims, 3, ("uniform", 3.0, 6.0), seed).numpy()
    cams = synth.random_sphere_cameras(dims, n_views, w, h, seed, fov_deg=60.0)
    c = np.array([(d - 1) / 2.0 for d in dims])
    inside = synth.look_at_camera(c + 0.3, c + np.array([5.0, -3.0, 2.0]), w, h, 90.0)
    return cube, np.concatenate([cams, synth.cameras([inside]).astype(cams.dtype)]), w, h


def check(cube, dtype, cams, w, h, got, table, ta, step, what, mode="composite",
          clip_ties=0.05):
    """``got`` (views, h, w[, 4]) against the oracle's acceptance sets at
    every pixel, the ties bounded, and the clip shown to matter."""
    lut, v_lo, v_hi, clip = table
    nz, ny, nx = cube.shape
    ovol = oracle_volume(cube, dtype)
    bands = bands_for((nx, ny, nz), cams, step, w, h)
    res = oracle.render(ovol, cams, w, h, OMODE[mode], step, oracle.TF(lut, v_lo, v_hi, clip, ta),
                        bands=bands)
    ch = 4 if mode == "composite" else 1
    scale = float(cube.max() - cube.min()) if mode == "mip" else 1.0
    rep = compare(res, np.asarray(got).reshape(-1, ch), OMODE[mode], TOL_FP32, scale, what=what)
    rep["ties"] = assert_ties(res, what, clip=clip_ties, term=0.05)
    if mode == "composite":
        # sensitivity: the same render without the clip
        free = oracle.render(ovol, cams, w, h, oracle.COMPOSITE, step,
                             oracle.TF(lut, v_lo, v_hi, -1e30, ta), bands=bands)
        hit = res.nsamples > 0
        moved = np.abs(free.primary - res.primary).max(axis=1) > 100 * TOL_FP32
        assert hit.sum() > 0 and moved[hit].mean() > 0.5, (what, moved[hit].mean())
        rep["clip_moves"] = float(moved[hit].mean())
    return rep, res


def render_one(cube, dtype, cams, w, h, table, ta, step, store="bricks", masks=False):
    vol = Volume(torch.from_numpy(cube).cuda(), dtype)
    if store == "texture":
        vol.attach_texture()
    elif store == "pair":
        vol.attach_pair_texture()
    if masks:
        vol.attach_masks()
    lut, v_lo, v_hi, clip = table
    vol.set_transfer(lut, v_lo, v_hi, clip, ta)
    out = vol.render(cams, w, h, "composite", step)
    torch.cuda.synchronize()
    return out.cpu().numpy(), vol


STORES = [("f32", "bricks"), ("f16", "bricks"), ("i8", "bricks"), ("f32", "texture"),
          ("f16", "texture"), ("i8", "texture"), ("f16", "pair"), ("i8", "pair")]


@pytest.mark.parametrize("table", sorted(TABLES))
@pytest.mark.parametrize("dtype,store", STORES)
def test_clip_changes_the_image_on_every_storage(dtype, store, table):
    dims = (37, 45, 70)
    cube, cams, w, h = noisy_case(dims, 41)
    tb = TABLES[table]()
    for masks in ((False, True) if store != "bricks" else (False,)):
        got, _ = render_one(cube, dtype, cams, w, h, tb, 0.95, 0.5, store, masks)
        check(cube, dtype, cams, w, h, got, tb, 0.95, 0.5,
              "%s %s %s masks=%s" % (dtype, store, table, masks))


@pytest.mark.parametrize("table", sorted(TABLES))
def test_masks_keep_the_clipped_image_bit_for_bit(table):
    # a cleared mask bit must lie below a clip that removes opacity
    dims = (61, 53, 90)
    cube, cams, w, h = noisy_case(dims, 43, n_views=6, w=41, h=31)
    tb = TABLES[table]()
    for dtype, store in (("f32", "texture"), ("f16", "pair"), ("i8", "pair"), ("i8", "texture")):
        plain, _ = render_one(cube, dtype, cams, w, h, tb, 0.99, 0.5, store, masks=False)
        masked, _ = render_one(cube, dtype, cams, w, h, tb, 0.99, 0.5, store, masks=True)
        assert np.array_equal(plain, masked), (dtype, store, table)
        check(cube, dtype, cams, w, h, masked, tb, 0.99, 0.5, "masks %s %s %s" % (
            dtype, store, table))


def test_clip_ties_are_reached_on_longer_rays():
    # a larger cube seen from an orbit at 2x its edge: rays of ~250 samples
    # at the clip level of the noise, so a few percent of the pixels carry
    # clip-tie alternatives and the GPU matches one member of each set
    dims = (96, 80, 120)
    cube = synth.make_cube(dims, 6, ("uniform", 3.0, 10.0), 77).numpy()
    cams = synth.orbit_cameras(dims, 8, 64, 48)
    tb = raised_table()
    reps = []
    for clip in (1.0, 0.5):
        t = (tb[0], tb[1], tb[2], clip)
        got, _ = render_one(cube, "f32", cams, 64, 48, t, 0.99, 0.5, "texture", masks=True)
        rep, res = check(cube, "f32", cams, 64, 48, got, t, 0.99, 0.5, "orbit clip %g" % clip)
        reps.append(rep["ties"]["clip"])
    assert sum(reps) >= 50, reps      # the tie path is exercised


@pytest.mark.parametrize("table", sorted(TABLES))
def test_batched_launch_honours_each_requests_clip(table):
    # one batch over three storages, every request with its own clipped
    # table (two clip levels), against the oracle
    dims = (37, 45, 70)
    cube, cams, w, h = noisy_case(dims, 47, n_views=4)
    tb = TABLES[table]()
    vols = {}
    for dtype, store in (("f32", "texture"), ("f16", "pair"), ("i8", "bricks")):
        v = Volume(torch.from_numpy(cube).cuda(), dtype)
        if store == "texture":
            v.attach_texture()
        elif store == "pair":
            v.attach_pair_texture()
        v.set_transfer(synth.default_lut(), 1.0, 9.0, 1.0, 0.99)
        vols[dtype] = v
    reqs, keys = [], []
    for dtype, v in vols.items():
        for clip in (tb[3], tb[3] + 0.5):
            for i, cam in enumerate(cams):
                reqs.append(Request(v, cam, w, h, "composite", 0.5,
                                    tf=(tb[0], tb[1], tb[2], clip, 0.97)))
                keys.append((dtype, clip, i))
    outs = render_batch(reqs)
    torch.cuda.synchronize()
    for dtype in vols:
        for clip in (tb[3], tb[3] + 0.5):
            idx = [j for j, k in enumerate(keys) if k[0] == dtype and k[1] == clip]
            got = torch.stack([outs[j] for j in idx]).cpu().numpy()
            check(cube, dtype, cams, w, h, got, (tb[0], tb[1], tb[2], clip), 0.97, 0.5,
                  "batch %s %s clip %g" % (table, dtype, clip))


@pytest.mark.parametrize("table", sorted(TABLES))
@pytest.mark.parametrize("dtype,pair", [("f32", False), ("f16", True), ("i8", False)])
def test_parts_and_subcubes_honour_the_clip(dtype, pair, table):
    # part by part (continuing sweeps) and as sub-cubes integrated in each
    # ray's order, with and without masks
    dims = (37, 45, 70)
    cube, cams, w, h = noisy_case(dims, 53)
    tb = TABLES[table]()
    lut, v_lo, v_hi, clip = tb
    dev = torch.from_numpy(cube).cuda()
    ovol = oracle_volume(cube, dtype)
    for masks in (False, True):
        ps = PartStream(dims, dtype, lambda z0, n: dev[z0:z0 + n], 17, pair=pair,
                        cache_parts=2, masks=masks)
        ps.set_transfer(lut, v_lo, v_hi, clip, 0.95)
        out = torch.empty((len(cams), h, w, 4), device="cuda")
        ps.render(cams, w, h, [("composite", out)], 0.5)
        sub = torch.empty_like(out)
        ps.render_subcubes(cams, w, h, [("composite", sub)], 0.5)
        torch.cuda.synchronize()
        what = "parts %s %s masks=%s" % (dtype, table, masks)
        check(cube, dtype, cams, w, h, out.cpu().numpy(), tb, 0.95, 0.5, what)
        res = oracle.render_subcubes(ovol, cams, w, h, oracle.COMPOSITE, 0.5,
                                     oracle.TF(lut, v_lo, v_hi, clip, 0.95),
                                     [p.cell_lo for p in ps.parts],
                                     bands=bands_for(dims, cams, 0.5, w, h))
        compare(res, sub.cpu().numpy().reshape(-1, 4), oracle.COMPOSITE, TOL_FP32,
                what="sub-cubes " + what)
        assert_ties(res, "sub-cubes " + what, clip=0.05, term=0.05)
        free = oracle.render_subcubes(ovol, cams, w, h, oracle.COMPOSITE, 0.5,
                                      oracle.TF(lut, v_lo, v_hi, -1e30, 0.95),
                                      [p.cell_lo for p in ps.parts])
        hit = np.abs(res.primary).max(axis=1) > 0
        moved = np.abs(free.primary - res.primary).max(axis=1) > 100 * TOL_FP32
        assert moved[hit].mean() > 0.5, (what, moved[hit].mean())
        ps.close()


def test_served_mix_honours_each_requests_clip():
    # the continuous-batching server over three cubes, each request with a
    # clipped table of its own: every served image against the oracle
    specs = {"a": ((48, 40, 64), "f16", "pair"), "b": ((40, 36, 90), "i8", "texture"),
             "c": ((36, 30, 44), "f32", "bricks")}
    vols, cubes = {}, {}
    for i, (name, (dims, dt, store)) in enumerate(specs.items()):
        cube = synth.make_cube(dims, 3, ("uniform", 3.0, 6.0), 90 + i).numpy()
        v = Volume(torch.from_numpy(cube).cuda(), dt)
        if store == "texture":
            v.attach_texture()
        elif store == "pair":
            v.attach_pair_texture()
        v.set_transfer(synth.default_lut(), 1.0, 9.0, 1.0, 0.99)
        vols[name], cubes[name] = v, (cube, dt)
    server = Server(vols, mem_budget=1 << 22, max_batch=16, streams=2, keep_outputs=True)
    rng = np.random.default_rng(7)
    jobs = []
    for i in range(36):
        name = sorted(specs)[i % 3]
        dims = specs[name][0]
        w, h = (int(x) for x in rng.integers(12, 40, 2))
        cam = synth.random_sphere_cameras(dims, 1, w, h, 500 + i)[0]
        tb = TABLES[sorted(TABLES)[i % 2]]()
        clip = float(rng.uniform(0.8, 1.5))
        jobs.append(RenderJob(name, cam, w, h, "composite", 0.5,
                              (tb[0], tb[1], tb[2], clip, 0.99)))
    for k in range(0, len(jobs), 6):
        for job in jobs[k:k + 6]:
            server.submit(job)
        server.step()
    server.drain()
    assert len(server.done) == len(jobs)
    for job in jobs:
        cube, dt = cubes[job.cube]
        lut, v_lo, v_hi, clip, ta = job.tf
        check(cube, dt, np.asarray([job.cam]), job.w, job.h, job.out.cpu().numpy(),
              (lut, v_lo, v_hi, clip), ta, 0.5, "served %s" % job.cube, clip_ties=0.2)
