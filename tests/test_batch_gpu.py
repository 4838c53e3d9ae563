"""The batched persistent launch (many requests, mixed cubes, storage
types, resolutions, modes and transfer functions) against per-view renders
and the oracle, its completion flags, splitting and CUDA-graph replay."""
import numpy as np
import pytest
import torch

import oracle
from oracle import quantize
from paper_1001_2049_b300 import Request, Volume, batch_workspace, render_batch, synth

from _util import TOL_FP32, bands_for, compare, sum_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    specs = [((40, 36, 50), "f32", True), ((33, 45, 70), "f16", False),
             ((30, 30, 2100), "i8", True), ((24, 20, 28), "f32", False),
             ((35, 30, 2200), "f16", "pair"), ((28, 33, 40), "i8", "pair")]
    vols = []
    for i, (dims, dt, tex) in enumerate(specs):
        cube = synth.make_cube(dims, 4, ("uniform", 3.0, 9.0), 60 + i)
        v = Volume(cube.cuda(), dt)
        if tex == "pair":
            v.attach_pair_texture()
        elif tex:
            v.attach_texture()
        v.set_transfer(synth.default_lut(), 1.0, 9.0, 1.0, 0.97)
        vols.append((v, cube.numpy(), dims, dt))
    torch.cuda.synchronize()
    return vols


def requests_for(scene, n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        v, cube, dims, dt = scene[i % len(scene)]
        w, h = (int(x) for x in rng.integers(5, 40, 2))
        cam = synth.random_sphere_cameras(dims, 1, w, h, seed * 100 + i)[0]
        mode = ["composite", "mip", "sum"][int(rng.integers(0, 3))]
        tf = None
        if mode == "composite" and rng.random() < 0.5:
            clip = float(rng.uniform(1.0, 4.0))
            tf = (synth.default_lut(), clip, 9.0, clip, 0.95)
        reqs.append(Request(v, cam, w, h, mode, 0.5, tf=tf))
    return reqs


def single(rq):
    """The same request through vr_render."""
    v = rq.volume
    if rq.tf is not None:
        v.set_transfer(*rq.tf)
    img = v.render(np.asarray([rq.cam]), rq.w, rq.h, rq.mode, rq.step)[0]
    if rq.tf is not None:
        v.set_transfer(synth.default_lut(), 1.0, 9.0, 1.0, 0.97)
    return img


def test_batch_equals_per_view_renders(scene):
    reqs = requests_for(scene, 40, 1)
    outs = render_batch(reqs)
    torch.cuda.synchronize()
    for rq, out in zip(reqs, outs):
        ref = single(rq)
        torch.cuda.synchronize()
        assert torch.allclose(out, ref, rtol=0, atol=1e-6, equal_nan=True), rq.mode


def test_batch_matches_oracle(scene):
    reqs = requests_for(scene, 12, 2)
    outs = render_batch(reqs)
    torch.cuda.synchronize()
    modes = {"mip": oracle.MIP, "composite": oracle.COMPOSITE, "sum": oracle.SUM}
    for rq, out in zip(reqs, outs):
        v, cube, dims, dt = next(s for s in scene if s[0] is rq.volume)
        ovol = (oracle.Volume(cube) if dt == "f32" else
                oracle.Volume(quantize.to_f16(cube)) if dt == "f16" else
                oracle.Volume(*quantize.quantize_i8(cube)))
        lut, lo, hi, clip, ta = rq.tf or (synth.default_lut(), 1.0, 9.0, 1.0, 0.97)
        cams = np.asarray([rq.cam])
        res = oracle.render(ovol, cams, rq.w, rq.h, modes[rq.mode], rq.step,
                            oracle.TF(lut, lo, hi, clip, ta), bands=bands_for(dims, cams, rq.step))
        got = out.cpu().numpy()
        scale = 1.0
        if rq.mode == "mip":
            scale = float(cube.max() - cube.min())
        elif rq.mode == "sum":
            scale = sum_scale(oracle.Volume(cube), cams, rq.w, rq.h, rq.step, got)
        compare(res, got, modes[rq.mode], TOL_FP32, scale, what="batch %s %s" % (dt, rq.mode))


def test_batch_splits_large_and_varied_batches(scene):
    # more than 64 requests and more than two distinct tables
    reqs = requests_for(scene, 150, 3)
    for i, rq in enumerate(reqs):
        if rq.mode == "composite":
            clip = 1.0 + 0.01 * i
            rq.tf = (synth.default_lut(), clip, 9.0, clip, 0.99)
    outs = render_batch(reqs)
    torch.cuda.synchronize()
    for rq, out in list(zip(reqs, outs))[::7]:
        assert torch.allclose(out, single(rq), rtol=0, atol=1e-6, equal_nan=True)


def test_done_flags_in_pinned_host_memory(scene):
    reqs = requests_for(scene, 20, 4)
    flags = torch.zeros(len(reqs), dtype=torch.int32).pin_memory()
    for i, rq in enumerate(reqs):
        rq.done = (flags, i)
        rq.done_value = 1000 + i
    counts = torch.zeros(1, dtype=torch.int64, device="cuda")
    for rq in reqs:
        rq.samples = counts
    render_batch(reqs)
    torch.cuda.synchronize()
    assert flags.tolist() == [1000 + i for i in range(len(reqs))]
    assert int(counts.item()) > 0


def test_batch_replays_from_a_cuda_graph(scene):
    reqs = requests_for(scene, 16, 5)
    ws = batch_workspace()
    outs = [torch.empty((rq.h, rq.w, 4) if rq.mode == "composite" else (rq.h, rq.w),
                        device="cuda") for rq in reqs]
    for rq, o in zip(reqs, outs):
        rq.out = o
    render_batch(reqs, ws)             # warm-up outside the capture
    torch.cuda.synchronize()
    refs = [o.clone() for o in outs]
    for o in outs:
        o.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            render_batch(reqs, ws, stream=s)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)


def test_batch_argument_errors(scene):
    from paper_1001_2049_b300 import VRError
    v = scene[0][0]
    cam = synth.random_sphere_cameras(scene[0][2], 1, 8, 8, 1)[0]
    with pytest.raises(VRError):
        render_batch([Request(v, cam, 8, 8, "mip", 0.0)])
    small = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(VRError):
        render_batch([Request(v, cam, 8, 8, "mip", 0.5)], workspace=small)
    # an empty batch is no work, not an error
    assert render_batch([]) == []
    torch.cuda.synchronize()
    # a bad request after good ones of another launch class: nothing is
    # enqueued (the good request's image keeps its old contents)
    good = torch.full((8, 8), float("nan"), device="cuda")
    bricks_vol = scene[1][0]                       # no texture storage: a later launch
    cam1 = synth.random_sphere_cameras(scene[1][2], 1, 8, 8, 2)[0]
    bad_tf = (synth.default_lut(), 5.0, 1.0, 5.0, 1.0)       # v_lo > v_hi
    with pytest.raises(VRError):
        render_batch([Request(v, cam, 8, 8, "mip", 0.5, out=good),
                      Request(bricks_vol, cam1, 8, 8, "composite", 0.5, tf=bad_tf)])
    torch.cuda.synchronize()
    assert torch.isnan(good).all()


def test_every_batch_shape_gives_identical_images(scene):
    # tile and ray-packet shapes only change which block renders which ray
    from paper_1001_2049_b300 import (batch_autotune, batch_shapes, get_batch_config,
                                      set_batch_config)
    shapes = batch_shapes()
    assert len(shapes) >= 4
    for tx, ty, px, py in shapes:
        assert tx * ty == 256 and px * py == 32
    reqs = requests_for(scene, 24, 7)
    saved = get_batch_config()
    try:
        ref = None
        for cfg in range(len(shapes)):
            set_batch_config(cfg)
            assert get_batch_config() == cfg
            outs = [o.clone() for o in render_batch(reqs)]
            torch.cuda.synchronize()
            if ref is None:
                ref = outs
            for a, b in zip(ref, outs):
                assert torch.equal(torch.nan_to_num(a), torch.nan_to_num(b)), shapes[cfg]
        best, ms = batch_autotune(reqs)
        assert 0 <= best < len(shapes) and ms > 0
        assert get_batch_config() == best
        outs = render_batch(reqs)
        torch.cuda.synchronize()
        for a, b in zip(ref, outs):
            assert torch.equal(torch.nan_to_num(a), torch.nan_to_num(b))
        with pytest.raises(Exception):
            set_batch_config(len(shapes))
    finally:
        set_batch_config(saved)


def test_batch_on_masked_volumes_equals_renders_without():
    # batched launches march every sample (the lockstep march over the masks
    # measured slower there); requests on volumes with built masks, at clips
    # below, at and above the masks' level, give the images of mask-free
    # twin volumes bit for bit, and so do the twins' per-view renders
    specs = [((40, 36, 50), "f32", False), ((33, 45, 70), "f16", True),
             ((30, 30, 2100), "i8", False), ((35, 30, 2200), "f16", True)]
    lut = synth.default_lut()
    masked, twins = [], []
    for i, (dims, dt, pair) in enumerate(specs):
        cube = synth.make_cube(dims, 6, ("uniform", 3.0, 9.0), 300 + i).cuda()
        for out in (masked, twins):
            v = Volume(cube, dt)
            v.attach_pair_texture() if pair else v.attach_texture()
            v.set_transfer(lut, 2.0, 9.0, 2.0, 0.97)
            out.append((v, dims))
        masked[-1][0].attach_masks()
        masked[-1][0].build_masks()
    rng = np.random.default_rng(17)
    reqs, twin_reqs = [], []
    for i in range(24):
        (v, dims), (t, _) = masked[i % len(masked)], twins[i % len(twins)]
        w, h = (int(x) for x in rng.integers(9, 48, 2))
        cam = synth.random_sphere_cameras(dims, 1, w, h, 900 + i)[0]
        mode = "mip" if i % 6 == 5 else "composite"
        clip = [1.5, 2.0, 3.0, 2.5][i % 4]          # 1.5: below the masks' level
        tf = (lut, clip, 9.0, clip, 0.95)
        reqs.append(Request(v, cam, w, h, mode, 0.5, tf=tf))
        twin_reqs.append(Request(t, cam, w, h, mode, 0.5, tf=tf))
    ref = render_batch(twin_reqs)
    got = render_batch(reqs)
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(zip(got, ref)):
        assert torch.equal(a, b), (k, reqs[k].mode, reqs[k].tf[1])
    for rq, img in zip(twin_reqs[:8], ref[:8]):
        assert torch.equal(single(rq), img)


def test_row_bands_give_the_whole_images_rows(scene):
    # a request limited to a band of rows renders exactly those rows of the
    # whole image (the same rays), whatever the band and the tile shape;
    # bands of one image can go to different launches
    reqs = requests_for(scene, 18, 9)
    whole = render_batch(reqs)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    band_reqs = []
    for rq in reqs:
        cuts = sorted({0, rq.h} | {int(x) for x in rng.integers(1, max(2, rq.h), 2)})
        for r0, r1 in zip(cuts[:-1], cuts[1:]):
            band_reqs.append(Request(rq.volume, rq.cam, rq.w, rq.h, rq.mode, rq.step, tf=rq.tf,
                                     band=(r0, r1 - r0)))
    outs = []
    for k in range(0, len(band_reqs), 7):                 # several launches
        outs += render_batch(band_reqs[k:k + 7])
    torch.cuda.synchronize()
    i = 0
    for rq, ref in zip(reqs, whole):
        got = []
        while i < len(band_reqs) and band_reqs[i].cam is rq.cam:
            got.append(outs[i])
            i += 1
        assert torch.equal(torch.cat(got), ref), rq.mode
    assert i == len(band_reqs)


def test_row_band_arguments_are_checked(scene):
    # through the C ABI: a band must lie inside the image, rows = 0 means the
    # whole image (with row0 = 0)
    from paper_1001_2049_b300 import _lib
    from paper_1001_2049_b300.api import _batch_args
    v = scene[0][0]
    cam = synth.random_sphere_cameras(scene[0][2], 1, 16, 12, 1)[0]
    arr, keep, outs = _batch_args([Request(v, cam, 16, 12, "mip", 0.5)])
    ws = batch_workspace()
    lib = _lib.load()
    for row0, rows in ((0, 13), (5, 8), (-1, 3), (2, -1), (3, 0)):
        arr[0].row0, arr[0].rows = row0, rows
        rc = lib.vr_render_batch(arr, 1, ws.data_ptr(), ws.numel(), None)
        assert rc == _lib.VR_ERR_ARG, (row0, rows)
        assert b"row band" in lib.vr_last_error()
    arr[0].row0, arr[0].rows = 4, 8
    assert lib.vr_render_batch(arr, 1, ws.data_ptr(), ws.numel(), None) == 0
    torch.cuda.synchronize()
    del keep
