"""The allocation-free batch call, for callers that cannot allocate device
memory (a fixed-budget real-time loop, a plugin given no allocator, a
process that may not grow after start-up): vr_render_batch_noalloc keeps
its work and tile counters in a fixed array inside the library instead of
asking for a workspace.  It must render exactly what vr_render_batch
renders, call after call (the array keeps the previous call's counters and
every launch clears them first), and refuse batches larger than the array.

Collected last on purpose: a failure here leaves every other test run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1001_2049_b300 import Volume, _lib, synth
from paper_1001_2049_b300.api import MODES, _Request, _Transfer, batch_workspace

pytestmark = pytest.mark.gpu


def _requests(n, seed):
    """n requests over four volumes (plain-texel, pair-texel and brick
    storage, three storage types), mixed sizes, modes, steps and transfer
    functions, with their C records and freshly allocated outputs."""
    # one volume per launch class of the batched kernel: plain texels,
    # brick gathers, plain texels again, pair texels
    specs = [((40, 36, 50), "f32", "texture"), ((33, 45, 70), "f16", "bricks"),
             ((30, 30, 60), "i8", "texture"), ((28, 34, 44), "f16", "pair")]
    vols = []
    for i, (dims, dt, store) in enumerate(specs):
        v = Volume(synth.make_cube(dims, 4, ("uniform", 3.0, 9.0), 90 + i).cuda(), dt)
        if store == "texture":
            v.attach_texture()
        elif store == "pair":
            v.attach_pair_texture()
        v.set_transfer(synth.default_lut(), 1.0, 9.0, 1.0, 0.97)
        vols.append((v, dims))
    rng = np.random.default_rng(seed)
    lut = np.ascontiguousarray(synth.default_lut())
    tfs = [_Transfer(lut.ctypes.data, lut.shape[0], 2.0, 9.0, 2.0, 0.95),
           _Transfer(lut.ctypes.data, lut.shape[0], 0.0, 9.0, 1.0, 0.99)]
    arr = (_Request * n)()
    outs = []
    for i in range(n):
        v, dims = vols[i % len(vols)]
        w, h = (int(x) for x in rng.integers(6, 40, 2))
        mode = ["composite", "mip"][i % 2]
        cam = synth.random_sphere_cameras(dims, 1, w, h, seed * 1000 + i)
        out = torch.empty((h, w, 4) if mode == "composite" else (h, w), device="cuda")
        r = arr[i]
        r.vol = v.handle.value
        ctypes.memmove(ctypes.addressof(r.cam), cam.ctypes.data, 64)
        # three steps: more distinct corrected tables than one launch holds
        r.w, r.h, r.mode, r.step = w, h, MODES[mode], (0.5, 0.37, 0.61)[i % 3]
        r.out = out.data_ptr()
        if mode == "composite" and i % 4 == 0:
            r.tf = ctypes.addressof(tfs[(i // 4) % 2])
        outs.append(out)
    return arr, outs, (vols, lut, tfs)


@pytest.mark.parametrize("n", [24, 64])
def test_no_alloc_batch_matches_the_workspace_batch_on_two_calls(n):
    # both calls take the batched launch path of vr_render_batch, so the
    # images are the same bit for bit; with 64 requests over four storage
    # kinds and several tables one call makes several launches on the
    # shared counters, each clearing them first
    lib = _lib.load()
    arr, outs, keep = _requests(n, 7)
    stream = torch.cuda.current_stream().cuda_stream
    ws = batch_workspace()
    _lib.check(lib.vr_render_batch(arr, n, ws.data_ptr(), ws.numel(), stream))
    torch.cuda.synchronize()
    refs = [o.clone() for o in outs]
    for call in range(2):
        for o in outs:
            o.fill_(float("nan"))
        _lib.check(lib.vr_render_batch_noalloc(arr, n, stream))
        torch.cuda.synchronize()
        for i, (o, ref) in enumerate(zip(outs, refs)):
            assert torch.equal(o, ref), (call, i)
    del keep


def test_no_alloc_batch_rejects_more_requests_than_its_array_holds():
    lib = _lib.load()
    arr = (_Request * 65)()
    rc = lib.vr_render_batch_noalloc(arr, 65, None)
    assert rc == _lib.VR_ERR_ARG
    assert b"at most" in lib.vr_last_error()
