"""The checked build (VR_DEBUG: kernels test every output index, brick
address, partial-image index, batched tile and staged sample they compute,
record failures and skip the access, never trapping) on the GPU: renders
through every checked kernel -- texture, pair-texture and brick storage,
masks, MIP bounds, object order, the batched launch with row bands, parts
and scene integration -- record no failed check, and give the regular
library's images bit for bit.  Runs in a child process, since a process
loads one of the two libraries."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

CHILD = r'''
import ctypes, hashlib, json, sys
sys.path.insert(0, ROOT)
import numpy as np, torch
from paper_1001_2049_b300 import Request, Volume, _lib, render_batch, synth
from paper_1001_2049_b300.stream import PartStream
dims = (37, 45, 70)
cube = synth.make_cube(dims, 3, ("uniform", 3.0, 8.0), 5).cuda()
cams = synth.random_sphere_cameras(dims, 3, 23, 17, 5, fov_deg=60.0)
digest = hashlib.sha256()
def add(t):
    torch.cuda.synchronize()
    digest.update(t.cpu().numpy().tobytes())
for dt, store in (("f32", "texture"), ("f16", "pair"), ("i8", "bricks")):
    v = Volume(cube, dt)
    if store == "texture":
        v.attach_texture(); v.attach_masks(); v.attach_mip_bounds()
    elif store == "pair":
        v.attach_pair_texture(); v.attach_masks()
    v.set_transfer(synth.default_lut(), 0.0, 8.0, 1.0, 0.95)
    for mode in ("composite", "mip"):
        add(v.render(cams, 23, 17, mode, 0.5))
    add(v.render_object_order(cams, 23, 17, "mip", 0.5))
    reqs = [Request(v, c, 23, 17, m, 0.5, band=b) for c in cams for m in ("mip", "composite")
            for b in (None, (3, 9))]
    for o in render_batch(reqs):
        add(o)
ps = PartStream(dims, "f32", lambda z0, n: cube[z0:z0 + n], 17, cache_parts=2, masks=True)
ps.set_transfer(synth.default_lut(), 0.0, 8.0, 1.0, 0.95)
out = torch.empty((len(cams), 17, 23, 4), device="cuda")
ps.render(cams, 23, 17, [("composite", out)], 0.5); add(out)
ps.render_subcubes(cams, 23, 17, [("composite", out)], 0.5); add(out)
flags = ctypes.c_uint(0)
rc = _lib.load().vr_debug_status(ctypes.byref(flags), 1)
print(json.dumps({"rc": rc, "flags": flags.value, "digest": digest.hexdigest()}))
'''


def _run(debug):
    env = dict(os.environ, VR_DEBUG="1" if debug else "0")
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_records_no_failed_check_and_renders_the_same_images():
    checked = _run(True)
    assert checked["rc"] == 0 and checked["flags"] == 0, checked
    regular = _run(False)
    assert regular["rc"] != 0                      # the regular build has no checks
    assert checked["digest"] == regular["digest"]
