"""Scene integration across ranks, on CPU with gloo (world sizes 2 and 3):
each rank renders its sub-cube's partial images with the FP64 oracle, the
exchange combines them (the collectives of paper_1001_2049_b300.exchange;
the composite's per-pixel "over" by a numpy stand-in for the library's
integration kernel, which needs a GPU), and every rank's images must be the
oracle's sub-cube rendering of the whole split.  The kernel itself is
checked against the same oracle on the GPU (tests/test_subcubes_gpu.py)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS = (23, 19, 41)
W, H = 13, 11


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    from paper_1001_2049_b300 import synth
    cube = synth.make_cube(DIMS, 4, ("uniform", 3.0, 8.0), 5).numpy()
    cams = synth.random_sphere_cameras(DIMS, 3, W, H, 5, fov_deg=60.0)
    c = np.array([(d - 1) / 2.0 for d in DIMS])
    recs = [synth.axis_camera(DIMS, W, H, axis=2, sign=1),
            synth.axis_camera(DIMS, W, H, axis=2, sign=-1),
            synth.look_at_camera(c + 0.3, c + np.array([4.0, -2.0, 3.0]), W, H, 90.0)]
    return cube, np.concatenate([cams, synth.cameras(recs).astype(cams.dtype)])


def _cell_lo(world):
    return [0, 9, 30][:world] if world <= 3 else list(range(0, 40, 40 // world))[:world]


def over_by_ray_order(stacked, cams, mode):
    """numpy stand-in for vr_integrate_partials: per pixel, "over" of the
    partials in ascending order when the ray goes up (the direction's
    height component before normalisation is >= 0), descending otherwise."""
    parts, views, h, w, _ = stacked.shape
    out = torch.zeros(stacked.shape[1:], dtype=stacked.dtype)
    py, px = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    u, v = px + 0.5 - w / 2.0, py + 0.5 - h / 2.0
    for vi, c in enumerate(cams):
        if int(c["proj"]) == 0:
            up = np.full((h, w), float(c["fwd"][2]) >= 0.0)
        else:
            up = (float(c["fwd"][2]) + u * float(c["du"][2]) + v * float(c["dv"][2])) >= 0.0
        acc = np.zeros((h, w, 4))
        for j in range(parts):
            pa = stacked[j, vi].numpy()
            pd = stacked[parts - 1 - j, vi].numpy()
            part = np.where(up[..., None], pa, pd)
            T = 1.0 - acc[..., 3:4]
            acc = acc + T * part
        out[vi] = torch.from_numpy(acc)
    return out


def _rank(rank, world, port, mode, root, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1001_2049_b300 import synth
    from paper_1001_2049_b300.exchange import exchange_partials
    cube, cams = _case()
    om = {"mip": oracle.MIP, "sum": oracle.SUM, "composite": oracle.COMPOSITE}[mode]
    tf = oracle.TF(synth.default_lut(64, alpha_max=0.8), 0.5, 8.0, 1.0, 0.9)
    lo = _cell_lo(world)
    mine = oracle.render_partial(oracle.Volume(cube), cams, W, H, om, 0.37, tf, lo, rank)
    shape = (len(cams), H, W, 4) if mode == "composite" else (len(cams), H, W)
    part = torch.from_numpy(mine.reshape(len(cams), H, W, 4) if mode == "composite"
                            else mine[:, 0].reshape(len(cams), H, W).copy())
    assert part.shape == shape
    got = exchange_partials(part, cams, mode, root=root, combine=over_by_ray_order)
    out[rank] = None if got is None else got.numpy()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("mode", ["composite", "mip", "sum"])
def test_exchange_gives_the_subcube_rendering_on_every_rank(world, mode):
    import oracle
    from paper_1001_2049_b300 import synth
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, mode, None, out), nprocs=world, join=True)
        got = dict(out)
    cube, cams = _case()
    om = {"mip": oracle.MIP, "sum": oracle.SUM, "composite": oracle.COMPOSITE}[mode]
    tf = oracle.TF(synth.default_lut(64, alpha_max=0.8), 0.5, 8.0, 1.0, 0.9)
    ref = oracle.render_subcubes(oracle.Volume(cube), cams, W, H, om, 0.37, tf,
                                 _cell_lo(world)).primary
    ch = 4 if mode == "composite" else 1
    for r in range(world):
        g = got[r].reshape(-1, ch)
        if mode == "mip":
            assert np.array_equal(g[:, 0], ref[:, 0])      # the maximum is exact
        else:
            assert np.allclose(g, ref[:, :ch], rtol=1e-12, atol=1e-12), (mode, r)
    if mode == "composite":
        # the split matters: partials stop at their own opacity
        assert (ref[:, 3] > 0.5).sum() > 10


def test_exchange_to_a_root_only():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, "composite", 1, out), nprocs=2, join=True)
        got = dict(out)
    assert got[0] is None and got[1] is not None


def test_partials_of_one_subcube_are_the_one_pass_render():
    # pins the oracle's partial: one sub-cube holding every cell is the whole
    # ray, from an empty start
    import oracle
    from paper_1001_2049_b300 import synth
    cube, cams = _case()
    tf = oracle.TF(synth.default_lut(64, alpha_max=0.8), 0.5, 8.0, 1.0, 0.9)
    vol = oracle.Volume(cube)
    for om in (oracle.COMPOSITE, oracle.MIP, oracle.SUM):
        one = oracle.render(vol, cams, W, H, om, 0.37, tf).primary
        part = oracle.render_partial(vol, cams, W, H, om, 0.37, tf, [0], 0)
        ch = 4 if om == oracle.COMPOSITE else 1
        assert np.array_equal(part[:, :ch], one[:, :ch])
