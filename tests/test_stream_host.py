"""Host logic of part-by-part rendering (no GPU): the parts' cell ranges
tile the cube's cells within each part's planes, and the sweeps a view set
needs follow the directions of its rays."""
import numpy as np
import pytest

from paper_1001_2049_b300 import synth
from paper_1001_2049_b300.stream import pick_volume, plan_parts, sweeps


@pytest.mark.parametrize("nz", [2, 3, 9, 70, 1024, 4500])
@pytest.mark.parametrize("planes", [2, 3, 9, 129, 5000])
def test_parts_tile_the_cells(nz, planes):
    parts = plan_parts(nz, planes)
    p = min(planes, nz)
    assert parts[0].cell_lo == 0 and parts[-1].cell_hi == nz - 1
    for a, b in zip(parts, parts[1:]):
        assert a.cell_hi == b.cell_lo                    # contiguous, in order
    for part in parts:
        assert part.cell_lo < part.cell_hi
        assert 0 <= part.z_first and part.z_first + p <= nz
        # both planes of every cell are in the part
        assert part.z_first <= part.cell_lo and part.cell_hi <= part.z_first + p - 1


def test_a_part_needs_two_planes():
    with pytest.raises(ValueError):
        plan_parts(10, 1)


def _dz_signs(cams, w, h):
    """Signs of the height component of every ray of the views (brute force)."""
    out = set()
    for c in cams:
        u = (np.arange(w) + 0.5 - w / 2.0)[None, :]
        v = (np.arange(h) + 0.5 - h / 2.0)[:, None]
        if int(c["proj"]) == 0:
            dz = np.full((h, w), float(c["fwd"][2]))
        else:
            dz = c["fwd"][2] + u * c["du"][2] + v * c["dv"][2]
        out |= {1 if x >= 0 else -1 for x in np.unique(np.sign(dz))}
    return out


def test_sweeps_cover_every_ray_direction():
    dims = (64, 48, 80)
    w, h = 31, 23
    cases = [synth.cameras([synth.axis_camera(dims, w, h, axis=2, sign=1)]),
             synth.cameras([synth.axis_camera(dims, w, h, axis=2, sign=-1)]),
             synth.cameras([synth.axis_camera(dims, w, h, axis=0, sign=1)]),   # level rays
             synth.orbit_cameras(dims, 8, w, h, elev_deg=20.0),
             synth.orbit_cameras(dims, 4, w, h, elev_deg=60.0),
             synth.orbit_cameras(dims, 4, w, h, elev_deg=-60.0),
             synth.random_sphere_cameras(dims, 16, w, h, 3)]
    for cams in cases:
        got = set(sweeps(cams, w, h))
        assert _dz_signs(cams, w, h) <= got, cams["fwd"]
    # views looking steeply down need the descending sweep only
    assert sweeps(synth.orbit_cameras(dims, 4, w, h, elev_deg=60.0), w, h) == [-1]
    assert sweeps(synth.orbit_cameras(dims, 4, w, h, elev_deg=-60.0), w, h) == [1]


def _hit_dz_signs(cams, w, h, dims):
    """Signs of the height component of the rays that enter the box
    [0, n - 1]^3 (brute force, FP64 slab test, a ray in a face's plane
    passing only when its coordinate lies between the faces)."""
    out = set()
    hi = np.array([d - 1.0 for d in dims])
    for c in cams:
        u = (np.arange(w) + 0.5 - w / 2.0)[None, :, None]
        v = (np.arange(h) + 0.5 - h / 2.0)[:, None, None]
        eye, fwd = np.asarray(c["eye"], float), np.asarray(c["fwd"], float)
        du, dv = np.asarray(c["du"], float), np.asarray(c["dv"], float)
        if int(c["proj"]) == 0:
            o = eye + u * du + v * dv
            d = np.broadcast_to(fwd, o.shape)
        else:
            d = fwd + u * du + v * dv
            o = np.broadcast_to(eye, d.shape)
        with np.errstate(divide="ignore", invalid="ignore"):
            t0, t1 = (0.0 - o) / d, (hi - o) / d
        inside = (o >= 0.0) & (o <= hi)
        tn = np.where(d == 0, np.where(inside, -np.inf, np.inf), np.minimum(t0, t1))
        tf = np.where(d == 0, np.where(inside, np.inf, -np.inf), np.maximum(t0, t1))
        te, tx = np.maximum(tn.max(axis=-1), 0.0), tf.min(axis=-1)
        hit = tx >= te
        out |= {1 if x >= 0 else -1 for x in d[..., 2][hit]}
    return out


def test_sweeps_leave_out_directions_whose_rays_miss_the_cube():
    dims = (64, 48, 80)
    w, h = 31, 23
    cases = [synth.orbit_cameras(dims, 8, w, h, elev_deg=20.0),
             synth.orbit_cameras(dims, 8, w, h, elev_deg=20.0, radius=60.0),
             synth.orbit_cameras(dims, 4, w, h, elev_deg=-20.0),
             synth.random_sphere_cameras(dims, 16, w, h, 3),
             synth.cameras([synth.axis_camera(dims, w, h, axis=2, sign=1)]),
             synth.cameras([synth.axis_camera(dims, w, h, axis=2, sign=-1)]),
             synth.cameras([synth.axis_camera(dims, w, h, axis=0, sign=1)]),
             synth.cameras([synth.look_at_camera((31.5, 23.5, 39.5), (40.0, 20.0, 45.0),
                                                 w, h, 90.0)])]
    for cams in cases:
        got = sweeps(cams, w, h, dims)
        assert _hit_dz_signs(cams, w, h, dims) <= set(got), cams["eye"]
        assert set(got) <= set(sweeps(cams, w, h))
    # the orbit cameras sit above the cube: their ascending rays (the top
    # rows of the images) never enter it, so one sweep serves them
    above = synth.orbit_cameras(dims, 8, w, h, elev_deg=20.0)
    assert sweeps(above, w, h) == [1, -1] and sweeps(above, w, h, dims) == [-1]
    below = synth.orbit_cameras(dims, 4, w, h, elev_deg=-20.0)
    assert sweeps(below, w, h, dims) == [1]
    inside = synth.cameras([synth.look_at_camera((31.5, 23.5, 39.5), (40.0, 20.0, 45.0),
                                                 w, h, 90.0)])
    assert sweeps(inside, w, h, dims) == [1, -1]


def _loads(n_parts, n_vols, order, renders):
    """Loads per render of a cache of ``n_vols`` part volumes (pick_volume
    choosing), and whether a load ever took the volume rendered last."""
    holds, last, uses, out, took_last = [None] * n_vols, [-1] * n_vols, 0, [], False
    for _ in range(renders):
        loads = 0
        for n, z in enumerate(order):
            if z in holds:
                i = holds.index(z)
            else:
                i = pick_volume(holds, last, order, n)
                took_last |= uses > 0 and last[i] == uses and n_vols > 1
                holds[i] = z
                loads += 1
            uses += 1
            last[i] = uses
        out.append(loads)
    return out, took_last


@pytest.mark.parametrize("n_parts", [3, 8, 9, 15])
@pytest.mark.parametrize("n_vols", [2, 3, 4, 5])
def test_part_volume_choice(n_parts, n_vols):
    if n_vols > n_parts:
        return
    up = list(range(n_parts))
    two = up + up[::-1]
    loads, took_last = _loads(n_parts, n_vols, two, 4)
    assert not took_last
    # two sweeps: the turn reuses the parts held, as the least recently
    # used choice would
    assert loads == [2 * n_parts - n_vols] + [2 * (n_parts - n_vols)] * 3
    one = up[::-1]
    loads, took_last = _loads(n_parts, n_vols, one, 12)
    assert not took_last and loads[0] == n_parts
    if n_vols == 2:
        assert loads == [n_parts] * 12       # nothing to keep: one volume loads, one renders
    else:
        # the least recently used choice loads every part of a repeated
        # sweep; keeping the parts a sweep starts with saves loads
        assert max(loads[1:]) < n_parts
        assert np.mean(loads[1:]) <= n_parts - n_vols + 2


def test_part_volume_choice_prefers_empty_volumes():
    assert pick_volume([None, 5, None], [-1, 3, -1], [5, 7, 9], 1) in (0, 2)
    # the volume rendered last is never taken, even when its part comes last
    assert pick_volume([1, 2], [1, 2], [1, 2, 3], 2) == 0
