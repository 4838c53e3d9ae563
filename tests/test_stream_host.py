"""Host logic of part-by-part rendering (no GPU): the parts' cell ranges
tile the cube's cells within each part's planes, and the sweeps a view set
needs follow the directions of its rays."""
import numpy as np
import pytest

from paper_1001_2049_b300 import synth
from paper_1001_2049_b300.stream import plan_parts, sweeps


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
