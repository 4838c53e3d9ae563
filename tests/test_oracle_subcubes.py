"""Pins for the oracle's sub-cube rendering (the paper's pipeline: the cube
split into sub-cubes along z, each rendered into its own partial result, the
partial results combined in the order each ray meets them; §3.1 items 1, 4,
5).  Checked against the one-pass oracle, which it must equal wherever the
combination is exact (one sub-cube; no early termination, by associativity
of the front-to-back operator; MIP always), and against the closed form of a
constant cube, where each sub-cube stops at its own opacity."""
import numpy as np
import pytest

import oracle
from paper_1001_2049_b300 import synth

MODES = (oracle.MIP, oracle.COMPOSITE, oracle.SUM)


def _case(seed, dims=(23, 19, 41)):
    cube = synth.make_cube(dims, 4, ("uniform", 3.0, 8.0), seed).numpy()
    w, h = 13, 11
    cams = synth.random_sphere_cameras(dims, 3, w, h, seed, fov_deg=60.0)
    c = np.array([(d - 1) / 2.0 for d in dims])
    recs = [synth.axis_camera(dims, w, h, axis=2, sign=1),
            synth.axis_camera(dims, w, h, axis=2, sign=-1),
            synth.look_at_camera(c + 0.3, c + np.array([4.0, -2.0, 3.0]), w, h, 90.0)]
    cams = np.concatenate([cams, synth.cameras(recs).astype(cams.dtype)])
    return oracle.Volume(cube), cams, w, h


def test_one_subcube_is_the_one_pass_result():
    vol, cams, w, h = _case(11)
    tf = oracle.TF(synth.default_lut(64), 1.0, 8.0, 1.0, 0.9)
    for mode in MODES:
        ref = oracle.render(vol, cams, w, h, mode, 0.37, tf)
        got = oracle.render_subcubes(vol, cams, w, h, mode, 0.37, tf, [0]).primary
        ch = 4 if mode == oracle.COMPOSITE else 1
        assert np.array_equal(got[:, :ch], ref.primary[:, :ch]), mode


@pytest.mark.parametrize("cell_lo", [[0, 20], [0, 7, 8, 30], [0, 1, 2, 3, 39]])
def test_without_termination_any_split_is_the_one_pass_result(cell_lo):
    # the front-to-back operator is associative: partial images combined in
    # each ray's order give the one-pass image up to FP64 rounding; the max
    # is exact.  A wrong order (or a partial that did not start empty) fails.
    vol, cams, w, h = _case(12 + len(cell_lo))
    tf = oracle.TF(synth.default_lut(64, alpha_max=0.9), 1.0, 8.0, 1.0, 2.0)
    for mode in MODES:
        ref = oracle.render(vol, cams, w, h, mode, 0.37, tf).primary
        got = oracle.render_subcubes(vol, cams, w, h, mode, 0.37, tf, cell_lo).primary
        if mode == oracle.MIP:
            assert np.array_equal(got[:, 0], ref[:, 0])
        else:
            ch = 4 if mode == oracle.COMPOSITE else 1
            assert np.allclose(got[:, :ch], ref[:, :ch], rtol=1e-12, atol=1e-12), mode
    # and the composite images are not trivial
    comp = oracle.render(vol, cams, w, h, oracle.COMPOSITE, 0.37, tf).primary
    assert (comp[:, 3] > 0.5).sum() > 10


@pytest.mark.parametrize("sign", [1, -1])
def test_constant_cube_each_subcube_stops_at_its_own_opacity(sign):
    # constant value c above the clip, orthographic rays along +z (or -z)
    # entering at the face, step 1/2: the samples sit at heights 0, 1/2, ...
    # (or nz - 1, nz - 3/2, ...); sub-cube 0 owns cells [0, m), sub-cube 1
    # the rest.  Sub-cube i's partial alpha after n samples is
    # 1 - (1 - a)^n with a the corrected alpha of c, stopping at the first n
    # with alpha >= term_alpha (or at its K_i samples); the combination is
    # A = 1 - (1 - A_0)(1 - A_1), C = rgb(c) A.
    dims, c, m, step = (6, 5, 20), 5.0, 6, 0.5
    vol = oracle.Volume(np.full(dims[::-1], c, dtype=np.float32))
    lut = synth.default_lut(64)
    probe = oracle.TF(lut, 1.0, 8.0, 1.0, 1.0)
    rgba = oracle.classify(probe, step, c)
    a = rgba[3]
    assert 0.05 < a < 0.5
    ta = 1.0 - (1.0 - a) ** 5.5                 # reached at the sixth sample
    tf = oracle.TF(lut, 1.0, 8.0, 1.0, ta)
    cams = synth.cameras([synth.axis_camera(dims, 4, 3, axis=2, sign=sign)])
    K = int(2 * (dims[2] - 1)) + 1
    K0 = 2 * m if sign > 0 else K - (2 * (dims[2] - 1 - m) + 1)
    Ks = [K0, K - K0]

    def partial(n_avail):
        n = next((j for j in range(1, n_avail + 1) if 1.0 - (1.0 - a) ** j >= ta), n_avail)
        return 1.0 - (1.0 - a) ** n
    A0, A1 = partial(Ks[0]), partial(Ks[1])
    A = 1.0 - (1.0 - A0) * (1.0 - A1)
    got = oracle.render_subcubes(vol, cams, 4, 3, oracle.COMPOSITE, step, tf, [0, m]).primary
    for p in range(got.shape[0]):
        assert abs(got[p, 3] - A) < 1e-12
        assert np.allclose(got[p, :3], rgba[:3] * A, rtol=1e-12, atol=1e-12)
    # the one-pass render stops inside the first sub-cube it meets
    one = oracle.render(vol, cams, 4, 3, oracle.COMPOSITE, step, tf).primary
    assert abs(one[0, 3] - partial(K)) < 1e-12 and one[0, 3] < A - 0.05


def test_subcube_arguments_are_checked():
    vol, cams, w, h = _case(3)
    tf = oracle.TF(synth.default_lut(64), 1.0, 8.0, 1.0, 0.9)
    for bad in ([1, 5], [0, 5, 5], [0, 40]):
        with pytest.raises(ValueError):
            oracle.render_subcubes(vol, cams, w, h, oracle.COMPOSITE, 0.5, tf, bad)
