"""Seeded synthetic inputs for the spectral-cube ray caster.

This module only *generates inputs*: noisy RA x Dec x frequency cubes with
Gaussian-ellipsoid line sources, camera descriptions and raw RGBA lookup
tables.  It holds none of the rendering arithmetic (ray generation, box
intersection, sampling, transfer function, compositing): the CUDA path and
the FP64 oracle each implement that on their own, and both are fed the same
arrays produced here.

Data model (paper §2): a spectral cube is a stack of sky images, each over a
small frequency interval, i.e. a scalar flux density on a 3-D grid with two
sky axes and one frequency axis.  Here it is a float32 array of shape
(nz, ny, nx): x = RA (fastest), y = Dec, z = frequency channel (slowest).

Input recipe (the paper gives none; chosen to look like a radio line survey):
  * background: i.i.d. N(0, sigma=1) noise,
  * sources: Gaussian ellipsoids, spatial width sigma_xy ~ U[2, 6] voxels,
    spectral width sigma_z ~ U[4, 20] channels, peak = SNR * sigma, with a
    linear velocity gradient: the line centre moves across the source as
    z_c(x, y) = z0 + g * ((x - x0) cos(theta) + (y - y0) sin(theta)),
    g ~ U[-1, 1] channels / voxel, theta ~ U[0, 2 pi); each source is
    evaluated inside a +-4 sigma box,
  * source centres uniform in the cube.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

# ---------------------------------------------------------------------------
# camera records
# ---------------------------------------------------------------------------
#: Memory layout of one camera record: 64 bytes, identical to the C struct
#: ``vr_camera`` (int32 projection, then eye, fwd, du, dv as float[3] each,
#: then three reserved floats).  Lengths are in voxel units.
CAMERA_DTYPE = np.dtype([
    ("proj", "<i4"), ("eye", "<f4", 3), ("fwd", "<f4", 3),
    ("du", "<f4", 3), ("dv", "<f4", 3), ("pad", "<f4", 3)])
assert CAMERA_DTYPE.itemsize == 64

ORTHO, PERSP = 0, 1


def cameras(records) -> np.ndarray:
    """Pack ``[(proj, eye, fwd, du, dv), ...]`` into a CAMERA_DTYPE array."""
    out = np.zeros(len(records), dtype=CAMERA_DTYPE)
    for i, (proj, eye, fwd, du, dv) in enumerate(records):
        out[i]["proj"] = proj
        out[i]["eye"] = eye
        out[i]["fwd"] = fwd
        out[i]["du"] = du
        out[i]["dv"] = dv
    return out


def axis_camera(dims, w, h, axis=2, spacing=(1.0, 1.0), eye_back=1.0,
                sign=+1, centre=None):
    """Orthographic camera looking along +axis (or -axis).

    ``dims`` = (nx, ny, nz).  The two other axes are spanned by du and dv in
    increasing index order; the image is centred on the cube centre (or on
    ``centre``).  The eye sits ``eye_back`` voxels outside the entry face.
    """
    n = [float(d) for d in dims]
    c = [(d - 1.0) / 2.0 for d in n] if centre is None else list(centre)
    a, b = [i for i in range(3) if i != axis]
    eye = list(c)
    eye[axis] = -eye_back if sign > 0 else (n[axis] - 1.0) + eye_back
    fwd = [0.0, 0.0, 0.0]
    fwd[axis] = float(sign)
    du = [0.0, 0.0, 0.0]
    dv = [0.0, 0.0, 0.0]
    du[a] = spacing[0]
    dv[b] = spacing[1]
    return (ORTHO, eye, fwd, du, dv)


def _normalize(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def look_at_camera(eye, target, w, h, fov_deg, up=(0.0, 0.0, 1.0)):
    """Perspective camera at ``eye`` looking at ``target``.

    Pixel rows run downward (row 0 at the top); ``fov_deg`` is the vertical
    field of view.  du and dv are the per-pixel offsets at unit distance.
    """
    eye = np.asarray(eye, dtype=np.float64)
    fwd = _normalize(np.asarray(target, dtype=np.float64) - eye)
    right = np.cross(fwd, np.asarray(up, dtype=np.float64))
    if np.linalg.norm(right) < 1e-9:  # looking along up: pick any right
        right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right = _normalize(right)
    upv = np.cross(right, fwd)
    s = 2.0 * math.tan(math.radians(fov_deg) / 2.0) / h
    return (PERSP, eye.tolist(), fwd.tolist(), (right * s).tolist(),
            (-upv * s).tolist())


def orbit_cameras(dims, n_views, w, h, elev_deg=20.0, radius=None,
                  fov_deg=52.0):
    """``n_views`` perspective cameras on a circle around the cube centre.

    Azimuths 2*pi*i/n_views, fixed elevation, looking at the centre, up=+z.
    Default radius is twice the largest cube edge.
    """
    c = np.array([(d - 1.0) / 2.0 for d in dims])
    r = 2.0 * max(dims) if radius is None else radius
    e = math.radians(elev_deg)
    recs = []
    for i in range(n_views):
        az = 2.0 * math.pi * i / n_views
        eye = c + r * np.array([math.cos(e) * math.cos(az),
                                math.cos(e) * math.sin(az), math.sin(e)])
        recs.append(look_at_camera(eye, c, w, h, fov_deg))
    return cameras(recs)


def random_sphere_cameras(dims, n_views, w, h, seed, radius=None,
                          fov_deg=52.0):
    """Perspective cameras at uniformly random directions around the cube."""
    rng = np.random.default_rng(seed)
    c = np.array([(d - 1.0) / 2.0 for d in dims])
    r = 2.0 * max(dims) if radius is None else radius
    recs = []
    for _ in range(n_views):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        recs.append(look_at_camera(c + r * v, c, w, h, fov_deg))
    return cameras(recs)


# ---------------------------------------------------------------------------
# lookup tables
# ---------------------------------------------------------------------------
def default_lut(n=256, alpha_max=0.5):
    """Raw RGBA lookup table (n, 4) float32, alpha per unit voxel length.

    alpha_i = alpha_max * i / (n - 1) (zero at the clip level, which is also
    the bottom of the table's value domain); colour is an analytic ramp of
    s = i / (n - 1): r = s, g = 1 - |2s - 1|, b = 1 - s.
    """
    s = np.arange(n, dtype=np.float64) / (n - 1)
    lut = np.stack([s, 1.0 - np.abs(2.0 * s - 1.0), 1.0 - s, alpha_max * s],
                   axis=1)
    return lut.astype(np.float32)


# ---------------------------------------------------------------------------
# cubes
# ---------------------------------------------------------------------------
@dataclass
class Source:
    x0: float
    y0: float
    z0: float
    sxy: float
    sz: float
    amp: float
    g: float
    theta: float


def draw_sources(dims, n_sources, snr, seed, sigma=1.0):
    """Draw source parameters.  ``snr`` = ("uniform"|"loguniform", lo, hi)."""
    rng = np.random.default_rng(seed)
    kind, lo, hi = snr
    out = []
    for _ in range(n_sources):
        x0, y0, z0 = (rng.uniform(0.0, d - 1.0) for d in dims)
        sxy = rng.uniform(2.0, 6.0)
        sz = rng.uniform(4.0, 20.0)
        if kind == "uniform":
            s = rng.uniform(lo, hi)
        else:
            s = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        g = rng.uniform(-1.0, 1.0)
        th = rng.uniform(0.0, 2.0 * math.pi)
        out.append(Source(x0, y0, z0, sxy, sz, s * sigma, g, th))
    return out


def add_sources_(cube: torch.Tensor, sources, z_offset=0):
    """Add Gaussian-ellipsoid sources to ``cube`` (nz, ny, nx) in place.

    ``z_offset`` is the global channel index of the first plane of ``cube``,
    so that a cube generated in z-chunks gets the same sources.
    """
    nz, ny, nx = cube.shape
    dev = cube.device
    for s in sources:
        rxy = 4.0 * s.sxy
        xa, xb = max(0, math.ceil(s.x0 - rxy)), min(nx - 1, math.floor(s.x0 + rxy))
        ya, yb = max(0, math.ceil(s.y0 - rxy)), min(ny - 1, math.floor(s.y0 + rxy))
        zr = 4.0 * s.sz + abs(s.g) * rxy * math.sqrt(2.0)
        za = max(z_offset, math.ceil(s.z0 - zr))
        zb = min(z_offset + nz - 1, math.floor(s.z0 + zr))
        if xa > xb or ya > yb or za > zb:
            continue
        x = torch.arange(xa, xb + 1, device=dev, dtype=torch.float32) - s.x0
        y = torch.arange(ya, yb + 1, device=dev, dtype=torch.float32) - s.y0
        z = torch.arange(za, zb + 1, device=dev, dtype=torch.float32)
        r2 = x[None, :] ** 2 + y[:, None] ** 2                       # (y, x)
        zc = s.z0 + s.g * (x[None, :] * math.cos(s.theta)
                           + y[:, None] * math.sin(s.theta))          # (y, x)
        dz = z[:, None, None] - zc[None]                              # (z, y, x)
        val = s.amp * torch.exp(-r2[None] / (2.0 * s.sxy ** 2)
                                - dz * dz / (2.0 * s.sz ** 2))
        cube[za - z_offset:zb - z_offset + 1, ya:yb + 1, xa:xb + 1] += val


def make_cube(dims, n_sources, snr, seed, device="cpu", sigma=1.0):
    """Noise + sources cube, float32 tensor of shape (nz, ny, nx)."""
    nx, ny, nz = dims
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    cube = torch.randn((nz, ny, nx), generator=gen, device=device,
                       dtype=torch.float32)
    if sigma != 1.0:
        cube.mul_(sigma)
    add_sources_(cube, draw_sources(dims, n_sources, snr, seed + 7919, sigma))
    return cube


# ---------------------------------------------------------------------------
# workloads (shapes, sources, transfer-function levels, seeds)
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    dims: tuple            # (nx, ny, nz)
    n_sources: int
    snr: tuple
    clip: float            # in units of sigma
    v_hi: float            # top of the lookup-table domain, units of sigma
    seed: int
    term_alpha: float = 1.0
    step: float = 0.5
    extra: dict = field(default_factory=dict)

    def cube(self, device="cpu"):
        return make_cube(self.dims, self.n_sources, self.snr, self.seed,
                         device=device)


#: 64x64x128 cube, 5 sources SNR 3-10, 256^2 orthographic view along the
#: frequency axis, clip 2 sigma, no early termination.
SMALL = Workload("cube64x64x128_ortho256", (64, 64, 128), 5,
                 ("uniform", 3.0, 10.0), clip=2.0, v_hi=10.0, seed=1001)

#: 1024^3 cube, 2000 sources SNR log-uniform 2-50, 32 orbiting 1920x1080
#: perspective views, clip 3 sigma, early termination at alpha 0.99.
LARGE = Workload("cube1024_orbit32_1080p", (1024, 1024, 1024), 2000,
                 ("loguniform", 2.0, 50.0), clip=3.0, v_hi=50.0, seed=1002,
                 term_alpha=0.99)


def small_camera(w=256, h=256):
    """The 256^2 orthographic view along +z of the 64x64x128 cube."""
    sp = 63.0 / 256.0
    return cameras([axis_camera(SMALL.dims, w, h, axis=2, spacing=(sp, sp))])


def large_cameras(n_views=32, w=1920, h=1080):
    """The orbiting perspective views of the 1024^3 cube."""
    return orbit_cameras(LARGE.dims, n_views, w, h)


# ---------------------------------------------------------------------------
# batched and served workloads (several resident cubes, mixed requests)
# ---------------------------------------------------------------------------
#: The four resident cubes of the batched workload: (name, dims, storage).
BATCH_CUBES = [("cube256_f32", (256, 256, 256), "f32"),
               ("cube512x512x2048_f16", (512, 512, 2048), "f16"),
               ("cube1024_f16", (1024, 1024, 1024), "f16"),
               ("cube768x768x3072_i8", (768, 768, 3072), "i8")]
BATCH_SEED = 1004
SERVE_SEED = 1005


def batch_cube(i, device="cpu"):
    """Cube i of the batched workload as float32 (noise + sources scaled to
    the cube's volume, SNR log-uniform 2-50)."""
    name, dims, _ = BATCH_CUBES[i]
    n_src = max(5, int(2000 * dims[0] * dims[1] * dims[2] / 1024 ** 3))
    return make_cube(dims, n_src, ("loguniform", 2.0, 50.0), BATCH_SEED + 10 * i,
                     device=device)


def batch_views(n_views=64, seed=BATCH_SEED):
    """(cube index, camera record, w, h, mode) for the batched workload: view
    i renders cube i mod 4 from an orbit position, at a resolution drawn from
    {256^2, 512^2, 1024^2, 2048^2} and a mode drawn from {mip, composite}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_views):
        c = i % len(BATCH_CUBES)
        res = int(rng.choice([256, 512, 1024, 2048]))
        mode = ["mip", "composite"][int(rng.integers(0, 2))]
        dims = BATCH_CUBES[c][1]
        cam = orbit_cameras(dims, 16, res, res)[(i // len(BATCH_CUBES)) % 16]
        out.append((c, cam, res, res, mode))
    return out


#: The resident cubes of the served workload: four 2048 x 2048 x 4096 cubes
#: and two 1024^3 cubes (as FP16: 4 x 32 GiB + 2 x 2 GiB = 146 GB).
SERVE_CUBES = ([("cube2048x2048x4096_%d" % i, (2048, 2048, 4096)) for i in range(4)]
               + [("cube1024_%d" % i, (1024, 1024, 1024)) for i in range(2)])


def cube_slabs(dims, n_sources, snr, seed, device="cpu", planes=256):
    """A noise + sources cube generated in z-slabs, for cubes too large to
    hold whole in float32: yields (z0, float32 tensor (n, ny, nx)).  The
    noise of each slab comes from its own generator (seeded from ``seed`` and
    the slab index); sources straddling slabs are added to each part."""
    nx, ny, nz = dims
    srcs = draw_sources(dims, n_sources, snr, seed + 7919)
    for i, z0 in enumerate(range(0, nz, planes)):
        n = min(planes, nz - z0)
        gen = torch.Generator(device=device)
        gen.manual_seed(seed * 1000003 + i)
        slab = torch.randn((n, ny, nx), generator=gen, device=device, dtype=torch.float32)
        add_sources_(slab, srcs, z_offset=z0)
        yield z0, slab


def serve_cube_slabs(i, device="cpu", planes=256):
    """Cube i of the served workload in z-slabs (sources at the density of
    the 1024^3 workload, SNR log-uniform 2-50)."""
    name, dims = SERVE_CUBES[i]
    n_src = int(2000 * dims[0] * dims[1] * dims[2] / 1024 ** 3)
    return cube_slabs(dims, n_src, ("loguniform", 2.0, 50.0), SERVE_SEED + 10 * i, device,
                      planes)


def serve_request(dims, rng):
    """One served request: a random direction around the cube, a resolution
    from {512^2, 1024^2, 1280x720, 1920x1080}, composite (80 %) or MIP, and a
    clip level U[2, 5] sigma (the table spans [clip, 50 sigma])."""
    w, h = [(512, 512), (1024, 1024), (1280, 720), (1920, 1080)][int(rng.integers(0, 4))]
    cam = random_sphere_cameras(dims, 1, w, h, int(rng.integers(0, 2 ** 31)))[0]
    mode = "composite" if rng.random() < 0.8 else "mip"
    clip = float(rng.uniform(2.0, 5.0))
    return cam, w, h, mode, (default_lut(), clip, 50.0, clip, 0.99)
