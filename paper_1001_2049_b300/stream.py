"""Rendering a cube part by part, for cubes larger than the device.

The paper's pipeline splits the cube into sub-cubes, renders each and
combines the images (§3.1 items 1, 4, 5), and aims at data larger than GPU
memory (abstract).  Here the cube stays with its source (page-locked host
memory, or a generator) and passes through a cache of part volumes on the
device: while one part renders on the compute stream, the next is packed
(into one brick buffer the part volumes share) and copied into a part
volume's texture on a copy stream.  Each part continues the
images from the state the earlier parts left (``vr_render_part``), so the
images are those of a one-pass render of the whole cube, bit for bit.

Rays going up in z take the parts in ascending order and rays going down
in descending order: a view set whose rays go both ways is rendered in two
sweeps (the turning part is not loaded twice), and a direction none of whose
rays can enter the cube (a camera above the top plane looking down sends no
ascending ray into it) is not swept.  The part volume that takes a part is
the one whose part is needed again last, assuming the next render repeats
this one's order, never the one rendered just before (whose render may still
run): the parts a render starts with stay resident from one render to the
next, and every load overlaps the renders of earlier parts.  All rendering
runs in the library's kernels; this module is host-side control.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from .api import MODES, Volume, integrate_partials, render_init
from ._lib import VR_COMPOSITE


def sweeps(cams: np.ndarray, w: int, h: int, dims=None):
    """The sweeps a view set needs: +1 when some ray may go up in z (or be
    level), -1 when some ray may go down.  The height components of a ray's
    direction and (orthographic views) origin are affine functions of the
    pixel position, so their extremes are at the image corners; a margin
    keeps near-level rays in both.  With ``dims`` (nx, ny, nz), a direction
    is left out when every ray going that way starts beyond the box's face
    in that direction (heights above nz - 1 going up, below 0 going down):
    such a ray never enters the cube (the ray-box test gives it no sample)."""
    need_up = need_down = False
    corners = [(u, v) for u in (0.5 - w / 2.0, w / 2.0 - 0.5) for v in (0.5 - h / 2.0, h / 2.0 - 0.5)]
    for c in np.asarray(cams):
        fz, ez = float(c["fwd"][2]), float(c["eye"][2])
        duz, dvz = float(c["du"][2]), float(c["dv"][2])
        if int(c["proj"]) == 0:
            dz = [fz]
            oz = [ez + u * duz + v * dvz for u, v in corners]
        else:
            dz = [fz + u * duz + v * dvz for u, v in corners]
            oz = [ez]
        scale = max(1e-30, max(abs(x) for x in dz), float(np.abs(c["fwd"]).max()))
        up = max(dz) >= -1e-5 * scale
        down = min(dz) < 1e-5 * scale
        if dims is not None:
            # FP32 rounding of the origins: a relative margin of their terms
            tol = 1e-5 * (1.0 + abs(ez) + (w / 2.0) * abs(duz) + (h / 2.0) * abs(dvz))
            up = up and min(oz) <= float(dims[2]) - 1.0 + tol
            down = down and max(oz) >= -tol
        need_up |= up
        need_down |= down
    return ([1] if need_up else []) + ([-1] if need_down else [])


def pick_volume(holds, last_use, order, n):
    """The part volume that takes visit ``n``'s part (``order``: the parts'
    z_first of a render's visits, in order; ``holds``: the z_first each part
    volume holds, or None; ``last_use``: when each was last rendered, larger
    = later).  The volume rendered last is never taken (its render may still
    be running, so a load into it would wait for it); of the others, an
    empty one, else the one whose part is needed again latest: in the rest of
    this render, then in the next, assumed to repeat this order (ties: the
    one used least recently)."""
    future = list(order[n + 1:]) + list(order)
    never = len(future) + 1

    def next_use(z):
        if z is None:
            return never + 1
        try:
            return future.index(z)
        except ValueError:
            return never

    cands = list(range(len(holds)))
    if len(cands) > 1:
        newest = max(cands, key=lambda j: last_use[j])
        cands.remove(newest)
    return max(cands, key=lambda j: (next_use(holds[j]), -last_use[j]))


@dataclass
class Part:
    z_first: int
    cell_lo: int
    cell_hi: int


def plan_parts(nz: int, planes: int):
    """Parts of ``planes`` planes (at most nz) whose cell ranges tile the
    cells [0, nz - 1) in order; the last part is moved down so it has as
    many planes as the others."""
    planes = min(planes, nz)
    if planes < 2:
        raise ValueError("a part needs at least two planes")
    cells = planes - 1
    return [Part(min(lo, nz - planes), lo, min(lo + cells, nz - 1))
            for lo in range(0, nz - 1, cells)]


class PartStream:
    """A cube of ``dims`` (nx, ny, nz) rendered in parts of ``part_planes``
    planes.  ``source(z0, n)`` returns planes [z0, z0 + n) as a float32
    tensor (n, ny, nx) on the device or in page-locked host memory; it is
    called on the copy stream.  ``dtype`` is the parts' storage, ``pair``
    selects pair-texel texture storage (FP16 / int8), ``bounds`` gives FP32
    part volumes MIP bounds (vr_volume_attach_mip_bounds: faster MIP, the
    same images) and ``masks`` empty-space masks, built for the clip at each
    part's upload (faster compositing, the same images; a lower clip later
    reloads the parts).  ``cache_parts`` part
    volumes (at least two, at most one per part) stay on the device
    (``pick_volume`` decides which takes a part); two sweeps load
    2 (parts - cache_parts) parts a render once the cache is warm; one sweep
    keeps the parts it starts with and loads about parts - cache_parts + 1
    (varying from render to render in a short cycle; all parts with two
    volumes).
    Device memory: one brick buffer and one staging buffer of a part, and
    ``cache_parts`` textures of a part."""

    def __init__(self, dims, dtype: str, source, part_planes: int, device=None,
                 pair: bool = False, cache_parts: int = 2, bounds: bool = False,
                 masks: bool = False):
        nx, ny, nz = (int(d) for d in dims)
        self.dims = (nx, ny, nz)
        self.source = source
        self.parts = plan_parts(nz, part_planes)
        self.planes = min(part_planes, nz)
        self.device = torch.device(device) if device is not None else torch.device("cuda")
        self.dtype, self.pair = dtype, bool(pair)
        n_vols = min(max(2, int(cache_parts)), len(self.parts))
        from .api import volume_bytes
        # zeroed: the part volumes' first bound fills read defined values (each
        # part load derives the MIP bounds' scale again from its planes)
        self.bricks = torch.zeros(volume_bytes((nx, ny, self.planes), dtype), dtype=torch.uint8,
                                  device=self.device)
        self.bounds = bool(bounds) and dtype == "f32" and not pair
        self.vols = []
        for _ in range(n_vols):
            v = Volume(dims=(nx, ny, self.planes), dtype=dtype, buffer=self.bricks)
            v.attach_pair_texture() if pair else v.attach_texture()
            if self.bounds:
                v.attach_mip_bounds()
            if masks:
                v.attach_masks()
            self.vols.append(v)
        self.masks = bool(masks)
        self.clip = None
        self.holds = [None] * len(self.vols)        # z_first of the part each volume holds
        self.last_use = [-1] * len(self.vols)       # when each volume last rendered
        self.uses = 0
        # device staging for parts that come from host memory: one DMA copy
        # per part, then packing from device memory (uploads are serialised
        # on the copy stream, so one staging buffer serves every volume)
        self.staging = None
        self.copy = torch.cuda.Stream(self.device)
        self.done = [torch.cuda.Event() for _ in self.vols]
        self.bytes_loaded = 0
        self.parts_loaded = 0

    def device_bytes(self) -> int:
        """Device memory the stream holds for the cube: the shared brick
        buffer, the staging buffer and the part volumes' textures."""
        nx, ny, _ = self.dims
        tex_slices = self.planes + 2                 # plain formats; pair: planes + 1
        texel = {"f32": 4, "f16": 2, "i8": 1}[self.dtype]
        if self.pair:
            tex_slices, texel = self.planes + 1, 2 * texel
        staging = nx * ny * self.planes * 4
        bounds = nx * ny * (self.planes + 1) * 2 if self.bounds else 0
        masks = self.vols[0].mask_bytes() if self.masks else 0
        return (self.bricks.numel() + staging
                + len(self.vols) * (nx * ny * tex_slices * texel + bounds + masks))

    def set_transfer(self, lut, v_lo, v_hi, clip, term_alpha=1.0):
        for v in self.vols:
            v.set_transfer(lut, v_lo, v_hi, clip, term_alpha)
        # masks hold for clips at or above the one they were built for: a
        # lower clip reloads the parts (their bricks are gone)
        if self.masks and self.clip is not None and clip < self.clip:
            self.holds = [None] * len(self.vols)
        self.clip = clip

    def _load(self, i: int, part: Part):
        v = self.vols[i]
        if self.holds[i] == part.z_first:
            return
        self.copy.wait_event(self.done[i])           # its last render has finished
        with torch.cuda.stream(self.copy):
            planes = self.source(part.z_first, self.planes)
            if not planes.is_cuda:
                if self.staging is None or self.staging.shape != planes.shape:
                    self.staging = torch.empty(planes.shape, dtype=torch.float32,
                                               device=self.device)
                self.staging.copy_(planes, non_blocking=True)
                planes = self.staging
            # packs into the shared bricks and refreshes this volume's texture;
            # the next load reuses the staging and brick buffers after it, in
            # the copy stream's order
            v.upload(0, planes, stream=self.copy)
            if self.masks:                           # while the bricks hold this part
                v.build_masks(stream=self.copy)
        self.bytes_loaded += planes.numel() * planes.element_size()
        self.parts_loaded += 1
        self.holds[i] = part.z_first

    def render(self, cams: np.ndarray, w: int, h: int, targets, step: float = 0.5,
               count: torch.Tensor | None = None, stream=None):
        """Render the views into every target: a list of (mode, out) pairs,
        out a float32 tensor (views, h, w) or (views, h, w, 4); each part is
        loaded once per sweep for all targets."""
        stream = stream or torch.cuda.current_stream(self.device)
        cams = np.ascontiguousarray(cams)
        for mode, out in targets:
            render_init(out, mode, stream)
        step_order = []
        for sw in sweeps(cams, w, h, self.dims):
            order = self.parts if sw > 0 else self.parts[::-1]
            step_order += [(sw, p) for p in order]
        visits = [p.z_first for _, p in step_order]
        for n, (sw, part) in enumerate(step_order):
            held = [i for i, z in enumerate(self.holds) if z == part.z_first]
            if held:
                i = held[0]
            else:
                i = pick_volume(self.holds, self.last_use, visits, n)
                self._load(i, part)
            self.uses += 1
            self.last_use[i] = self.uses
            loaded = torch.cuda.Event()
            loaded.record(self.copy)
            stream.wait_event(loaded)
            for mode, out in targets:
                self.vols[i].render_part(self.dims, part.z_first, part.cell_lo, part.cell_hi,
                                         cams, w, h, mode, step, sw, out, count=count,
                                         stream=stream)
            self.done[i].record(stream)
        return targets

    def render_subcubes(self, cams: np.ndarray, w: int, h: int, targets, step: float = 0.5,
                        count: torch.Tensor | None = None, stream=None):
        """The paper's sub-cube pipeline (§3.1 items 1, 4, 5): every part
        rendered on its own into a partial image set (vr_render_part with
        sweep 0 from an empty start, so the parts go in any order: here the
        held ones first, each loaded at most once), then the partial images
        integrated per pixel in the order its ray meets the parts
        (vr_integrate_partials).  ``targets`` as in render.  Without early
        termination the images are the one-pass ones up to FP32 rounding;
        with it, each part stops at its own opacity.  Device memory: one
        partial image set per part and target."""
        stream = stream or torch.cuda.current_stream(self.device)
        cams = np.ascontiguousarray(cams)
        parts = sorted(range(len(self.parts)),
                       key=lambda j: self.parts[j].z_first not in self.holds)
        partials = []
        for mode, out in targets:
            pt = torch.empty((len(self.parts),) + tuple(out.shape), dtype=torch.float32,
                             device=out.device)
            render_init(pt.view((-1,) + tuple(out.shape[1:])), mode, stream)
            partials.append(pt)
        visits = [self.parts[j].z_first for j in parts]
        for n, j in enumerate(parts):
            part = self.parts[j]
            held = [i for i, z in enumerate(self.holds) if z == part.z_first]
            if held:
                i = held[0]
            else:
                i = pick_volume(self.holds, self.last_use, visits, n)
                self._load(i, part)
            self.uses += 1
            self.last_use[i] = self.uses
            loaded = torch.cuda.Event()
            loaded.record(self.copy)
            stream.wait_event(loaded)
            for (mode, _), pt in zip(targets, partials):
                self.vols[i].render_part(self.dims, part.z_first, part.cell_lo, part.cell_hi,
                                         cams, w, h, mode, step, 0, pt[j], count=count,
                                         stream=stream)
            self.done[i].record(stream)
        for (mode, out), pt in zip(targets, partials):
            integrate_partials(pt, cams, mode, out=out, stream=stream)
        return targets

    def close(self):
        for v in self.vols:
            v.close()
        self.vols = []
