"""Benchmark: samples/s and frames/s of the ray caster on the 1024^3 workload.

Workload (one "step"): a 1024^3 float32 cube of sigma = 1 noise plus 2000
Gaussian line sources (SNR log-uniform 2-50) is resident in HBM; the step
renders 32 perspective 1920x1080 views orbiting the cube (step 0.5 voxel)
with front-to-back compositing (RGBA table clipped below 3 sigma, early
termination at alpha 0.99) and then a maximum-intensity pass on the same
views: 64 frames, two kernel launches.

``python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]``

Under torchrun (N > 1) every rank renders its own replica of the workload
(views are independent; no collective on the data path): weak scaling, and
the value is the samples of all ranks over the slowest rank's time.

The reference arm (``--impl reference``) times the FP64 CPU oracle as it
stands on the host cores, on a bounded sample of pixels of the same views.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1001_2049_b300 import Volume, synth  # noqa: E402
from paper_1001_2049_b300.api import launch_shapes  # noqa: E402

METRIC = "samples/s & fps (1080p, 1024³ cube), FP32 plain vs FP16/int8 batched; p99 ms"
W, H = 1920, 1080


def workload(args):
    """The benchmark workload, or (for profiling captures) a smaller cube
    with the same framing and ray density (edge E, resolution scaled by
    E/1024)."""
    wl = synth.LARGE
    if args.cube_edge == 1024 and args.views == 32 and args.res is None:
        return wl, synth.large_cameras(), W, H
    e = args.cube_edge
    w, h = (int(v) for v in args.res.split("x")) if args.res else (W * e // 1024, H * e // 1024)
    sub = synth.Workload("cube%d_orbit%d_%dx%d" % (e, args.views, w, h), (e, e, e),
                         max(1, wl.n_sources * e ** 3 // 1024 ** 3), wl.snr, wl.clip, wl.v_hi,
                         wl.seed, wl.term_alpha, wl.step)
    return sub, synth.orbit_cameras(sub.dims, args.views, w, h), w, h


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d["hbm_gbs"], "measured"
    return 6400.0, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r]
        os.unlink(self.f.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for n, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes: storage bytes of every voxel some sample's corners touch
# ---------------------------------------------------------------------------
# DRAM traffic of the two headline launches, per algorithmic byte, from one
# ncu capture of the small case of the same kernels (512^3 FP32 cube, 4
# orbit views at 960x540: inputs 4x the L2, a few GB on the device;
# dram__bytes_read.sum + dram__bytes_write.sum over the algorithmic bytes of
# that launch), scaled here to the full-size launch by its algorithmic bytes.
# At 512^3 the cube is 4x the L2 against 34x at 1024^3, so a kernel that
# re-reads voxels across a view re-reads a little more at full size (the
# MIP march without bounds: 0.95 at 512^3, 1.11 at 1024^3).  The ratios
# hold for the kernel sources they were taken on: KERNEL_SHA is the digest
# of every CUDA/C++ source of the library (kernel_sources_sha); when the
# sources differ the bench reports no traffic rather than a stale one.
TRAFFIC_CAPTURE = {
    "capture": "prof_final: bench.py --cube-edge 512 --views 4 --steps 1 --warmup 1 "
               "--shapes 7,3 (ncu --set full; profiles/tex_kernel_f32_cube1024_orbit32.md)",
    "kernel_sha": "96a7a1cab272c21e",
    # MIP with 8-bit bound codes, shape 3: (1.534231 + 0.021571) GB over 2.130716 GB
    "mip_bounds": (1.534231e9 + 0.021571e9) / 2.130716e9,
    # composite with masks, windowed march, shape 7: (0.366143 + 0.033616) GB over 2.153293 GB
    "composite_masks": (0.366143e9 + 0.033616e9) / 2.153293e9,
}


def kernel_sources_sha() -> str:
    """Digest of the library's CUDA/C++ sources and public header."""
    import hashlib
    root = os.path.dirname(os.path.abspath(__file__))
    csrc = os.path.join(root, "paper_1001_2049_b300", "csrc")
    files = sorted(os.path.join(csrc, f) for f in os.listdir(csrc)
                   if f.endswith((".cu", ".cuh", ".cpp", ".h")))
    h = hashlib.sha256()
    for f in files + [os.path.join(root, "include", "vr.h")]:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def touched_voxels(cam, dims, step, w, h, device):
    """Number of distinct voxels referenced by the eight corners of every
    sample of one view (float64 geometry; measurement only)."""
    nx, ny, nz = dims
    hi = torch.tensor([nx - 1.0, ny - 1.0, nz - 1.0], dtype=torch.float64, device=device)
    py, px = torch.meshgrid(torch.arange(h, device=device, dtype=torch.float64),
                            torch.arange(w, device=device, dtype=torch.float64), indexing="ij")
    u = (px + 0.5 - w / 2.0).reshape(-1, 1)
    v = (py + 0.5 - h / 2.0).reshape(-1, 1)
    t = lambda a: torch.tensor(np.asarray(a, dtype=np.float64), device=device)
    eye, fwd, du, dv = t(cam["eye"]), t(cam["fwd"]), t(cam["du"]), t(cam["dv"])
    if int(cam["proj"]) == 0:
        o = eye + u * du + v * dv
        d = fwd.expand_as(o) / torch.linalg.norm(fwd)
    else:
        o = eye.expand(u.shape[0], 3)
        d = fwd + u * du + v * dv
        d = d / torch.linalg.norm(d, dim=1, keepdim=True)
    with torch.no_grad():
        inv = 1.0 / d
        ta = (0.0 - o) * inv
        tb = (hi - o) * inv
        tn = torch.minimum(ta, tb).amax(dim=1).clamp_min(0.0)
        tf = torch.maximum(ta, tb).amin(dim=1)
        hit = tf >= tn
        K = torch.where(hit, torch.floor((tf - tn) / step) + 1, torch.zeros_like(tf)).long()
        o, d, tn, K = o[hit], d[hit], tn[hit], K[hit]
        bitmap = torch.zeros(nx * ny * nz, dtype=torch.bool, device=device)
        kmax = int(K.max().item()) if K.numel() else 0
        chunk = max(1, (1 << 23) // max(kmax, 1))
        ks = torch.arange(kmax, device=device, dtype=torch.float64)
        for s in range(0, o.shape[0], chunk):
            oo, dd, tt, kk = o[s:s + chunk], d[s:s + chunk], tn[s:s + chunk], K[s:s + chunk]
            valid = ks[None, :] < kk[:, None]
            tk = tt[:, None] + ks[None, :] * step
            p = oo[:, None, :] + tk[..., None] * dd[:, None, :]
            p = torch.minimum(torch.maximum(p, torch.zeros_like(p)), hi)[valid]
            i0 = torch.minimum(torch.floor(p).long(), (hi - 1).long())
            for c in range(8):
                ix = i0[:, 0] + (c & 1)
                iy = i0[:, 1] + ((c >> 1) & 1)
                iz = i0[:, 2] + ((c >> 2) & 1)
                bitmap[(iz * ny + iy) * nx + ix] = True
        return int(bitmap.sum().item())


# ---------------------------------------------------------------------------
# the reference arm and the CPU baseline: the FP64 oracle on host cores
# ---------------------------------------------------------------------------
def cpu_model() -> str:
    """The host CPU's model name (Linux /proc/cpuinfo), or the platform's."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or "unknown"


def oracle_throughput(host_cube, cams, wl, budget_s, seed=5, w=W, h=H, nthreads=0):
    """Run the oracle on random pixels of the views (composite then MIP) for
    about budget_s seconds (nthreads: OpenMP threads, 0 = all); returns
    (samples/s, frames/s, threads, sample)."""
    import oracle
    vol = oracle.Volume(host_cube)
    tf = oracle.TF(synth.default_lut(), wl.clip, wl.v_hi, wl.clip, wl.term_alpha)
    nb = oracle.Bands(0.0, 0.0, 0.0, 0.0)
    rng = np.random.default_rng(seed)
    samples, secs, pixels_done, n = 0, 0.0, 0, 2048
    while secs < budget_s:
        pix = np.stack([rng.integers(0, len(cams), n), rng.integers(0, w, n),
                        rng.integers(0, h, n)], axis=1).astype(np.int32)
        for mode in (oracle.COMPOSITE, oracle.MIP):
            t0 = time.perf_counter()
            r = oracle.render(vol, cams, w, h, mode, wl.step, tf, pixels=pix, bands=nb,
                              nthreads=nthreads)
            secs += time.perf_counter() - t0
            samples += int(r.nsamples.sum())
            pixels_done += n
        n = min(n * 2, 1 << 18)
    # a frame = W*H pixels; the two modes each count as frames
    fps = pixels_done / (w * h) / secs
    sample = "%d random pixels of the %d views (composite and MIP), %.1f s" % (
        pixels_done, len(cams), secs)
    return samples / secs, fps, nthreads if nthreads > 0 else oracle.num_threads(), sample


def precision_leg(cube, cams, W, H, wl, lut, pixels, reps=3, touched=None, peak=None):
    """The same cube and views stored as FP16 and as int8 with per-plane
    scale and offset, in both texture formats (one texel per voxel, and
    pair texels: a voxel with its neighbour in the next plane; the same
    images bit for bit), empty-space masks for the composite launch: launch
    times of each format, the faster format's as the row's, its roofline at
    the storage's own bytes (``touched`` voxels a view at 2 or 1 bytes, plus
    the images; int8 adds its two per-plane tables), and the images' values at
    ``pixels`` for the error against the oracle (evaluated in the CPU leg)."""
    out, values = {}, {}
    stream = torch.cuda.current_stream()
    comp = torch.empty((len(cams), H, W, 4), dtype=torch.float32, device=cube.device)
    mip = torch.empty((len(cams), H, W), dtype=torch.float32, device=cube.device)
    idx = torch.from_numpy(pixels.astype(np.int64)).to(cube.device)
    for dt in ("f16", "i8"):
        formats = {}
        for fmt in ("texture", "pair texture"):
            v = Volume(cube, dt)
            v.attach_texture() if fmt == "texture" else v.attach_pair_texture()
            v.attach_masks()
            v.set_transfer(lut, wl.clip, wl.v_hi, wl.clip, wl.term_alpha)
            row = {"storage": dt + " " + fmt}
            for mode, img in (("composite", comp), ("mip", mip)):
                cfg, _ = v.autotune(cams, W, H, mode, wl.step, out=img)
                ms = event_ms(lambda: v.render(cams, W, H, mode, wl.step, out=img), reps, stream)
                row[mode + "_ms_per_launch"] = ms
                row[mode + "_shape"] = cfg
                values[(dt, mode)] = img[idx[:, 0], idx[:, 2], idx[:, 1]].cpu().numpy()
            formats[fmt] = row
            v.close()
        best = min(formats.values(),
                   key=lambda r: r["composite_ms_per_launch"] + r["mip_ms_per_launch"])
        out[dt] = dict(best, formats=formats)
        if touched and peak:
            vb = {"f16": 2, "i8": 1}[dt]
            tables = 2 * 4 * wl.dims[2] if dt == "i8" else 0
            roof = {}
            for mode, px_bytes in (("composite", 16), ("mip", 4)):
                alg = (touched * vb + W * H * px_bytes + tables) * len(cams)
                gbs = alg / (best[mode + "_ms_per_launch"] / 1000.0) / 1e9
                roof[mode] = {"algorithmic_bytes_per_launch": alg, "achieved_gbs": gbs,
                              "frac": gbs / peak}
            out[dt]["roofline_at_storage_bytes"] = roof
    return out, values


def oracle_errors(host_cube, cams, wl, pixels, values, w=W, h=H):
    """The oracle at ``pixels`` (view, px, py) on the float32 source cube and
    on each storage's decoded cube; the largest error of each GPU image there
    against the oracle's acceptance set (max abs per channel; MIP divided by
    the cube's max - min), and how many pixels exceed the stated tolerance."""
    import oracle
    from oracle import quantize
    bands = oracle.fp32_bands(wl.dims, cams, wl.step, w, h)
    tf = oracle.TF(synth.default_lut(), wl.clip, wl.v_hi, wl.clip, wl.term_alpha)
    vols = {"f32": oracle.Volume(host_cube)}
    if any(dt == "f16" for dt, _ in values):
        vols["f16"] = oracle.Volume(quantize.to_f16(host_cube))
    if any(dt == "i8" for dt, _ in values):
        vols["i8"] = oracle.Volume(*quantize.quantize_i8(host_cube))
    tol = {"f32": 1e-4, "f16": 2e-3, "i8": 1e-2}
    mip_scale = float(host_cube.max() - host_cube.min())
    res = {}
    for mode_name, mode in (("composite", oracle.COMPOSITE), ("mip", oracle.MIP)):
        ch = 4 if mode == oracle.COMPOSITE else 1
        scale = 1.0 if mode == oracle.COMPOSITE else mip_scale
        ref = {k: oracle.render(vol, cams, w, h, mode, wl.step, tf, pixels=pixels, bands=bands)
               for k, vol in vols.items()}
        for (dt, m), got in values.items():
            if m != mode_name:
                continue
            row = res.setdefault(dt, {}).setdefault(mode_name, {})
            for against in ("f32", dt) if dt != "f32" else ("f32",):
                t = 1e-4 if against == dt else tol[dt]
                ok, err = oracle.match(ref[against], got.reshape(-1, ch), t, ch, scale)
                fin = err[np.isfinite(err)]
                key = "vs_float32_source" if against == "f32" else "vs_decoded_storage"
                row[key] = {"max_err": float(fin.max()) if fin.size else 0.0, "tol": t,
                            "pixels_over_tol": int((~ok).sum())}
    return {"pixels": int(len(pixels)), "errors": res}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = synth.LARGE
    cams = synth.large_cameras()
    cube = wl.cube("cuda" if torch.cuda.is_available() else "cpu").cpu().numpy()
    per_step = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        sps, fps, threads, sample = oracle_throughput(cube, cams, wl, args.ref_budget, seed=i)
        if i >= args.warmup:
            per_step.append((sps, fps, time.perf_counter() - t0))
    sps = statistics.mean(s for s, _, _ in per_step)
    fps = statistics.mean(f for _, f, _ in per_step)
    line = {
        "impl": "reference", "metric": METRIC, "value": sps, "unit": "samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # each step is a bounded sample of the workload: its measured time;
        # the whole 64-frame step at this rate is in config
        "ms_per_step": 1000.0 * statistics.mean(t for _, _, t in per_step),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "cube": "1024^3 float32", "views": 32,
                   "resolution": "1920x1080", "modes": ["composite", "mip"], "step": wl.step,
                   "fps": fps,
                   "projected_ms_per_full_step": 1000.0 * 64 / fps if fps else None},
        "cpu_baseline": {"value": sps, "unit": "samples/s", "cores": threads, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": sps, "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# batched and served legs (reported beside the headline number)
# ---------------------------------------------------------------------------
def aggregate_ranks(samples, elapsed, dist=None, device=None):
    """Whole-job figures of a timed region run by every rank: the samples of
    all ranks (sum) and the slowest rank's time (max), after which the ranks
    meet at a barrier.  One rank: the figures as given."""
    if dist is None:
        return samples, elapsed
    t = torch.tensor([float(samples), float(elapsed)], dtype=torch.float64, device=device)
    s = t[:1].clone()
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    e = t[1:].clone()
    dist.all_reduce(e, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(s.item()), float(e.item())


def run_leg(fn):
    """One secondary leg of the line: its figures, or the error that ended
    it (recorded in the line, so that the headline measured before it is
    still reported)."""
    try:
        return fn()
    except Exception as e:             # noqa: BLE001 -- reported, not hidden
        torch.cuda.empty_cache()
        return {"error": "%s: %s" % (type(e).__name__, str(e)[:300])}


def event_ms(fn, reps, stream):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def batched_leg(dev, reps=3):
    """64 mixed views of four resident cubes (f32, f16, f16, int8; texture
    storage, pair texels for f16 and int8): one persistent launch (replayed
    from a CUDA graph, tile and packet shape from the batch autotuner)
    against the plain FP32 path (the same views as 64 per-request renders of
    FP32 copies with texture storage, launch shapes from the per-view
    autotuner)."""
    from paper_1001_2049_b300 import (Request, batch_autotune, batch_shapes, batch_workspace,
                                      render_batch)
    lut = synth.default_lut()
    vols, f32 = [], []
    for i, (name, dims, dt) in enumerate(synth.BATCH_CUBES):
        cube = synth.batch_cube(i, dev)
        v = Volume(cube, dt)
        v.attach_pair_texture() if dt != "f32" else v.attach_texture()
        v.set_transfer(lut, 3.0, 50.0, 3.0, 0.99)
        p = Volume(cube, "f32")
        p.attach_texture()
        p.set_transfer(lut, 3.0, 50.0, 3.0, 0.99)
        del cube
        vols.append(v)
        f32.append(p)
    views = synth.batch_views()
    stream = torch.cuda.current_stream(dev)
    outs = [torch.empty((h, w, 4) if m == "composite" else (h, w), device=dev)
            for (_, _, w, h, m) in views]
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    reqs = [Request(vols[c], cam, w, h, m, 0.5, out=o, samples=cnt)
            for (c, cam, w, h, m), o in zip(views, outs)]
    ws = batch_workspace(dev)
    render_batch(reqs, ws)
    torch.cuda.synchronize()
    samples = int(cnt.item())
    for r in reqs:
        r.samples = None
    # tile and ray-packet shape of the batched launch, by the batch autotuner
    # on this very batch; the plain path's launch shapes by the per-view
    # autotuner, per cube and mode on that cube's largest view
    cfg, tune_ms = batch_autotune(reqs, ws)
    for c, p in enumerate(f32):
        for mode in ("composite", "mip"):
            mine = [(w * h, cam, w, h) for (cc, cam, w, h, m) in views if cc == c and m == mode]
            if mine:
                _, cam, w, h = max(mine, key=lambda x: x[0])
                p.autotune(np.asarray([cam]), w, h, mode, 0.5)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        render_batch(reqs, ws, stream=side)
        with torch.cuda.graph(g, stream=side):
            render_batch(reqs, ws, stream=side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    batch_ms = event_ms(g.replay, reps, stream)
    launch_ms = event_ms(lambda: render_batch(reqs, ws), reps, stream)

    def per_request():
        for (c, cam, w, h, m), o in zip(views, outs):
            f32[c].render(np.asarray([cam]), w, h, m, 0.5, out=o.view((1,) + tuple(o.shape)))
    per_request()
    plain_ms = event_ms(per_request, reps, stream)
    n = len(views)
    res = {"views": n, "cubes": [c[0] for c in synth.BATCH_CUBES],
           "samples_per_batch": samples,
           "batched_graph_ms": batch_ms, "batched_fps": n / (batch_ms / 1000.0),
           "batched_samples_per_s": samples / (batch_ms / 1000.0),
           "batched_launch_ms": launch_ms,
           "batch_shape": {"config": cfg, "tile_and_packet": list(batch_shapes()[cfg]),
                           "ms": tune_ms},
           "plain_f32_per_request_ms": plain_ms, "plain_f32_fps": n / (plain_ms / 1000.0),
           "speedup_vs_plain_f32": plain_ms / batch_ms}
    for v in vols + f32:
        v.close()
    return res


def small_workload_leg(dev, reps=50, check=True):
    """The 64x64x128 workload: its 256^2 orthographic view along the
    frequency axis and the 32 orbit views at 256^2 (the precision variants'
    views), stored as FP32, FP16 and int8 (texture storage; empty-space
    masks for compositing; MIP bounds for FP32), MIP and composite: ms per
    launch, frames/s and samples/s (launch-bound at this size: no roofline
    figure).  With ``check``, each image's largest error at every pixel
    against the FP64 oracle on the decoded storage and on the float32
    source, acceptance sets as in the tests."""
    wl = synth.SMALL
    lut = synth.default_lut()
    cube = wl.cube(dev)
    host = cube.cpu().numpy()
    views = {"ortho_256": (synth.small_camera(), 256, 256),
             "orbit32_256": (synth.orbit_cameras(wl.dims, 32, 256, 256), 256, 256)}
    stream = torch.cuda.current_stream(dev)
    out = {"workload": wl.name, "cube": "64x64x128 float32, 5 sources SNR 3-10", "step": wl.step,
           "clip_sigma": wl.clip, "rows": {}}
    if check:
        import oracle
        from oracle import quantize
        ovols = {"f32": oracle.Volume(host), "f16": oracle.Volume(quantize.to_f16(host)),
                 "i8": oracle.Volume(*quantize.quantize_i8(host))}
        tf = oracle.TF(lut, wl.clip, wl.v_hi, wl.clip, wl.term_alpha)
        tol = {"f32": 1e-4, "f16": 2e-3, "i8": 1e-2}
        mip_scale = float(host.max() - host.min())
    for dt in ("f32", "f16", "i8"):
        v = Volume(cube, dt)
        v.attach_texture()
        v.attach_masks()
        if dt == "f32":
            v.attach_mip_bounds()
        v.set_transfer(lut, wl.clip, wl.v_hi, wl.clip, wl.term_alpha)
        for vname, (cams, w, h) in views.items():
            row = {}
            for mode in ("composite", "mip"):
                img = torch.empty((len(cams), h, w, 4) if mode == "composite" else
                                  (len(cams), h, w), device=dev)
                cnt = torch.zeros(1, dtype=torch.int64, device=dev)
                v.render(cams, w, h, mode, wl.step, out=img, count=cnt)
                torch.cuda.synchronize()
                ms = event_ms(lambda: v.render(cams, w, h, mode, wl.step, out=img), reps,
                              stream)
                r = {"ms_per_launch": ms, "fps": len(cams) / (ms / 1000.0),
                     "samples_per_s": int(cnt.item()) / (ms / 1000.0)}
                if check:
                    got = img.cpu().numpy().reshape(-1, 4 if mode == "composite" else 1)
                    om = oracle.COMPOSITE if mode == "composite" else oracle.MIP
                    bands = oracle.fp32_bands(wl.dims, cams, wl.step, w, h)
                    sc = mip_scale if mode == "mip" else 1.0
                    for ref, key in ((dt, "vs_decoded"), ("f32", "vs_source")):
                        if dt == "f32" and key == "vs_source":
                            continue
                        res = oracle.render(ovols[ref], cams, w, h, om, wl.step, tf, bands=bands)
                        ok, err = oracle.match(res, got, 1e-4 if key == "vs_decoded" else tol[dt],
                                               got.shape[1], sc)
                        fin = err[np.isfinite(err)]
                        r["max_err_" + key] = float(fin.max()) if fin.size else 0.0
                        r["pixels_over_tol_" + key] = int((~ok).sum())
                row[mode] = r
            out["rows"]["%s %s" % (dt, vname)] = row
        v.close()
    return out


def object_order_leg(vol, cams, W, H, wl, mip, mip_ms, reps=3):
    """MIP of the same views in object order (sub-cubes of 32^3 cells staged
    in shared memory once for all views, read from the bricks): its launch
    time against the texture march's, and whether its images and sample
    count are the texture march's bit for bit."""
    dev = mip.device
    out = torch.empty_like(mip)
    n = torch.zeros(1, dtype=torch.int64, device=dev)
    vol.render_object_order(cams, W, H, "mip", wl.step, out=out, count=n)
    torch.cuda.synchronize()
    n_tex = torch.zeros(1, dtype=torch.int64, device=dev)
    vol.render(cams, W, H, "mip", wl.step, out=torch.empty_like(mip), count=n_tex)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    ms = event_ms(lambda: vol.render_object_order(cams, W, H, "mip", wl.step, out=out), reps, s)
    return {"ms_per_launch": ms, "texture_mip_ms_per_launch": mip_ms,
            "vs_texture": mip_ms / ms,
            "images_identical_to_texture_mip": bool(torch.equal(out, mip)),
            "samples": int(n.item()), "samples_identical": int(n.item()) == int(n_tex.item()),
            "sub_cubes": int(np.prod([(d - 2) // 32 + 1 for d in wl.dims])),
            "reads": "bricks (no texture storage)"}


def tf_edit_leg(vol, cams, W, H, wl, lut):
    """Interactive transfer-function editing: a sequence of clip levels, each
    set and followed by one 1080p composite view; latency from the
    vr_set_transfer call to the finished image (host clock), with the
    empty-space masks (rebuilt only when the clip drops below the level they
    were built for) and without them."""
    clips = [3.0, 3.25, 3.5, 2.75, 4.0, 2.5, 3.0, 5.0, 2.0, 3.0, 3.5, 4.5] * 3
    out = torch.empty((1, H, W, 4), dtype=torch.float32, device=vol.device)
    res = {}
    for label, masks in (("with_masks", True), ("without_masks", False)):
        if masks:
            vol.attach_masks()
        else:
            vol.detach_masks()
        lat, level, rebuilt = [], None, 0
        for i, c in enumerate(clips):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            vol.set_transfer(lut, c, wl.v_hi, c, wl.term_alpha)
            vol.render(cams[i % len(cams):i % len(cams) + 1], W, H, "composite", wl.step, out=out)
            torch.cuda.synchronize()
            lat.append(1000.0 * (time.perf_counter() - t0))
            if masks and (level is None or c < level):
                level, rebuilt = c, rebuilt + 1
        lat = np.array(lat[1:])                 # the first edit also builds the first masks
        res[label] = {"edits": int(lat.size), "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
                      "mask_builds": rebuilt if masks else 0}
    vol.attach_masks()
    vol.set_transfer(lut, wl.clip, wl.v_hi, wl.clip, wl.term_alpha)
    return res


def out_of_core_leg(cube, cams, W, H, wl, lut, comp_ref, mip_ref, part_planes=129, cache_parts=4,
                    reps=6):
    """The 1024^3 workload rendered part by part from page-locked host memory
    (the cube never resident on the device: a cache of ``cache_parts`` part
    volumes of ``part_planes`` planes sharing one brick buffer, each with MIP
    bounds and empty-space masks built as it loads), composite and MIP in one
    pass over the parts
    per sweep; the images are compared with the resident render's.  The
    loads vary from render to render in a short cycle (the part volumes keep
    the parts a sweep starts with), so time and loads are means over
    ``reps`` renders after a warm-up render."""
    from paper_1001_2049_b300.stream import PartStream, sweeps
    host = torch.empty(cube.shape, dtype=torch.float32, pin_memory=True)
    host.copy_(cube)
    ps = PartStream(wl.dims, "f32", lambda z0, n: host[z0:z0 + n], part_planes,
                    cache_parts=cache_parts, bounds=True, masks=True)
    ps.set_transfer(lut, wl.clip, wl.v_hi, wl.clip, wl.term_alpha)
    comp = torch.empty_like(comp_ref)
    mip = torch.empty_like(mip_ref)
    targets = [("composite", comp), ("mip", mip)]
    ps.render(cams, W, H, targets, wl.step)
    torch.cuda.synchronize()
    same = bool(torch.equal(comp, comp_ref) and torch.equal(mip, mip_ref))
    times, loaded, parts = [], [], []
    for _ in range(reps):
        b0, p0 = ps.bytes_loaded, ps.parts_loaded
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ps.render(cams, W, H, targets, wl.step)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        loaded.append(ps.bytes_loaded - b0)
        parts.append(ps.parts_loaded - p0)
    same = same and bool(torch.equal(comp, comp_ref) and torch.equal(mip, mip_ref))
    sub = subcube_leg(ps, cams, W, H, wl, comp, mip, comp_ref, mip_ref, reps)
    res = {"parts": len(ps.parts), "planes_per_part": ps.planes,
           "cache_parts": len(ps.vols), "mip_bounds": True, "empty_space_masks": True,
           "sweeps": len(sweeps(cams, W, H, wl.dims)),
           "ms_per_step": 1000.0 * sum(times) / len(times),
           "ms_per_step_min": 1000.0 * min(times), "renders_timed": len(times),
           "part_loads_per_step": sum(parts) / len(parts),
           "host_bytes_read_per_step": sum(loaded) / len(loaded),
           "device_bytes_for_the_cube": ps.device_bytes(),
           "cube_bytes": cube.numel() * 4, "images_identical_to_resident": same,
           "subcubes": sub}
    ps.close()
    del host
    return res


def subcube_leg(ps, cams, W, H, wl, comp, mip, comp_ref, mip_ref, reps):
    """The paper's own pipeline on the same part cache: every part rendered
    on its own into partial images (any order, each loaded at most once),
    then the partial images integrated per pixel in each ray's order.  MIP
    is the resident image bit for bit; composite differs where a part
    reaches the termination alpha (each part stops at its own opacity).
    The integration kernel is also timed alone on a partial image set of
    this size: it reads every partial image once and writes one image."""
    from paper_1001_2049_b300 import integrate_partials
    targets = [("composite", comp), ("mip", mip)]
    ps.render_subcubes(cams, W, H, targets, wl.step)
    torch.cuda.synchronize()
    times, loads = [], []
    for _ in range(reps):
        p0 = ps.parts_loaded
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ps.render_subcubes(cams, W, H, targets, wl.step)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        loads.append(ps.parts_loaded - p0)
    mip_same = bool(torch.equal(mip, mip_ref))
    dA = float((comp[..., 3] - comp_ref[..., 3]).abs().max().item())
    n_parts = len(ps.parts)
    partials = torch.zeros((n_parts,) + tuple(comp.shape), device=comp.device)
    stream = torch.cuda.current_stream()
    integrate_partials(partials, cams, "composite", out=comp)
    ms = event_ms(lambda: integrate_partials(partials, cams, "composite", out=comp), 5, stream)
    nbytes = (n_parts + 1) * comp.numel() * 4
    del partials
    torch.cuda.empty_cache()
    return {"ms_per_step": 1000.0 * sum(times) / len(times),
            "part_loads_per_step": sum(loads) / len(loads),
            "mip_identical_to_resident": mip_same,
            "composite_max_alpha_difference_to_resident": dA,
            "integrate_composite_ms": ms, "integrate_bytes": nbytes,
            "integrate_gb_s": nbytes / ms / 1e6}


def _served_volume(i, dt, dev):
    """Served cube i stored as ``dt`` with texture storage only (built slab
    by slab through one brick buffer, which is freed afterwards)."""
    name, dims = synth.SERVE_CUBES[i]
    v = Volume(dims=dims, dtype=dt, device=dev)
    for z0, slab in synth.serve_cube_slabs(i, dev):
        v.upload(z0, slab)
        del slab
    v.attach_texture()
    v.drop_bricks()
    v.set_transfer(synth.default_lut(), 3.0, 50.0, 3.0, 0.99)
    return v


#: Continuous batching splits images into row bands of about BAND_RAYS rays
#: and gives a launch at most LAUNCH_RAYS rays, so no launch -- and none of
#: the requests that arrive while it runs -- waits on one large view.
BAND_RAYS = 1 << 19
LAUNCH_RAYS = 1 << 22


def _serve(vols, names, rate, duration, batched, seed, split=True):
    from paper_1001_2049_b300.serve import RenderJob, Server, latency_stats, run_poisson
    rng = np.random.default_rng(seed)
    dims = {n: vols[n].dims for n in names}

    def make(i):
        name = names[int(rng.integers(0, len(names)))]
        cam, w, h, mode, tf = synth.serve_request(dims[name], rng)
        return RenderJob(name, cam, w, h, mode, 0.5, tf)
    if batched:
        server = Server(vols, mem_budget=8 << 30, max_batch=64, streams=2,
                        band_rays=BAND_RAYS if split else 0,
                        launch_rays=LAUNCH_RAYS if split else 0)
    else:
        server = Server(vols, mem_budget=8 << 30, max_batch=1, streams=1, per_request=True)
    done, wall, n = run_poisson(server, make, rate, duration, seed=seed)
    st = latency_stats(done)
    st["throughput_req_s"] = n / wall
    st["launches"] = server.launches
    return st


def serving_leg(dev, rates=(50.0, 100.0, 200.0, 500.0), duration=20.0, saturated=5.0):
    """The served workload: Poisson arrivals of random requests (a random
    direction, a resolution from 512^2 to 1920x1080, 80 % composite, clip
    U[2,5] sigma) over six resident cubes (four 2048x2048x4096 and two
    1024^3, FP16, texture storage only: 146 GB of cube data), served with
    continuous batching (images split into row bands, launches capped in
    rays; at 200 req/s also without splitting, for comparison).  Each rate
    runs ``duration`` seconds, except 500 req/s, above what one GPU serves,
    which runs ``saturated`` seconds: there the queue only grows, and the
    figure of interest is the throughput, not the latency of a backlog.  Head to
    head with the plain FP32 path (one single-view render per request) on
    the cubes whose FP32 copies fit together in memory (two large, two
    small): the same request streams on those four cubes, served both
    ways."""
    t0 = time.perf_counter()
    names = [n for n, _ in synth.SERVE_CUBES]
    sub = [names[0], names[1], names[4], names[5]]
    vols = {n: _served_volume(i, "f16", dev) for i, n in enumerate(names)}
    torch.cuda.synchronize()
    build_f16 = time.perf_counter() - t0
    out = {"cubes": names, "storage": "f16 layered textures, bricks dropped",
           "resident_cube_bytes": sum(2 * d[0] * d[1] * d[2] for _, d in synth.SERVE_CUBES),
           "resident_device_bytes": {n: dict(zip(("library", "caller"), vols[n].device_bytes()))
                                     for n in names},
           "band_rays": BAND_RAYS, "launch_rays": LAUNCH_RAYS,
           "duration_s_per_rate": duration, "duration_s_at_500": saturated,
           "build_s": build_f16, "rates": {},
           "head_to_head": {"cubes": sub, "rates": {}}}
    for rate in rates:
        secs = saturated if rate >= 500.0 else duration
        out["rates"][str(int(rate))] = _serve(vols, names, rate, secs, True,
                                             synth.SERVE_SEED + int(rate))
        if rate == 200.0:
            out["rates"]["200_without_splitting"] = _serve(
                vols, names, rate, duration, True, synth.SERVE_SEED + int(rate), split=False)
        out["head_to_head"]["rates"][str(int(rate))] = {
            "continuous_batching_f16": _serve(vols, sub, rate, secs, True,
                                              synth.SERVE_SEED + 1000 + int(rate))}
    for v in vols.values():
        v.close()
    del vols
    torch.cuda.empty_cache()
    f32 = {n: _served_volume(names.index(n), "f32", dev) for n in sub}
    for rate in rates:
        secs = saturated if rate >= 500.0 else duration
        out["head_to_head"]["rates"][str(int(rate))]["plain_f32_per_request"] = _serve(
            f32, sub, rate, secs, False, synth.SERVE_SEED + 1000 + int(rate))
    for v in f32.values():
        v.close()
    del f32
    torch.cuda.empty_cache()
    out["total_s"] = time.perf_counter() - t0
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0,
                    help="seconds of oracle work for the CPU baseline (0: skip)")
    ap.add_argument("--ref-budget", type=float, default=10.0,
                    help="seconds of oracle work per step of the reference arm")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="steps of the end-to-end leg (default: --steps)")
    ap.add_argument("--cube-edge", type=int, default=1024,
                    help="profiling captures only: smaller cube, same framing")
    ap.add_argument("--views", type=int, default=32)
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--shapes", default=None,
                    help="launch shapes C,M (composite, MIP) instead of the autotuner's")
    ap.add_argument("--no-masks", action="store_true",
                    help="composite without the empty-space masks")
    ap.add_argument("--no-bounds", action="store_true",
                    help="MIP without the MIP bounds")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched and served legs")
    ap.add_argument("--storage", default="texture", choices=["texture", "bricks"],
                    help="render from layered textures (default) or gather from the bricks")
    ap.add_argument("--res", default=None, help="WxH (default scales with the cube)")
    args = ap.parse_args()
    if args.e2e_steps is None:
        args.e2e_steps = args.steps
    if args.impl == "reference":
        return run_reference(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    wl, cams, W, H = workload(args)
    n_views = len(cams)
    lut = synth.default_lut()
    cube = wl.cube(dev)
    vol = Volume(cube, "f32")
    if args.storage == "texture":
        vol.attach_texture()
        if not args.no_masks:
            vol.attach_masks()
        if not args.no_bounds:
            vol.attach_mip_bounds()
    masks_on = args.storage == "texture" and not args.no_masks
    bounds_on = args.storage == "texture" and not args.no_bounds
    vol.set_transfer(lut, wl.clip, wl.v_hi, wl.clip, wl.term_alpha)
    comp = torch.empty((n_views, H, W, 4), dtype=torch.float32, device=dev)
    mip = torch.empty((n_views, H, W), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # launch shapes chosen by the autotuner on these very views (untimed)
    tuned = {}
    if args.storage == "texture" and args.shapes:
        for mode, cfg in zip(("composite", "mip"), (int(c) for c in args.shapes.split(","))):
            vol.set_launch_config(mode, cfg)
            tuned[mode] = {"config": cfg, "shape": list(launch_shapes()[cfg]), "ms": None}
    elif args.storage == "texture" and not args.no_tune:
        for mode, out in (("composite", comp), ("mip", mip)):
            cfg, ms = vol.autotune(cams, W, H, mode, wl.step, out=out)
            tuned[mode] = {"config": cfg, "shape": list(launch_shapes()[cfg]), "ms": ms}

    # samples per step (untimed): counted by the kernels themselves
    cnt = torch.zeros(2, dtype=torch.int64, device=dev)
    vol.render(cams, W, H, "composite", wl.step, out=comp, count=cnt[0:1])
    vol.render(cams, W, H, "mip", wl.step, out=mip, count=cnt[1:2])
    torch.cuda.synchronize()
    samples_comp, samples_mip = (int(x) for x in cnt.tolist())
    samples_step = samples_comp + samples_mip

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        vol.render(cams, W, H, "composite", wl.step, out=comp)
        if ev is not None:
            ev[1].record(stream)
        vol.render(cams, W, H, "mip", wl.step, out=mip)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed = t0.elapsed_time(t1) / 1000.0
    total_samples, elapsed = aggregate_ranks(samples_step * args.steps, elapsed, dist, dev)
    comp_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    mip_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)

    # context only (outside the timed region): the composite launch without
    # the empty-space masks, the MIP launch without the MIP bounds
    def one_launch_ms(mode, out):
        vol.render(cams, W, H, mode, wl.step, out=out)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        vol.render(cams, W, H, mode, wl.step, out=out)
        e[1].record(stream)
        torch.cuda.synchronize()
        return e[0].elapsed_time(e[1])
    no_masks = no_bounds = None
    if masks_on:
        vol.detach_masks()
        no_masks = {"composite_ms_per_launch": one_launch_ms("composite", comp)}
        vol.attach_masks()
    if bounds_on:
        vol.detach_mip_bounds()
        no_bounds = {"mip_ms_per_launch": one_launch_ms("mip", mip)}
        vol.attach_mip_bounds()

    # end to end through the public API: cameras in, every step's images back
    # to pinned host memory.  The copies run on a second stream from two
    # alternating sets of output buffers, so a step's copies overlap the next
    # step's renders; a render waits until the copies that read its buffers
    # two steps earlier have finished, and the clock stops when the last
    # step's copies have landed.
    host_comp = torch.empty(comp.shape, dtype=torch.float32, pin_memory=True)
    host_mip = torch.empty(mip.shape, dtype=torch.float32, pin_memory=True)
    outs = [(comp, mip)]
    if args.e2e_steps > 1:
        outs.append((torch.empty_like(comp), torch.empty_like(mip)))
    copy_stream = torch.cuda.Stream(dev)
    copied = [None] * len(outs)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for i in range(args.e2e_steps):
        slot = i % len(outs)
        c_out, m_out = outs[slot]
        if copied[slot] is not None:
            stream.wait_event(copied[slot])
        for mode, out, host in (("composite", c_out, host_comp), ("mip", m_out, host_mip)):
            vol.render(cams, W, H, mode, wl.step, out=out, stream=stream)
            done = torch.cuda.Event()
            done.record(stream)
            copy_stream.wait_event(done)
            with torch.cuda.stream(copy_stream):
                host.copy_(out, non_blocking=True)
        copied[slot] = torch.cuda.Event()
        copied[slot].record(copy_stream)
    copy_stream.synchronize()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - e0) / max(1, args.e2e_steps)
    del outs
    d2h = host_comp.numel() * 4 + host_mip.numel() * 4
    h2d = 2 * cams.nbytes

    result = None
    if rank == 0:
        # algorithmic bytes of the dominant (composite) launch: per view, the
        # storage bytes of every voxel a sample's corners touch (measured on
        # view 0, the views being rotations of one another about the cube's
        # vertical axis), plus the RGBA output and the table
        touched = touched_voxels(cams[0], wl.dims, wl.step, W, H, dev)
        full = samples_mip
        frac_run = samples_comp / full if full else 1.0
        per_view = touched * 4 * frac_run + W * H * 16 + 256 * 16
        comp_bytes = per_view * n_views
        mip_bytes = (touched * 4 + W * H * 4) * n_views
        peak, peak_kind = peaks()
        dom_ms, dom_bytes, dom = (comp_ms, comp_bytes, "composite") if comp_ms >= mip_ms else \
            (mip_ms, mip_bytes, "mip")
        achieved = dom_bytes / (dom_ms / 1000.0) / 1e9

        sha = kernel_sources_sha()
        fresh = TRAFFIC_CAPTURE["kernel_sha"] == sha

        def measured(kind, alg):
            if args.storage != "texture" or kind is None or not fresh or \
                    TRAFFIC_CAPTURE.get(kind) is None:
                return None
            return TRAFFIC_CAPTURE[kind] * alg
        kinds = {"mip": "mip_bounds" if bounds_on else None,
                 "composite": "composite_masks" if masks_on else None}
        traffic = measured(kinds[dom], dom_bytes)
        comp_traffic = measured(kinds["composite"], comp_bytes)
        value = total_samples / elapsed
        fps = 2 * n_views * args.steps * world / elapsed
        # precision variants of the same cube and views (FP16, int8), and the
        # f32 images' values at the pixels where the oracle checks them
        rng = np.random.default_rng(synth.LARGE.seed + 7)
        pixels = np.stack([rng.integers(0, n_views, 20000), rng.integers(0, W, 20000),
                           rng.integers(0, H, 20000)], axis=1).astype(np.int32)
        prec, values = None, {}
        if args.storage == "texture" and not args.no_extra and W == 1920:
            idx = torch.from_numpy(pixels.astype(np.int64)).to(dev)
            values[("f32", "composite")] = comp[idx[:, 0], idx[:, 2], idx[:, 1]].cpu().numpy()
            values[("f32", "mip")] = mip[idx[:, 0], idx[:, 2], idx[:, 1]].cpu().numpy()
            prec, pv = precision_leg(cube, cams, W, H, wl, lut, pixels, touched=touched,
                                     peak=peak)
            values.update(pv)
            for dt, row in prec.items():
                ms = row["composite_ms_per_launch"] + row["mip_ms_per_launch"]
                row["fps"] = 2 * n_views / (ms / 1000.0)
                row["fps_vs_f32"] = (comp_ms + mip_ms) / ms
        cpu = None
        if args.cpu_budget > 0:
            host_cube = cube.cpu().numpy()
            sps, cfps, threads, sample = oracle_throughput(host_cube, cams, wl,
                                                           args.cpu_budget, w=W, h=H)
            cpu = {"value": sps, "unit": "samples/s", "cores": threads, "kind": "oracle",
                   "sample": sample, "fps": cfps, "cpu_model": cpu_model(),
                   "nproc": os.cpu_count()}
            # the same oracle on one thread, on a smaller sample
            sps1, _, _, sample1 = oracle_throughput(host_cube, cams, wl,
                                                    max(2.0, args.cpu_budget / 5), seed=11,
                                                    w=W, h=H, nthreads=1)
            cpu["one_thread"] = {"value": sps1, "unit": "samples/s", "sample": sample1}
            if values:
                # the oracle's results at the checked pixels also give the
                # error of every storage's images against FP64
                cpu["errors_at_checked_pixels"] = oracle_errors(host_cube, cams, wl, pixels,
                                                                values, w=W, h=H)
            del host_cube
        extra = {}
        if not args.no_extra and W == 1920:
            extra["object_order"] = run_leg(
                lambda: object_order_leg(vol, cams, W, H, wl, mip, mip_ms))
            if args.storage == "texture" and not args.no_masks:
                extra["tf_edit"] = run_leg(lambda: tf_edit_leg(vol, cams, W, H, wl, lut))
            if args.storage == "texture":
                vol.close()
                torch.cuda.empty_cache()
                r = run_leg(lambda: out_of_core_leg(cube, cams, W, H, wl, lut, comp, mip))
                r["resident_ms_per_step"] = comp_ms + mip_ms
                extra["out_of_core"] = r
            del comp, mip, host_comp, host_mip
            vol.close()
            del vol, cube
            torch.cuda.empty_cache()
            extra["small_workload"] = run_leg(
                lambda: small_workload_leg(dev, check=args.cpu_budget > 0))
            extra["batched"] = run_leg(lambda: batched_leg(dev))
            torch.cuda.empty_cache()
            extra["serving"] = run_leg(lambda: serving_leg(dev))
        result = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {
                "workload": wl.name,
                "cube": "%dx%dx%d float32, %d sources, sigma=1 noise" % (wl.dims + (wl.n_sources,)),
                "storage": "f32 32^3 bricks" + (" + layered textures" if args.storage == "texture"
                                                else ""),
                "views": n_views, "resolution": "%dx%d" % (W, H),
                "modes": ["composite (clip 3 sigma, early termination 0.99)", "mip"],
                "step": wl.step, "fps": fps, "frames_per_step": 2 * n_views,
                "samples_per_step": samples_step, "samples_composite": samples_comp,
                "samples_mip": samples_mip, "composite_ms_per_launch": comp_ms,
                "mip_ms_per_launch": mip_ms, "parallelism": "replica per GPU (views)",
                "empty_space_masks": masks_on,
                "without_masks": no_masks,
                "mip_bounds": bounds_on,
                "without_bounds": no_bounds,
                "autotuned": tuned,
                "l2": "inputs larger than L2 (a %.2f GiB cube per view pass, L2 126 MB)"
                      % (4.0 * wl.dims[0] * wl.dims[1] * wl.dims[2] / 2 ** 30)},
            "roofline": {"bound": "hbm",
                         "kernel": ("tex_kernel" if args.storage == "texture"
                                    else "march kernel") + " %s f32" % dom
                                   + (" (8-bit MIP bound codes)" if dom == "mip" and bounds_on
                                      else ""),
                         "achieved": achieved,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "traffic_source": (
                             "ncu dram__bytes_read.sum + dram__bytes_write.sum per algorithmic "
                             "byte of the small case (%s), times this launch's algorithmic "
                             "bytes" % TRAFFIC_CAPTURE["capture"]) if traffic else (
                             "null: the kernel sources (%s) differ from those of the capture "
                             "(%s)" % (sha, TRAFFIC_CAPTURE["kernel_sha"])),
                         "kernel_sources_sha": sha,
                         "algorithmic_bytes_per_launch": dom_bytes, "dominant": dom,
                         "touched_voxels_per_view": touched,
                         # the whole step: both launches' algorithmic bytes over
                         # the timed step
                         "step": {"achieved": (comp_bytes + mip_bytes) * args.steps
                                  / elapsed / 1e9,
                                  "frac": (comp_bytes + mip_bytes) * args.steps
                                  / elapsed / 1e9 / peak,
                                  "algorithmic_bytes": comp_bytes + mip_bytes,
                                  "ms": 1000.0 * elapsed / args.steps},
                         "composite": {"achieved": comp_bytes / (comp_ms / 1000.0) / 1e9,
                                       "frac": comp_bytes / (comp_ms / 1000.0) / 1e9 / peak,
                                       "algorithmic_bytes_per_launch": comp_bytes,
                                       "traffic": comp_traffic,
                                       "empty_space_masks": masks_on}},
            "cpu_baseline": cpu,
            "e2e": ({"value": samples_step / e2e_s * world, "unit": "samples/s",
                     "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                     "ms_per_step": 1000.0 * e2e_s} if args.e2e_steps > 0 else None),
            "gpu_launches": 2 * args.steps,
            "clocks": clk,
        }
        if prec is not None:
            result["precision"] = prec
        result.update(extra)
        print(json.dumps(result))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
