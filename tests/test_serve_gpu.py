"""The continuous-batching server: every request's image is the same served
in a mix as rendered alone, admission never exceeds the memory budget, and
latencies are recorded."""
import numpy as np
import pytest
import torch

from paper_1001_2049_b300 import Volume, synth
from paper_1001_2049_b300.serve import RenderJob, Server, latency_stats, run_poisson

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cubes():
    specs = {"a": ((48, 40, 64), "f16", True), "b": ((40, 40, 2100), "i8", True),
             "c": ((36, 30, 44), "f32", False)}
    vols = {}
    for i, (name, (dims, dt, tex)) in enumerate(specs.items()):
        v = Volume(synth.make_cube(dims, 4, ("uniform", 3.0, 9.0), 70 + i).cuda(), dt)
        if tex:
            v.attach_texture()
        v.set_transfer(synth.default_lut(), 1.0, 9.0, 1.0, 0.99)
        vols[name] = (v, dims)
    torch.cuda.synchronize()
    return vols


def make_jobs(cubes, n, seed):
    rng = np.random.default_rng(seed)
    names = sorted(cubes)
    jobs = []
    for i in range(n):
        name = names[i % len(names)]
        dims = cubes[name][1]
        w, h = (int(x) for x in rng.integers(8, 64, 2))
        cam = synth.random_sphere_cameras(dims, 1, w, h, seed * 1000 + i)[0]
        mode = "mip" if rng.random() < 0.2 else "composite"
        clip = float(rng.uniform(2.0, 5.0))
        tf = (synth.default_lut(), clip, 9.0, clip, 0.99) if mode == "composite" else None
        jobs.append(RenderJob(name, cam, w, h, mode, 0.5, tf))
    return jobs


def alone(cubes, job):
    v = cubes[job.cube][0]
    if job.tf is not None:
        v.set_transfer(*job.tf)
    img = v.render(np.asarray([job.cam]), job.w, job.h, job.mode, job.step)[0]
    v.set_transfer(synth.default_lut(), 1.0, 9.0, 1.0, 0.99)
    return img


def test_each_request_is_the_same_alone_and_in_the_mix(cubes):
    server = Server({k: v[0] for k, v in cubes.items()}, mem_budget=1 << 22, max_batch=16,
                    streams=2, keep_outputs=True)
    jobs = make_jobs(cubes, 60, 1)
    for k in range(0, len(jobs), 7):          # arrivals while earlier work runs
        for job in jobs[k:k + 7]:
            server.submit(job)
        server.step()
    server.drain()
    assert len(server.done) == len(jobs) and server.launches >= 2
    for job in jobs:
        ref = alone(cubes, job)
        assert torch.allclose(job.out, ref, rtol=0, atol=1e-6), (job.cube, job.mode)


def test_admission_respects_the_memory_budget(cubes):
    budget = 64 * 64 * 16 * 3                  # about three large images at a time
    server = Server({k: v[0] for k, v in cubes.items()}, mem_budget=budget, max_batch=64,
                    streams=2)
    jobs = make_jobs(cubes, 40, 2)
    for job in jobs:
        server.submit(job)
    peak = 0
    while not server.idle():
        server.step()
        peak = max(peak, server.mem_in_use)
        assert server.mem_in_use <= budget
    assert len(server.done) == 40 and peak > 0
    too_big = RenderJob("a", jobs[0].cam, 4096, 4096)
    with pytest.raises(ValueError):
        server.submit(too_big)


def test_poisson_serving_reports_latencies(cubes):
    server = Server({k: v[0] for k, v in cubes.items()}, mem_budget=1 << 26, max_batch=32)
    pool = make_jobs(cubes, 50, 3)
    done, wall, n = run_poisson(server, lambda i: RenderJob(**{
        k: getattr(pool[i % len(pool)], k) for k in ("cube", "cam", "w", "h", "mode", "step",
                                                      "tf")}), rate=200.0, duration=1.0)
    st = latency_stats(done)
    assert st["n"] == n > 50
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    assert all(j.finished >= j.admitted >= j.arrival for j in done)


def test_per_request_server_gives_the_same_images(cubes):
    # the plain path the batched one is compared with: one single-view render
    # call per request, in arrival order
    server = Server({k: v[0] for k, v in cubes.items()}, mem_budget=1 << 22, max_batch=1,
                    streams=1, keep_outputs=True, per_request=True)
    jobs = make_jobs(cubes, 24, 4)
    for job in jobs:
        server.submit(job)
    server.drain()
    assert len(server.done) == len(jobs) and server.launches == len(jobs)
    for job in jobs:
        assert job.out.shape[0] == 1
        ref = alone(cubes, job)
        assert torch.allclose(job.out[0], ref, rtol=0, atol=1e-6), (job.cube, job.mode)


def test_split_requests_are_the_same_alone_and_in_the_mix(cubes):
    # images split into row bands of about 300 rays, launches of at most
    # 2000 rays: every band of a request may run in a different launch, and
    # the assembled image is the single-view render's
    server = Server({k: v[0] for k, v in cubes.items()}, mem_budget=1 << 22, max_batch=16,
                    streams=2, keep_outputs=True, band_rays=300, launch_rays=2000)
    jobs = make_jobs(cubes, 40, 5)
    for k in range(0, len(jobs), 6):
        for job in jobs[k:k + 6]:
            server.submit(job)
        server.step()
    server.drain()
    assert len(server.done) == len(jobs)
    assert server.launches > len(jobs) // 4
    assert server.mem_in_use == 0
    for job in jobs:
        ref = alone(cubes, job)
        assert torch.allclose(job.out, ref, rtol=0, atol=1e-6), (job.cube, job.mode)
        assert job.finished >= job.admitted >= job.arrival


def test_cancelled_requests_leave_the_server(cubes):
    server = Server({k: v[0] for k, v in cubes.items()}, mem_budget=1 << 20, max_batch=4,
                    streams=1, keep_outputs=True, band_rays=256, launch_rays=1024)
    jobs = make_jobs(cubes, 24, 6)
    tickets = [server.submit(j) for j in jobs]
    server.step()                                  # some admitted and one launch out
    cancel = tickets[1::3]
    assert all(server.cancel(t) for t in cancel)
    assert not server.cancel(10 ** 6)
    server.drain()
    assert sorted(j.ticket for j in server.cancelled) == sorted(cancel)
    assert sorted(j.ticket for j in server.done) == sorted(set(tickets) - set(cancel))
    assert server.mem_in_use == 0 and server.idle()
    for job in server.done:
        assert torch.allclose(job.out, alone(cubes, job), rtol=0, atol=1e-6)
