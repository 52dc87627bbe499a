#!/usr/bin/env python3
"""Benchmark of the renderer's per-frame hot path on B300.

One step = one frame of the headline workload: fire_bvh_refit (64 rigid
bodies moved by that frame's poses) + fire_render (7,299,072 triangles,
1920x1080, 4 spp, 2 lights).  Frame 0 (the LBVH build) is in the warm-up.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as independent replicas (the path has no exchange
step): each rank renders its own frames; the time is the max over ranks and
the value is the whole job's ms per frame.  Prints ONE JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenegen as sg  # noqa: E402

METRIC = "ms/frame & Grays/s at 7.3M tris 1080p 4spp; batched & backward vs plain"
UNIT = "ms/frame"


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def workload_config(w, nframes):
    cam = w.camera
    return {"workload": (f"frame7m: {w.scene.nt:,} triangles (1,400 icospheres of 5,120 + 256x256-cell "
                         f"terrain), 64 rigid bodies moved every frame, refit + render per frame, "
                         f"{cam.width}x{cam.height}, {cam.spp} spp rotated grid, {len(w.lights)} point lights"),
            "triangles": w.scene.nt, "width": cam.width, "height": cam.height, "spp": cam.spp,
            "lights": len(w.lights), "bodies": w.scene.nbody - 1, "frames": nframes,
            "l2": "inputs larger than L2: every refit rewrites 445 MB of 4-wide nodes + 350 MB of triangles",
            "parallelism": "replicas"}


# ----------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling during the timed region (read-only queries)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------- roofline
KERNEL_NAMES = {"refit": "k_refit_leaves+k_refit_tl+k_refit_top", "primary": "k_primary",
                "queue": "k_qsum+k_qperm", "shadow": "k_shadow", "resolve": "k_shade<resolve>"}


def render_tasks(width: int, height: int, spp: int) -> int:
    """Warp tasks of one image: 4 x 2 pixels at 4 spp, 8 x 4 at 1 spp."""
    tw, th = (4, 2) if spp == 4 else (8, 4)
    return -(-width // tw) * -(-height // th)


def algorithmic_bytes(nt: int, nv: int, n4: int, samples: int, pixels: int, shadow_rays: int,
                      queue_counts: int = 0):
    """Minimum bytes each kernel family must move per frame
    (queue_counts = lights x tasks):
    refit   -- read rest vertices (16 B) + body ids (2 B) per vertex, the
               sorted index record (16 B) and material (4 B) per triangle;
               write its 48-B record and its 24-B box, read the box back
               (its treelet); per 4-wide node read its 8-B list entry and
               16-B child slots and write its 96 B of boxes once
    primary -- read the traversal tree once (128 B per 4-wide node + 48 B
               per triangle) + write a 16-B record per sample, a 32-B
               queued shadow ray and a 4-B ray count per task and light
    queue   -- read the counts twice (block sums, then the scan) and write a
               4-B slot per shadow ray
    shadow  -- read the traversal tree once + each ray's 4-B slot, its 32-B
               queue entry, its 4-B skip id and a 4-B visibility update
    resolve -- read the 16-B record per sample + 32 B of its triangle for the
               hit frame + write a 16-B pixel."""
    tree = 128 * n4 + 48 * nt
    return {"refit": nv * 18 + nt * (16 + 4 + 48 + 24 + 24) + n4 * (8 + 16 + 96),
            "primary": tree + 16 * samples + 32 * shadow_rays + 4 * queue_counts,
            "queue": 8 * queue_counts + 4 * shadow_rays,
            "shadow": tree + 44 * shadow_rays,
            "resolve": 16 * samples + 32 * samples + 16 * pixels}


def committed_counter(kind: str, kernel: str):
    """Per-launch ncu counter of the current kernels from the committed
    summary: kind "dram_bytes" (dram__bytes_read.sum + dram__bytes_write.sum),
    "warp_inst" (smsp__inst_executed.sum) or "l2_bytes" (lts__t_bytes.sum);
    None if not captured."""
    p = os.path.join(ROOT, "profiles", "counters_frame7m.txt")
    if os.path.exists(p):
        lines = [l for l in open(p) if not l.startswith("#")]
        return json.loads("".join(lines)).get(kind, {}).get(kernel)
    return None


def l2_read_probe(fb, torch, sizes_mb=(24, 48, 80), reps=40):
    """L2 read bandwidth, measured the way the kernels are timed (CUDA events
    on the launching stream, after a warm-up launch): fire_probe_read over a
    buffer that fits in L2 (126 MB), `reps` reads per launch, best over the
    buffer sizes and 5 launches each.  GB/s of bytes read."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.zeros(4 * sms, dtype=torch.int32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    best, where = 0.0, None
    for mb in sizes_mb:
        buf = torch.ones(mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")
        fb.fire.probe_read(buf, reps, sink)
        for _ in range(5):
            e0.record(stream)
            fb.fire.probe_read(buf, reps, sink)
            e1.record(stream)
            torch.cuda.synchronize()
            gbs = buf.numel() * 4 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9
            if gbs > best:
                best, where = gbs, mb
        del buf
    return {"gbs": best, "buffer_mb": where, "reps": reps,
            "how": "fire_probe_read: (SMs x 4) blocks x 256 threads, 16-B ld.global.cg loads of an "
                   "L2-resident buffer, best of 5 launches per size, CUDA events"}


def camera_rays(cam, x, y, k):
    """Pinhole rays of samples (x, y, k) in float32, the render's camera
    formula (4 spp: the rotated grid); for traversal statistics only."""
    pos, tgt, up = (np.array(v, np.float64) for v in (cam.pos, cam.target, cam.up))
    f = tgt - pos
    f /= np.linalg.norm(f)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    f, r, u = (v.astype(np.float32) for v in (f, r, u))
    sy = np.float32(np.tan(np.float64(cam.vfov_deg) * np.pi / 360.0))
    sx = sy * np.float32(np.float32(cam.width) / np.float32(cam.height))
    if cam.spp == 4:
        ox = np.array([-0.125, 0.375, -0.375, 0.125], np.float32)[k]
        oy = np.array([-0.375, -0.125, 0.125, 0.375], np.float32)[k]
    else:
        ox = oy = np.zeros(len(k), np.float32)
    ndx = (np.float32(2) * (x.astype(np.float32) + (np.float32(0.5) + ox))) / np.float32(cam.width) - np.float32(1)
    ndy = np.float32(1) - (np.float32(2) * (y.astype(np.float32) + (np.float32(0.5) + oy))) / np.float32(cam.height)
    d = (ndx * sx)[:, None] * r + (ndy * sy)[:, None] * u + f
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    o = np.tile(np.array(cam.pos, np.float32), (len(d), 1))
    return o, d


def traversal_demand(G, cam, gb_host, nwarps=2048):
    """Node steps, triangle tests and warp demand per ray of the frame's
    primary and shadow passes, from the render kernels' traversal code run on
    the host (fire_debug_trace_stats) over `nwarps` warps of each pass spread
    evenly over it: a primary warp's task (4x2 pixels x 4 samples, or 8x4 x
    1), and 32 consecutive shadow rays of the dense queue of the last render
    (fire_debug_dump 12).  Demand bytes of a warp: distinct 4-wide nodes x
    128 B + distinct triangle records x 48 B."""
    spp = cam.spp
    tw, rows = (4, 2) if spp == 4 else (8, 4)
    tiles_x, tiles_y = -(-cam.width // tw), -(-cam.height // rows)
    tasks = np.unique(np.linspace(0, tiles_x * tiles_y - 1, nwarps).astype(np.int64))
    lane = np.arange(32)
    q = lane >> 2 if spp == 4 else lane
    k = lane & 3 if spp == 4 else np.zeros(32, np.int64)
    x = ((tasks % tiles_x)[:, None] * tw + (q % tw)[None, :]).ravel()
    y = ((tasks // tiles_x)[:, None] * rows + (q // tw)[None, :]).ravel()
    kk = np.tile(k, len(tasks))
    full = ((x < cam.width) & (y < cam.height)).reshape(-1, 32).all(1)  # tasks without idle lanes
    keep = np.repeat(full, 32)
    o, d = camera_rays(cam, x[keep], y[keep], kk[keep])
    out = {}
    prim = G.trace_stats(o, d, group=32, per_ray=True)
    q_rays = G.dump("shadow_rays")
    sid = q_rays[:, 7].view(np.int32) >> 3
    nq = len(q_rays) // 32
    starts = np.unique(np.linspace(0, max(nq - 1, 0), min(nwarps, max(nq, 1))).astype(np.int64)) * 32
    idx = (starts[:, None] + np.arange(32)[None, :]).ravel()
    idx = idx[idx < len(q_rays)]
    qs = q_rays[idx]
    shad = G.trace_stats(qs[:, 0:3], qs[:, 4:7], tmax=qs[:, 3], skip=gb_host[sid[idx], 0], any_hit=True, group=32,
                         per_ray=True)
    for name, st in (("primary", prim), ("shadow", shad)):
        n = max(st["rays"], 1)
        # node steps a warp runs (its longest ray) against its lanes' steps
        w = st["steps"][: len(st["steps"]) // 32 * 32].reshape(-1, 32)
        busy = float(w.sum() / max(32 * w.max(1).sum(), 1))
        out[name] = {"rays_sampled": st["rays"], "warps_sampled": st["groups"],
                     "node_steps_per_ray": st["node_steps"] / n, "tri_tests_per_ray": st["tri_tests"] / n,
                     "warp_distinct_nodes_per_ray": st["group_nodes"] / n,
                     "warp_distinct_tris_per_ray": st["group_tris"] / n,
                     "demand_bytes_per_ray": (128 * st["group_nodes"] + 48 * st["group_tris"]) / n,
                     "lanes_busy_by_length": busy,
                     "check": {"bad_loads": st["bad_loads"], "err": st["err"]}}
    return out


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ------------------------------------------------------------------ CPU baseline
def host_threads() -> int:
    """Host threads for the oracle's split runs: std::thread::hardware_concurrency()
    as Python sees it (os.cpu_count), limited to the cores this process may use."""
    n = os.cpu_count() or 1
    if hasattr(os, "sched_getaffinity"):
        n = min(n, len(os.sched_getaffinity(0)))
    return max(1, n)


def oracle_samples(S, cam, lights, ids, threads: int):
    """The oracle's sample renderer over `ids`, split into contiguous chunks
    over `threads` host threads (ctypes releases the GIL; the oracle's render
    only reads the scene)."""
    if threads <= 1:
        S.render_samples(cam, lights, ids, want_t2=False)
        return
    from concurrent.futures import ThreadPoolExecutor
    chunks = np.array_split(np.sort(ids), threads)
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda c: S.render_samples(cam, lights, c, want_t2=False), chunks))


def cpu_oracle_frame(S, w, xf_frame, nsamples: int, threads: int, seed: int = 7):
    """The oracle as it stands on the host (S: an oracle scene built at the
    first pose): one refit of the frame (timed, single-threaded: the
    oracle's refit is a serial post-order walk) plus a bounded random sample
    of the frame's samples (timed), scaled to a whole frame, on `threads`
    host threads."""
    t0 = time.perf_counter()
    S.update(xf_frame, rebuild=False)
    t_refit = time.perf_counter() - t0
    cam = w.camera
    n = cam.width * cam.height * cam.spp
    ids = np.random.default_rng(seed).choice(n, nsamples, replace=False)
    t0 = time.perf_counter()
    oracle_samples(S, cam, w.lights, ids, threads)
    t_samp = time.perf_counter() - t0
    ms = 1e3 * (t_refit + t_samp * n / nsamples)
    return ms, {"refit_s": t_refit, "sample_s": t_samp, "samples": nsamples, "threads": threads}


def reference_arm(args, rank, world):
    """--impl reference: the oracle timed on the host cores, rank 0 only."""
    if rank != 0:
        return
    w = sg.workload_frame7m()
    xf0 = w.motion.xforms()
    frames = [w.motion.step() for _ in range(args.warmup + args.steps)]
    import oracle
    S = oracle.OracleScene(w.scene)
    S.update(xf0, rebuild=True)
    cam = w.camera
    n = cam.width * cam.height * cam.spp
    threads = host_threads()
    per = max(200, args.ref_samples) * threads
    rng = np.random.default_rng(11)
    times = []
    for i, xf in enumerate(frames):
        t0 = time.perf_counter()
        S.update(xf, rebuild=False)
        t1 = time.perf_counter()
        ids = rng.choice(n, per, replace=False)
        oracle_samples(S, cam, w.lights, ids, threads)
        t2 = time.perf_counter()
        if i >= args.warmup:
            times.append(1e3 * ((t1 - t0) + (t2 - t1) * n / per))
    ms = float(np.mean(times))
    sample = (f"each step: oracle refit of the frame (one thread) + {per} random samples of its "
              f"{n:,} split over {threads} host threads, scaled to the frame")
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(w, args.steps),
            "cpu_baseline": {"value": ms, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------- side runs
def batch_ratio(fb, torch, reps=5):
    """Batched (three launches for the whole batch, one CUDA graph) vs the same 64 frames
    rendered by 64 fire_render calls; same images."""
    scenes, cams, cam_scene, lights = sg.batch16()
    G = []
    for sc in scenes:
        g = fb.Scene.from_numpy(sc)
        g.build(sc.identity_xforms())
        G.append(g)
    outs = [torch.zeros((c.height, c.width, 4), device="cuda") for c in cams]
    fb.render_batch(G, cams, cam_scene, lights, outs)  # autotune + capture
    cfg = fb.batch_last_config()
    tuning = fb.fire.batch_last_tuning()
    for _ in range(2):
        fb.render_batch(G, cams, cam_scene, lights, outs)
    seq = [torch.zeros_like(o) for o in outs]
    for c, si, o in zip(cams, cam_scene, seq):
        G[si].render(c, lights[si], out=o)
    same = all(torch.equal(a, b) for a, b in zip(outs, seq))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fb.render_batch(G, cams, cam_scene, lights, outs)
    e1.record()
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / reps
    e0.record()
    for _ in range(reps):
        for c, si, o in zip(cams, cam_scene, seq):
            G[si].render(c, lights[si], out=o)
    e1.record()
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / reps
    tris = [s.nt for s in scenes]
    return {"batched_ms": t_batch, "sequential_ms": t_seq, "ratio": t_seq / t_batch, "identical": bool(same),
            "cameras": len(cams), "scenes": len(scenes), "tris_min": min(tris), "tris_max": max(tris),
            "tuned": cfg, "tuning": tuning,
            "tuning_spread": tuning["worst_ms"] / tuning["best_ms"] if tuning["best_ms"] > 0 else None}


def two_level_compare(fb, torch, w, xf_build, xf_dev, ropts, single_seq):
    """The paper's two-level structure (a bottom level per body built once
    at rest, the top level rebuilt every frame) on the headline workload:
    serial stage times over 20 frames and the 99-frame sequence in the
    pipelined mode of the headline (top-level rebuild of frame i on its own
    stream while frame i-1 renders), beside the single-level refit's."""
    cam, lights = w.camera, w.lights
    G = fb.Scene.from_numpy(w.scene)
    G.set_two_level(True)
    stream = torch.cuda.current_stream()
    side = torch.cuda.Stream(priority=0)
    out = torch.zeros((cam.height, cam.width, 4), dtype=torch.float32, device="cuda")
    G.build(xf_build)
    G.profile(True)
    for i in range(5):
        G.refit(xf_dev[i])
        G.render(cam, lights, out=out)
    torch.cuda.synchronize()
    G.profile_read()
    for i in range(5, 25):
        G.refit(xf_dev[i])
        G.render(cam, lights, out=out)
    p = G.profile_read()
    G.profile(False)
    stages = {k: p[k][0] / 20 for k in ("primary", "queue", "shadow", "resolve")}
    G.build(xf_build)
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(100)]
    ends[0].record(stream)
    for i in range(99):
        G.refit(xf_dev[i], stream=side)
        G.render(cam, lights, out=out, opts=ropts)
        ends[i + 1].record(stream)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    assert G.sync_status() == 0
    seq = np.array([ends[i].elapsed_time(ends[i + 1]) for i in range(99)])
    G.destroy()
    return {"stages_ms": stages, "median_ms": float(np.median(seq)), "p95_ms": float(np.percentile(seq, 95)),
            "frames_5_24_ms": float(seq[4:24].mean()),
            "single_level_median_ms": single_seq["median_ms"], "single_level_p95_ms": single_seq["p95_ms"],
            "mode": "pipelined: top level of frame i rebuilt on its own stream while frame i-1 renders; no "
                    "per-frame triangle work"}


def frame_filling_view(fb, torch, G, w, xf_dev, first, reps=10):
    """The headline scene seen from (0, 4, 12) towards the origin, a view
    that geometry fills (the headline view keeps the whole scene in sight,
    so most of its rays miss): refit + render per frame on one stream,
    per-stage times, rays traced and Grays/s over the covered image."""
    cam = sg.Camera((0.0, 4.0, 12.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, w.camera.width, w.camera.height,
                    w.camera.spp)
    lights = w.lights
    out = torch.zeros((cam.height, cam.width, 4), dtype=torch.float32, device="cuda")
    gb = torch.zeros((cam.width * cam.height * cam.spp, 4), dtype=torch.int32, device="cuda")
    G.build(xf_dev[first - 1])  # a tree of the frames measured here (the sequences rebuilt it elsewhere)
    for i in range(3):
        G.refit(xf_dev[first + i])
        G.render(cam, lights, out=out)
    torch.cuda.synchronize()
    G.profile_read()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    for i in range(reps):
        G.refit(xf_dev[first + 3 + i])
        G.render(cam, lights, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    p = G.profile_read()
    G.render(cam, lights, out=out, gbuf=gb)
    vis = gb[:, 2].to(torch.int64)
    shadow = int(sum(((vis >> (8 + j)) & 1).sum().item() for j in range(len(lights))))
    hits = int((gb[:, 0] >= 0).sum().item())
    prim_rays = cam.width * cam.height * cam.spp
    st = {k: p[k][0] / reps for k in ("refit", "primary", "queue", "shadow", "resolve")}
    trace = st["primary"] + st["queue"] + st["shadow"] + st["resolve"]
    return {"camera": {"pos": list(cam.pos), "target": list(cam.target)}, "ms_per_frame_serial": e0.elapsed_time(e1) / reps,
            "stages_ms": st, "rays": {"primary": prim_rays, "shadow": shadow, "hit_samples": hits},
            "hit_fraction": hits / prim_rays, "grays_per_s": (prim_rays + shadow) / (trace * 1e-3) / 1e9}


def static_workloads(fb, torch):
    """The static workloads of the measurement plan: tiny41k (40,962
    triangles, 256^2, 1 spp, 1 light; 100 renders after 10 warm-up renders)
    and mid1m (1,155,072 triangles, 1280x720, 4 spp, 3 lights; build time
    reported separately, then 100 renders): median and p95 ms per render
    (CUDA events around each render), and the one-time build (GPU time of
    a second build, and wall clock of the first with its allocations)."""
    res = {}
    for name in ("tiny41k", "mid1m"):
        w = sg.WORKLOADS[name]()
        cam, lights = w.camera, w.lights
        G = fb.Scene.from_numpy(w.scene)
        xf = w.scene.identity_xforms()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.build(xf)
        torch.cuda.synchronize()
        first_build = (time.perf_counter() - t0) * 1e3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        e0.record(stream)
        G.build(xf)
        e1.record(stream)
        torch.cuda.synchronize()
        build = e0.elapsed_time(e1)
        out = torch.zeros((cam.height, cam.width, 4), dtype=torch.float32, device="cuda")
        for _ in range(10):
            G.render(cam, lights, out=out)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(100)]
        for a, b in evs:
            a.record(stream)
            G.render(cam, lights, out=out)
            b.record(stream)
        torch.cuda.synchronize()
        assert G.sync_status() == 0
        t = np.array([a.elapsed_time(b) for a, b in evs])
        res[name] = {"triangles": w.scene.nt, "image": f"{cam.width}x{cam.height}x{cam.spp}spp",
                     "lights": len(lights), "render_median_ms": float(np.median(t)),
                     "render_p95_ms": float(np.percentile(t, 95)), "build_ms": build,
                     "first_build_wall_ms": first_build,
                     "mrays_primary_per_s": cam.width * cam.height * cam.spp / (np.median(t) * 1e-3) / 1e6}
        G.destroy()
    return res


def backward_ratio(fb, torch, reps=20):
    """Backward of the shading stage vs its forward (512x512, 1 spp, 32
    materials, 2 lights, 499,712 triangles)."""
    w = sg.workload_grad500k()
    cam, lights = w.camera, w.lights
    G = fb.Scene.from_numpy(w.scene)
    G.build(w.scene.identity_xforms())
    gb = torch.zeros((cam.width * cam.height * cam.spp, 4), dtype=torch.int32, device="cuda")
    G.render(cam, lights, gbuf=gb)
    P = np.zeros((len(w.scene.mats), 5), np.float32)
    for i, m in enumerate(w.scene.mats):
        P[i, :3], P[i, 3], P[i, 4] = m["albedo"], m["roughness"], m["metallic"]
    params = torch.from_numpy(P).cuda()
    inten = torch.tensor([l.intensity for l in lights], dtype=torch.float32, device="cuda")
    dimg = torch.randn((cam.height, cam.width, 4), device="cuda")
    dP, dI = torch.zeros_like(params), torch.zeros_like(inten)
    G.profile(True)
    for _ in range(3):
        G.shade(gb, cam, lights, params, inten)
        G.shade_backward(gb, cam, lights, params, inten, dimg, dP, dI)
    G.profile_read()
    out = torch.zeros((cam.height, cam.width, 4), device="cuda")
    for _ in range(reps):
        G.shade(gb, cam, lights, params, inten, out=out)
        G.shade_backward(gb, cam, lights, params, inten, dimg, dP, dI)
    p = G.profile_read()
    fwd = p["shade_gbuf"][0] / max(1, p["shade_gbuf"][1])
    bwd = p["backward"][0] / max(1, p["backward"][1])
    return {"forward_shade_ms": fwd, "backward_ms": bwd, "ratio": bwd / fwd, "pixels": cam.width * cam.height}


# --------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-samples", type=int, default=40000,
                    help="oracle samples per host thread for the CPU baseline")
    ap.add_argument("--ref-samples", type=int, default=4000,
                    help="oracle samples per host thread per reference step")
    ap.add_argument("--no-side", action="store_true", help="skip the batched and backward side runs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline (profiling runs)")
    ap.add_argument("--render-bps", type=int, default=7,
                    help="blocks per SM of the primary pass in the pipelined frames (0 = occupancy limit; 7 leaves room for the next frame's refit blocks beside it)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank, local_rank, world = env_rank()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    import paper_2410_05095_b300 as fb
    from paper_2410_05095_b300 import _build
    from paper_2410_05095_b300.replicas import max_over_ranks
    _build.build()
    torch.cuda.set_device(local_rank)
    # the render runs on a high-priority stream and the refit of the next
    # frame on a normal one: when a render kernel ends, the next render
    # kernel's blocks go first, and the refit fills the room the render
    # leaves (pipelined frame7m: 2.43 ms against 2.47 with the priorities
    # the other way round)
    torch.cuda.set_stream(torch.cuda.Stream(priority=-1))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    w = sg.workload_frame7m()
    K, W = args.steps, args.warmup
    xf_build = w.motion.xforms()
    frames = np.stack([w.motion.step() for _ in range(max(W + 2 * K, 99))])
    cam, lights = w.camera, w.lights
    G = fb.Scene.from_numpy(w.scene)
    xf_dev = torch.from_numpy(frames).cuda()
    xf_pinned = torch.from_numpy(frames).pin_memory()
    torch.cuda.synchronize()
    t_build = time.perf_counter()
    G.build(xf_build)
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t_build) * 1e3  # wall clock: the collapse synchronises per depth
    out = torch.zeros((cam.height, cam.width, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    G.profile(True)
    for i in range(W):
        G.refit(xf_dev[i])
        G.render(cam, lights, out=out)
    torch.cuda.synchronize()
    build_stats = G.profile_read()
    assert G.sync_status() == 0

    # --- timed region: K frames, inputs resident in HBM -----------------------------
    # Frames are pipelined as the library allows: the refit of frame i runs on
    # its own stream into the second frame buffer while frame i-1 renders
    # (the paper's async compute queue, §IV-B-3); the render of frame i waits
    # for its refit.  The serial order (refit, render, refit, ...) on one
    # stream is timed as well, and gives the per-stage split.
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    refit_stream = torch.cuda.Stream(priority=0)  # below the render stream's priority
    ropts = fb.fire.make_opts(blocks_per_sm=args.render_bps) if args.render_bps > 0 else None

    def timed_frames(first, pipelined):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(K):
            if pipelined:
                G.refit(xf_dev[first + i], stream=refit_stream)
                G.render(cam, lights, out=out, opts=ropts)
            else:
                G.refit(xf_dev[first + i])
                G.render(cam, lights, out=out)
        stream.wait_stream(refit_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return e0.elapsed_time(e1)

    with Clocks(local_rank) as clk:
        t_serial = timed_frames(W, False)
        stages = G.profile_read()
        # the pipelined frames as a caller runs them: stage events off (the
        # serial loop above launched the same kernels, K frames of them)
        G.profile(False)
        for i in range(W):  # warm the pipelined order
            G.refit(xf_dev[i], stream=refit_stream)
            G.render(cam, lights, out=out, opts=ropts)
        torch.cuda.synchronize()
        t_ms = timed_frames(W, True)  # the same poses as the serial loop
    primary_info = G.render_info()
    launches = sum(n for (_, n) in stages.values())
    assert G.sync_status() == 0
    t_ms = max_over_ranks(t_ms, device="cuda")
    t_serial = max_over_ranks(t_serial, device="cuda")
    ms_frame_rank = t_ms / K
    value = t_ms / (K * world)

    # --- end to end through the public API with host buffers ----------------------
    # Every frame: host poses -> refit -> render -> image to pinned host memory,
    # pipelined like the timed loop: the refit (host poses, own stream) of
    # frame i overlaps the render of frame i-1, and with two output buffers the
    # image of frame i is copied on a third stream while frame i+1 renders
    # (events order the reuse of each buffer).
    host_img = [torch.empty((cam.height, cam.width, 4), dtype=torch.float32).pin_memory() for _ in range(2)]
    outs = [out, torch.zeros_like(out)]
    copy_stream = torch.cuda.Stream()
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]

    def e2e_frame(i, xf_host):
        b = i % 2
        stream.wait_event(copied[b])          # the copy of frame i-2 has left buffer b
        G.refit(xf_host, stream=refit_stream)
        G.render(cam, lights, out=outs[b], opts=ropts)
        rendered[b].record(stream)
        copy_stream.wait_event(rendered[b])
        with torch.cuda.stream(copy_stream):
            host_img[b].copy_(outs[b], non_blocking=True)
        copied[b].record(copy_stream)

    for i in range(W):  # warm the host path (pinned buffers, copy engines)
        e2e_frame(i, xf_pinned[i].numpy())
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0.record(stream)
    t0 = time.perf_counter()
    for i in range(K):
        e2e_frame(i, xf_pinned[W + K + i].numpy())
    stream.wait_stream(copy_stream)
    stream.wait_stream(refit_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t0))
    t_e2e = max_over_ranks(t_e2e, device="cuda")
    G.profile(True)  # stage events again for the side measurements below
    G.profile_read()
    e2e = {"value": t_e2e / (K * world), "unit": UNIT, "h2d_bytes_per_step": int(frames[0].nbytes),
           "d2h_bytes_per_step": int(host_img[0].numel() * 4), "host_pinned": bool(host_img[0].is_pinned()),
           "pipelining": "refit of frame i (own stream) overlaps the render of frame i-1; the image copy of "
                         "frame i (third stream, two output buffers) overlaps frame i+1"}
    host_img = host_img[0]
    # where the end-to-end time goes (a separate, untimed pass of 3 frames)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    parts = np.zeros(3)
    for i in range(3):
        ev[0].record(stream)
        G.refit(xf_pinned[W + i].numpy())
        ev[1].record(stream)
        G.render(cam, lights, out=out)
        ev[2].record(stream)
        host_img.copy_(out, non_blocking=True)
        ev[3].record(stream)
        torch.cuda.synchronize()
        parts += [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])]
    e2e["breakdown_ms"] = dict(zip(["refit_from_host", "render", "d2h_image"], (parts / 3).tolist()))
    G.profile_read()

    # --- the 100-frame sequence of the workload: build at frame 0, refit 1..99 --------
    # In the headline's mode (pipelined, refit only): a frame's time is the
    # interval between the ends of consecutive renders on the render stream,
    # so the median and p95 cover the tree's decay under motion over the
    # whole sequence, not only the first frames after the build.
    G.build(xf_build)
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(100)]
    ends[0].record(stream)
    for i in range(99):
        G.refit(xf_dev[i], stream=refit_stream)
        G.render(cam, lights, out=out, opts=ropts)
        ends[i + 1].record(stream)
    stream.wait_stream(refit_stream)
    torch.cuda.synchronize()
    seqp = np.array([ends[i].elapsed_time(ends[i + 1]) for i in range(99)])
    G.profile_read()

    def seq_summary(x):
        return {"median_ms": float(np.median(x)), "p95_ms": float(np.percentile(x, 95)), "mean_ms": float(x.mean()),
                "first_ms": float(x[0]), "last_ms": float(x[-1])}

    sequence = {"frames": 99, "mode": "pipelined, refit only (the mode of the headline value)", **seq_summary(seqp),
                "by_decile_ms": [float(np.median(c)) for c in np.array_split(seqp, 10)],
                "note": "frame time = interval between the ends of consecutive renders; refit + render per "
                        "frame after a build at frame 0 (tree quality decays with motion)"}
    # the same frames serially on one stream (refit, render, refit, ...)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(99)]
    G.build(xf_build)
    for i in range(99):
        evs[i][0].record(stream)
        G.refit(xf_dev[i])
        G.render(cam, lights, out=out)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    seq = np.array([a.elapsed_time(b) for a, b in evs])
    G.profile_read()
    sequence["serial"] = seq_summary(seq)
    # serial, with a full rebuild (fire_bvh_build) in place of the refit every
    # 25th frame: the rebuild frames cost more, the others stay near the
    # frame-1 quality
    G.build(xf_build)
    for i in range(99):
        evs[i][0].record(stream)
        if (i + 1) % 25 == 0:
            G.build(xf_dev[i])
        else:
            G.refit(xf_dev[i])
        G.render(cam, lights, out=out)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    seq2 = np.array([a.elapsed_time(b) for a, b in evs])
    G.profile_read()
    sequence["serial_rebuild_every_25"] = {**seq_summary(seq2),
                                           "rebuild_frames_ms": [float(seq2[i]) for i in range(24, 99, 25)]}

    # --- the same scene from a view that geometry fills (second reported line) -------
    filling = frame_filling_view(fb, torch, G, w, xf_dev, W)

    # --- rays traced per frame (shadow rays counted from the G-buffer) ------------
    gb = torch.zeros((cam.width * cam.height * cam.spp, 4), dtype=torch.int32, device="cuda")
    G.render(cam, lights, out=out, gbuf=gb)
    vis = gb[:, 2].to(torch.int64)
    shadow_rays = int(sum(((vis >> (8 + j)) & 1).sum().item() for j in range(len(lights))))
    primary_rays = cam.width * cam.height * cam.spp
    hits = int((gb[:, 0] >= 0).sum().item())
    # traversal work and warp demand of this frame (host run of the kernels' traversal code)
    demand = None
    if rank == 0:
        try:
            demand = traversal_demand(G, cam, gb.cpu().numpy())
        except Exception as e:  # a measurement aid: never costs the bench line
            demand = {"error": f"{type(e).__name__}: {e}"}
    del gb

    avg = {k: stages[k][0] / K for k in ("refit", "primary", "queue", "shadow", "resolve")}  # one of each per frame
    trace_ms = avg["primary"] + avg["queue"] + avg["shadow"] + avg["resolve"]
    grays = (primary_rays + shadow_rays) / (trace_ms * 1e-3) / 1e9
    grays_frame = (primary_rays + shadow_rays) / (ms_frame_rank * 1e-3) / 1e9
    alg = algorithmic_bytes(w.scene.nt, w.scene.nv, G.info()["n4"], primary_rays, cam.width * cam.height,
                            shadow_rays, len(lights) * render_tasks(cam.width, cam.height, cam.spp))
    dom = max(avg, key=avg.get)
    peak, peak_kind = load_peaks()
    achieved = alg[dom] / (avg[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": KERNEL_NAMES[dom], "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": committed_counter("dram_bytes", dom),
                "peak_source": f"{peak_kind} hbm_gbs (of measured)" if peak_kind == "measured" else "fallback",
                "algorithmic_bytes": alg[dom],
                "all_kernels": {k: {"ms": avg[k], "algorithmic_bytes": alg[k],
                                    "gbs": alg[k] / (avg[k] * 1e-3) / 1e9 if avg[k] > 0 else None}
                                for k in avg}}
    # the traversal kernels reuse the tree through L1 and L2: their L2 traffic
    # (ncu lts__t_bytes.sum per launch) over the live launch time, against the
    # L2 read bandwidth measured here with the same kind of timing
    l2b = committed_counter("l2_bytes", dom)
    if l2b:
        probe = l2_read_probe(fb, torch)
        got = l2b / (avg[dom] * 1e-3) / 1e9
        roofline["l2"] = {"bytes_per_launch": l2b, "achieved": got, "peak": probe["gbs"], "unit": "GB/s",
                          "frac": got / probe["gbs"], "peak_source": probe["how"],
                          "peak_buffer_mb": probe["buffer_mb"]}
    # demand traffic of the traversal kernels: per warp, each distinct node and
    # triangle record fetched once (what the warp asks of L2 if L1 kept
    # nothing between warps), scaled to the frame's rays, over the live time
    if demand is not None and "error" in demand:
        roofline["demand"] = demand
    elif demand is not None:
        probe_gbs = roofline.get("l2", {}).get("peak") or l2_read_probe(fb, torch)["gbs"]
        for name, rays in (("primary", primary_rays), ("shadow", shadow_rays)):
            dm = demand[name]
            dm["demand_bytes_per_launch"] = dm["demand_bytes_per_ray"] * rays
            dm["achieved_gbs"] = dm["demand_bytes_per_launch"] / (avg[name] * 1e-3) / 1e9
            dm["l2_frac"] = dm["achieved_gbs"] / probe_gbs
            dm["hbm_frac"] = dm["achieved_gbs"] / peak
        roofline["demand"] = {**demand, "l2_peak_gbs": probe_gbs,
                              "bytes": "per warp: distinct 4-wide nodes x 128 B + distinct triangle records x 48 B",
                              "sample": "2048 warps of each pass spread evenly over the frame (a primary task of "
                                        "32 samples; 32 consecutive rays of the shadow queue in the shadow pass's "
                                        "order); the render kernels' traversal code run on the host over copies "
                                        "of the frame's tree (fire_debug_trace_stats)"}
    # the traversal kernels are issue-bound: warp instructions per launch (ncu)
    # over the live launch time, against 4 schedulers x 1 warp-inst/clock per SM
    clocks = clk.summary()
    inst = committed_counter("warp_inst", dom)
    if inst:
        mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2032.0
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        peak_gi = sms * 4 * float(mhz) * 1e6 / 1e9
        got_gi = inst / (avg[dom] * 1e-3) / 1e9
        roofline["issue"] = {"warp_inst_per_launch": inst, "achieved": got_gi, "peak": peak_gi,
                             "unit": "G warp-inst/s", "frac": got_gi / peak_gi,
                             "peak_source": f"{sms} SMs x 4 schedulers x {float(mhz):.0f} MHz (median under load)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_frame_rank, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded icospheres + value-noise terrain, random rigid motion)",
            "config": workload_config(w, K), "gpu_launches": int(launches),
            "grays_per_s": grays, "grays_per_s_frame": grays_frame,
            "samples_per_s": primary_rays / (ms_frame_rank * 1e-3),
            "rays_per_frame": {"primary": primary_rays, "shadow": shadow_rays, "hit_samples": hits},
            "stages_ms": {**avg, "build_once": build_ms},
            "serial_ms_per_frame": t_serial / K,
            "frame_loop": "pipelined: refit of frame i (own stream, second frame buffer) overlaps the render of "
                          "frame i-1; stages_ms from the serial loop",
            "primary_pass": {"method": "raster" if primary_info["raster"] else "traversal",
                             "fallback_bits": primary_info["fallback"], "pieces": primary_info["pieces"]},
            "roofline": roofline, "clocks": clocks, "e2e": e2e, "sequence_100": sequence,
            "frame_filling_view": filling,
            # the paper's own timings (§V-A, Table I), context only: another GPU
            # (RTX 4090), a rasterised main pass with RT-core shadow queries, and
            # no stated resolution, sample count or light count
            "paper_context": {"frame_ms": "within 2", "frame_what": "total GPU time per frame (TLAS build, "
                              "rasterised main pass, post-processing, UI), scenes duplicated past 7M triangles",
                              "main_pass_ms": {"scene1_223k_tris": 0.55, "scene2_550k_tris": 0.56},
                              "hardware": "RTX 4090 (Vulkan)", "comparable": False}}

    if rank == 0 and not args.no_side:
        line["batched"] = batch_ratio(fb, torch)
        line["backward"] = backward_ratio(fb, torch)
        line["two_level"] = two_level_compare(fb, torch, w, xf_build, xf_dev, ropts, sequence)
        line["static_workloads"] = static_workloads(fb, torch)
    if rank == 0 and not args.no_cpu:
        import oracle
        threads = host_threads()
        S = oracle.OracleScene(w.scene)
        S.update(xf_build, rebuild=True)
        ms_mt, info = cpu_oracle_frame(S, w, frames[0], args.cpu_samples * threads, threads)
        ms_1, info1 = cpu_oracle_frame(S, w, frames[1], args.cpu_samples, 1)
        line["cpu_baseline"] = {"value": ms_mt, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": (f"oracle refit of one frame (one thread) + {info['samples']} random "
                                           f"samples of its {primary_rays:,} split over {threads} host threads "
                                           f"(hardware_concurrency), scaled to the frame"),
                                "single_thread": {"value": ms_1, "unit": UNIT, "cores": 1,
                                                  "sample": f"the same with {info1['samples']} samples on one thread"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
