"""Host-side logic of the benchmark (no GPU): the clock-sample summary that
decides whether a run is kept, the algorithmic-byte model behind the
roofline, and the committed ncu counters it reads."""
import json
import os

import numpy as np

import bench
import scenegen as sg


def _clocks_from(lines):
    c = bench.Clocks(0)
    fd, c.path = bench.tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    return c.summary()


def test_clock_summary_median_under_load_and_reasons():
    # index, sm, max sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    rows = ["0, 345, 2032, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # idle: dropped
            "0, 2032, 2032, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2032, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2032, 2032, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    s = _clocks_from(rows)
    assert s["sm_mhz"] == 2032.0 and s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4


def test_clock_summary_reports_throttling():
    rows = ["0, 1500, 2032, 700.0, 0x40, Not Active, Active, Not Active, Not Active"] * 3
    s = _clocks_from(rows)
    assert s["reasons"] == ["hw_thermal_slowdown"] and s["sm_mhz"] == 1500.0


def test_clock_summary_without_samples():
    assert _clocks_from([""])["reasons"] == ["no samples"]


def test_algorithmic_bytes_model():
    nt, nv, n4, samples, pixels, rays, counts = 1000, 600, 400, 80, 20, 30, 6
    b = bench.algorithmic_bytes(nt, nv, n4, samples, pixels, rays, counts)
    tree = 128 * n4 + 48 * nt
    assert b["shadow"] == tree + 44 * rays
    assert b["primary"] == tree + 16 * samples + 32 * rays + 4 * counts
    assert b["queue"] == 8 * counts + 4 * rays
    assert b["resolve"] == 48 * samples + 16 * pixels
    assert b["refit"] == 18 * nv + 116 * nt + 120 * n4
    # the headline frame: 7,299,072 triangles, 3,652,849 vertices
    full = bench.algorithmic_bytes(7_299_072, 3_652_849, 3_476_669, 8_294_400, 2_073_600, 3_842_521)
    assert 0.9e9 < full["shadow"] < 1.0e9
    # 4 x 2-pixel tasks at 4 spp, 8 x 4 at 1 spp, ragged edges rounded up
    assert bench.render_tasks(1920, 1080, 4) == 480 * 540
    assert bench.render_tasks(5, 3, 4) == 2 * 2 and bench.render_tasks(9, 5, 1) == 2 * 2


def test_committed_counters_are_per_launch_integers():
    for kernel in ("shadow", "primary", "resolve"):
        v = bench.committed_counter("dram_bytes", kernel)
        w = bench.committed_counter("warp_inst", kernel)
        assert isinstance(v, int) and 1e7 < v < 2e9
        assert isinstance(w, int) and 1e7 < w < 2e9
    assert bench.committed_counter("dram_bytes", "refit") is None
    assert bench.committed_counter("dram_bytes", "no such kernel") is None


def test_workload_config_names_the_headline_frame():
    import scenegen as sg
    w = sg.workload_frame7m(nspheres=4, cells=4)   # small stand-in: the fields, not the sizes
    cfg = bench.workload_config(w, 20)
    assert cfg["workload"].startswith("frame7m") and cfg["frames"] == 20
    assert cfg["parallelism"] == "replicas" and "L2" in cfg["l2"]
    json.dumps(cfg)


def test_host_threads_and_split_sample():
    """The CPU baseline's thread count is the cores this process may use, and
    the split oracle run covers every requested sample once (chunks are
    contiguous in sorted order)."""
    n = bench.host_threads()
    assert 1 <= n <= (os.cpu_count() or 1)
    seen = []

    class FakeScene:
        def render_samples(self, cam, lights, ids, want_t2=False):
            seen.append(list(ids))

    import numpy as np
    ids = np.random.default_rng(0).choice(1000, 97, replace=False)
    bench.oracle_samples(FakeScene(), None, [], ids, 4)
    assert sorted(sum(seen, [])) == sorted(ids.tolist()) and len(seen) == 4
    seen.clear()
    bench.oracle_samples(FakeScene(), None, [], ids, 1)
    assert seen == [list(ids)]


def test_demand_sample_rays_are_the_render_camera():
    """The rays bench.py replays for the warp-demand count (its float32
    pinhole camera with the 4-spp rotated grid) are the oracle's camera rays
    to a few ulp, so the sampled warps trace the render's rays."""
    import oracle
    w = sg.workload_frame7m(nspheres=4, cells=8)
    for spp in (1, 4):
        cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 37, 23, spp)
        rng = np.random.default_rng(spp)
        x, y = rng.integers(0, cam.width, 200), rng.integers(0, cam.height, 200)
        k = rng.integers(0, spp, 200)
        o, d = bench.camera_rays(cam, x, y, k)
        for i in range(len(x)):
            ro, rd = oracle.camera_ray(cam, int(x[i]), int(y[i]), int(k[i]))
            assert np.allclose(o[i], ro, rtol=0, atol=0)
            assert np.allclose(d[i], rd, rtol=0, atol=4e-7)
