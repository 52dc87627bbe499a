"""The raster primary pass against the traversal primary pass: both compute
the nearest hit of every sample with the same ray-triangle test and the
same (t, original index) tie-break, so images and G-buffers must be equal
bit for bit -- across cameras outside, inside and grazing the scene, both
sample counts, row bands, the fallback cases and the headline frame after
motion.  The raster path itself is checked against the oracle by the
agreement rule for hits and visibility and 1e-4 radiance."""
import numpy as np
import pytest

import scenegen as sg
from gpu_common import (assert_radiance_close, build_pair, compare_samples, gbuf_of, pixel_ok_mask, torch_cuda,
                        THREADS)

pytestmark = pytest.mark.gpu

TRACE, RASTER = 2, 4


@pytest.fixture(scope="module")
def fb():
    import paper_2410_05095_b300 as fb
    torch_cuda()
    return fb


def _gpu_scene(scene, xf=None):
    import paper_2410_05095_b300 as fb
    G = fb.Scene.from_numpy(scene)
    G.build(scene.identity_xforms() if xf is None else xf)
    return G


def _pair(fb, G, cam, lights, **opts):
    """(image, gbuf) by traversal and by raster, plus the raster render's info."""
    torch = torch_cuda()
    res = []
    info = None
    for flags in (TRACE, RASTER):
        gb = torch.zeros((cam.width * cam.height * cam.spp, 4), dtype=torch.int32, device="cuda")
        out = torch.zeros((cam.height, cam.width, 4), dtype=torch.float32, device="cuda")
        G.render(cam, lights, out=out, gbuf=gb, opts=fb.fire.make_opts(flags=flags, **opts))
        assert G.sync_status() == 0
        info = G.render_info()
        assert info["raster"] == (flags == RASTER)
        res.append((out, gb))
    return res[0], res[1], info


def _same(tg, rg, cam):
    """Equal G-buffers, else a message naming the differing samples."""
    torch = torch_cuda()
    if torch.equal(tg, rg):
        return True
    d = (tg != rg).any(1).nonzero().flatten()[:8].tolist()
    rows = [(i, tg[i].tolist(), rg[i].tolist()) for i in d]
    raise AssertionError(f"{int((tg != rg).any(1).sum())} samples differ for {cam}: {rows}")


def _cameras(W, H, spp):
    rng = sg.Rng(4242)
    cams = [sg.orbit_camera(rng, W, H, spp, radius=r) for r in (3.0, 6.0, 9.0, 14.0, 25.0, 60.0)]
    cams += [sg.Camera((0.5, 0.3, 0.5), (5.0, 0.2, -3.0), (0.0, 1.0, 0.0), 75.0, W, H, spp),  # inside, low
             sg.Camera((0.0, 0.05, 14.0), (0.0, 0.05, 0.0), (0.0, 1.0, 0.0), 60.0, W, H, spp),  # grazing ground
             sg.Camera((0.0, 30.0, 0.01), (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), 20.0, W, H, spp),  # top down, narrow
             sg.Camera((-14.0, 2.0, -14.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 120.0, W, H, spp)]  # wide
    return cams


@pytest.mark.parametrize("spp", [1, 4])
def test_raster_equals_traversal_tiny(fb, spp):
    w = sg.workload_tiny41k()
    G = _gpu_scene(w.scene)
    for cam in _cameras(97, 61, spp):
        (ti, tg), (ri, rg), info = _pair(fb, G, cam, w.lights)
        assert info["fallback"] == 0, cam
        assert _same(tg, rg, cam)
        assert torch_cuda().equal(ti, ri), cam


def test_raster_equals_traversal_mid(fb):
    w = sg.workload_mid1m(320, 180, 4)
    G = _gpu_scene(w.scene)
    for cam in [w.camera] + _cameras(320, 180, 4)[::3]:
        (ti, tg), (ri, rg), info = _pair(fb, G, cam, w.lights)
        assert info["fallback"] == 0
        assert _same(tg, rg, cam)
        assert torch_cuda().equal(ti, ri)


def test_raster_against_oracle(fb):
    """The raster path alone against the oracle (agreement rule, radiance)."""
    torch = torch_cuda()
    w = sg.workload_tiny41k()
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 128, 96, 4)
    G, S = build_pair(w.scene)
    gb = torch.zeros((cam.width * cam.height * cam.spp, 4), dtype=torch.int32, device="cuda")
    img = G.render(cam, w.lights, gbuf=gb, opts=fb.fire.make_opts(flags=RASTER)).cpu().numpy()
    assert G.render_info()["raster"]
    g = gbuf_of(gb)
    ref = S.render_all_samples(cam, w.lights, threads=THREADS)
    _, bad = compare_samples(g, ref)
    assert np.array_equal(g["t"][~bad], ref["t"][~bad])
    ok = pixel_ok_mask(bad, cam.width, cam.height, 4)
    assert_radiance_close(img, S.render_image(cam, w.lights, threads=THREADS), ok)


def test_raster_row_bands(fb):
    torch = torch_cuda()
    w = sg.workload_tiny41k()
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 96, 61, 4)
    G = _gpu_scene(w.scene)
    full = G.render(cam, w.lights, opts=fb.fire.make_opts(flags=TRACE))
    part = torch.full_like(full, -1.0)
    G.render(cam, w.lights, out=part, opts=fb.fire.make_opts(row_begin=0, row_end=29, flags=RASTER))
    G.render(cam, w.lights, out=part, opts=fb.fire.make_opts(row_begin=29, row_end=61, flags=RASTER))
    assert torch.equal(full, part)


def test_raster_fallback_cases(fb):
    """Geometry touching the camera (a camera on the ground plane) makes the
    raster pass hand the frame to traversal: same result, reason bit 1."""
    w = sg.workload_tiny41k()
    G = _gpu_scene(w.scene)
    cam = sg.Camera((3.0, 0.0, 14.0), (0.0, 1.0, 0.0), (0.0, 1.0, 0.0), 60.0, 64, 48, 4)
    (ti, tg), (ri, rg), info = _pair(fb, G, cam, w.lights)
    assert info["fallback"] & 1
    assert _same(tg, rg, cam) and torch_cuda().equal(ti, ri)


def test_raster_default_choice(fb):
    """Default: traversal; the raster pass only when asked for."""
    w = sg.workload_mid1m(640, 480, 1)
    G = _gpu_scene(w.scene)
    G.render(w.camera, w.lights)
    assert not G.render_info()["raster"]
    G.render(w.camera, w.lights, opts=fb.fire.make_opts(flags=RASTER))
    assert G.render_info()["raster"]


def test_raster_frame7m_after_motion(fb):
    """The headline frame (7.3M triangles, 1920x1080, 4 spp) after 3 refit
    frames: raster and traversal agree bit for bit."""
    w = sg.workload_frame7m()
    G = _gpu_scene(w.scene, w.motion.xforms())
    for _ in range(3):
        G.refit(w.motion.step())
    (ti, tg), (ri, rg), info = _pair(fb, G, w.camera, w.lights)
    assert info["fallback"] == 0 and info["pieces"] > 0
    assert _same(tg, rg, w.camera)
    assert torch_cuda().equal(ti, ri)
