"""Smooth shading normals and sRGB albedo on the GPU (§IV-A-1 vertex normals
and colour decode) against the oracle: hits and visibility by the agreement
rule, t exact, radiance within 1e-4, under rigid motion and refits, through
the pipelined (double-buffered), batched, G-buffer shading and backward
paths; switching the normals off restores the flat image bit for bit."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from gpu_common import (assert_radiance_close, build_pair, compare_samples, gbuf_of, pixel_ok_mask, torch_cuda,
                        THREADS)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fb():
    import paper_2410_05095_b300 as fb
    torch_cuda()
    return fb


def _render(G, cam, lights):
    torch = torch_cuda()
    gb = torch.zeros((cam.width * cam.height * cam.spp, 4), dtype=torch.int32, device="cuda")
    img = G.render(cam, lights, gbuf=gb)
    assert G.sync_status() == 0
    return img.cpu().numpy(), gbuf_of(gb), gb


def _check(G, S, cam, lights):
    img, g, gb = _render(G, cam, lights)
    ref = S.render_all_samples(cam, lights, threads=THREADS)
    _, bad = compare_samples(g, ref)
    assert np.array_equal(g["t"][~bad], ref["t"][~bad])
    ok = pixel_ok_mask(bad, cam.width, cam.height, cam.spp)
    assert_radiance_close(img, S.render_image(cam, lights, threads=THREADS), ok)
    return img, g, gb


def _small():
    w = sg.workload_frame7m(nspheres=40, cells=16)
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 96, 64, 4)
    return w, cam


def test_smooth_tiny_matches_oracle(fb):
    w = sg.workload_tiny41k()
    cam = sg.Camera((0.0, 4.0, 12.0), (0, 0, 0), (0, 1, 0), 60.0, 96, 64, 4)
    lights = sg.LIGHTS_MAIN[:2]
    G, S = build_pair(w.scene)
    flat, _, _ = _render(G, cam, lights)
    nrm = sg.vertex_normals(w.scene)
    G.set_normals(nrm)
    S.set_normals(nrm)
    img, g, _ = _check(G, S, cam, lights)
    assert (g["prim"] >= 0).mean() > 0.3
    assert not np.array_equal(img, flat)          # the normals were used
    G.set_normals(None)                            # back to flat, bit for bit
    again, _, _ = _render(G, cam, lights)
    assert np.array_equal(again, flat)


def test_smooth_under_motion_matches_oracle(fb):
    """Bodies rotate every frame: the normals turn with the frame's body
    matrices (refit keeps them per frame buffer)."""
    w, cam = _small()
    sc = w.scene
    xf0 = w.motion.xforms()
    G, S = build_pair(sc, xf0)
    nrm = sg.vertex_normals(sc)
    G.set_normals(nrm)
    S.set_normals(nrm)
    for _ in range(3):
        xf = w.motion.step()
        G.refit(xf)
        S.update(xf, rebuild=False)
        _check(G, S, cam, w.lights)


def test_smooth_pipelined_frames_equal_serial(fb):
    torch = torch_cuda()
    w, cam = _small()
    xf0 = w.motion.xforms()
    poses = [w.motion.step() for _ in range(5)]
    nrm = sg.vertex_normals(w.scene)
    G1, G2 = fb.Scene.from_numpy(w.scene), fb.Scene.from_numpy(w.scene)
    for G in (G1, G2):
        G.build(xf0)
        G.set_normals(nrm)
    serial = []
    for xf in poses:
        G1.refit(xf)
        serial.append(G1.render(cam, w.lights).clone())
    outs = [torch.zeros_like(serial[0]) for _ in poses]
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    for i, xf in enumerate(poses):
        G2.refit(xf, stream=side)
        G2.render(cam, w.lights, out=outs[i])
    torch.cuda.synchronize()
    assert G2.sync_status() == 0
    for a, b in zip(serial, outs):
        assert torch.equal(a, b)


def test_smooth_batch_equals_sequential(fb):
    torch = torch_cuda()
    rng = sg.Rng(77)
    G = []
    for s in range(2):
        sc = sg.scene_icospheres_terrain(rng, 4 + 3 * s, 16, 8)
        g = fb.Scene.from_numpy(sc)
        g.build(sc.identity_xforms())
        if s == 0:
            g.set_normals(sg.vertex_normals(sc))   # one smooth, one flat scene
        G.append(g)
    cams = [sg.orbit_camera(rng, 48, 32, 4), sg.orbit_camera(rng, 40, 24, 1), sg.orbit_camera(rng, 33, 17, 4)]
    cam_scene = [0, 1, 0]
    lights = [sg.LIGHTS_MAIN[:2], sg.LIGHTS_MAIN[:1]]
    outs = [torch.zeros((c.height, c.width, 4), device="cuda") for c in cams]
    fb.render_batch(G, cams, cam_scene, lights, outs)
    for c, si, o in zip(cams, cam_scene, outs):
        assert torch.equal(o, G[si].render(c, lights[si]))


def test_smooth_shade_and_backward(fb):
    """fire_shade from the G-buffer equals the render; the backward kernel
    matches the oracle's FP64 analytic gradient with smooth normals."""
    torch = torch_cuda()
    w = sg.workload_grad500k(96, 96)
    cam, lights = w.camera, w.lights
    G, S = build_pair(w.scene)
    nrm = sg.vertex_normals(w.scene)
    G.set_normals(nrm)
    S.set_normals(nrm)
    img, g, gb = _render(G, cam, lights)
    ref = S.render_all_samples(cam, lights, threads=THREADS)
    _, bad = compare_samples(g, ref)
    P0 = oracle.params_of(w.scene.mats)
    I0 = np.array([l.intensity for l in lights], np.float64)
    params = torch.from_numpy(P0.astype(np.float32)).cuda()
    inten = torch.from_numpy(I0.astype(np.float32)).cuda()
    img2 = G.shade(gb, cam, lights, params, inten)
    assert np.array_equal(img, img2.cpu().numpy())
    if bad.any():
        pytest.skip("gradient check needs identical visibility")
    tm, ti = sg.perturbed_params(w.scene.mats, I0)
    target = S.shade_f64(cam, lights, ref, oracle.params_of(tm), ti.astype(np.float64))
    npx = cam.width * cam.height * 3
    dimg = torch.zeros_like(img2)
    dimg[..., :3] = 2.0 * (img2[..., :3] - torch.from_numpy(target.astype(np.float32)).cuda()) / npx
    dP, dI = torch.zeros_like(params), torch.zeros_like(inten)
    G.shade_backward(gb, cam, lights, params, inten, dimg, dP, dI)
    img64 = S.shade_f64(cam, lights, ref, P0, I0)
    rP, rI = S.grad_f64(cam, lights, ref, P0, I0, 2.0 * (img64 - target) / npx)
    got = np.concatenate([dP.cpu().numpy().ravel(), dI.cpu().numpy()]).astype(np.float64)
    want = np.concatenate([rP.ravel(), rI])
    err = np.abs(got - want) / np.maximum(np.abs(want), 1e-3 * np.abs(want).max())
    assert err.max() <= 1e-4, err.max()


def test_srgb_materials_match_oracle(fb):
    w = sg.workload_tiny41k()
    cam = sg.Camera((0.0, 4.0, 12.0), (0, 0, 0), (0, 1, 0), 60.0, 64, 48, 4)
    G, S = build_pair(w.scene)
    lin, _, _ = _render(G, cam, w.lights)
    G.set_materials(w.scene.mats, srgb=True)
    S.set_materials_srgb(w.scene.mats)
    img, _, _ = _check(G, S, cam, w.lights)
    assert not np.array_equal(img, lin)
    G.set_materials(w.scene.mats)                   # linear again: the first image
    again, _, _ = _render(G, cam, w.lights)
    assert np.array_equal(again, lin)


def test_normals_errors(fb):
    w = sg.workload_tiny41k()
    G = fb.Scene.from_numpy(w.scene)
    G.build(w.scene.identity_xforms())
    bad = sg.vertex_normals(w.scene)
    bad[5, 1] = np.nan
    with pytest.raises(fb.FireError):
        G.set_normals(bad)
    mats = fb.fire.make_materials(w.scene.mats)
    L = fb.fire.lib()
    assert L.fire_scene_set_materials_ex(G.h, fb.fire.C.cast(mats, fb.fire.C.c_void_p), len(mats), 2) != 0
    assert L.fire_scene_set_materials_ex(G.h, fb.fire.C.cast(mats, fb.fire.C.c_void_p), len(mats) + 1, 1) != 0
    assert L.fire_scene_set_normals(None, None, 0, None) != 0
    G.set_normals(None)                             # clearing twice is fine
    G.set_normals(None)


def test_smooth_device_normals_zero_fallback_and_empty(fb):
    """Normals given as a CUDA tensor render like the same host array; a
    triangle whose three normals are zero falls back to its geometric
    normal on both sides; an empty scene takes normals and renders black."""
    torch = torch_cuda()
    w = sg.workload_tiny41k()
    cam = sg.Camera((0.0, 4.0, 12.0), (0, 0, 0), (0, 1, 0), 60.0, 64, 48, 4)
    nrm = sg.vertex_normals(w.scene)
    nrm[w.scene.idx[::3].ravel()] = 0.0           # every third triangle: all-zero normals
    G, S = build_pair(w.scene)
    S.set_normals(nrm)
    G.set_normals(torch.from_numpy(nrm).cuda())
    img_dev, _, _ = _check(G, S, cam, w.lights)
    G.set_normals(nrm)
    img_host, _, _ = _render(G, cam, w.lights)
    assert np.array_equal(img_dev, img_host)
    empty = sg.Scene(verts=np.zeros((0, 4), np.float32), idx=np.zeros((0, 3), np.uint32),
                     tri_mat=np.zeros(0, np.uint32), vert_body=np.zeros(0, np.uint16),
                     mats=sg.random_materials(sg.Rng(5), 1), nbody=1)
    E = fb.Scene.from_numpy(empty)
    E.build(empty.identity_xforms())
    E.set_normals(np.zeros((0, 4), np.float32))
    img = E.render(cam, w.lights)
    assert E.sync_status() == 0 and float(img.abs().sum()) == 0.0
