"""GPU parity: the CUDA path (called through the C ABI) against the oracle on
the same seeded inputs, at sizes the oracle finishes in seconds, spanning
several tiles and ragged tails, plus the edge cases of the method."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from gpu_common import (assert_lbvh_equal, assert_radiance_close, assert_tris_equal, build_pair,
                        compare_samples, gbuf_of, pixel_ok_mask, torch_cuda, THREADS)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fb():
    import paper_2410_05095_b300 as fb
    torch_cuda()
    return fb


def _gbuf(cam):
    torch = torch_cuda()
    return torch.zeros((cam.width * cam.height * cam.spp, 4), dtype=torch.int32, device="cuda")


def _render(G, cam, lights, **opts):
    import paper_2410_05095_b300 as fb
    torch = torch_cuda()
    gb = _gbuf(cam)
    out = torch.zeros((cam.height, cam.width, 4), dtype=torch.float32, device="cuda")
    G.render(cam, lights, out=out, gbuf=gb, opts=fb.fire.make_opts(**opts) if opts else None)
    assert G.sync_status() == 0
    return out.cpu().numpy(), gbuf_of(gb)


# ----------------------------------------------------------------------------- LBVH
@pytest.mark.parametrize("name", ["tiny41k", "mid1m"])
def test_lbvh_bitexact(fb, name):
    w = sg.WORKLOADS[name]()
    G, S = build_pair(w.scene)
    assert_lbvh_equal(G, S, w.scene)
    assert G.info()["height"] >= 2


def test_lbvh_duplicate_keys_and_tiny_counts(fb):
    """Many equal Morton codes (index-augmented topology); 1, 2 and 3 triangles."""
    rng = sg.Rng(77)
    for n in (1, 2, 3, 5000):
        tris = []
        for _ in range(n):
            c = np.array([float(int(rng.u() * 4)) for _ in range(3)])
            tris.append(np.stack([c - 0.1, c, c + np.array([0.1, -0.05, 0.1])]))
        sc = sg.assemble([(np.concatenate(tris), np.arange(3 * n).reshape(n, 3))], 1,
                         sg.random_materials(rng, 1))
        G, S = build_pair(sc)
        assert_lbvh_equal(G, S, sc)


def _xf_rot(rng, nbody):
    """Rigid 3x4 matrices: a rotation about a random unit axis and a shift."""
    out = np.zeros((nbody, 12), np.float32)
    for b in range(nbody):
        ax = rng.unit_vector()
        ang = rng.uniform(-0.6, 0.6)
        K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        R = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K
        shift = np.array([[rng.uniform(-0.5, 0.5)] for _ in range(3)])
        out[b] = np.concatenate([R, shift], 1).reshape(12)
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 17, 33, 34, 100, 5000])
def test_refit_tiny_and_treelet_edges(fb, n):
    """The per-frame refit (by treelets of at most 32 4-wide nodes and the top
    nodes above them) at triangle counts around one treelet and below it:
    after two frames of motion of two bodies the boxes and triangle records
    equal the oracle's refit bit for bit, and a render agrees with it."""
    rng = sg.Rng(91 + n)
    meshes, mesh_body = [], []
    for i in range(n):
        c = np.array([rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(-3, 3)])
        size = 3.0 if n < 100 else 0.4  # few triangles: big ones, so that the image shows them
        e = [np.array([rng.uniform(-size, size) for _ in range(3)]) for _ in range(2)]
        meshes.append((np.stack([c, c + e[0], c + e[1]]), np.array([[0, 1, 2]])))
        mesh_body.append(i % 2)
    sc = sg.assemble(meshes, 2, sg.random_materials(rng, 2), mesh_body=mesh_body, nbody=2)
    G, S = build_pair(sc)
    for _ in range(2):
        xf = _xf_rot(rng, 2)
        G.refit(xf)
        S.update(xf, rebuild=False)
        assert np.array_equal(G.dump("boxes"), S.get("boxes"))
        assert_tris_equal(G, S, sc)
    assert G.sync_status() == 0
    cam = sg.Camera((0.3, 0.7, 9.0), (0, 0, 0), (0, 1, 0), 50.0, 24, 16, 4)
    lights = [sg.Light(0, (2.0, 6.0, 3.0), 40.0)]
    img, g = _render(G, cam, lights)
    ref = S.render_all_samples(cam, lights)
    _, bad = compare_samples(g, ref)
    assert bad.mean() < 0.01


@pytest.mark.parametrize("nbody", [1000, 65536])
def test_lbvh_many_bodies_bitexact(fb, nbody):
    """Keys with a wide body field (B = 10 and 16 bits, m = 17 and 15 bits per
    axis): a soup of small triangles spread over the bodies, posed by random
    rigid matrices -- build, refit, sampled render, all against the oracle."""
    rng = np.random.default_rng(nbody)
    nt = 3000 if nbody == 1000 else 70000
    c = rng.uniform(-4, 4, (nt, 3))
    tris = np.stack([c, c + rng.uniform(-0.2, 0.2, (nt, 3)), c + rng.uniform(-0.2, 0.2, (nt, 3))], 1)
    body = rng.integers(0, nbody, nt)
    from test_oracle_lbvh import _scene_from_tris
    sc = _scene_from_tris(tris, nbody=nbody, vbody=np.repeat(body, 3).astype(np.uint16))

    def poses(seed):
        r = np.random.default_rng(seed)
        xf = np.zeros((nbody, 12), np.float32)
        for b in range(nbody):
            q = r.normal(size=4)
            q /= np.linalg.norm(q)
            w, x, y, z = q
            R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                          [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                          [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]]) if b % 7 else np.eye(3)
            xf[b] = np.concatenate([R, r.uniform(-0.5, 0.5, (3, 1))], 1).reshape(12)
        return xf
    G, S = build_pair(sc, poses(1))
    assert_lbvh_equal(G, S, sc)
    xf = poses(2)
    G.refit(xf)
    S.update(xf, rebuild=False)
    assert np.array_equal(G.dump("boxes"), S.get("boxes"))
    cam = sg.Camera((0.5, 9.0, 11.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 50.0, 64, 48, 4)
    img, g = _render(G, cam, [sg.LIGHTS_MAIN[0]])
    ref = S.render_all_samples(cam, [sg.LIGHTS_MAIN[0]], threads=THREADS)
    _, bad = compare_samples(g, ref)
    assert_radiance_close(img, S.render_image(cam, [sg.LIGHTS_MAIN[0]], threads=THREADS), pixel_ok_mask(bad, 64, 48, 4))
    assert (ref["prim"] >= 0).mean() > 0.03


def test_refit_frames_bitexact(fb):
    w = sg.workload_frame7m(nspheres=120, cells=64)
    sc = w.scene
    G, S = build_pair(sc, w.motion.xforms())
    order = G.dump("order")
    for frame in range(3):
        xf = w.motion.step()
        G.refit(xf)
        S.update(xf, rebuild=False)
        assert np.array_equal(G.dump("order"), order)
        assert np.array_equal(G.dump("boxes"), S.get("boxes"))
        assert_tris_equal(G, S, sc)
    # device-resident transforms give the same result
    torch = torch_cuda()
    xf = w.motion.step()
    G.refit(torch.from_numpy(xf).cuda())
    S.update(xf, rebuild=False)
    assert np.array_equal(G.dump("boxes"), S.get("boxes"))
    # a rebuild after motion re-derives everything
    G.build(xf)
    S.update(xf, rebuild=True)
    assert_lbvh_equal(G, S, sc)


# --------------------------------------------------------------------------- render
def test_render_tiny_full_image(fb):
    w = sg.workload_tiny41k()
    G, S = build_pair(w.scene)
    img, g = _render(G, w.camera, w.lights)
    ref = S.render_all_samples(w.camera, w.lights, threads=THREADS)
    frac, bad = compare_samples(g, ref)
    assert np.array_equal(g["t"][~bad], ref["t"][~bad])
    img_ref = S.render_image(w.camera, w.lights, threads=THREADS)
    ok = pixel_ok_mask(bad, w.camera.width, w.camera.height, 1)
    assert_radiance_close(img, img_ref, ok)
    assert np.array_equal(img[..., 3][ok], img_ref[..., 3][ok])
    assert (g["prim"] >= 0).mean() > 0.5


def test_render_info_counts_the_shadow_rays(fb):
    """fire_render_info's shadow-ray count equals the cast bits of the
    G-buffer (rays queued over all lights' segments)."""
    w = sg.workload_mid1m(160, 90, 4)
    G, _ = build_pair(w.scene)
    img, g = _render(G, w.camera, w.lights)
    cast = sum(int(((g["vis"] >> (8 + j)) & 1).sum()) for j in range(len(w.lights)))
    info = G.render_info()
    assert cast > 0 and info["shadow_rays"] == cast and not info["raster"]


def test_render_mid_4spp_three_lights(fb):
    w = sg.workload_mid1m(320, 180, 4)
    G, S = build_pair(w.scene)
    img, g = _render(G, w.camera, w.lights)
    ref = S.render_all_samples(w.camera, w.lights, threads=THREADS)
    frac, bad = compare_samples(g, ref)
    img_ref = S.render_image(w.camera, w.lights, threads=THREADS)
    assert_radiance_close(img, img_ref, pixel_ok_mask(bad, 320, 180, 4))
    lit = (ref["vis"] & 0xFF) != 0
    shadowed = ((ref["vis"] >> 8) & ~ref["vis"] & 0xFF) != 0
    assert lit.mean() > 0.2 and shadowed.mean() > 0.01  # all three light kinds exercised


@pytest.mark.parametrize("W,H,spp", [(37, 23, 4), (37, 23, 1), (8, 4, 1), (1, 1, 4), (129, 3, 1)])
def test_render_ragged_sizes(fb, W, H, spp):
    w = sg.workload_tiny41k()
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, W, H, spp)
    G, S = build_pair(w.scene)
    img, g = _render(G, cam, w.lights)
    ref = S.render_all_samples(cam, w.lights)
    _, bad = compare_samples(g, ref)
    assert_radiance_close(img, S.render_image(cam, w.lights), pixel_ok_mask(bad, W, H, spp))


def test_row_bands_equal_full_render(fb):
    """Image partition by row bands (the replica split): two band renders
    into one buffer equal the full render bit for bit."""
    torch = torch_cuda()
    w = sg.workload_tiny41k()
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 96, 61, 4)
    G, _ = build_pair(w.scene)
    full = G.render(cam, w.lights)
    part = torch.full_like(full, -1.0)
    G.render(cam, w.lights, out=part, opts=fb.fire.make_opts(row_begin=0, row_end=29))
    G.render(cam, w.lights, out=part, opts=fb.fire.make_opts(row_begin=29, row_end=61))
    assert torch.equal(full, part)


def test_empty_scene_and_single_triangle(fb):
    torch = torch_cuda()
    mats = sg.random_materials(sg.Rng(1), 2)
    empty = sg.Scene(verts=np.zeros((0, 4), np.float32), idx=np.zeros((0, 3), np.uint32),
                     tri_mat=np.zeros(0, np.uint32), vert_body=np.zeros(0, np.uint16), mats=mats, nbody=1)
    G = fb.Scene.from_numpy(empty)
    G.build(empty.identity_xforms())
    cam = sg.Camera((0, 0, 5), (0, 0, 0), (0, 1, 0), 60.0, 16, 8, 4)
    out = G.render(cam, [sg.LIGHTS_MAIN[0]])
    assert torch.count_nonzero(out) == 0
    one = sg.assemble([(np.array([[-1.0, -1, 0], [1, -1, 0], [0, 1, 0]]), np.array([[0, 1, 2]]))], 2, mats)
    G1, S1 = build_pair(one)
    assert_lbvh_equal(G1, S1, one)
    cam = sg.Camera((0.1, 0.2, 5), (0, 0, 0), (0, 1, 0), 40.0, 33, 17, 4)
    img, g = _render(G1, cam, [sg.Light(0, (0.0, 0.0, 4.0), 10.0)])
    ref = S1.render_all_samples(cam, [sg.Light(0, (0.0, 0.0, 4.0), 10.0)])
    _, bad = compare_samples(g, ref)
    assert not bad.any()
    assert_radiance_close(img, S1.render_image(cam, [sg.Light(0, (0.0, 0.0, 4.0), 10.0)]))


# ---------------------------------------------------------------------- error paths
def test_error_paths(fb):
    torch = torch_cuda()
    w = sg.workload_tiny41k()
    sc = w.scene
    G = fb.Scene.from_numpy(sc)
    cam = w.camera
    with pytest.raises(fb.FireError) as e:
        G.refit(sc.identity_xforms())
    assert e.value.code == -6                        # refit before build
    with pytest.raises(fb.FireError) as e:
        G.render(cam, w.lights)
    assert e.value.code == -6
    bad = sc.identity_xforms()
    bad[0, 3] = np.nan
    with pytest.raises(fb.FireError) as e:
        G.build(bad)
    assert e.value.code == -1                        # non-finite transform
    G.build(sc.identity_xforms())
    for bad_cam in (sg.Camera(cam.pos, cam.target, cam.up, 60.0, 16, 16, 2),
                    sg.Camera(cam.pos, cam.pos, cam.up, 60.0, 16, 16, 1),
                    sg.Camera(cam.pos, cam.target, cam.up, 180.0, 16, 16, 1)):
        with pytest.raises(fb.FireError) as e:
            G.render(bad_cam, w.lights)
        assert e.value.code == -1
    with pytest.raises(fb.FireError) as e:
        G.render(cam, [sg.LIGHTS_MAIN[0]] * 9)
    assert e.value.code == -1
    with pytest.raises(fb.FireError):
        G.render(cam, w.lights, opts=fb.fire.make_opts(row_begin=5, row_end=3))
    with pytest.raises(fb.FireError):
        G.render(cam, w.lights, opts=fb.fire.make_opts(stack_depth=2))  # below the tree height
    # out-of-range index / material / body -> counted on the device, rejected
    for field, val in (("idx", sc.nv), ("tri_mat", 9), ("vert_body", 3)):
        bad_sc = sg.Scene(verts=sc.verts, idx=sc.idx.copy(), tri_mat=sc.tri_mat.copy(),
                          vert_body=sc.vert_body.copy(), mats=sc.mats, nbody=1)
        getattr(bad_sc, field).reshape(-1)[7] = val
        with pytest.raises(fb.FireError) as e:
            fb.Scene.from_numpy(bad_sc)
        assert e.value.code == -1
    # injected allocation failure -> OOM, and the next create works
    fb.fire.fail_next_alloc(3)
    with pytest.raises(fb.FireError) as e:
        fb.Scene.from_numpy(sc)
    assert e.value.code == -2
    fb.Scene.from_numpy(sc).destroy()


def test_device_error_flags(fb):
    """Stack overflow and the iteration cap are reported through the sticky
    device error word (no trap): a forced 8-entry stack on a deep tree, and
    a cap of 3 node visits per ray."""
    w = sg.workload_mid1m(64, 36, 1)
    G, _ = build_pair(w.scene)
    assert G.info()["height"] > 8
    G.render(w.camera, w.lights, opts=fb.fire.make_opts(stack_depth=8, flags=1))
    assert G.sync_status() == -4
    assert G.sync_status() == 0                       # cleared by the read
    G.set_iteration_cap(3)
    G.render(w.camera, w.lights)
    assert G.sync_status() == -5
    G.set_iteration_cap(0)
    G.render(w.camera, w.lights)
    assert G.sync_status() == 0


# ---------------------------------------------------------------------------- batch
def test_batch_equals_sequential(fb):
    torch = torch_cuda()
    rng = sg.Rng(2024)
    scenes, G = [], []
    for s in range(3):
        sc = sg.scene_icospheres_terrain(rng, 3 + 4 * s, 32, 32)
        scenes.append(sc)
        g = fb.Scene.from_numpy(sc)
        g.build(sc.identity_xforms())
        G.append(g)
    res = [(64, 64, 1), (37, 23, 4), (128, 96, 1), (20, 11, 1), (33, 9, 4), (96, 64, 1)]
    cams, cam_scene = [], []
    for i, (W, H, spp) in enumerate(res):
        c = sg.orbit_camera(rng, W, H, spp)
        cams.append(c)
        cam_scene.append(i % 3)
    lights = [sg.LIGHTS_MAIN[:1], sg.LIGHTS_MAIN[:2], sg.LIGHTS_MAIN[:3]]
    outs = [torch.zeros((c.height, c.width, 4), device="cuda") for c in cams]
    fb.render_batch(G, cams, cam_scene, lights, outs)
    cfg = fb.batch_last_config()
    assert cfg["tuned"] == 1 and cfg["threads"] in (64, 128, 256)
    tun = fb.fire.batch_last_tuning()
    assert tun["tuned_now"] and tun["tried"] >= 11 and 0 < tun["best_ms"] <= tun["worst_ms"]
    assert (tun["tile_w_1spp"], tun["tile_w_4spp"]) in ((8, 4), (4, 2), (16, 8)) and tun["grab"] in (1, 2)
    for c, si, o in zip(cams, cam_scene, outs):
        ref = G[si].render(c, lights[si])
        assert torch.equal(o, ref)
    # every tile shape and grab size the search may pick gives the same
    # images (fixed threads / blocks per SM skip the search; the flags force
    # the shape)
    for tile in (1, 2, 3):
        for grab in (0, 1024):
            outs_fixed = [torch.zeros_like(o) for o in outs]
            fb.render_batch(G, cams, cam_scene, lights, outs_fixed,
                            opts=fb.fire.make_opts(block_threads=64, blocks_per_sm=2, flags=(tile << 8) | grab))
            t = fb.fire.batch_last_tuning()
            assert t["tried"] == 0 and t["grab"] == (2 if grab else 1)
            assert t["tile_w_1spp"] == (8, 4, 16)[tile - 1] and t["tile_w_4spp"] == (4, 2, 8)[tile - 1]
            for a, b in zip(outs, outs_fixed):
                assert torch.equal(a, b), (tile, grab)
    # graph replay gives the same images
    outs2 = [o.clone().fill_(-1) for o in outs]
    fb.render_batch(G, cams, cam_scene, lights, outs2)
    assert fb.batch_last_config()["tuned"] == 0
    for a, b in zip(outs, outs2):
        assert torch.equal(a, b)
    # and after a refit of one scene (new poses, same buffers) the replay reflects it
    xf = scenes[1].identity_xforms()
    xf[0, 3] = 0.25
    G[1].refit(xf)
    fb.render_batch(G, cams, cam_scene, lights, outs2)
    for c, si, o in zip(cams, cam_scene, outs2):
        assert torch.equal(o, G[si].render(c, lights[si]))
    for g in G:
        assert g.sync_status() == 0


# ------------------------------------------------------------------- differentiable
def test_shade_gbuffer_equals_render(fb):
    torch = torch_cuda()
    w = sg.workload_tiny41k(64, 48)
    cam = sg.Camera(**{**w.camera.__dict__, "spp": 4})
    lights = [sg.LIGHTS_MAIN[0], sg.LIGHTS_MAIN[1]]
    G, _ = build_pair(w.scene)
    gb = _gbuf(cam)
    img = G.render(cam, lights, gbuf=gb)
    params = torch.from_numpy(oracle.params_of(w.scene.mats).astype(np.float32)).cuda()
    inten = torch.tensor([l.intensity for l in lights], dtype=torch.float32, device="cuda")
    img2 = G.shade(gb, cam, lights, params, inten)
    assert torch.equal(img, img2)


def test_pipelined_frames_equal_serial(fb):
    """Double-buffered frames: refits on their own stream (into the buffer
    the last render did not read) interleaved with renders on another stream
    give the images of the serial order, frame by frame."""
    torch = torch_cuda()
    w = sg.workload_frame7m(nspheres=120, cells=64)
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 160, 96, 4)
    xf0 = w.motion.xforms()
    poses = [w.motion.step() for _ in range(6)]
    G1, G2 = fb.Scene.from_numpy(w.scene), fb.Scene.from_numpy(w.scene)
    G1.build(xf0)
    G2.build(xf0)
    serial = []
    for xf in poses:
        G1.refit(xf)
        serial.append(G1.render(cam, w.lights).clone())
    dev = [torch.from_numpy(xf).cuda() for xf in poses]
    outs = [torch.zeros_like(serial[0]) for _ in poses]
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    for i, xf in enumerate(dev):
        G2.refit(xf if i % 2 else poses[i], stream=side)   # device and host poses
        G2.render(cam, w.lights, out=outs[i])
    torch.cuda.synchronize()
    assert G2.sync_status() == 0
    for a, b in zip(serial, outs):
        assert torch.equal(a, b)
