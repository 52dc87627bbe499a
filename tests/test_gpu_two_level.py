"""The two-level acceleration structure on the GPU (fire_scene_set_two_level:
a bottom level per rigid body built once over the rest pose, a top level
over subtrees of the bodies' bottom levels rebuilt every frame, §IV-B-3)
against the oracle's
two-level mode (bodies as instances of rest-space geometry, rays met in
each body's frame).

Order matters in this file: the first tests build the structure on the GPU
and run the traversal code on the host (fire_debug_trace_host: every load
checked against the copied arrays' bounds and alignment) before any test
launches the two-level render kernels; run with -x, a failure there stops
the file before the device traversal runs."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from gpu_common import (THREADS, TIE_REL, assert_radiance_close, compare_samples, gbuf_of, pixel_ok_mask,
                        torch_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fb():
    import paper_2410_05095_b300 as fb
    torch_cuda()
    return fb


def _moving(nspheres=120, cells=64, frames=4):
    w = sg.workload_frame7m(nspheres=nspheres, cells=cells)
    poses = [w.motion.step() for _ in range(frames)]
    return w, poses


def _pair2(fb, sc, xf):
    G = fb.Scene.from_numpy(sc)
    G.set_two_level(True)
    G.build(xf)
    S = oracle.OracleScene(sc)
    S.set_two_level(True)
    S.update(xf, rebuild=True)
    return G, S


def _camera_rays(cam):
    n = cam.width * cam.height * cam.spp
    o = np.zeros((n, 3), np.float32)
    d = np.zeros((n, 3), np.float32)
    for i in range(n):
        k, p = i % cam.spp, i // cam.spp
        o[i], d[i] = oracle.camera_ray(cam, p % cam.width, p // cam.width, k)
    return o, d


def _segments(rng, n, lo, hi):
    o = rng.uniform(lo, hi, (n, 3)).astype(np.float32)
    e = rng.uniform(lo, hi, (n, 3)).astype(np.float32)
    v = e - o
    L = np.linalg.norm(v, axis=1).astype(np.float32)
    d = (v / L[:, None]).astype(np.float32)
    return o, d, L


# ------------------------------------------------------------- build, then host emulation
def test_top_entries_cut_bodies(fb):
    """The top level is built over subtrees of the bodies' bottom levels:
    every triangle of a body lies under exactly one of that body's entries,
    the entries come in body order within each body's share of the 1,024
    slots (the unused slots after them), a body of spheres spread over the
    scene gets more than one entry, and an entry's rest box holds its
    subtree's triangles and is tight around them."""
    w, _ = _moving(nspheres=40, cells=32, frames=1)
    G = fb.Scene.from_numpy(w.scene)
    G.set_two_level(True)
    G.build(w.motion.xforms())
    E, N, R = G.dump("top_entries"), G.dump("nodes4"), G.dump("tris")
    roots, nb, nt = G.dump("blas_root"), G.nbody, G.nt
    k = int((E[:, 0] >= 0).sum())
    assert (E[:k] >= 0).all() and (E[k:] == -1).all()
    assert np.all(np.diff(E[:k, 1]) >= 0)
    share = max(1, min(64, 1024 // int((roots >= 0).sum())))
    counts = np.bincount(E[:k, 1], minlength=nb)
    assert counts.max() <= share and k > int((roots >= 0).sum())
    assert np.array_equal(counts > 0, roots >= 0)
    links = N[:, 24:28].copy().view(np.int32)
    lo_n, hi_n = N[:, 0:12].reshape(-1, 3, 4), N[:, 12:24].reshape(-1, 3, 4)
    body = R[:, 11].copy().view(np.int32)
    v0 = R[:, 0:3].astype(np.float64)
    tri_lo = np.minimum(v0, np.minimum(v0 + R[:, 4:7], v0 + R[:, 8:11]))
    tri_hi = np.maximum(v0, np.maximum(v0 + R[:, 4:7], v0 + R[:, 8:11]))
    seen = np.zeros(nt, np.int64)
    box = {}  # rest box of each node from its parent's slot
    for q in range(len(N)):
        for c in range(4):
            if links[q, c] >= 0:
                box[int(links[q, c])] = (lo_n[q, :, c], hi_n[q, :, c])
    for q, b in E[:k]:
        stack, under = [int(q)], []
        while stack:
            v = stack.pop()
            for l in links[v]:
                if l == -2**31:
                    continue
                (under.append(~int(l)) if l < 0 else stack.append(int(l)))
        under = np.array(under)
        seen[under] += 1
        assert (body[under] == b).all()
        lo, hi = tri_lo[under].min(0), tri_hi[under].max(0)
        tol = 1e-5 * (1.0 + np.abs(np.concatenate([lo, hi])).max())
        if int(q) in box:
            blo, bhi = box[int(q)]
            assert (blo <= lo + tol).all() and (bhi >= hi - tol).all()
            assert (np.abs(blo - lo) <= tol).all() and (np.abs(bhi - hi) <= tol).all()
    assert (seen == 1).all()


def test_emulated_traversal_matches_oracle(fb):
    """Built on the GPU (bottom levels at rest, top level for frame 3's
    poses), walked on the host by the render kernels' traversal code: every
    load in bounds and aligned, no error bit, nearest hits equal to the
    oracle's (up to near ties), any-hit answers equal."""
    w, poses = _moving()
    G, S = _pair2(fb, w.scene, poses[0])
    for xf in poses[1:]:
        G.refit(xf)
        S.update(xf, rebuild=False)
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 96, 54, 4)
    o, d = _camera_rays(cam)
    prim, t, _, err = G.trace_host(o, d)
    assert err == 0, hex(err)
    rp, rt, _, _, rt2 = S.trace(o, d, want_t2=True)
    bad = (prim != rp) | ((prim >= 0) & (t != rt))
    with np.errstate(invalid="ignore"):
        tie = np.isfinite(rt2) & (np.abs(rt2 - rt) <= TIE_REL * np.abs(rt))
    assert bad.mean() <= 1e-4 and not (bad & ~tie).any(), int(bad.sum())
    assert (rp >= 0).mean() > 0.2
    # any hit: segments across the scene, with and without a skipped triangle
    rng = np.random.default_rng(5)
    so, sd, sl = _segments(rng, 6000, [-12, -3, -12], [12, 5, 12])
    skip = np.where(rng.uniform(size=6000) < 0.5, rng.integers(0, w.scene.nt, 6000), -1).astype(np.int32)
    _, _, hit, err = G.trace_host(so, sd, tmax=sl, skip=skip, any_hit=True)
    assert err == 0, hex(err)
    ref = S.occluded(so, sd, sl, skip)
    assert np.array_equal(hit, ref), int((hit != ref).sum())
    assert 0.1 < ref.mean() < 0.95


def test_emulated_degenerate_bodies(fb):
    """Bodies of one triangle, bodies without triangles, and a scene whose
    triangles are all in one body: the host walk stays in bounds and
    matches the oracle."""
    rng = sg.Rng(17)
    tris, vb = [], []
    for b in range(9):
        if b in (2, 5):
            continue  # bodies without triangles
        n = 1 if b in (0, 7) else 40
        for _ in range(n):
            c = np.array([rng.uniform(-3, 3), rng.uniform(-1, 1), rng.uniform(-3, 3)])
            tris.append(np.stack([c, c + [0.3, 0.0, 0.1], c + [0.0, 0.25, 0.2]]))
            vb += [b] * 3
    from test_oracle_lbvh import _scene_from_tris
    for nbody, vbody in ((9, np.array(vb, np.uint16)), (1, np.zeros(len(vb), np.uint16))):
        sc = _scene_from_tris(np.array(tris), nbody=nbody, vbody=vbody)
        xf = np.tile(np.eye(3, 4, dtype=np.float32).reshape(1, 12), (nbody, 1))
        xf[:, 3] += np.linspace(0, 0.5, nbody, dtype=np.float32)
        G, S = _pair2(fb, sc, xf)
        rr = np.random.default_rng(nbody)
        o, d, L = _segments(rr, 3000, [-4, -2, -4], [4, 2, 4])
        prim, t, _, err = G.trace_host(o, d)
        assert err == 0
        rp, rt, _, _ = S.trace(o, d)
        assert np.array_equal(prim, rp) and np.array_equal(t[rp >= 0], rt[rp >= 0])
        _, _, hit, err = G.trace_host(o, d, tmax=L, any_hit=True)
        assert err == 0 and np.array_equal(hit, S.occluded(o, d, L))


def test_emulated_fullsize(fb, frame7m_two):
    """The headline workload at full size (7,299,072 triangles, 65 bodies),
    frame 2: 2,000 sampled camera rays and 2,000 segments walked on the
    host, in bounds, equal to the oracle."""
    w, G, S, _ = frame7m_two
    cam = w.camera
    rng = np.random.default_rng(77)
    ids = rng.choice(cam.width * cam.height * cam.spp, 2000, replace=False)
    o = np.zeros((len(ids), 3), np.float32)
    d = np.zeros((len(ids), 3), np.float32)
    for i, sid in enumerate(ids):
        k, p = int(sid % 4), int(sid // 4)
        o[i], d[i] = oracle.camera_ray(cam, p % cam.width, p // cam.width, k)
    prim, t, _, err = G.trace_host(o, d)
    assert err == 0, hex(err)
    rp, rt, _, _, rt2 = S.trace(o, d, want_t2=True)
    bad = (prim != rp) | ((prim >= 0) & (t != rt))
    with np.errstate(invalid="ignore"):
        tie = np.isfinite(rt2) & (np.abs(rt2 - rt) <= TIE_REL * np.abs(rt))
    assert not (bad & ~tie).any()
    so, sd, sl = _segments(rng, 2000, [-12, -3, -12], [12, 5, 12])
    _, _, hit, err = G.trace_host(so, sd, tmax=sl, any_hit=True)
    assert err == 0 and np.array_equal(hit, S.occluded(so, sd, sl))


@pytest.fixture(scope="module")
def frame7m_two():
    """The full-size moving workload in two-level mode on both sides, two
    frames after the build (top level rebuilt per frame)."""
    import paper_2410_05095_b300 as fb
    torch_cuda()
    w = sg.workload_frame7m()
    G, S = _pair2(fb, w.scene, w.motion.xforms())
    poses = []
    for _ in range(2):
        xf = w.motion.step()
        poses.append(xf)
        G.refit(xf)
        S.update(xf, rebuild=False)
    return w, G, S, poses


# --------------------------------------------------------------- device kernels
def test_fullsize_two_level_sampled_render(fb, frame7m_two):
    """The GPU two-level render of that frame: 20,000 sampled samples by the
    agreement rule, 2,000 sampled pixels' radiance within 1e-4."""
    torch = torch_cuda()
    w, G, S, _ = frame7m_two
    cam = w.camera
    gb = torch.zeros((cam.width * cam.height * cam.spp, 4), dtype=torch.int32, device="cuda")
    img = G.render(cam, w.lights, gbuf=gb).cpu().numpy()
    assert G.sync_status() == 0
    g = gbuf_of(gb)
    rng = np.random.default_rng(2411)
    from concurrent.futures import ThreadPoolExecutor

    def ref_of(ids):
        chunks = np.array_split(np.asarray(ids, np.int64), THREADS * 2)
        with ThreadPoolExecutor(THREADS) as ex:
            parts = list(ex.map(lambda c: S.render_samples(cam, w.lights, c), chunks))
        return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    ids = rng.choice(cam.width * cam.height * cam.spp, 20000, replace=False)
    compare_samples(g, ref_of(ids), ids)
    pix = rng.choice(cam.width * cam.height, 2000, replace=False)
    pid = (pix[:, None] * 4 + np.arange(4)[None, :]).ravel()
    rs = ref_of(pid)
    _, bad = compare_samples(g, rs, pid)
    acc = np.zeros((len(pix), 3), np.float32)
    for k in range(4):
        acc = acc + rs["rgb"][k::4]
    ref_px = np.concatenate([acc / np.float32(4), (rs["prim"].reshape(-1, 4) >= 0).mean(1, keepdims=True)], 1)
    ok = ~bad.reshape(-1, 4).any(1)
    assert_radiance_close(img.reshape(-1, 4)[pix][None], ref_px[None].astype(np.float32), ok[None])
    assert (g["prim"] >= 0).mean() > 0.3
def _render(fb, G, cam, lights, **opts):
    torch = torch_cuda()
    gb = torch.zeros((cam.width * cam.height * cam.spp, 4), dtype=torch.int32, device="cuda")
    out = torch.zeros((cam.height, cam.width, 4), dtype=torch.float32, device="cuda")
    G.render(cam, lights, out=out, gbuf=gb, opts=fb.fire.make_opts(**opts) if opts else None)
    assert G.sync_status() == 0
    return out.cpu().numpy(), gbuf_of(gb)


def test_two_level_render_matches_oracle(fb):
    """Frames 1-3 of the moving workload (reduced), 4 spp, two point lights:
    hits and visibility by the agreement rule, radiance within 1e-4."""
    w, poses = _moving()
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 192, 108, 4)
    G, S = _pair2(fb, w.scene, poses[0])
    for xf in poses[1:]:
        G.refit(xf)
        S.update(xf, rebuild=False)
        img, g = _render(fb, G, cam, w.lights)
        ref = S.render_all_samples(cam, w.lights, threads=THREADS)
        _, bad = compare_samples(g, ref)
        img_ref = S.render_image(cam, w.lights, threads=THREADS)
        assert_radiance_close(img, img_ref, pixel_ok_mask(bad, cam.width, cam.height, 4))
    assert (ref["prim"] >= 0).mean() > 0.2 and ((ref["vis"] >> 8) & ~ref["vis"] & 3).any()


def test_two_level_single_body_and_directional_light(fb):
    """A static single-body scene (tiny41k) in two-level mode with a point
    and a directional light, ragged 4-spp image."""
    w = sg.workload_tiny41k()
    lights = [sg.LIGHTS_MAIN[0], sg.LIGHTS_MAIN[2]]
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 77, 45, 4)
    xf = w.scene.identity_xforms()
    G, S = _pair2(fb, w.scene, xf)
    img, g = _render(fb, G, cam, lights)
    ref = S.render_all_samples(cam, lights)
    _, bad = compare_samples(g, ref)
    assert_radiance_close(img, S.render_image(cam, lights), pixel_ok_mask(bad, cam.width, cam.height, 4))


def test_two_level_pipelined_frames_and_shading(fb):
    """Top levels rebuilt on their own stream into the second frame buffer
    while the previous frame renders: frames 2 and 4 against the oracle; the
    G-buffer shading and its backward run on the two-level hit frame."""
    torch = torch_cuda()
    w, poses = _moving(frames=4)
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 160, 90, 4)
    G = fb.Scene.from_numpy(w.scene)
    G.set_two_level(True)
    G.build(poses[0])
    n = cam.width * cam.height * cam.spp
    gbs = [torch.zeros((n, 4), dtype=torch.int32, device="cuda") for _ in poses]
    outs = [torch.zeros((cam.height, cam.width, 4), device="cuda") for _ in poses]
    side = torch.cuda.Stream(priority=-1)
    dev = [torch.from_numpy(x).cuda() for x in poses]
    torch.cuda.synchronize()
    for i in range(1, len(poses)):
        G.refit(dev[i], stream=side)
        G.render(cam, w.lights, out=outs[i], gbuf=gbs[i], opts=fb.fire.make_opts(blocks_per_sm=6))
    torch.cuda.synchronize()
    assert G.sync_status() == 0
    S = oracle.OracleScene(w.scene)
    S.set_two_level(True)
    S.update(poses[0], rebuild=True)
    for i in range(1, len(poses)):
        S.update(poses[i], rebuild=False)
        if i % 2:
            continue
        ref = S.render_all_samples(cam, w.lights, threads=THREADS)
        _, bad = compare_samples(gbuf_of(gbs[i]), ref)
        assert_radiance_close(outs[i].cpu().numpy(), S.render_image(cam, w.lights, threads=THREADS),
                              pixel_ok_mask(bad, cam.width, cam.height, 4))
    # shading of the last G-buffer with the scene's own parameters = the render
    params = torch.from_numpy(oracle.params_of(w.scene.mats).astype(np.float32)).cuda()
    inten = torch.tensor([l.intensity for l in w.lights], dtype=torch.float32, device="cuda")
    img2 = G.shade(gbs[-1], cam, w.lights, params, inten)
    assert torch.equal(img2, outs[-1])
    dP, dI = torch.zeros_like(params), torch.zeros_like(inten)
    G.shade_backward(gbs[-1], cam, w.lights, params, inten, torch.ones_like(img2), dP, dI)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(dP).all()) and float(dI.abs().sum()) > 0


def test_two_level_error_paths(fb):
    torch = torch_cuda()
    w = sg.workload_tiny41k(32, 32)
    G = fb.Scene.from_numpy(w.scene)
    G.build(w.scene.identity_xforms())
    G.set_two_level(True)
    with pytest.raises(fb.FireError) as e:
        G.render(w.camera, w.lights)
    assert e.value.code == -6                          # mode change leaves the scene unbuilt
    G.build(w.scene.identity_xforms())
    with pytest.raises(fb.FireError) as e:
        G.render(w.camera, w.lights, opts=fb.fire.make_opts(flags=4))
    assert e.value.code == -1                          # no raster pass in two-level mode
    out = torch.zeros((32, 32, 4), device="cuda")
    with pytest.raises(fb.FireError) as e:
        fb.render_batch([G], [w.camera], [0], [w.lights], [out])
    assert e.value.code == -1                          # no batch in two-level mode
    with pytest.raises(fb.FireError) as e:
        G.set_normals(sg.vertex_normals(w.scene))
        G.render(w.camera, w.lights)
    assert e.value.code == -1                          # no smooth normals in two-level mode
    G.set_normals(None)
    G.set_two_level(False)
    G.build(w.scene.identity_xforms())
    G.render(w.camera, w.lights)
    # a triangle across two bodies cannot be an instance's
    sc = sg.assemble([(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0.0]]), np.array([[0, 1, 2]]))], 1,
                     sg.random_materials(sg.Rng(3), 1))
    sc.vert_body[:] = [0, 1, 0]
    sc.nbody = 2
    G2 = fb.Scene.from_numpy(sc)
    with pytest.raises(fb.FireError) as e:
        G2.set_two_level(True)
    assert e.value.code == -1
