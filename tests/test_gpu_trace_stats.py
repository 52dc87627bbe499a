"""Host emulation of the single-level traversal and the traversal statistics
(fire_debug_trace_host, fire_debug_trace_stats), and the dump of a render's
shadow rays (fire_debug_dump 12).

The emulation runs the render kernels' own traversal code on host copies of
the scene's 4-wide tree and triangle records, so on the same rays it must
give exactly the device's answers: the primary hits of a render (camera
rays of the oracle, which equal the kernel's bit for bit) and the
visibility bits its shadow pass wrote for the dumped shadow rays.  The
statistics are pinned on a scene whose counts follow from its layout."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from gpu_common import TIE_REL, gbuf_of, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fb():
    import paper_2410_05095_b300 as fb
    torch_cuda()
    return fb


def _camera_rays(cam):
    n = cam.width * cam.height * cam.spp
    o = np.zeros((n, 3), np.float32)
    d = np.zeros((n, 3), np.float32)
    for i in range(n):
        k, p = i % cam.spp, i // cam.spp
        o[i], d[i] = oracle.camera_ray(cam, p % cam.width, p // cam.width, k)
    return o, d


def _moving_scene(fb, frames=3):
    w = sg.workload_frame7m(nspheres=120, cells=64)
    G = fb.Scene.from_numpy(w.scene)
    G.build(w.motion.xforms())
    for _ in range(frames):
        G.refit(w.motion.step())
    return w, G


def test_emulated_single_level_matches_render_and_oracle(fb):
    """After three refits: the host walk of the device tree gives the
    render's primary records exactly (same code, same rays), every load in
    bounds, no error bit; and the oracle's nearest hits up to near ties."""
    import torch
    w, G = _moving_scene(fb)
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 80, 45, 4)
    gb = torch.zeros((cam.width * cam.height * cam.spp, 4), dtype=torch.int32, device="cuda")
    out = torch.zeros((cam.height, cam.width, 4), device="cuda")
    G.render(cam, w.lights, out=out, gbuf=gb)
    g = gbuf_of(gb)
    o, d = _camera_rays(cam)
    prim, t, _, err = G.trace_host(o, d)
    assert err == 0, hex(err)
    assert np.array_equal(prim, g["prim"])
    hit = prim >= 0
    assert np.array_equal(t[hit].view(np.uint32), g["t"][hit].view(np.uint32))
    assert 0.2 < hit.mean() < 0.95
    S = oracle.OracleScene(w.scene)
    S.update(w.motion.xforms(), rebuild=True)
    rp, rt, _, _, rt2 = S.trace(o, d, want_t2=True)
    bad = (prim != rp) | (hit & (t != rt))
    with np.errstate(invalid="ignore"):
        tie = np.isfinite(rt2) & (np.abs(rt2 - rt) <= TIE_REL * np.abs(rt))
    assert bad.mean() <= 1e-4 and not (bad & ~tie).any(), int(bad.sum())


def test_dumped_shadow_rays_reproduce_the_visibility_bits(fb):
    """The dump holds the render's shadow rays in the shadow pass's order:
    one per (hit sample, light with n.l > 0) -- the render's cast bits --,
    light by light, unit directions; traced on the host with the sample's
    own triangle skipped they give exactly the visibility bits the device
    wrote."""
    import torch
    w, G = _moving_scene(fb)
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 72, 40, 4)
    nsamp = cam.width * cam.height * cam.spp
    gb = torch.zeros((nsamp, 4), dtype=torch.int32, device="cuda")
    out = torch.zeros((cam.height, cam.width, 4), device="cuda")
    G.render(cam, w.lights, out=out, gbuf=gb)
    g = gbuf_of(gb)
    q = G.dump("shadow_rays")
    tag = q[:, 7].view(np.int32)
    sid, light = tag >> 3, tag & 7
    assert len(q) == G.render_info()["shadow_rays"] > 100
    assert (sid >= 0).all() and (sid < nsamp).all() and (light < len(w.lights)).all()
    assert (np.diff(light) >= 0).all()  # light by light
    cast = np.zeros((nsamp, len(w.lights)), bool)
    cast[sid, light] = True
    want = np.stack([(g["vis"] >> (8 + j)) & 1 for j in range(len(w.lights))], 1).astype(bool)
    assert np.array_equal(cast, want)
    assert len(np.unique(tag)) == len(tag)
    assert np.allclose(np.linalg.norm(q[:, 4:7], axis=1), 1.0, atol=1e-5)
    _, _, occ, err = G.trace_host(q[:, 0:3], q[:, 4:7], tmax=q[:, 3], skip=g["prim"][sid], any_hit=True)
    assert err == 0, hex(err)
    vis = ((g["vis"][sid] >> light) & 1).astype(bool)
    assert np.array_equal(~occ, vis)
    assert 0.05 < occ.mean() < 0.95


def test_trace_stats_on_separated_boxes(fb):
    """Three triangles far apart under one 4-wide root: a ray fetches the
    root once; a ray through one triangle's box tests that triangle, a ray
    that misses every box tests none; per group the distinct nodes are the
    root alone and the distinct records the triangles its rays tested."""
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    tris = np.stack([tri + [x, 0.0, 0.0] for x in (0.0, 10.0, 20.0)])
    from test_oracle_lbvh import _scene_from_tris
    sc = _scene_from_tris(tris)
    G = fb.Scene.from_numpy(sc)
    G.build(sc.identity_xforms())
    assert G.info()["n4"] == 1
    # 4 rays per triangle through (x + 0.25, 0.25) along -z, then 4 rays above every box
    o = np.array([[x + 0.25, 0.25, 5.0] for x in (0.0, 10.0, 20.0) for _ in range(4)] +
                 [[x, 5.0, 5.0] for x in (0.0, 10.0, 20.0, 30.0)], np.float32)
    d = np.tile(np.array([[0.0, 0.0, -1.0]], np.float32), (len(o), 1))
    st = G.trace_stats(o, d, group=4)
    assert st["rays"] == 16 and st["groups"] == 4 and st["bad_loads"] == 0 and st["err"] == 0
    assert st["node_steps"] == 16
    assert st["tri_tests"] == 12
    assert st["group_nodes"] == 4
    assert st["group_tris"] == 3
    st1 = G.trace_stats(o, d, group=1, per_ray=True)
    assert st1["groups"] == 16 and st1["group_nodes"] == 16 and st1["group_tris"] == 12
    assert (st1["steps"] == 1).all()
    prim, _, _, _ = G.trace_host(o, d)
    assert (prim[:12] >= 0).all() and (prim[12:] == -1).all()


def test_trace_stats_invariants_on_camera_rays(fb):
    """Camera rays of a moving scene in warps of 32: counts add up, the
    distinct nodes and records per warp never exceed its fetches, warps
    share nodes (fewer distinct nodes than steps), and the any-hit counts
    of the dumped shadow rays follow the same rules."""
    import torch
    w, G = _moving_scene(fb, frames=2)
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 64, 32, 4)
    o, d = _camera_rays(cam)
    st = G.trace_stats(o, d, group=32)
    n = len(o)
    assert st["rays"] == n and st["groups"] == -(-n // 32) and st["bad_loads"] == 0 and st["err"] == 0
    assert n <= st["node_steps"] and st["group_nodes"] < st["node_steps"]
    assert st["group_tris"] <= st["tri_tests"]
    one = G.trace_stats(o, d, group=1, per_ray=True)
    assert one["node_steps"] == st["node_steps"] and one["tri_tests"] == st["tri_tests"]
    assert int(one["steps"].sum()) == one["node_steps"] and (one["steps"] >= 1).all()
    # a ray fetches a node and tests a triangle at most once (a tree)
    assert st["group_nodes"] < one["group_nodes"] == one["node_steps"]
    assert one["group_tris"] == one["tri_tests"]
    gb = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    G.render(cam, w.lights, out=torch.zeros((cam.height, cam.width, 4), device="cuda"), gbuf=gb)
    g = gbuf_of(gb)
    q = G.dump("shadow_rays")
    sid = q[:, 7].view(np.int32) >> 3
    ss = G.trace_stats(q[:, 0:3], q[:, 4:7], tmax=q[:, 3], skip=g["prim"][sid], any_hit=True, group=32)
    assert ss["rays"] == len(q) and ss["err"] == 0 and ss["bad_loads"] == 0
    assert len(q) <= ss["node_steps"] and ss["group_nodes"] < ss["node_steps"]
    assert ss["group_tris"] <= ss["tri_tests"]


def test_trace_stats_edges(fb):
    """No rays: all counts zero; a group longer than the input: one group
    (a one-triangle tree holds its triangle on both sides of its only node:
    two tests per ray, one distinct record); a group size below 1 is
    refused."""
    tri = np.array([[[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]])
    from test_oracle_lbvh import _scene_from_tris
    sc = _scene_from_tris(tri)
    G = fb.Scene.from_numpy(sc)
    G.build(sc.identity_xforms())
    e = np.zeros((0, 3), np.float32)
    st = G.trace_stats(e, e, group=32)
    assert all(v == 0 for v in st.values()), st
    o = np.array([[0.25, 0.25, 1.0]] * 5, np.float32)
    d = np.array([[0.0, 0.0, -1.0]] * 5, np.float32)
    st = G.trace_stats(o, d, group=64)
    assert st["groups"] == 1 and st["rays"] == 5 and st["tri_tests"] == 10 and st["group_tris"] == 1
    with pytest.raises(fb.FireError):
        G.trace_stats(o, d, group=0)


def test_two_level_dump_and_stats(fb):
    """Two-level scene: the dumped shadow rays, walked on the host with the
    sample's triangle skipped, give the device's visibility bits; the
    statistics count top-level and bottom-level node fetches alike (at
    least one per ray: the top root) and keep their invariants."""
    import torch
    w = sg.workload_frame7m(nspheres=120, cells=64)
    G = fb.Scene.from_numpy(w.scene)
    G.set_two_level(True)
    G.build(w.motion.xforms())
    for _ in range(2):
        G.refit(w.motion.step())
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 64, 36, 4)
    n = cam.width * cam.height * cam.spp
    gb = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    G.render(cam, w.lights, out=torch.zeros((cam.height, cam.width, 4), device="cuda"), gbuf=gb)
    g = gbuf_of(gb)
    q = G.dump("shadow_rays")
    tag = q[:, 7].view(np.int32)
    sid, light = tag >> 3, tag & 7
    assert len(q) == G.render_info()["shadow_rays"] > 50
    _, _, occ, err = G.trace_host(q[:, 0:3], q[:, 4:7], tmax=q[:, 3], skip=g["prim"][sid], any_hit=True)
    assert err == 0, hex(err)
    assert np.array_equal(~occ, ((g["vis"][sid] >> light) & 1).astype(bool))
    o, d = _camera_rays(cam)
    st = G.trace_stats(o, d, group=32, per_ray=True)
    assert st["rays"] == n and st["err"] == 0 and st["bad_loads"] == 0
    assert (st["steps"] >= 1).all() and int(st["steps"].sum()) == st["node_steps"]
    assert st["group_nodes"] < st["node_steps"] and st["group_tris"] <= st["tri_tests"]


def test_axis_aligned_rays_match_oracle(fb):
    """Rays along the coordinate axes (two direction components exactly 0,
    their reciprocals clamped to +-1e30, so the children's order keys are
    huge): nearest hits and any-hit answers of the kernels' traversal code
    equal the oracle's, and no error bit is set."""
    w, G = _moving_scene(fb, frames=1)
    S = oracle.OracleScene(w.scene)
    S.update(w.motion.xforms(), rebuild=True)
    rng = np.random.default_rng(11)
    n = 3000
    o = rng.uniform([-12, -3, -12], [12, 5, 12], (n, 3)).astype(np.float32)
    d = np.zeros((n, 3), np.float32)
    axis = rng.integers(0, 3, n)
    d[np.arange(n), axis] = np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    prim, t, _, err = G.trace_host(o, d)
    assert err == 0, hex(err)
    rp, rt, _, _, rt2 = S.trace(o, d, want_t2=True)
    bad = (prim != rp) | ((prim >= 0) & (t != rt))
    with np.errstate(invalid="ignore"):
        tie = np.isfinite(rt2) & (np.abs(rt2 - rt) <= TIE_REL * np.abs(rt))
    assert not (bad & ~tie).any(), int(bad.sum())
    assert 0.05 < (rp >= 0).mean() < 0.95
    L = rng.uniform(0.5, 20.0, n).astype(np.float32)
    _, _, hit, err = G.trace_host(o, d, tmax=L, any_hit=True)
    assert err == 0, hex(err)
    assert np.array_equal(hit, S.occluded(o, d, L, np.full(n, -1, np.int32)))


def test_shadow_dump_edges(fb):
    """Before any render the shadow-ray dump is empty; a byte count that is
    not the exact size is refused."""
    import ctypes as C

    from paper_2410_05095_b300 import fire
    tri = np.array([[[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]])
    from test_oracle_lbvh import _scene_from_tris
    sc = _scene_from_tris(tri)
    G = fb.Scene.from_numpy(sc)
    G.build(sc.identity_xforms())
    assert G.dump("shadow_rays").shape == (0, 8)
    buf = np.zeros(8, np.float32)
    rc = fire.lib().fire_debug_dump(G.h, 12, buf.ctypes.data_as(C.c_void_p), 32)
    assert fire.ERRORS.get(rc) == "FIRE_ERR_INVALID_ARG"
