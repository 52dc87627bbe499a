"""Pins of the oracle's smooth shading normals and sRGB albedo decode (§IV-A-1:
the main pass shades with per-vertex normals and decodes sRGB colour inputs
to linear).  Each pin checks the oracle against something it does not
compute itself: barycentric interpolation of a linear field (exact for any
correct weights), equivariance under a body rotation, the flat special case,
the analytic normal of a sphere, the published sRGB transfer values and the
display stage's independent encoder."""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg


def _patch_scene(seed=7, cells=6, half=2.0):
    v, f = sg.terrain(sg.Rng(seed), cells, half=half, y_offset=0.0)
    return sg.assemble([(v, f)], 1, sg.random_materials(sg.Rng(seed + 1), 1))


def _down_rays(rng, n, half=1.6):
    o = np.array([[rng.uniform(-half, half), 6.0, rng.uniform(-half, half)] for _ in range(n)], np.float32)
    d = np.array([sg.Rng(i + 99).unit_vector() * 0.15 + np.array([0, -1.0, 0]) for i in range(n)])
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    return o, d


def _facing_geometric(sc, xf, prim, d):
    """FP64 geometric normal of the world-space triangle, turned against d."""
    M = np.asarray(xf, np.float64).reshape(-1, 3, 4)[0]
    R, t = M[:, :3], M[:, 3]
    p = sc.verts[sc.idx[prim], :3].astype(np.float64) @ R.T + t
    n = np.cross(p[1] - p[0], p[2] - p[0])
    n /= np.linalg.norm(n)
    return -n if n @ d > 0 else n


def _linear_normals(sc, A, b):
    out = np.zeros((sc.nv, 4), np.float32)
    out[:, :3] = sc.verts[:, :3].astype(np.float64) @ A.T + b
    return out


def test_linear_field_is_interpolated_exactly():
    """Vertex normals n_i = A v_i + b (a linear field, not unit): at the hit
    point p, barycentric interpolation must give A p + b, whatever the
    triangle -- a swapped weight or a wrong w0 breaks it."""
    sc = _patch_scene()
    rng = np.random.default_rng(3)
    A, b = rng.normal(size=(3, 3)), np.array([0.3, 2.5, -0.4])
    S = oracle.OracleScene(sc)
    xf = sc.identity_xforms()
    S.update(xf, rebuild=True)
    S.set_normals(_linear_normals(sc, A, b))
    o, d = _down_rays(sg.Rng(11), 200)
    prim, t, _, _ = S.trace(o, d)
    assert (prim >= 0).sum() > 150
    worst = 0.0
    for i in np.flatnonzero(prim >= 0):
        p = o[i].astype(np.float64) + float(t[i]) * d[i].astype(np.float64)
        want = A @ p + b
        want /= np.linalg.norm(want)
        ng = _facing_geometric(sc, xf, prim[i], d[i].astype(np.float64))
        if want @ ng < 0:
            want = -want
        got = S.shading_normal(prim[i], o[i], d[i]).astype(np.float64)
        worst = max(worst, np.abs(got - want).max())
    assert worst < 2e-5, worst


def test_normals_turn_with_the_body():
    """Same field in the rest frame, body posed with a rotation R and a
    translation: the shading normal is R times the rest-frame one (R^T, or
    a translated normal, would fail)."""
    sc = _patch_scene(seed=21)
    rng = np.random.default_rng(5)
    A, b = rng.normal(size=(3, 3)), np.array([0.1, 3.0, 0.2])
    ax = rng.normal(size=3)
    ax /= np.linalg.norm(ax)
    ang = 0.7
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    R = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)
    tr = np.array([0.4, -0.2, 0.3])
    xf = np.zeros((1, 12), np.float32)
    xf[0] = np.concatenate([R, tr[:, None]], axis=1).reshape(-1)
    S = oracle.OracleScene(sc)
    S.update(xf, rebuild=True)
    S.set_normals(_linear_normals(sc, A, b))
    # rays aimed at the posed patch from above its (rotated) normal side
    up = R @ np.array([0.0, 1.0, 0.0])
    o0, _ = _down_rays(sg.Rng(12), 200, half=1.2)
    o = ((o0.astype(np.float64) - [0, 6.0, 0]) @ R.T + tr + 6.0 * up).astype(np.float32)
    d = np.tile((-up).astype(np.float32), (len(o), 1))
    prim, t, _, _ = S.trace(o, d)
    hits = np.flatnonzero(prim >= 0)
    assert len(hits) > 150
    worst = 0.0
    for i in hits:
        pw = o[i].astype(np.float64) + float(t[i]) * d[i].astype(np.float64)
        pr = R.T @ (pw - tr)
        want = R @ (A @ pr + b)
        want /= np.linalg.norm(want)
        ng = _facing_geometric(sc, xf, prim[i], d[i].astype(np.float64))
        if want @ ng < 0:
            want = -want
        got = S.shading_normal(prim[i], o[i], d[i]).astype(np.float64)
        worst = max(worst, np.abs(got - want).max())
    assert worst < 5e-5, worst


def test_face_normals_reduce_to_flat_shading():
    """Unshared vertices whose normals are their triangle's face normal:
    smooth shading equals flat shading up to rounding, sample by sample."""
    v, idx = sg.random_soup(sg.Rng(31), 300, extent=1.5, size=0.5)
    sc = sg.Scene(verts=v, idx=idx, tri_mat=np.zeros(len(idx), np.uint32),
                  vert_body=np.zeros(len(v), np.uint16), mats=sg.random_materials(sg.Rng(32), 1), nbody=1)
    p = v[:, :3].astype(np.float64)
    fn = np.cross(p[1::3] - p[0::3], p[2::3] - p[0::3])
    fn /= np.linalg.norm(fn, axis=1, keepdims=True)
    nrm = np.zeros((len(v), 4), np.float32)
    nrm[:, :3] = np.repeat(fn, 3, axis=0)
    cam = sg.Camera((0.5, 1.0, 6.0), (0, 0, 0), (0, 1, 0), 50.0, 48, 40, 4)
    lights = [sg.Light(0, (3.0, 4.0, 5.0), 60.0), sg.Light(1, (-0.3, 1.0, 0.4), 1.5)]
    S = oracle.OracleScene(sc)
    S.update(sc.identity_xforms(), rebuild=True)
    flat = S.render_all_samples(cam, lights)
    S.set_normals(nrm)
    smooth = S.render_all_samples(cam, lights)
    assert np.array_equal(flat["prim"], smooth["prim"])
    hit = flat["prim"] >= 0
    assert hit.mean() > 0.2
    # the normals themselves: the FP64 face normal, facing the ray, to rounding
    ids = np.flatnonzero(hit)[::7]
    for i in ids:
        k = int(i % cam.spp)
        x, y = int((i // cam.spp) % cam.width), int((i // cam.spp) // cam.width)
        o3, d3 = oracle.camera_ray(cam, x, y, k)
        ns = S.shading_normal(flat["prim"][i], o3, d3).astype(np.float64)
        ng = _facing_geometric(sc, sc.identity_xforms(), flat["prim"][i], d3.astype(np.float64))
        assert np.abs(ns - ng).max() < 1e-6
    # the cast decision can flip only where n.l is within rounding of 0; the
    # radiance moves by the BRDF's sensitivity to a ~1e-7 rad normal change
    # (GGX peaks sharply at roughness 0.05)
    same_vis = flat["vis"] == smooth["vis"]
    assert same_vis.mean() > 0.999
    d = np.abs(flat["rgb"] - smooth["rgb"])[same_vis]
    assert d.max() <= 1e-3 * max(1.0, np.abs(flat["rgb"]).max())


def test_sphere_normals_are_radial():
    """Vertices on a sphere with their exact radial normals: at a point p of
    a flat triangle the interpolated normal is sum w_i (v_i - c) / r =
    (p - c) / r, so the shading normal is the radial direction of p itself,
    to FP32 rounding.  (The area-weighted normals of the scene generator
    stay within 1e-2 of radial on the same mesh.)"""
    v, f = sg.icosphere(4)
    c, r = np.array([0.2, -0.1, 0.3]), 1.7
    sc = sg.assemble([(v * r + c, f)], 1, sg.random_materials(sg.Rng(41), 1))
    S = oracle.OracleScene(sc)
    S.update(sc.identity_xforms(), rebuild=True)
    radial_n = np.zeros((sc.nv, 4), np.float32)
    radial_n[:, :3] = (sc.verts[:, :3].astype(np.float64) - c) / r
    gen = sg.vertex_normals(sc)
    assert np.abs(gen[:, :3] - radial_n[:, :3]).max() < 1e-2
    S.set_normals(radial_n)
    rng = sg.Rng(42)
    o = np.array([c + 5.0 * rng.unit_vector() for _ in range(300)], np.float32)
    tgt = np.array([c + 0.8 * r * rng.unit_vector() for _ in range(300)])
    d = tgt - o
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    prim, t, _, _ = S.trace(o, d)
    assert (prim >= 0).all()
    worst = 0.0
    for i in range(len(o)):
        p = o[i].astype(np.float64) + float(t[i]) * d[i].astype(np.float64)
        radial = (p - c) / np.linalg.norm(p - c)
        worst = max(worst, np.abs(S.shading_normal(prim[i], o[i], d[i]) - radial).max())
    assert worst < 2e-5, worst


def test_shading_normal_is_unit_and_faces_the_viewer_side():
    w = sg.workload_tiny41k()
    sc = w.scene
    S = oracle.OracleScene(sc)
    S.update(sc.identity_xforms(), rebuild=True)
    S.set_normals(sg.vertex_normals(sc))
    o, d = sg.random_rays(sg.Rng(51), 400, (-6, 1, -6), (6, 8, 6), (-3, -2, -3), (3, 2, 3))
    prim, t, _, _ = S.trace(o, d)
    xf = sc.identity_xforms()
    n_hit = 0
    for i in np.flatnonzero(prim >= 0):
        ns = S.shading_normal(prim[i], o[i], d[i]).astype(np.float64)
        assert abs(np.linalg.norm(ns) - 1.0) < 1e-6
        assert ns @ _facing_geometric(sc, xf, prim[i], d[i].astype(np.float64)) >= 0.0
        n_hit += 1
    assert n_hit > 100


def test_shadow_rays_are_cast_by_the_shading_normal():
    """One upward-facing triangle seen from above; a directional light just
    below its plane.  Flat: n.l < 0, no shadow ray, black.  Vertex normals
    tilted toward the light: n_s.l > 0, the ray is cast (bit 8), meets
    nothing (the hit triangle is skipped) and the sample is lit."""
    v = np.array([[-2, 0, -2, 1], [2, 0, -2, 1], [0, 0, 2, 1]], np.float32)
    idx = np.array([[0, 2, 1]], np.uint32)
    sc = sg.Scene(verts=v, idx=idx, tri_mat=np.zeros(1, np.uint32), vert_body=np.zeros(3, np.uint16),
                  mats=sg.random_materials(sg.Rng(61), 1), nbody=1)
    cam = sg.Camera((0.0, 5.0, 0.3), (0, 0, 0), (0, 0, -1), 20.0, 8, 8, 1)
    lights = [sg.Light(1, (1.0, -0.2, 0.0), 2.0)]
    S = oracle.OracleScene(sc)
    S.update(sc.identity_xforms(), rebuild=True)
    flat = S.render_all_samples(cam, lights)
    hit = flat["prim"] >= 0
    assert hit.mean() > 0.5
    assert (flat["vis"] == 0).all() and (flat["rgb"] == 0).all()
    tilt = np.zeros((3, 4), np.float32)
    tilt[:, :3] = np.array([1.0, 0.5, 0.0]) / math.sqrt(1.25)
    S.set_normals(tilt)
    sm = S.render_all_samples(cam, lights)
    assert (sm["vis"][hit] == (1 << 8) | 1).all() and (sm["vis"][~hit] == 0).all()
    assert (sm["rgb"][hit] > 0).all()


@pytest.mark.parametrize("c,want", [(0.0, 0.0), (1.0, 1.0), (0.5, 0.21404114),
                                    (128 / 255, 0.21586050), (64 / 255, 0.05126946),
                                    (0.04045, 0.0031308)])
def test_srgb_decode_published_values(c, want):
    """IEC 61966-2-1 transfer values (0.5 -> 0.2140, 128/255 -> 0.2159,
    64/255 -> 0.0513, and the breakpoint pair 0.04045 <-> 0.0031308)."""
    assert abs(oracle.srgb_decode(c) - want) <= 2e-7 + 1e-6 * want


def test_srgb_decode_inverts_the_display_encoder():
    """The display stage's encoder (its own Newton 12th root, pinned in
    test_oracle_display.py) undoes the decode across [0, 1]."""
    for c in np.linspace(0.0, 1.0, 2001):
        lin = oracle.srgb_decode(float(c))
        assert abs(oracle.srgb_encode(lin) - c) < 3e-6
    xs = np.linspace(0.0, 1.0, 4001)
    ys = np.array([oracle.srgb_decode(float(x)) for x in xs])
    assert (np.diff(ys) > 0).all()


def test_srgb_materials_decode_albedo_only():
    """sRGB materials render exactly like linear materials holding the
    decoded albedo (roughness and metallic are not colours)."""
    w = sg.workload_tiny41k()
    sc = w.scene
    cam = sg.Camera((0.0, 4.0, 12.0), (0, 0, 0), (0, 1, 0), 60.0, 40, 24, 1)
    S = oracle.OracleScene(sc)
    S.update(sc.identity_xforms(), rebuild=True)
    S.set_materials_srgb(sc.mats)
    a = S.render_image(cam, w.lights)
    lin = sc.mats.copy()
    for i in range(len(lin)):
        lin[i]["albedo"] = [oracle.srgb_decode(float(x)) for x in sc.mats[i]["albedo"]]
    S.set_materials(lin)
    b = S.render_image(cam, w.lights)
    assert np.array_equal(a, b)
    S.set_materials(sc.mats)
    c = S.render_image(cam, w.lights)
    assert not np.array_equal(a, c)
