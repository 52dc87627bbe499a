"""Pins for the oracle's visibility path: BVH traversal against brute force,
ray/triangle closed forms, the camera model, and analytic hard-shadow
boundaries (§IV-B-3: a point is in shadow iff the segment to the light hits
opaque geometry)."""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg
from test_oracle_lbvh import _scene_from_tris


def _soup_scene(n, seed):
    v, idx = sg.random_soup(sg.Rng(seed), n)
    mats = sg.random_materials(sg.Rng(1), 1)
    return sg.Scene(verts=v, idx=idx, tri_mat=np.zeros(n, np.uint32),
                    vert_body=np.zeros(len(v), np.uint16), mats=mats, nbody=1)


@pytest.mark.parametrize("n", [1, 2, 10, 300, 2000])
def test_bvh_equals_brute_force_on_soups(n):
    S = oracle.OracleScene(_soup_scene(n, 10 + n))
    S.update(np.eye(3, 4, dtype=np.float32).reshape(1, 12), rebuild=True)
    o, d = sg.random_rays(sg.Rng(99 + n), 3000 if n < 2000 else 1500, [-2, -2, -2], [2, 2, 2])
    a = S.trace(o, d, bvh=True, want_t2=True)
    b = S.trace(o, d, bvh=False, want_t2=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert (a[0] >= 0).sum() > 50 or n < 10
    tmax = np.abs(np.array([sg.Rng(3).uniform(0.1, 3) for _ in range(len(o))], np.float32))
    skip = np.where(a[0] >= 0, a[0], -1).astype(np.int32)
    occ_bvh = S.occluded(o, d, tmax, skip, bvh=True)
    occ_brute = S.occluded(o, d, tmax, skip, bvh=False)
    assert np.array_equal(occ_bvh, occ_brute)


def test_quad_closed_form_and_shared_edge():
    """Ray straight down onto a horizontal quad at y = 0 from height 5: t = 5
    exactly; a ray through the shared diagonal hits both triangles at the
    same t and the smaller original index wins."""
    quad = np.array([[[-1, 0, -1], [1, 0, -1], [1, 0, 1]], [[-1, 0, -1], [1, 0, 1], [-1, 0, 1]]], np.float32)
    S = oracle.OracleScene(_scene_from_tris(quad))
    S.update(np.eye(3, 4, dtype=np.float32).reshape(1, 12), rebuild=True)
    o = np.array([[0.5, 5, -0.25], [-0.5, 5, 0.25], [0.25, 5, 0.25], [3, 5, 0]], np.float32)
    d = np.tile(np.array([[0, -1, 0]], np.float32), (4, 1))
    for bvh in (True, False):
        prim, t, u, v, t2 = S.trace(o, d, bvh=bvh, want_t2=True)
        assert prim.tolist() == [0, 1, 0, -1]
        assert t[:3].tolist() == [5.0, 5.0, 5.0]
        assert t2[2] == 5.0  # both triangles hit on the diagonal
        assert math.isinf(t2[0])
    # tmin excludes hits at or before it
    prim, t, _, _ = S.trace(o[:1], d[:1], tmin=5.0)
    assert prim[0] == -1


def test_tiny_scene_bvh_equals_brute(tiny41k):
    sc = tiny41k.scene
    S = oracle.OracleScene(sc)
    S.update(sc.identity_xforms(), rebuild=True)
    cam = sg.Camera(**{**tiny41k.camera.__dict__, "width": 24, "height": 24, "spp": 4})
    ids = np.arange(24 * 24 * 4)
    a = S.render_samples(cam, tiny41k.lights, ids, bvh=True)
    b = S.render_samples(cam, tiny41k.lights, ids, bvh=False)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert (a["prim"] >= 0).mean() > 0.5
    assert ((a["vis"] & 1) == 0).sum() > 0 and ((a["vis"] & 1) == 1).sum() > 0  # shadows and light


def test_camera_centre_and_edges():
    """Odd image: the centre sample's ray is the forward vector; the centre of
    the top row is tilted by atan((1 - 1/H) tan(fov/2)); the camera sits at
    its position."""
    cam = sg.Camera((1.0, 2.0, 3.0), (-2.0, 0.5, -1.0), (0.0, 1.0, 0.0), 50.0, 31, 21, 1)
    f = np.array(cam.target) - np.array(cam.pos)
    f /= np.linalg.norm(f)
    o, d = oracle.camera_ray(cam, 15, 10, 0)
    assert np.allclose(o, cam.pos)
    assert np.abs(d - f).max() < 3e-7
    _, d0 = oracle.camera_ray(cam, 15, 0, 0)
    ang = math.acos(min(1.0, float(np.dot(d0.astype(np.float64), f))))
    want = math.atan((1 - 1 / 21) * math.tan(math.radians(25)))
    assert abs(ang - want) < 1e-5
    assert np.dot(d0, [0, 1, 0]) > np.dot(d, [0, 1, 0])  # row 0 is the top
    _, dl = oracle.camera_ray(cam, 0, 10, 0)
    right = np.cross(f, [0, 1, 0])
    assert np.dot(dl, right) < 0  # column 0 is the left
    # 4-spp rotated grid: the four offsets average to the pixel centre
    cam4 = sg.Camera(cam.pos, cam.target, cam.up, cam.vfov_deg, cam.width, cam.height, 4)
    ds = np.array([oracle.camera_ray(cam4, 15, 10, k)[1] for k in range(4)], np.float64)
    assert np.abs(ds.mean(0) / np.linalg.norm(ds.mean(0)) - f).max() < 1e-6
    assert len({tuple(x) for x in ds}) == 4


def _plane_scene(extra_tris, half=50.0):
    plane = np.array([[[-half, 0, -half], [half, 0, -half], [half, 0, half]],
                      [[-half, 0, -half], [half, 0, half], [-half, 0, half]]])
    tris = np.concatenate([plane, np.asarray(extra_tris, np.float64).reshape(-1, 3, 3)])
    return _scene_from_tris(tris)


def _plane_hits(S, cam, lights):
    n = cam.width * cam.height
    out = S.render_samples(cam, lights, np.arange(n), bvh=True)
    pts = []
    for i in range(n):
        o, d = oracle.camera_ray(cam, i % cam.width, i // cam.width, 0)
        pts.append(o.astype(np.float64) + float(out["t"][i]) * d.astype(np.float64))
    return out, np.array(pts)


def test_triangle_shadow_is_central_projection():
    occ = np.array([[-1.0, 2.0, -1.0], [1.5, 2.0, -0.5], [0.0, 2.0, 1.2]])
    S = oracle.OracleScene(_plane_scene(occ))
    S.update(np.eye(3, 4, dtype=np.float32).reshape(1, 12), rebuild=True)
    eps = S.shadow_eps()
    light = np.array([0.3, 8.0, 0.2])
    cam = sg.Camera((5.0, 9.0, 5.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 40.0, 61, 61, 1)
    out, P = _plane_hits(S, cam, [sg.Light(0, tuple(light), 100.0)])
    # occluder projected from the light onto the plane y = eps (the shadow-ray origins)
    proj = light + (occ - light) * ((light[1] - eps) / (light[1] - occ[:, 1]))[:, None]
    a, b, c = proj[:, [0, 2]]
    checked = inside_n = 0
    for i in np.nonzero(out["prim"] <= 1)[0]:
        if out["prim"][i] < 0:
            continue
        p = P[i, [0, 2]]
        def edge(u, w):
            e = w - u
            return (e[0] * (p - u)[1] - e[1] * (p - u)[0]) / np.linalg.norm(e)
        ds = [edge(a, b), edge(b, c), edge(c, a)]
        inside = all(x > 0 for x in ds) or all(x < 0 for x in ds)
        if min(abs(x) for x in ds) < 1e-4:
            continue
        assert out["vis"][i] & 0x100
        assert bool(out["vis"][i] & 1) == (not inside), i
        checked += 1
        inside_n += inside
    assert checked > 1000 and inside_n > 50


def test_sphere_shadow_disc_radius():
    """Light at height H over a sphere of radius r centred at height h: the
    shadow on the plane is a disc of radius D r / sqrt((H-h)^2 - r^2), D the
    depth of the plane below the light; the tessellated sphere's shadow lies
    between the discs of its inscribed and circumscribed spheres."""
    uv, uf = sg.icosphere(4)
    H, h, r = 10.0, 2.0, 1.0
    verts = uv * r + [0, h, 0]
    tris = verts[uf]
    nrm = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r_in = np.abs(np.einsum("ij,ij->i", tris[:, 0] - [0, h, 0], nrm)).min()
    S = oracle.OracleScene(_plane_scene(tris))
    S.update(np.eye(3, 4, dtype=np.float32).reshape(1, 12), rebuild=True)
    eps = S.shadow_eps()
    D = H - eps
    R_out = D * r / math.sqrt((H - h) ** 2 - r ** 2)
    R_in = D * r_in / math.sqrt((H - h) ** 2 - r_in ** 2)
    cam = sg.Camera((4.0, 7.0, 0.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 35.0, 81, 81, 1)
    out, P = _plane_hits(S, cam, [sg.Light(0, (0.0, H, 0.0), 100.0)])
    n_in = n_out = 0
    for i in np.nonzero((out["prim"] >= 0) & (out["prim"] <= 1))[0]:
        rho = math.hypot(P[i, 0], P[i, 2])
        lit = bool(out["vis"][i] & 1)
        if rho < R_in * (1 - 1e-4):
            assert not lit
            n_in += 1
        elif rho > R_out * (1 + 1e-4):
            assert lit
            n_out += 1
    assert n_in > 100 and n_out > 1000
