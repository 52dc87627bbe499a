"""Pins for three legs of the oracle that the GPU parity tests lean on:

* directional lights (§IV-B-3 shadow rays, Fig. 5 several lights): radiance
  (f_d + f_s) I (n.l) with no distance falloff, the light direction
  normalised, and a shadow that is the PARALLEL projection of an occluder
  (shadow rays of unbounded length);
* the 4-sample rotated grid (§IV-B-2 multisampling): every sample's ray
  equals the pinhole ray through its own sub-pixel offset, computed here in
  FP64 from the camera definition, in sample order k = 0..3;
* the 4-spp box resolve (§IV-B-2 resolve): a pixel is the mean of its four
  sample radiances and its alpha the fraction of samples that hit, checked on
  a quad whose edges cross the image.

Each expected value is computed here from the definitions in FP64; nothing
is read back from the oracle except the image or ray under test.
"""
import math

import numpy as np

import oracle
import scenegen as sg
from test_oracle_lbvh import _scene_from_tris

GRID4 = [(-0.125, -0.375), (0.375, -0.125), (-0.375, 0.125), (0.125, 0.375)]


def _pinhole(cam, x, y, ox, oy):
    """FP64 ray of the point (x + 0.5 + ox, y + 0.5 + oy) of the image plane:
    f = normalize(target - pos), r = normalize(f x up), u = r x f,
    s_x = (2 fx / W - 1) tan(fov/2) W/H, s_y = (1 - 2 fy / H) tan(fov/2)."""
    pos = np.array(cam.pos, np.float64)
    f = np.array(cam.target, np.float64) - pos
    f /= np.linalg.norm(f)
    r = np.cross(f, np.array(cam.up, np.float64))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = math.tan(math.radians(cam.vfov_deg) / 2)
    sx = (2 * (x + 0.5 + ox) / cam.width - 1) * th * cam.width / cam.height
    sy = (1 - 2 * (y + 0.5 + oy) / cam.height) * th
    d = sx * r + sy * u + f
    return pos, d / np.linalg.norm(d)


def _plane(half=50.0, extra=()):
    plane = [[[-half, 0, -half], [half, 0, -half], [half, 0, half]],
             [[-half, 0, -half], [half, 0, half], [-half, 0, half]]]
    tris = np.concatenate([np.array(plane, np.float64), np.asarray(extra, np.float64).reshape(-1, 3, 3)])
    return _scene_from_tris(tris)


def _ident(S):
    S.update(np.eye(3, 4, dtype=np.float32).reshape(1, 12), rebuild=True)


# --------------------------------------------------------------------------- grid
def test_rotated_grid_sample_rays():
    """Each of the four samples of a pixel is the pinhole ray through its own
    offset: (-1/8,-3/8), (3/8,-1/8), (-3/8,1/8), (1/8,3/8) pixels for k = 0..3
    (x to the right, y down).  A non-square, tilted camera, so a swapped
    (x, y), a mirrored grid or a permuted sample order moves some ray by
    about a quarter pixel (~1e-2 rad here), far above the FP32 rounding."""
    cam = sg.Camera((1.0, 2.5, 7.0), (-0.5, 0.3, -1.0), (0.2, 1.0, 0.1), 55.0, 37, 23, 4)
    worst = 0.0
    for (x, y) in [(0, 0), (36, 0), (0, 22), (36, 22), (18, 11), (5, 17), (29, 3)]:
        for k, (ox, oy) in enumerate(GRID4):
            o, d = oracle.camera_ray(cam, x, y, k)
            _, want = _pinhole(cam, x, y, ox, oy)
            assert np.allclose(o, cam.pos)
            worst = max(worst, float(np.abs(d.astype(np.float64) - want).max()))
            # and no other grid position is as close (the ray is identified)
            for k2, (ox2, oy2) in enumerate(GRID4 + [(oy, ox) for (ox, oy) in GRID4]):
                if (ox2, oy2) == (ox, oy):
                    continue
                _, other = _pinhole(cam, x, y, ox2, oy2)
                assert np.abs(d.astype(np.float64) - other).max() > 1e-3
    assert worst < 1e-6, worst
    # one sample per pixel: the pixel centre
    cam1 = sg.Camera(cam.pos, cam.target, cam.up, cam.vfov_deg, cam.width, cam.height, 1)
    _, d = oracle.camera_ray(cam1, 7, 9, 0)
    _, want = _pinhole(cam1, 7, 9, 0.0, 0.0)
    assert np.abs(d - want).max() < 1e-6


def test_sample_ids_follow_grid_order():
    """render_samples' sample id (y W + x) spp + k is sample k of pixel
    (x, y): the hit distance on the plane y = 0 equals -o_y / d_y of the FP64
    ray through offset k."""
    S = oracle.OracleScene(_plane())
    _ident(S)
    cam = sg.Camera((0.3, 6.0, 0.1), (0.8, 0.0, -0.4), (0.0, 1.0, 0.0), 50.0, 21, 15, 4)
    ids = np.arange(cam.width * cam.height * 4)
    out = S.render_samples(cam, [], ids, want_t2=False)
    assert (out["prim"] >= 0).all()
    worst = 0.0
    for i in ids[::7]:
        k, pix = int(i % 4), int(i // 4)
        x, y = pix % cam.width, pix // cam.width
        o, d = _pinhole(cam, x, y, *GRID4[k])
        worst = max(worst, abs(float(out["t"][i]) - (-o[1] / d[1])) / (-o[1] / d[1]))
    assert worst < 2e-6, worst


# ------------------------------------------------------------------ directional
def _dir_light(v, intensity=2.0):
    return sg.Light(1, tuple(float(a) for a in v), intensity)


def test_directional_light_closed_form():
    """Camera above a large plane, one directional light given by an
    UNNORMALISED direction towards the light: every pixel equals
    (f_d + f_s)(n, v, l) I (n.l) in FP64 with l = v/|v| and no 1/d^2 --
    the same value at every distance from any point."""
    sc = _plane()
    sc.mats[0]["albedo"] = [0.6, 0.35, 0.15]
    v_raw = np.array([0.6, 2.0, 1.0])
    l = v_raw / np.linalg.norm(v_raw)
    n = np.array([0.0, 1.0, 0.0])
    for rough, metal in ((0.45, 0.0), (0.75, 1.0), (0.2, 0.0)):
        sc.mats[0]["roughness"], sc.mats[0]["metallic"] = rough, metal
        S = oracle.OracleScene(sc)
        _ident(S)
        cam = sg.Camera((0.37, 10.0, 0.21), (0.37, 0.0, 0.21), (0.0, 0.0, -1.0), 60.0, 31, 25, 1)
        img = S.render_image(cam, [_dir_light(v_raw, 2.0)])
        worst = 0.0
        for y in range(cam.height):
            for x in range(cam.width):
                o, d = _pinhole(cam, x, y, 0.0, 0.0)
                fd, fs = oracle.brdf_f64(n, -d, l, sc.mats[0]["albedo"], rough, metal)
                want = (fd + fs) * 2.0 * l[1]
                h = (l - d) / np.linalg.norm(l - d)
                dd = h[1] ** 2 * (rough ** 4 - 1) + 1
                tol = 1e-5 + 2.0 ** -21 / dd  # FP32 conditioning of D near its peak
                worst = max(worst, float(np.max(np.abs(img[y, x, :3] - want) / want)) / tol)
                assert img[y, x, 3] == 1.0
        assert worst < 1.0, (rough, metal, worst)
    # a light below the horizon casts nothing: black, still covered
    S = oracle.OracleScene(sc)
    _ident(S)
    img = S.render_image(sg.Camera((0.37, 10.0, 0.21), (0.37, 0.0, 0.21), (0.0, 0.0, -1.0), 60.0, 9, 7, 1),
                         [_dir_light(-v_raw)])
    assert np.all(img[..., :3] == 0.0) and np.all(img[..., 3] == 1.0)


def test_directional_shadow_is_parallel_projection():
    """A triangle occluder at height 3 over the plane, lit by a directional
    light: the shadow is the occluder projected ALONG l onto the plane of the
    lifted shadow-ray origins (y = eps) -- parallel, not central -- and the
    shadow rays reach it at any distance (t_max = inf: an occluder further
    than |v| = 1 still shadows).  Samples outside a 1e-4 band around the
    projected edges must agree."""
    occ = np.array([[-1.2, 3.0, -0.9], [1.6, 3.0, -0.4], [0.1, 3.0, 1.3]])
    S = oracle.OracleScene(_plane(extra=occ))
    _ident(S)
    eps = S.shadow_eps()
    v_raw = np.array([0.9, 2.5, -0.6])
    l = v_raw / np.linalg.norm(v_raw)
    cam = sg.Camera((2.0, 12.0, 4.0), (-0.9, 0.0, 0.7), (0.0, 1.0, 0.0), 30.0, 71, 61, 1)
    n = cam.width * cam.height
    out = S.render_samples(cam, [_dir_light(v_raw)], np.arange(n), want_t2=False)
    proj = occ - ((occ[:, 1] - eps) / l[1])[:, None] * l
    a, b, c = proj[:, [0, 2]]
    checked = inside_n = 0
    for i in range(n):
        if out["prim"][i] not in (0, 1):  # the plane only (the occluder itself is lit)
            continue
        o, d = _pinhole(cam, i % cam.width, i // cam.width, 0.0, 0.0)
        p = (o + float(out["t"][i]) * d)[[0, 2]]

        def edge(u, w):
            e = w - u
            return (e[0] * (p - u)[1] - e[1] * (p - u)[0]) / np.linalg.norm(e)
        ds = [edge(a, b), edge(b, c), edge(c, a)]
        if min(abs(x) for x in ds) < 1e-4:
            continue
        inside = all(x > 0 for x in ds) or all(x < 0 for x in ds)
        assert out["vis"][i] & 0x100, i            # cast (n.l > 0 everywhere on the plane)
        assert bool(out["vis"][i] & 1) == (not inside), i
        checked += 1
        inside_n += inside
    assert checked > 2500 and inside_n > 150, (checked, inside_n)


# ---------------------------------------------------------------------- resolve
def test_four_sample_resolve_closed_form():
    """A 3 x 2 quad on y = 0, turned 20 degrees about y, seen from above at 4 spp with one point light;
    the quad's edges cross the image.  Expected pixel = the mean of the four
    FP64 sample radiances (f_d + f_s) I cos / d^2 at the rotated-grid
    sample points (0 for a sample that misses), alpha = hits / 4.  Edge
    pixels have alpha 1/4, 1/2 or 3/4, so a wrong grid, a wrong sample
    count or a wrong divisor changes them."""
    cth, sth = math.cos(0.35), math.sin(0.35)  # edges oblique to the pixel grid
    rot = np.array([[cth, 0, -sth], [0, 1, 0], [sth, 0, cth]])  # local (x, z) -> world
    quad = np.array([[[-1.5, 0, -1], [1.5, 0, -1], [1.5, 0, 1]], [[-1.5, 0, -1], [1.5, 0, 1], [-1.5, 0, 1]]])
    sc = _scene_from_tris(quad @ rot.T)
    sc.mats[0]["albedo"], sc.mats[0]["roughness"], sc.mats[0]["metallic"] = [0.55, 0.4, 0.25], 0.5, 0.0
    S = oracle.OracleScene(sc)
    _ident(S)
    eps = S.shadow_eps()
    cam = sg.Camera((0.13, 4.0, 0.07), (0.13, 0.0, 0.07), (0.0, 0.0, -1.0), 60.0, 41, 29, 4)
    light = np.array([2.0, 6.0, -1.5])
    img = S.render_image(cam, [sg.Light(0, tuple(light), 80.0)])
    nrm = np.array([0.0, 1.0, 0.0])
    mat = sc.mats[0]
    checked = 0
    partial = set()
    for y in range(cam.height):
        for x in range(cam.width):
            acc, hits, ambiguous = np.zeros(3), 0, False
            for (ox, oy) in GRID4:
                o, d = _pinhole(cam, x, y, ox, oy)
                p = o + (-o[1] / d[1]) * d
                q = rot.T @ p  # quad-local coordinates
                mx, mz = 1.5 - abs(q[0]), 1.0 - abs(q[2])
                # (the shared diagonal z = 2x/3 may be missed by both triangles
                # of a non-watertight test; an edge within 1e-5 is undecided)
                if min(abs(mx), abs(mz)) < 1e-5 or abs(q[2] - q[0] / 1.5) < 1e-5:
                    ambiguous = True
                if mx < 0 or mz < 0:
                    continue
                hits += 1
                po = p + eps * nrm
                L = light - po
                d2 = L @ L
                lv = L / math.sqrt(d2)
                fd, fs = oracle.brdf_f64(nrm, -d, lv, mat["albedo"], mat["roughness"], mat["metallic"])
                acc += (fd + fs) * 80.0 * lv[1] / d2
            if ambiguous:
                continue
            want = acc / 4.0
            assert img[y, x, 3] == hits / 4.0, (x, y, img[y, x, 3], hits)
            if hits:
                assert np.all(np.abs(img[y, x, :3] - want) <= 1e-5 * want + 1e-7), (x, y, img[y, x, :3], want)
                if hits < 4:
                    partial.add(hits)
            else:
                assert np.all(img[y, x, :3] == 0.0)
            checked += 1
    assert checked > 0.9 * cam.width * cam.height
    assert partial == {1, 2, 3}, partial
