"""Pins for the oracle's shading (§IV-B-1: Cook-Torrance with GGX D, Schlick
F, Schlick-GGX G; Lambert diffuse for the metallic-roughness workflow) and
its FP64 gradient: closed forms, normalisation integrals, a closed-form
image, and central finite differences."""
import math
import os

import numpy as np
import pytest

import oracle
import scenegen as sg
from test_oracle_trace import _plane_scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hemi_quad(fn, n_theta=400, n_phi=64):
    """Integral over the hemisphere of fn(direction) dOmega (midpoint rule in
    mu = cos theta and phi)."""
    tot = 0.0
    for i in range(n_theta):
        mu = (i + 0.5) / n_theta
        s = math.sqrt(1 - mu * mu)
        for j in range(n_phi):
            ph = 2 * math.pi * (j + 0.5) / n_phi
            tot += fn(np.array([s * math.cos(ph), mu, s * math.sin(ph)]))
    return tot * (1.0 / n_theta) * (2 * math.pi / n_phi)


@pytest.mark.parametrize("alpha", [0.0025, 0.04, 0.25, 0.6, 1.0])
def test_ggx_normalisation(alpha):
    """Integral of D(h) (n.h) dOmega_h = 1 (Walter et al. 2007); substitute
    u = tan^2(theta) so the narrow lobes integrate accurately:
    dOmega cos = 2 pi sin cos dtheta = pi / (1+u)^2 du."""
    def integrand(u):
        c2 = 1.0 / (1.0 + u)
        return oracle.ggx_d(math.sqrt(c2), alpha) * math.pi / (1.0 + u) ** 2
    # integrate u in [0, inf) with u = a2 * tan(w)^2-ish mapping: u = a2 * s/(1-s)
    a2 = alpha * alpha
    N = 20000
    tot = 0.0
    for i in range(N):
        s = (i + 0.5) / N
        u = a2 * s / (1 - s)
        tot += integrand(u) * a2 / (1 - s) ** 2 / N
    assert abs(tot - 1.0) < 1e-6
    assert abs(oracle.ggx_d(1.0, alpha) - 1.0 / (math.pi * alpha * alpha)) < 1e-9 / alpha ** 2


def test_schlick_and_smith_closed_forms():
    for f0 in (0.04, 0.5, 0.95):
        assert oracle.schlick_f(1.0, f0) == f0
        assert oracle.schlick_f(0.0, f0) == 1.0
        assert abs(oracle.schlick_f(0.5, f0) - (f0 + (1 - f0) / 32)) < 1e-15
    # G1(1) = 1 for any k; r = 1 -> k = 1/2 -> G1(1/2) = 2/3; kmode 1, r = 1 -> k = 1/2 too
    for r in (0.05, 0.5, 1.0):
        assert oracle.smith_g(1.0, 1.0, r) == 1.0
    assert abs(oracle.smith_g(0.5, 1.0, 1.0) - 2.0 / 3.0) < 1e-15
    assert abs(oracle.smith_g(0.5, 0.5, 1.0, kmode=1) - 4.0 / 9.0) < 1e-15
    # r = 0.5 -> k = 2.25/8 = 0.28125
    assert abs(oracle.smith_g(0.25, 1.0, 0.5) - 0.25 / (0.25 * 0.71875 + 0.28125)) < 1e-15
    rng = sg.Rng(3)
    for _ in range(200):
        g = oracle.smith_g(rng.u(), rng.u(), rng.uniform(0.05, 1))
        assert 0.0 <= g <= 1.0


def _golden_brdf():
    rows = []
    for line in open(os.path.join(GOLDEN, "brdf_normal_incidence.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return rows


def test_brdf_normal_incidence_golden():
    """At l = v = n: h = n, D = 1/(pi a^2), F = F0, G = 1, so
    f_s = F0 / (4 pi a^2) and f_d = (1 - F0)(1 - m) albedo / pi; values of
    tests/golden/brdf_normal_incidence.txt."""
    n = np.array([0.0, 1.0, 0.0])
    for alb, r, m, fd_want, fs_want in _golden_brdf():
        fd, fs = oracle.brdf_f64(n, n, n, [alb] * 3, r, m)
        assert abs(fd[0] - fd_want) <= 1e-12 * max(1, fd_want)
        # (a2 - 1) + 1 cancels: relative rounding ~ 2^-53 / a2
        assert abs(fs[0] - fs_want) <= 1e-9 * fs_want
        mat = np.zeros(1, sg.MATERIAL_DTYPE)[0]
        mat["albedo"], mat["roughness"], mat["metallic"] = [alb] * 3, r, m
        f32 = oracle.brdf_f32(n, n, n, mat)
        # FP32: dd = fma(nh^2, a2 - 1, 1) loses ~2^-24 absolute to the rounding
        # of a2 - 1, i.e. 2^-24 / a2 relative, doubled by dd^2
        tol = 2e-6 + 3 * 2.0 ** -24 / (r ** 4)
        assert abs(f32[0] - (fd_want + fs_want)) <= tol * (fd_want + fs_want)


def _rand_dirs(rng, n, upper=True):
    out = []
    while len(out) < n:
        v = rng.unit_vector()
        if upper and v[1] < 0.02:
            continue
        out.append(v)
    return np.array(out)


def test_cancelled_form_equals_plain_product():
    """G/(4 nl nv) written as 1/(4 (nl(1-k)+k)(nv(1-k)+k)) equals the plain
    D F G / (4 nl nv) for nl, nv >= 1e-3."""
    rng = sg.Rng(11)
    n = np.array([0.0, 1.0, 0.0])
    for _ in range(300):
        v, l = _rand_dirs(rng, 2)
        r, m, a = rng.uniform(0.05, 1), float(rng.u() < 0.5), rng.uniform(0.05, 0.95)
        nl, nv = l[1], v[1]
        if nl < 1e-3 or nv < 1e-3:
            continue
        h = (l + v) / np.linalg.norm(l + v)
        f0 = 0.04 * (1 - m) + a * m
        plain = (oracle.ggx_d(h[1], r * r) * oracle.schlick_f(float(np.dot(v, h)), f0)
                 * oracle.smith_g(nl, nv, r) / (4 * nl * nv))
        fd, fs = oracle.brdf_f64(n, v, l, [a] * 3, r, m)
        assert abs(fs[0] - plain) <= 1e-12 * max(plain, 1e-12)
        fdp = (1 - oracle.schlick_f(float(np.dot(v, h)), f0)) * (1 - m) * a / math.pi
        assert abs(fd[0] - fdp) <= 1e-14


def test_fp32_brdf_matches_fp64_twin():
    rng = sg.Rng(12)
    n = np.array([0.0, 1.0, 0.0])
    worst = 0.0
    for _ in range(2000):
        v, l = _rand_dirs(rng, 2)
        mat = np.zeros(1, sg.MATERIAL_DTYPE)[0]
        mat["albedo"] = [rng.uniform(0.05, 0.95) for _ in range(3)]
        mat["roughness"] = rng.uniform(0.05, 1.0)
        mat["metallic"] = float(rng.u() < 0.3)
        f32 = oracle.brdf_f32(n.astype(np.float32), v.astype(np.float32), l.astype(np.float32), mat)
        fd, fs = oracle.brdf_f64(n, v.astype(np.float32).astype(np.float64), l.astype(np.float32).astype(np.float64),
                                 mat["albedo"].astype(np.float64), float(mat["roughness"]), float(mat["metallic"]))
        ref = fd + fs
        # conditioning of D: dd = (n.h)^2 (a2 - 1) + 1 carries ~2^-23 absolute
        # FP32 error (roundings of n.h, (n.h)^2 and a2 - 1), so D's relative
        # error is up to ~2^-22 / dd
        h = (l + v) / np.linalg.norm(l + v)
        a2 = float(mat["roughness"]) ** 4
        dd = h[1] ** 2 * (a2 - 1) + 1
        tol = 2e-5 + 2.0 ** -21 / dd
        worst = max(worst, float(np.max(np.abs(f32 - ref) / ref)) / tol)
    assert worst < 1.0, worst


def test_white_furnace_lambert_and_energy_bound():
    """Lambert part: f_d / ((1-F)(1-m)) = albedo / pi, whose cosine-weighted
    hemisphere integral is the albedo.  Whole BRDF: directional albedo stays
    near or below 1 (the measured maximum over the grid is recorded)."""
    n = np.array([0.0, 1.0, 0.0])
    for a in (0.2, 0.9):
        for vth in (0.1, 0.7, 1.4):
            v = np.array([math.sin(vth), math.cos(vth), 0.0])

            def lam(l):
                fd, _ = oracle.brdf_f64(n, v, l, [a] * 3, 0.5, 0.0)
                h = (l + v) / np.linalg.norm(l + v)
                F = oracle.schlick_f(max(float(np.dot(v, h)), 0.0), 0.04)
                return fd[0] / (1 - F) * l[1]
            assert abs(_hemi_quad(lam, 100, 32) - a) < 1e-3
    worst = 0.0
    for r in (0.05, 0.3, 0.7, 1.0):
        for m in (0.0, 1.0):
            for vth in (0.0, 0.8, 1.3, 1.5):
                v = np.array([math.sin(vth), math.cos(vth), 0.0])

                def full(l):
                    fd, fs = oracle.brdf_f64(n, v, l, [1.0] * 3, r, m)
                    return (fd[0] + fs[0]) * l[1]
                worst = max(worst, _hemi_quad(full, 120, 48))
    # reported bound: this Schlick-GGX direct-light variant is not exactly
    # energy conserving at grazing view; it must stay close to 1
    assert worst < 1.1, worst


def test_closed_form_image():
    """Camera straight above a large horizontal quad, one point light: each
    pixel = (f_d + f_s) I cos(theta) / d^2 evaluated in FP64 at the exact
    ray/plane point, with the shadow-ray origin lifted by eps = 1e-4 x the
    scene-box diagonal."""
    sc = _plane_scene(np.zeros((0, 3, 3)))
    sc.mats[0]["albedo"] = [0.5, 0.3, 0.2]
    for rough, metal in ((0.4, 0.0), (0.7, 1.0), (0.08, 0.0)):
        sc.mats[0]["roughness"], sc.mats[0]["metallic"] = rough, metal
        S = oracle.OracleScene(sc)
        S.update(np.eye(3, 4, dtype=np.float32).reshape(1, 12), rebuild=True)
        # (off the quad's diagonal: a ray exactly through the shared edge may
        # miss both triangles of a non-watertight ray/triangle test)
        cam = sg.Camera((0.37, 10.0, 0.21), (0.37, 0.0, 0.21), (0.0, 0.0, -1.0), 60.0, 33, 33, 1)
        light = np.array([3.0, 8.0, -2.0])
        img = S.render_image(cam, [sg.Light(0, tuple(light), 100.0)])
        eps = 1e-4 * math.sqrt(100.0 ** 2 + 100.0 ** 2)
        n = np.array([0.0, 1.0, 0.0])
        worst = 0.0
        for y in range(33):
            for x in range(33):
                o, d = (a.astype(np.float64) for a in oracle.camera_ray(cam, x, y, 0))
                p = o + (-o[1] / d[1]) * d
                po = p + eps * n
                L = light - po
                d2 = L @ L
                l = L / math.sqrt(d2)
                fd, fs = oracle.brdf_f64(n, -d, l, [0.5, 0.3, 0.2], rough, metal)
                want = (fd + fs) * 100.0 * l[1] / d2
                # FP32 conditioning of D near its peak (see the BRDF test)
                h = (l - d) / np.linalg.norm(l - d)
                dd = h[1] ** 2 * (rough ** 4 - 1) + 1
                tol = 1e-5 + 2.0 ** -21 / dd
                worst = max(worst, float(np.max(np.abs(img[y, x, :3] - want) / want)) / tol)
                assert img[y, x, 3] == 1.0
        assert worst < 1.0, (rough, metal, worst)


def _grad_setup(spp=1, W=20, H=20):
    w = sg.workload_tiny41k(W, H)
    cam = sg.Camera(**{**w.camera.__dict__, "spp": spp})
    lights = [sg.LIGHTS_MAIN[0], sg.LIGHTS_MAIN[1]]
    S = oracle.OracleScene(w.scene)
    S.update(w.scene.identity_xforms(), rebuild=True)
    samples = S.render_all_samples(cam, lights)
    return w, cam, lights, S, samples


@pytest.mark.parametrize("spp", [1, 4])
def test_gradient_matches_central_differences(spp):
    """dL/d(albedo, roughness, metallic, intensity) of L = mean((I - I*)^2)
    (visibility fixed): the FP64 analytic gradient equals FP64 central
    differences (step 1e-4 relative, 1e-6 absolute minimum) to 1e-6."""
    w, cam, lights, S, samples = _grad_setup(spp)
    P0 = oracle.params_of(w.scene.mats)
    I0 = np.array([l.intensity for l in lights], np.float64)
    tm, ti = sg.perturbed_params(w.scene.mats, I0)
    target = S.shade_f64(cam, lights, samples, oracle.params_of(tm), ti.astype(np.float64))
    npx = cam.width * cam.height * 3

    def loss(P, I):
        img = S.shade_f64(cam, lights, samples, P, I)
        return float(np.sum((img - target) ** 2) / npx)

    img = S.shade_f64(cam, lights, samples, P0, I0)
    dimg = 2 * (img - target) / npx
    gP, gI = S.grad_f64(cam, lights, samples, P0, I0, dimg)
    fd = np.zeros_like(gP)
    for i in range(P0.shape[0]):
        for j in range(5):
            h = max(1e-4 * abs(P0[i, j]), 1e-6)
            Pp, Pm = P0.copy(), P0.copy()
            Pp[i, j] += h
            Pm[i, j] -= h
            fd[i, j] = (loss(Pp, I0) - loss(Pm, I0)) / (2 * h)
    fdI = np.zeros_like(gI)
    for j in range(len(I0)):
        h = 1e-4 * I0[j]
        Ip, Im = I0.copy(), I0.copy()
        Ip[j] += h
        Im[j] -= h
        fdI[j] = (loss(P0, Ip) - loss(P0, Im)) / (2 * h)
    g, f = np.concatenate([gP.ravel(), gI]), np.concatenate([fd.ravel(), fdI])
    floor = 1e-3 * np.abs(f).max()
    assert np.all(np.abs(g - f) <= 1e-6 * np.maximum(np.abs(f), floor)), np.abs(g - f).max()
    assert np.count_nonzero(gP) > 20


def test_fp32_render_matches_fp64_shading():
    """The FP32 forward radiance equals the FP64 twin on the same hits to
    within a few FP32 roundings (pins the FP32 operation order to the
    definitions)."""
    w, cam, lights, S, samples = _grad_setup(4, 24, 24)
    P0 = oracle.params_of(w.scene.mats)
    I0 = np.array([l.intensity for l in lights], np.float64)
    img64 = S.shade_f64(cam, lights, samples, P0, I0)
    img32 = S.render_image(cam, lights)[..., :3]
    rel = np.abs(img32 - img64) / np.maximum(np.abs(img64), 1e-6)
    assert np.max(rel) < 1e-3 and np.median(rel[img64 > 1e-3]) < 1e-5, (rel.max(),)


def test_fresh_fp64_frame_closed_form():
    """shade_f64_fresh on the quad under the camera: each pixel is
    (f_d + f_s) I cos(theta) g at the exact FP64 ray/plane point (g = 1/d^2
    for the point light, 1 for the directional one), the shadow origin lifted
    by eps along the plane's normal; FP64 agreement (1e-9 relative)."""
    sc = _plane_scene(np.zeros((0, 3, 3)))
    sc.mats[0]["albedo"] = [0.5, 0.3, 0.2]
    sc.mats[0]["roughness"], sc.mats[0]["metallic"] = 0.35, 0.4
    S = oracle.OracleScene(sc)
    S.update(np.eye(3, 4, dtype=np.float32).reshape(1, 12), rebuild=True)
    cam = sg.Camera((0.37, 10.0, 0.21), (0.37, 0.0, 0.21), (0.0, 0.0, -1.0), 60.0, 17, 13, 1)
    lights = [sg.Light(0, (3.0, 8.0, -2.0), 100.0), sg.Light(1, (0.3, 1.0, 0.2), 2.0)]
    samples = S.render_all_samples(cam, lights)
    assert np.all(samples["prim"] >= 0)
    P = oracle.params_of(sc.mats)
    I = np.array([100.0, 2.0])
    img = S.shade_f64_fresh(cam, lights, samples, P, I)
    eps = float(S.shadow_eps())
    n = np.array([0.0, 1.0, 0.0])
    worst = 0.0
    for y in range(cam.height):
        for x in range(cam.width):
            o, d = (a.astype(np.float64) for a in oracle.camera_ray(cam, x, y, 0))
            p = o + (-o[1] / d[1]) * d
            po = p + eps * n
            v = -d / np.linalg.norm(d)
            want = np.zeros(3)
            vis = int(samples["vis"][y * cam.width + x])
            for j, L in enumerate(lights):
                if L.type == 0:
                    lv = np.array(L.v, np.float32).astype(np.float64) - po
                    g, l = 1.0 / (lv @ lv), lv / np.linalg.norm(lv)
                else:
                    lv = np.array(L.v, np.float32).astype(np.float64)  # the light record is FP32
                    g, l = 1.0, lv / np.linalg.norm(lv)
                if not (vis >> j) & 1:
                    continue
                fd, fs = oracle.brdf_f64(n, v, l, P[0, :3], P[0, 3], P[0, 4])  # (params_of rounds to FP32)
                want += (fd + fs) * I[j] * l[1] * g
            worst = max(worst, float(np.max(np.abs(img[y, x] - want) / want)))
    assert worst < 1e-9, worst


def test_fresh_fp64_frame_near_fp32_frame():
    """On the tiny scene the FP64 frame from scratch and the FP32 frame give
    the same image to FP32 frame precision (GGX peaks amplify the angle
    rounding, hence the 1e-3 bound on the largest difference)."""
    w, cam, lights, S, samples = _grad_setup(4, 24, 24)
    P0 = oracle.params_of(w.scene.mats)
    I0 = np.array([l.intensity for l in lights], np.float64)
    a = S.shade_f64(cam, lights, samples, P0, I0)
    b = S.shade_f64_fresh(cam, lights, samples, P0, I0)
    rel = np.abs(a - b) / np.maximum(np.abs(b), 1e-6)
    assert np.max(rel) < 1e-3 and np.median(rel[b > 1e-3]) < 1e-5, (rel.max(),)
    assert np.count_nonzero(b) > 100
