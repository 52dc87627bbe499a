"""Differentiable shading on the GPU at the size of the gradient workload
(499,712 triangles, 512 x 512, 1 spp, 32 materials, 2 lights): the
hand-written backward kernel against the oracle's FP64 analytic gradient
(1e-4) and FP64 central finite differences (1e-3), both with
|delta| <= tol * max(|g_ref|, 1e-3 ||g_ref||_inf), and the
torch.autograd.Function wrapper."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from gpu_common import build_pair, compare_samples, gbuf_of, torch_cuda, THREADS

pytestmark = pytest.mark.gpu


def _close(g, ref, tol):
    g, ref = np.asarray(g, np.float64).ravel(), np.asarray(ref, np.float64).ravel()
    floor = 1e-3 * np.abs(ref).max()
    err = np.abs(g - ref) / np.maximum(np.abs(ref), floor)
    return float(err.max())


@pytest.fixture(scope="module")
def setup():
    torch = torch_cuda()
    import paper_2410_05095_b300 as fb
    w = sg.workload_grad500k()  # 512 x 512, 1 spp, 32 materials, 2 lights
    cam, lights = w.camera, w.lights
    G, S = build_pair(w.scene)
    gb = torch.zeros((cam.width * cam.height * cam.spp, 4), dtype=torch.int32, device="cuda")
    G.render(cam, lights, gbuf=gb)
    g = gbuf_of(gb)
    ref = S.render_all_samples(cam, lights, threads=THREADS)
    _, bad = compare_samples(g, ref)
    # the loss covers the pixels whose samples agree (a near tie allowed by
    # the agreement rule would give the two sides different fixed
    # visibility); both sides use the same mask
    keep = (~bad).reshape(cam.height, cam.width, cam.spp).all(axis=2)
    assert keep.mean() >= 0.9999
    P0 = oracle.params_of(w.scene.mats)
    I0 = np.array([l.intensity for l in lights], np.float64)
    tm, ti = sg.perturbed_params(w.scene.mats, I0)
    Pt = oracle.params_of(tm)
    target = S.shade_f64(cam, lights, ref, Pt, ti.astype(np.float64))
    return dict(torch=torch, fb=fb, w=w, cam=cam, lights=lights, G=G, S=S, gb=gb, ref=ref, P0=P0, I0=I0,
                target=target, keep=keep)


def _upstream64(s, P, I):
    """dL/dimage of L = sum over kept pixels of (I - I*)^2 / (3 W H), from the
    oracle's FP64 image: the same upstream for both sides of a comparison.
    (Taken from the GPU's FP32 image instead it differs at the GGX peak, where
    FP32 radiance is ~1e-3 relative off FP64 (the forward check below), and
    those pixels weigh most in the roughness gradients.)"""
    cam = s["cam"]
    img64 = s["S"].shade_f64(cam, s["lights"], s["ref"], P, I)
    npx = cam.width * cam.height * 3
    return 2.0 * (img64 - s["target"]) / npx * s["keep"][..., None]


def _gpu_grad(s, P, I, upstream=None):
    """GPU forward image and backward at (P, I).  upstream: [H, W, 3] dL/dimage
    (FP64, rounded to FP32 for the kernel), or None for the gradient of the
    same loss taken at the GPU's own image."""
    torch = s["torch"]
    cam = s["cam"]
    params = torch.from_numpy(P.astype(np.float32)).cuda()
    inten = torch.from_numpy(I.astype(np.float32)).cuda()
    img = s["G"].shade(s["gb"], cam, s["lights"], params, inten)
    npx = cam.width * cam.height * 3
    dimg = torch.zeros_like(img)
    if upstream is None:
        tgt = torch.from_numpy(s["target"].astype(np.float32)).cuda()
        dimg[..., :3] = 2.0 * (img[..., :3] - tgt) / npx
        dimg[..., :3] *= torch.from_numpy(s["keep"].astype(np.float32)).cuda()[..., None]
    else:
        dimg[..., :3] = torch.from_numpy(upstream.astype(np.float32)).cuda()
    dP = torch.zeros_like(params)
    dI = torch.zeros_like(inten)
    s["G"].shade_backward(s["gb"], cam, s["lights"], params, inten, dimg, dP, dI)
    return img, dimg, dP.cpu().numpy().astype(np.float64), dI.cpu().numpy().astype(np.float64)


def test_backward_matches_oracle_analytic(setup):
    s = setup
    # both sides chain the same upstream gradient (from the FP64 forward image)
    d64 = _upstream64(s, s["P0"], s["I0"])
    img, dimg, gP, gI = _gpu_grad(s, s["P0"], s["I0"], d64)
    img64 = s["S"].shade_f64(s["cam"], s["lights"], s["ref"], s["P0"], s["I0"])
    rP, rI = s["S"].grad_f64(s["cam"], s["lights"], s["ref"], s["P0"], s["I0"], d64)
    err = _close(np.concatenate([gP.ravel(), gI]), np.concatenate([rP.ravel(), rI]), 1e-4)
    assert err <= 1e-4, err
    # the forward image agrees with the FP64 twin too
    a = img.cpu().numpy()[..., :3].astype(np.float64)
    assert np.max((np.abs(a - img64) / np.maximum(np.abs(img64), 1e-6))[s["keep"]]) < 2e-3


def test_backward_matches_finite_differences(setup):
    s = setup
    _, _, gP, gI = _gpu_grad(s, s["P0"], s["I0"], _upstream64(s, s["P0"], s["I0"]))
    S, cam, lights, ref = s["S"], s["cam"], s["lights"], s["ref"]
    npx = cam.width * cam.height * 3

    keep = s["keep"][..., None]

    def loss(P, I):
        return float(np.sum(((S.shade_f64(cam, lights, ref, P, I) - s["target"]) ** 2) * keep) / npx)

    used = np.unique(s["w"].scene.tri_mat[ref["prim"][ref["prim"] >= 0]])
    fd, g = [], []
    for m in used[:12]:
        for j in range(5):
            h = max(1e-4 * abs(s["P0"][m, j]), 1e-6)
            Pp, Pm = s["P0"].copy(), s["P0"].copy()
            Pp[m, j] += h
            Pm[m, j] -= h
            fd.append((loss(Pp, s["I0"]) - loss(Pm, s["I0"])) / (2 * h))
            g.append(gP[m, j])
    for j in range(len(s["I0"])):
        h = 1e-4 * s["I0"][j]
        Ip, Im = s["I0"].copy(), s["I0"].copy()
        Ip[j] += h
        Im[j] -= h
        fd.append((loss(s["P0"], Ip) - loss(s["P0"], Im)) / (2 * h))
        g.append(gI[j])
    err = _close(g, fd, 1e-3)
    assert err <= 1e-3, err


def test_backward_matches_fd_of_fp64_frame_from_scratch(setup):
    """The kernel's gradient against central differences of the loss shaded
    with an FP64 hit frame recomputed from the ray and the world triangle
    (t, p, n, v, l, h, 1/d^2 in FP64; the oracle's shade_f64_fresh), not from
    the FP32 frame the forward used: agreement to 1e-3 (the FP32 frame's
    angle rounding moves the roughness gradient by ~3e-4 at GGX peaks)."""
    s = setup
    S, cam, lights, ref = s["S"], s["cam"], s["lights"], s["ref"]
    npx = cam.width * cam.height * 3
    keep = s["keep"][..., None]
    target = S.shade_f64_fresh(cam, lights, ref, *_target_params(s))

    def loss(P, I):
        return float(np.sum(((S.shade_f64_fresh(cam, lights, ref, P, I) - target) ** 2) * keep) / npx)

    up = 2.0 * (S.shade_f64_fresh(cam, lights, ref, s["P0"], s["I0"]) - target) / npx * keep
    _, _, gP, gI = _gpu_grad(s, s["P0"], s["I0"], up)
    used = np.unique(s["w"].scene.tri_mat[ref["prim"][ref["prim"] >= 0]])
    fd, g = [], []
    for m in used[:8]:
        for j in range(5):
            h = max(1e-4 * abs(s["P0"][m, j]), 1e-6)
            Pp, Pm = s["P0"].copy(), s["P0"].copy()
            Pp[m, j] += h
            Pm[m, j] -= h
            fd.append((loss(Pp, s["I0"]) - loss(Pm, s["I0"])) / (2 * h))
            g.append(gP[m, j])
    for j in range(len(s["I0"])):
        h = 1e-4 * s["I0"][j]
        Ip, Im = s["I0"].copy(), s["I0"].copy()
        Ip[j] += h
        Im[j] -= h
        fd.append((loss(s["P0"], Ip) - loss(s["P0"], Im)) / (2 * h))
        g.append(gI[j])
    err = _close(g, fd, 1e-3)
    assert err <= 1e-3, err


def _target_params(s):
    tm, ti = sg.perturbed_params(s["w"].scene.mats, s["I0"])
    return oracle.params_of(tm), ti.astype(np.float64)


def test_autograd_function_and_descent(setup):
    """FireShade.apply gives the kernel's gradient; a few steps of gradient
    descent on the perturbed start reduce the loss."""
    s = setup
    torch = s["torch"]
    from paper_2410_05095_b300.autograd import FireShade
    P = torch.from_numpy(s["P0"].astype(np.float32)).cuda().requires_grad_(True)
    I = torch.from_numpy(s["I0"].astype(np.float32)).cuda().requires_grad_(True)
    tgt = torch.from_numpy(s["target"].astype(np.float32)).cuda()
    keep = torch.from_numpy(s["keep"].astype(np.float32)).cuda()[..., None]
    img = FireShade.apply(P, I, s["G"], s["gb"], s["cam"], s["lights"])
    loss = (((img[..., :3] - tgt) ** 2) * keep).sum() / (3 * keep.numel())
    loss.backward()
    _, _, gP, gI = _gpu_grad(s, s["P0"], s["I0"])
    assert np.allclose(P.grad.cpu().numpy(), gP, rtol=1e-5, atol=1e-12)
    assert np.allclose(I.grad.cpu().numpy(), gI, rtol=1e-5, atol=1e-12)
    # descent from the perturbed parameters towards the target
    tm, ti = sg.perturbed_params(s["w"].scene.mats, s["I0"])
    P = torch.from_numpy(oracle.params_of(s["w"].scene.mats).astype(np.float32)).cuda().requires_grad_(True)
    I = torch.from_numpy(s["I0"].astype(np.float32)).cuda().requires_grad_(True)
    opt = torch.optim.Adam([P, I], lr=1e-2)
    losses = []
    for _ in range(20):
        opt.zero_grad()
        img = FireShade.apply(P, I, s["G"], s["gb"], s["cam"], s["lights"])
        l = ((img[..., :3] - tgt) ** 2).mean()
        l.backward()
        opt.step()
        with torch.no_grad():
            P[:, :3].clamp_(0.01, 0.99)
            P[:, 3].clamp_(0.05, 1.0)
            I.clamp_(min=1e-3)
        losses.append(float(l))
    assert losses[-1] < 0.5 * losses[0]
