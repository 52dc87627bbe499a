"""The display stage (Reinhard + sRGB encode + FXAA + 8-bit rounding) on the
GPU against the oracle, byte for byte: rendered frames, random HDR images
with ragged sizes and extreme values, exposures, FXAA on and off."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from gpu_common import build_pair, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fb():
    import paper_2410_05095_b300 as fb
    torch_cuda()
    return fb


def _check(fb, img: np.ndarray, exposure: float, fxaa: bool):
    torch = torch_cuda()
    dev = torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda()
    got = fb.display(dev, exposure=exposure, fxaa=fxaa).cpu().numpy()
    ref = oracle.display(img, exposure=exposure, fxaa=fxaa)
    bad = np.argwhere(got != ref)
    assert bad.size == 0, (bad[:5].tolist(), got[tuple(bad[0][:2])].tolist(), ref[tuple(bad[0][:2])].tolist())


@pytest.mark.parametrize("W,H", [(1, 1), (7, 3), (64, 33), (257, 129)])
def test_display_random_images(fb, W, H):
    rng = np.random.default_rng(W * 1000 + H)
    img = (rng.random((H, W, 4)) ** 3 * 20).astype(np.float32)
    img[..., 3] = rng.random((H, W))
    img[rng.random((H, W)) < 0.1, :3] = 0.0          # background
    img[rng.random((H, W)) < 0.02, :3] = 1e6          # blown-out highlights
    for e in (1.0, 0.3, 7.0):
        for fxaa in (False, True):
            _check(fb, img, e, fxaa)


def test_display_rendered_frame(fb):
    torch = torch_cuda()
    w = sg.workload_tiny41k()
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 192, 128, 4)
    G, _ = build_pair(w.scene)
    img = G.render(cam, w.lights).cpu().numpy()
    for fxaa in (False, True):
        _check(fb, img, 1.0, fxaa)


def test_display_errors(fb):
    torch = torch_cuda()
    x = torch.zeros((4, 4, 4), device="cuda")
    with pytest.raises(fb.FireError):
        fb.display(x, exposure=0.0)
    with pytest.raises(fb.FireError):
        fb.display(x, exposure=float("nan"))
