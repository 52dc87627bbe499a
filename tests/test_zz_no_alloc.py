"""The allocation-free shading backward (fire_shade_backward_noalloc).

It serves callers that cannot call cudaMalloc while they run -- a frame loop
whose device memory is fixed at start-up, or a host that must not pay the
device synchronisation an allocation can cause.  Its scratch is a fixed
array inside the library, so it must give the same gradients as
fire_shade_backward, call after call, allocate nothing (the library's
allocation-failure hook stays armed through the calls and the scene's device
bytes do not change), and refuse a parameter count that does not fit that
array.

The file is named to be collected last: it is the newest addition, and a run
that stops at the first failure has then already run every other test.  It
does not depend on running last: each test builds its own scene, and the
fixture below disarms the allocation-failure hook whatever happened before or
during the test."""
import numpy as np
import pytest

import scenegen as sg

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4  # the gradient tolerance of the parity tests


def _close(g, ref):
    g, ref = np.asarray(g, np.float64).ravel(), np.asarray(ref, np.float64).ravel()
    floor = 1e-3 * np.abs(ref).max()
    return float(np.max(np.abs(g - ref) / np.maximum(np.abs(ref), floor)))


@pytest.fixture(autouse=True)
def disarmed_alloc_hook():
    import paper_2410_05095_b300 as fb
    fb.fire.fail_next_alloc(0)
    yield
    fb.fire.fail_next_alloc(0)


def test_noalloc_backward_matches_fire_shade_backward():
    import torch

    import paper_2410_05095_b300 as fb
    w = sg.workload_tiny41k(64, 48)
    cam = sg.Camera(**{**w.camera.__dict__, "spp": 4})
    lights = [sg.LIGHTS_MAIN[0], sg.LIGHTS_MAIN[1]]
    G = fb.Scene.from_numpy(w.scene)
    G.build(w.scene.identity_xforms())
    gb = torch.zeros((cam.width * cam.height * cam.spp, 4), dtype=torch.int32, device="cuda")
    G.render(cam, lights, gbuf=gb)
    P = np.zeros((len(w.scene.mats), 5), np.float32)
    for i, m in enumerate(w.scene.mats):
        P[i, :3], P[i, 3], P[i, 4] = m["albedo"], m["roughness"], m["metallic"]
    params = torch.from_numpy(P).cuda()
    inten = torch.tensor([l.intensity for l in lights], dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(5)
    dimg = torch.randn((cam.height, cam.width, 4), device="cuda", generator=gen)

    dP_ref, dI_ref = torch.zeros_like(params), torch.zeros_like(inten)
    G.shade_backward(gb, cam, lights, params, inten, dimg, dP_ref, dI_ref)
    torch.cuda.synchronize()
    assert float(dP_ref.abs().sum()) > 0

    outs = [(torch.zeros_like(params), torch.zeros_like(inten)) for _ in range(2)]  # caller-owned
    torch.cuda.synchronize()
    bytes_before = G.info()["bytes"]
    # the next library allocation would fail: the calls below must make none
    fb.fire.fail_next_alloc(1)
    for dP, dI in outs:  # two calls in a row share (and must re-clear) the scratch
        G.shade_backward_noalloc(gb, cam, lights, params, inten, dimg, dP, dI)
    torch.cuda.synchronize()
    fb.fire.fail_next_alloc(0)
    assert G.info()["bytes"] == bytes_before
    for dP, dI in outs:
        assert _close(dP.cpu(), dP_ref.cpu()) <= REL_TOL
        assert _close(dI.cpu(), dI_ref.cpu()) <= REL_TOL
    assert G.sync_status() == 0


def test_noalloc_backward_rejects_more_parameters_than_its_scratch():
    import torch

    import paper_2410_05095_b300 as fb
    rng = sg.Rng(9)
    mats = sg.random_materials(rng, 900)  # 900 * 5 + 1 = 4501 > 4096
    sc = sg.assemble([(np.array([[-1.0, -1, 0], [1, -1, 0], [0, 1, 0]]), np.array([[0, 1, 2]]))], 900, mats)
    G = fb.Scene.from_numpy(sc)
    G.build(sc.identity_xforms())
    cam = sg.Camera((0.0, 0.0, 5.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 40.0, 16, 16, 1)
    lights = [sg.Light(0, (0.0, 0.0, 4.0), 10.0)]
    gb = torch.zeros((16 * 16, 4), dtype=torch.int32, device="cuda")
    G.render(cam, lights, gbuf=gb)
    params = torch.zeros((900, 5), device="cuda")
    inten = torch.ones(1, device="cuda")
    dimg = torch.ones((16, 16, 4), device="cuda")
    dP, dI = torch.zeros_like(params), torch.zeros_like(inten)
    with pytest.raises(fb.FireError) as e:
        G.shade_backward_noalloc(gb, cam, lights, params, inten, dimg, dP, dI)
    assert e.value.code == -1 and "4096" in str(e.value)


def test_noalloc_backward_is_timed_as_the_backward_stage():
    import torch

    import paper_2410_05095_b300 as fb
    w = sg.workload_tiny41k(32, 32)
    cam = sg.Camera(**{**w.camera.__dict__, "spp": 1})
    lights = [sg.LIGHTS_MAIN[0]]
    G = fb.Scene.from_numpy(w.scene)
    G.build(w.scene.identity_xforms())
    gb = torch.zeros((cam.width * cam.height, 4), dtype=torch.int32, device="cuda")
    G.render(cam, lights, gbuf=gb)
    params = torch.ones((len(w.scene.mats), 5), device="cuda") * 0.5
    inten = torch.tensor([lights[0].intensity], dtype=torch.float32, device="cuda")
    dimg = torch.ones((cam.height, cam.width, 4), device="cuda")
    dP, dI = torch.zeros_like(params), torch.zeros_like(inten)
    G.profile(True)
    G.profile_read()  # drop what the build and render recorded
    for _ in range(3):
        G.shade_backward_noalloc(gb, cam, lights, params, inten, dimg, dP, dI)
    prof = G.profile_read()
    G.profile(False)
    ms, launches = prof["backward"]
    assert launches == 3 and ms > 0
    assert G.sync_status() == 0
