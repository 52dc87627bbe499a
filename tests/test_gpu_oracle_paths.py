"""The CUDA paths that have their own kernels or their own ordering, each
compared with the oracle directly (not with another CUDA path):

* the batch (fire_render_batch: its own primary, shadow and resolve kernels
  over many cameras and scenes) on a mix shaped like the batched workload --
  scenes of uneven size drawn log-uniformly, orbit cameras of 128^2 up to
  640x480, 1 to 3 lights (point and directional);
* pipelined frames (fire_bvh_refit on its own stream into the second frame
  buffer while the previous frame renders) on a reduced copy of the moving
  7.3M-triangle workload, frames 1, 3 and 5 against the oracle refit to the
  same poses."""
import numpy as np
import pytest

import scenegen as sg
from gpu_common import (THREADS, assert_radiance_close, compare_images, compare_samples, gbuf_of,
                        pixel_ok_mask, torch_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fb():
    import paper_2410_05095_b300 as fb
    torch_cuda()
    return fb


def test_batch_matches_oracle(fb):
    import oracle
    torch = torch_cuda()
    scenes, cams, cam_scene, lights = sg.batch16(nscenes=4, ncams_per=2, tmin=20e3, tmax=600e3, seed_offset=13)
    # the mix must hold a 640x480 camera and every light count 1..3
    cams[0] = sg.Camera(cams[0].pos, cams[0].target, cams[0].up, cams[0].vfov_deg, 640, 480, 1)
    lights = [sg.LIGHTS_MAIN[:n] for n in (1, 2, 3, 3)]
    G, S = [], []
    for sc in scenes:
        g = fb.Scene.from_numpy(sc)
        g.build(sc.identity_xforms())
        G.append(g)
        o = oracle.OracleScene(sc)
        o.update(sc.identity_xforms(), rebuild=True)
        S.append(o)
    outs = [torch.zeros((c.height, c.width, 4), device="cuda") for c in cams]
    fb.render_batch(G, cams, cam_scene, lights, outs)
    fb.render_batch(G, cams, cam_scene, lights, outs)  # graph replay
    torch.cuda.synchronize()
    for g in G:
        assert g.sync_status() == 0
    lit = 0
    for c, si, o in zip(cams, cam_scene, outs):
        ref = S[si].render_all_samples(c, lights[si], threads=THREADS)
        img_ref = S[si].render_image(c, lights[si], threads=THREADS)
        compare_images(o.cpu().numpy(), img_ref, ref, c.spp)
        lit += int(((ref["vis"] & 0xFF) != 0).sum())
    assert lit > 1000
    assert (cams[0].width, cams[0].height) == (640, 480)
    assert min(sc.nt for sc in scenes) >= 20_000


def test_pipelined_frames_match_oracle(fb):
    import oracle
    torch = torch_cuda()
    w = sg.workload_frame7m(nspheres=120, cells=64)
    cam = sg.Camera(w.camera.pos, w.camera.target, w.camera.up, 60.0, 192, 108, 4)
    xf0 = w.motion.xforms()
    poses = [w.motion.step() for _ in range(5)]
    G = fb.Scene.from_numpy(w.scene)
    G.build(xf0)
    dev = [torch.from_numpy(xf).cuda() for xf in poses]
    n = cam.width * cam.height * cam.spp
    gbs = [torch.zeros((n, 4), dtype=torch.int32, device="cuda") for _ in poses]
    outs = [torch.zeros((cam.height, cam.width, 4), device="cuda") for _ in poses]
    side = torch.cuda.Stream(priority=-1)
    torch.cuda.synchronize()
    for i in range(len(poses)):   # refit of frame i overlaps the render of frame i-1
        G.refit(dev[i], stream=side)
        G.render(cam, w.lights, out=outs[i], gbuf=gbs[i], opts=fb.fire.make_opts(blocks_per_sm=6))
    torch.cuda.synchronize()
    assert G.sync_status() == 0
    S = oracle.OracleScene(w.scene)
    S.update(xf0, rebuild=True)
    for i, xf in enumerate(poses):
        S.update(xf, rebuild=False)
        if i % 2:
            continue  # frames 1, 3, 5
        ref = S.render_all_samples(cam, w.lights, threads=THREADS)
        _, bad = compare_samples(gbuf_of(gbs[i]), ref)
        img_ref = S.render_image(cam, w.lights, threads=THREADS)
        assert_radiance_close(outs[i].cpu().numpy(), img_ref, pixel_ok_mask(bad, cam.width, cam.height, 4))
