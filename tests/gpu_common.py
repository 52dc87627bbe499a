"""Shared helpers of the GPU parity tests: build the same seeded scene on the
CUDA path (through the C ABI) and in the oracle, and compare by the
tolerances of the method (bit-exact integers; for hits and visibility the
agreement rule: >= 99.99 % of samples agree and every disagreement is a near
tie of the two nearest hits; 1e-4 relative radiance)."""
from __future__ import annotations

import os

import numpy as np

import oracle
import scenegen as sg

THREADS = max(1, min(32, os.cpu_count() or 1))
REL_TOL_RADIANCE = 1e-4     # relative, max over pixels whose samples agree
AGREE_MIN = 0.9999           # fraction of samples whose hit id and visibility agree
TIE_REL = 1e-5               # a disagreement needs the oracle's two nearest hits this close


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test without a GPU"
    return torch


def build_pair(scene: sg.Scene, xf=None):
    """(gpu Scene built, oracle scene built) for the same input."""
    import paper_2410_05095_b300 as fb
    xf = scene.identity_xforms() if xf is None else xf
    G = fb.Scene.from_numpy(scene)
    G.build(xf)
    S = oracle.OracleScene(scene)
    S.update(xf, rebuild=True)
    return G, S


def assert_lbvh_equal(G, S, scene: sg.Scene):
    """Bit-exact Morton codes, sorted order, topology, node boxes, triangle records."""
    assert np.array_equal(G.dump("morton"), S.get("morton"))
    assert np.array_equal(G.dump("order"), S.get("order"))
    assert np.array_equal(G.dump("children"), S.get("children"))
    assert np.array_equal(G.dump("parent"), S.get("parent"))
    assert np.array_equal(G.dump("boxes"), S.get("boxes"))
    assert np.array_equal(G.dump("centroid_bounds"), S.get("centroid_bounds"))
    assert_tris_equal(G, S, scene)


def assert_tris_equal(G, S, scene: sg.Scene):
    tr = G.dump("tris")
    order = S.get("order")
    w = S.get("world")
    idx = scene.idx.astype(np.int64)[order]
    v0, v1, v2 = w[idx[:, 0]], w[idx[:, 1]], w[idx[:, 2]]
    assert np.array_equal(tr[:, 0:3], v0)
    assert np.array_equal(tr[:, 4:7], v1 - v0)   # float32 subtraction, one rounding
    assert np.array_equal(tr[:, 8:11], v2 - v0)
    assert np.array_equal(tr[:, 3].view(np.uint32), order)
    assert np.array_equal(tr[:, 7].view(np.uint32), scene.tri_mat[order])


def gbuf_of(gbuf_tensor):
    g = gbuf_tensor.cpu().numpy()
    return dict(prim=g[:, 0].copy(), t=g[:, 1].view(np.float32).copy(), vis=g[:, 2].astype(np.uint32))


def compare_samples(gpu: dict, ref: dict, ids=None):
    """Agreement rule: hit id and visibility bits agree on >= 99.99% of samples, and
    every disagreement is a sample whose oracle two nearest hits lie within
    1e-5 relative distance.  Returns (agree fraction, bad mask)."""
    gp, gv = gpu["prim"], gpu["vis"]
    if ids is not None:
        gp, gv = gp[ids], gv[ids]
    rp, rv, rt, rt2 = ref["prim"], ref["vis"].astype(np.uint32), ref["t"], ref["t2"]
    bad = (gp != rp) | (gv != rv)
    frac = 1.0 - bad.mean() if len(bad) else 1.0
    with np.errstate(invalid="ignore"):
        tie = np.isfinite(rt2) & (np.abs(rt2 - rt) <= TIE_REL * np.abs(rt))
    unexplained = bad & ~tie
    assert frac >= AGREE_MIN, f"agreement {frac:.6f} < {AGREE_MIN}"
    assert not unexplained.any(), f"{int(unexplained.sum())} disagreements without a near tie"
    return frac, bad


def assert_radiance_close(img_gpu: np.ndarray, img_ref: np.ndarray, ok_pixels: np.ndarray | None = None):
    """|delta| <= 1e-4 max(|ref|, 1e-6), max over the pixels whose samples agree."""
    a, b = img_gpu[..., :3].astype(np.float64), img_ref[..., :3].astype(np.float64)
    rel = np.abs(a - b) / np.maximum(np.abs(b), 1e-6)
    if ok_pixels is not None:
        rel = rel[ok_pixels]
    worst = float(rel.max()) if rel.size else 0.0
    assert worst <= REL_TOL_RADIANCE, worst
    return worst


def pixel_ok_mask(bad_samples: np.ndarray, W: int, H: int, spp: int) -> np.ndarray:
    return ~bad_samples.reshape(H, W, spp).any(axis=2)


def compare_images(img_gpu: np.ndarray, img_ref: np.ndarray, ref: dict, spp: int):
    """Image-level form of the agreement rule, for paths that return images
    only (the batch): a pixel agrees when its coverage (alpha) is equal and
    its radiance is within 1e-4 relative; >= 99.99 % of the pixels agree, and
    every pixel that does not holds a sample whose oracle two nearest hits
    lie within 1e-5 relative distance.  Returns the disagreeing-pixel mask."""
    H, W = img_ref.shape[:2]
    a, b = img_gpu[..., :3].astype(np.float64), img_ref[..., :3].astype(np.float64)
    rel = (np.abs(a - b) / np.maximum(np.abs(b), 1e-6)).max(axis=2)
    ok = (img_gpu[..., 3] == img_ref[..., 3]) & (rel <= REL_TOL_RADIANCE)
    rt, rt2 = ref["t"], ref["t2"]
    with np.errstate(invalid="ignore"):
        tie = (np.isfinite(rt2) & (np.abs(rt2 - rt) <= TIE_REL * np.abs(rt))).reshape(H, W, spp).any(axis=2)
    bad = ~ok
    assert bad.mean() <= 1.0 - AGREE_MIN, f"pixel agreement {1 - bad.mean():.6f}"
    assert not (bad & ~tie).any(), f"{int((bad & ~tie).sum())} disagreeing pixels without a near tie"
    return bad
