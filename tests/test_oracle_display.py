"""Pins of the oracle's display stage (§IV-A-1 Reinhard tone mapping and
gamma correction, §IV-B-2 FXAA) against closed forms and invariants."""
import numpy as np

import oracle


def test_root12_pow5_against_fp64():
    rs = np.concatenate([np.geomspace(2.0 ** -9, 1.0, 20001, endpoint=False), [2.0 ** -9, 0.5, 0.25, 0.999999]])
    rs = rs.astype(np.float32)
    got = np.array([oracle.root12_pow5(float(r)) for r in rs], np.float64)
    ref = rs.astype(np.float64) ** (5.0 / 12.0)
    assert np.max(np.abs(got - ref) / ref) < 32 * 2.0 ** -24


def test_srgb_encode_curve():
    # linear segment, exact
    for r in (0.0, 1e-6, 1e-3, 0.003):
        assert oracle.srgb_encode(r) == np.float32(np.float32(12.92) * np.float32(r))
    # the two branches meet at the threshold (IEC 61966-2-1)
    t = 0.0031308
    assert abs(12.92 * t - (1.055 * t ** (1 / 2.4) - 0.055)) < 1e-6
    assert abs(oracle.srgb_encode(np.nextafter(np.float32(t), np.float32(1))) - 12.92 * t) < 1e-5
    # the power branch against the FP64 formula, and monotone
    rs = np.linspace(0.0032, 0.9999999, 5001).astype(np.float32)
    got = np.array([oracle.srgb_encode(float(r)) for r in rs])
    ref = 1.055 * rs.astype(np.float64) ** (1 / 2.4) - 0.055
    # r^(5/12) within 32 ulp (pinned above), times 1.055, plus two roundings
    assert np.max(np.abs(got - ref)) < 1.055 * 32 * 2.0 ** -24 + 2 * 2.0 ** -24
    assert np.all(np.diff(got) >= 0)
    assert oracle.srgb_encode(np.float32(1 - 2 ** -24)) > 0.99999


def _bytes_ref(c, exposure=1.0):
    """FP64 tone map + encode + rounding of one channel value."""
    x = exposure * c
    r = x / (1 + x)
    s = 12.92 * r if r <= 0.0031308 else 1.055 * r ** (1 / 2.4) - 0.055
    return s * 255 + 0.5


def test_reinhard_and_quantisation_without_fxaa():
    vals = np.array([0.0, 1e-4, 0.01, 0.2, 1.0, 3.0, 50.0, 1e4], np.float32)
    img = np.zeros((1, len(vals), 4), np.float32)
    img[0, :, 0] = vals
    img[0, :, 1] = vals * 0.5
    img[0, :, 2] = vals * 2
    img[0, :, 3] = np.linspace(0, 1, len(vals))
    for e in (1.0, 0.25, 4.0):
        out = oracle.display(img, exposure=e, fxaa=False)
        for ch, scale in ((0, 1.0), (1, 0.5), (2, 2.0)):
            for i, v in enumerate(vals):
                w = _bytes_ref(float(np.float32(v * scale)), e)
                if abs((w % 1.0) - 0.0) > 1e-3:  # not on a rounding boundary
                    assert out[0, i, ch] == int(np.floor(w)), (e, ch, v)
        # coverage is quantised as is
        assert np.array_equal(out[0, :, 3], np.floor(np.linspace(0, 1, len(vals)).astype(np.float32) * 255 + 0.5))
    # c = 1 at exposure 1 maps to r = 1/2
    assert oracle.display(np.full((1, 1, 4), 1.0, np.float32), fxaa=False)[0, 0, 0] == int(np.floor(_bytes_ref(1.0)))


def test_fxaa_invariants():
    rng = np.random.default_rng(5)
    # a constant image is unchanged
    const = np.full((9, 11, 4), 0.7, np.float32)
    assert np.array_equal(oracle.display(const, fxaa=True), oracle.display(const, fxaa=False))
    # a straight vertical or horizontal step is unchanged (taps run along it)
    step = np.zeros((12, 16, 4), np.float32)
    step[:, 8:, :3] = 5.0
    assert np.array_equal(oracle.display(step, fxaa=True), oracle.display(step, fxaa=False))
    assert np.array_equal(oracle.display(step.transpose(1, 0, 2).copy(), fxaa=True),
                          oracle.display(step.transpose(1, 0, 2).copy(), fxaa=False))
    # a diagonal staircase edge is blended next to the edge and nowhere else
    H, W = 32, 32
    yy, xx = np.mgrid[0:H, 0:W]
    diag = np.zeros((H, W, 4), np.float32)
    inside = yy > 0.5 * xx + 6
    diag[inside, :3] = 4.0
    a, b = oracle.display(diag, fxaa=True), oracle.display(diag, fxaa=False)
    changed = np.any(a[..., :3] != b[..., :3], axis=2)
    assert changed.any()
    edge = np.zeros_like(inside)
    edge[:-1] |= inside[:-1] != inside[1:]
    edge[1:] |= inside[1:] != inside[:-1]
    edge[:, :-1] |= inside[:, :-1] != inside[:, 1:]
    edge[:, 1:] |= inside[:, 1:] != inside[:, :-1]
    near = edge.copy()
    for _ in range(2):  # within two pixels of the edge
        n2 = near.copy()
        n2[:-1] |= near[1:]
        n2[1:] |= near[:-1]
        n2[:, :-1] |= near[:, 1:]
        n2[:, 1:] |= near[:, :-1]
        near = n2
    assert not (changed & ~near).any()
    # output stays within the image's range (convex combinations of taps)
    noise = rng.random((20, 24, 4)).astype(np.float32) * 3
    o, g = oracle.display(noise, fxaa=True, want_gamma=True)
    lo = np.floor(g[..., :3].min() * 255 + 0.5)
    hi = np.floor(g[..., :3].max() * 255 + 0.5)
    assert o[..., :3].min() >= lo and o[..., :3].max() <= hi
    # FXAA off: bytes are the rounded gamma-space image
    o2, g2 = oracle.display(noise, fxaa=False, want_gamma=True)
    assert np.array_equal(o2[..., :3], np.floor(np.clip(g2[..., :3], 0, 1) * np.float32(255) + np.float32(0.5)))
