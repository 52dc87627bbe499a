"""Differentiable shading of a G-buffer (torch.autograd.Function).

Forward = fire_shade (visibility held fixed, shading inputs recomputed from
the G-buffer); backward = fire_shade_backward (hand-written kernel giving
dL/d(albedo, roughness, metallic) per material and dL/d(intensity) per
light).  Both run in libfire's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import fire


class FireShade(torch.autograd.Function):
    """image[H,W,4] = shade(params[nmat,5], inten[nlights]; scene, gbuf, cam, lights)."""

    @staticmethod
    def forward(ctx, params, inten, scene, gbuf, cam, lights):
        params = params.contiguous()
        inten = inten.contiguous()
        out = scene.shade(gbuf, cam, lights, params, inten)
        ctx.save_for_backward(params, inten)
        ctx.scene, ctx.gbuf, ctx.cam, ctx.lights = scene, gbuf, cam, lights
        return out

    @staticmethod
    def backward(ctx, grad_out):
        params, inten = ctx.saved_tensors
        dparams = torch.zeros_like(params)
        dinten = torch.zeros_like(inten)
        ctx.scene.shade_backward(ctx.gbuf, ctx.cam, ctx.lights, params, inten, grad_out.contiguous(),
                                 dparams, dinten)
        return dparams, dinten, None, None, None, None


def shade(params, inten, scene, gbuf, cam, lights):
    return FireShade.apply(params, inten, scene, gbuf, cam, lights)
