"""B300-native per-frame hot path of the FIRE-3DV renderer (arXiv 2410.05095).

LBVH build/refit from per-body rigid transforms, supersampled primary
visibility, any-hit shadow rays, Cook-Torrance GGX shading and box-filter
resolve, batched multi-scene rendering and a differentiable shading stage --
all in hand-written CUDA for sm_103a behind the C ABI of include/fire.h.

Python is argument marshalling only (fire.py); PyTorch supplies device
memory and streams.
"""
from . import fire  # noqa: F401
from .fire import FireError, Scene, display, render_batch, batch_last_config  # noqa: F401
