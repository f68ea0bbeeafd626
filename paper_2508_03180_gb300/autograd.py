"""torch.autograd.Function over render / render_backward.

The differentiable inputs are the Gaussian parameters in the ABI layout
(CUDA float32): mean [G,3], scale [G,3] (linear), quat [G,4], logit [G],
sh [G,C,3].  Forward writes them into the resident scene (dgs_scene_update),
renders with a kept state; backward calls dgs_render_backward, which returns
dL/dscale directly (and dL/dlog-scale for callers that parameterise scales
in log space).  All arithmetic runs in libdgs.so.
"""
from __future__ import annotations

import torch

from .renderer import Context


class DuplexRender(torch.autograd.Function):
    @staticmethod
    def forward(fctx, rctx: Context, scene_id: int, N: int, K: int, deg: int, cams, mean, scale, quat, logit, sh):
        rctx.update_scene(scene_id, N, K, deg, g_mean=mean, g_scale=scale, g_quat=quat, g_logit=logit, g_sh=sh)
        img, state, _ = rctx.render(scene_id, cams, want_state=True)
        fctx.rctx, fctx.state = rctx, state
        fctx.shapes = (mean.shape, scale.shape, quat.shape, logit.shape, sh.shape)
        return img

    @staticmethod
    def backward(fctx, dimg):
        rctx, state = fctx.rctx, fctx.state
        dev = dimg.device
        shapes = fctx.shapes
        g = {name: torch.empty(shp, dtype=torch.float32, device=dev)
             for name, shp in zip(("g_mean", "g_scale", "g_quat", "g_logit", "g_sh"), shapes)}
        rctx.backward(state, dimg.contiguous(), g)
        rctx.release_state(state)
        fctx.state = None
        return (None, None, None, None, None, None, g["g_mean"], g["g_scale"], g["g_quat"], g["g_logit"], g["g_sh"])


def render(rctx: Context, scene_id: int, N: int, K: int, deg: int, cams, mean, scale, quat, logit, sh):
    """Differentiable render of views `cams`; returns the flat image tensor."""
    return DuplexRender.apply(rctx, scene_id, N, K, deg, cams, mean, scale, quat, logit, sh)
