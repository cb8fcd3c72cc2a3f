"""torch.autograd over the CUDA rasteriser: render (RGB, depth, alpha) of a
submap moved by one pose per camera, with gradients to every Gaussian
parameter and to the pose (as a left twist about a pivot), all computed by
libgsreg's kernels (gs_render, gs_render_backward).  Argument marshalling
only."""
from __future__ import annotations

import torch

from . import gsreg


class Rasterize(torch.autograd.Function):
    """(means4, log_scales4, quats4, logits, rgb4, twist) -> (rgb, depth,
    alpha), concatenated per camera as gs_render returns them.  ``twist``
    [n_cams, 6] is the left perturbation (w, v) of each pose about its
    pivot, evaluated at zero: its value is not read (the render is taken at
    the given poses), and its gradient is the pose gradient of the
    registration.  The forward keeps its projection and tile lists
    (gs_render_saved), so the backward neither projects nor bins again."""

    @staticmethod
    def forward(fctx, gsctx, cams, poses, pivots, means4, log_scales4, quats4, logits, rgb4, twist):
        g = gsreg.Gaussians(means4.contiguous(), log_scales4.contiguous(), quats4.contiguous(), logits.contiguous(),
                            rgb4.contiguous())
        out, saved = gsreg.gs_render_saved(gsctx, g, poses, cams)
        fctx.gsctx, fctx.saved = gsctx, saved
        fctx.save_for_backward(pivots)
        return out["rgb"], out["depth"], out["alpha"]

    @staticmethod
    def backward(fctx, d_rgb, d_depth, d_alpha):
        (pivots,) = fctx.saved_tensors
        pg, gr = gsreg.gs_render_backward_saved(fctx.gsctx, fctx.saved, d_rgb.contiguous(), d_depth.contiguous(),
                                                d_alpha.contiguous(), pivots, params=True)
        fctx.saved.close()
        return (None, None, None, None, gr["means4"], gr["log_scales4"], gr["quats4"], gr["logits"], gr["rgb4"], pg)


def rasterize(gsctx, g, poses, cams, pivots=None, twist=None):
    """Differentiable render; returns (rgb, depth, alpha)."""
    nc = len(cams)
    if pivots is None:
        pivots = torch.zeros((nc, 3), dtype=torch.float32, device=g.means4.device)
    if twist is None:
        twist = torch.zeros((nc, 6), dtype=torch.float32, device=g.means4.device, requires_grad=True)
    return Rasterize.apply(gsctx, cams, poses.contiguous(), pivots.contiguous(), g.means4, g.log_scales4, g.quats4,
                           g.logits, g.rgb4, twist)
