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
    pivot, evaluated at zero: it must be zero, and its gradient is the pose
    gradient of the registration."""

    @staticmethod
    def forward(fctx, gsctx, cams, poses, pivots, means4, log_scales4, quats4, logits, rgb4, twist):
        if torch.any(twist != 0):
            raise ValueError("the twist input is evaluated at zero")
        g = gsreg.Gaussians(means4.contiguous(), log_scales4.contiguous(), quats4.contiguous(), logits.contiguous(),
                            rgb4.contiguous())
        out = gsreg.gs_render(gsctx, g, poses, cams)
        fctx.gsctx, fctx.cams = gsctx, cams
        fctx.save_for_backward(g.means4, g.log_scales4, g.quats4, g.logits, g.rgb4, poses, pivots, out["t_final"],
                               out["last"])
        return out["rgb"], out["depth"], out["alpha"]

    @staticmethod
    def backward(fctx, d_rgb, d_depth, d_alpha):
        m, s, q, lg, c, poses, pivots, tf, last = fctx.saved_tensors
        g = gsreg.Gaussians(m, s, q, lg, c)
        pg, gr = gsreg.gs_render_backward(fctx.gsctx, g, poses, fctx.cams, tf, last, d_rgb.contiguous(),
                                          d_depth.contiguous(), d_alpha.contiguous(), pivots, params=True)
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
