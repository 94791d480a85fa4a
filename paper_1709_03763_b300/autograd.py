"""torch.autograd.Function over the integration + loss kernels and the hand-written adjoint.

SurfaceLoss.apply(xi, depths, ...) integrates every keyframe k at pose
exp(xi_k^) T_k into a freshly reset volume, evaluates the SDF loss, and in the
backward pass runs the adjoint kernel, which recomputes each voxel's projection
instead of storing it.  The pose gradient is that of the left se(3) perturbation
at the integrated pose (equal to d L / d xi at xi = 0).
"""
from __future__ import annotations

import numpy as np
import torch

from .volume import Volume, pose_exp_left


class SurfaceLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xi: torch.Tensor, depths: torch.Tensor, vol: Volume, kf_ids, poses0, rgbas, intr,
                points: torch.Tensor, lam: float):
        xs = xi.detach().double().cpu().numpy().reshape(-1, 6)
        poses = np.stack([pose_exp_left(poses0[k], xs[k]) for k in range(len(kf_ids))])
        vol.reset()
        for k, kid in enumerate(kf_ids):
            vol.integrate(int(kid), depths[k].detach().contiguous(), rgbas[k], intr, poses[k])
        out, grad_D = vol.sdf_loss(points, lam)
        ctx.vol = vol
        ctx.kf_ids = list(kf_ids)
        ctx.poses = poses
        ctx.intr = intr
        ctx.save_for_backward(depths.detach(), grad_D)
        ctx.xi_dtype, ctx.xi_device = xi.dtype, xi.device
        return out[0].clone()

    @staticmethod
    def backward(ctx, gL):
        depths, grad_D = ctx.saved_tensors
        gx, gd = ctx.vol.sdf_adjoint(ctx.kf_ids, [depths[k] for k in range(len(ctx.kf_ids))], ctx.poses,
                                     ctx.intr, grad_D, with_depth=ctx.needs_input_grad[1])
        gxi = (gx * gL.to(gx.dtype)).to(device=ctx.xi_device, dtype=ctx.xi_dtype) if ctx.needs_input_grad[0] else None
        gdep = (gd * gL.to(gd.dtype)) if (gd is not None and ctx.needs_input_grad[1]) else None
        return gxi, gdep, None, None, None, None, None, None, None


def surface_loss(xi, depths, vol, kf_ids, poses0, rgbas, intr, points, lam=0.1):
    return SurfaceLoss.apply(xi, depths, vol, kf_ids, poses0, rgbas, intr, points, lam)
