"""torch.autograd binding of the rasterizer: one view rendered through the C
ABI (gs2d_project, gs2d_bin_sort, gs2d_render_fwd) with gs2d_render_bwd as
its backward, so a loss written with torch ops on the rendered images
differentiates to every surfel parameter and to the camera pose (Sec. III-B).

The pose enters as a base world-to-camera pose T (12 floats, not
differentiated) and a tangent tau = (rho, theta) of the left perturbation:
the view is rendered at Exp(tau) T and the pose gradient returned for tau is
dL/dtau at tau = 0 (exact when tau is zero, first order otherwise) -- the
usual pattern is tau = 0 during the backward, an optimiser step on tau, then
T <- Exp(tau) T and tau <- 0.

The rasterizer holds the forward's records, bins and per-pixel compositing
state until the backward, so one Rasterizer serves one forward / backward
pair at a time.
"""
from __future__ import annotations

import torch

from . import gs2d


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, quat, scale, opacity, rgb, tau, pose, rast):
        surf = gs2d.DeviceSurfels.from_tensors(mu, quat, scale, opacity, rgb)
        p = pose.detach().reshape(1, 12).clone()
        if bool(torch.any(tau != 0)):
            gs2d.gs2d_net_apply((tau.detach().float() / gs2d.NET_TAU_SCALE).reshape(1, 6).contiguous(), p)
        p = p.reshape(12)
        out = rast.forward(surf, p)
        ctx.rast = rast
        ctx.surf = surf
        ctx.pose = p
        return (out["rgb"].clone(), out["depth"].clone(), out["normal"].clone(),
                out["opacity"].clone())

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_normal, g_opac):
        z = lambda g, like: torch.zeros_like(like) if g is None else g.contiguous()
        r = ctx.rast
        g = r.backward(ctx.surf, ctx.pose, z(g_rgb, r.rgb), z(g_depth, r.depth),
                       z(g_normal, r.normal), z(g_opac, r.opacity), full=True)
        return g["mu"], g["quat"], g["scale"], g["opacity"], g["rgb"], g["pose6"], None, None


def render(mu, quat, scale, opacity, rgb, tau, pose, rast):
    """Images (rgb, depth, normal, opacity) of one view; differentiable
    w.r.t. the surfel tensors and tau."""
    return RenderFunction.apply(mu, quat, scale, opacity, rgb, tau, pose, rast)
