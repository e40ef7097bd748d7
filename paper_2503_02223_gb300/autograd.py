"""The rasterizer and the quadric bbox loss as differentiable torch operations.

The adjoints are the library's hand-written backward kernels (dqo_render_backward,
dqo_quadric_bbox_loss); torch only routes gradients.  The render's forward keeps no
per-pixel list of blended Gaussians: the library context holds T_final and the blended
count per pixel, and the backward walks each pixel's list again back to front,
recomputing every Gaussian's alpha and transmittance.  If another forward on the same
Rasterizer ran in between, the backward first re-runs this forward to rebuild that state.
"""
from __future__ import annotations

import torch

from . import dqo

_PARAMS = ("means", "log_scales", "quats", "opacity_logit", "rgb")


class Rasterizer:
    """One keyframe camera, its settings and a library context (workspace).

    render(means, log_scales, quats, opacity_logit, rgb, obj_id, flags, targets=None)
    returns (rgb [H,W,3], depth [H,W], alpha [H,W], ins [H,W]), differentiable w.r.t. the five
    float parameter tensors.  `targets` (dict of rgb, depth, gt_id CUDA tensors) defines the
    pixel labels of the instance channel (Eq. 15)."""

    def __init__(self, camera: dict, num_objects: int, device: int | None = None, **settings):
        self.ctx = dqo.Context(device)
        self.camera = camera
        self.cs = dqo.camera(camera)
        self.st = dqo.settings(**settings)
        self.num_objects = num_objects
        self.generation = 0   # forwards run on this context

    def render(self, means, log_scales, quats, opacity_logit, rgb, obj_id, flags, targets=None):
        return _RenderFn.apply(means, log_scales, quats, opacity_logit, rgb, obj_id, flags, self, targets)

    # -- plumbing used by _RenderFn
    def _forward(self, g: dict, targets):
        W, H = self.camera["width"], self.camera["height"]
        dev = g["means"].device
        out = dqo.alloc_outputs(W, H, dev, loss=False, id_map=False)
        gs = dqo.gaussians(g, self.num_objects)
        dqo.dqo_render_forward(self.ctx, self.st, gs, self.cs, dqo.targets(targets), dqo.render_out(out))
        self.generation += 1
        return out, gs

    def close(self):
        self.ctx.close()


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, means, log_scales, quats, opacity_logit, rgb, obj_id, flags, raster, targets):
        g = dict(means=means.detach().contiguous(), log_scales=log_scales.detach().contiguous(),
                 quats=quats.detach().contiguous(), opacity_logit=opacity_logit.detach().contiguous(),
                 rgb=rgb.detach().contiguous(), obj_id=obj_id.contiguous(), flags=flags.contiguous())
        out, _ = raster._forward(g, targets)
        fctx.raster = raster
        fctx.targets = targets
        fctx.generation = raster.generation
        fctx.g = g
        return out["rgb"], out["depth"], out["alpha"], out["ins"]

    @staticmethod
    def backward(fctx, g_rgb, g_depth, g_alpha, g_ins):
        raster, g = fctx.raster, fctx.g
        if raster.generation != fctx.generation:   # the context holds another forward's state
            raster._forward(g, fctx.targets)
        n = g["means"].shape[0]
        grads = dqo.alloc_grads(n, g["means"].device)
        pg = {}
        for k, t in (("rgb", g_rgb), ("depth", g_depth), ("alpha", g_alpha), ("ins", g_ins)):
            pg[k] = None if t is None else t.contiguous()
        dqo.dqo_render_backward(raster.ctx, raster.st, dqo.gaussians(g, raster.num_objects), raster.cs,
                                dqo.targets(fctx.targets), dqo.pixel_grads(pg), dqo.gaussian_grads(grads))
        return (grads["means"], grads["log_scales"], grads["quats"], grads["opacity_logit"], grads["rgb"],
                None, None, None, None)


class QuadricBBoxLoss:
    """Eq. 12 bbox loss per quadric as a differentiable torch op over params [Q,9]."""

    def __init__(self, P: torch.Tensor, q_ptr: torch.Tensor, pair_v: torch.Tensor, obs: torch.Tensor,
                 device: int | None = None):
        self.ctx = dqo.Context(device)
        self.P, self.q_ptr, self.pair_v, self.obs = P, q_ptr, pair_v, obs

    def __call__(self, params: torch.Tensor) -> torch.Tensor:
        return _QuadricLossFn.apply(params, self)

    def close(self):
        self.ctx.close()


class _QuadricLossFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params, op):
        p = params.detach().contiguous()
        loss = torch.zeros(p.shape[0], device=p.device)
        dpar = torch.zeros_like(p)
        dqo.dqo_quadric_bbox_loss(op.ctx, p, op.P, op.q_ptr, op.pair_v, op.obs, loss, dpar)
        fctx.save_for_backward(dpar)
        return loss

    @staticmethod
    def backward(fctx, g_loss):
        (dpar,) = fctx.saved_tensors
        return dpar * g_loss[:, None], None
