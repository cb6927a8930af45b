"""``GaussianRasterize``: the differentiable render as a torch.autograd.Function.

Forward runs projection, binning/sort and compositing through the C ABI
(gs_project, gs_bin_sort, gs_render_fwd); backward runs the hand-written
adjoint (gs_render_bwd), which recomputes each pixel's blend state from the
stored final transmittance and last-contributor index instead of keeping
per-fragment state.  Sec. 3.2.3: the model is refined "by differentiable
rendering"; Sec. 3.1: the optimiser renders the model from the reference
views, compares with the captured images and updates the parameters.
"""
from __future__ import annotations

import torch

from . import (Context, _lib, cameras_to_device, gs_bin_sort, gs_project, gs_render_bwd, gs_render_fwd,
               pack_cameras, total_pixels)


class RenderSetup:
    """Cameras, context and key capacity shared by forward and backward."""

    def __init__(self, cams, sh_degree: int, n: int, keys_cap: int, bg=(0.0, 0.0, 0.0), ctx: Context | None = None,
                 device="cuda"):
        self.packed = pack_cameras(cams) if not hasattr(cams, "dtype") else cams
        self.V = len(self.packed)
        self.sh = sh_degree
        self.n = n
        self.bg = tuple(bg)
        self.ctx = ctx or Context(torch.device(device).index or 0, 0)
        self.keys_cap = int(keys_cap)
        self.ctx.reserve(self.ctx.workspace_size(self.packed, n, self.keys_cap))
        self.d_cams = cameras_to_device(self.packed, device)
        self.total_tiles = self.ctx.total_tiles(self.packed)
        self.npix = total_pixels(self.packed)


class GaussianRasterize(torch.autograd.Function):
    """images = GaussianRasterize.apply(params, setup): params float32 [15, n, 4]
    on the device; images float32, views concatenated, each planar [3, H, W]."""

    @staticmethod
    def forward(ctx, params, setup: RenderSetup):
        s = setup
        proj = gs_project(s.ctx, params, s.sh, s.d_cams, s.V)
        _, vals, ranges, nk = gs_bin_sort(s.ctx, proj, s.d_cams, s.V, s.n, s.total_tiles, s.keys_cap,
                                          want_keys=False)
        image, T, nc = gs_render_fwd(s.ctx, proj, s.d_cams, s.V, s.n, s.total_tiles, vals, ranges, s.npix, bg=s.bg)
        ctx.setup = s
        ctx.save_for_backward(params, proj, vals, ranges, T, nc)
        return image

    @staticmethod
    def backward(ctx, grad_image):
        params, proj, vals, ranges, T, nc = ctx.saved_tensors
        s = ctx.setup
        _, dparams = gs_render_bwd(s.ctx, params, s.sh, s.d_cams, s.V, s.total_tiles, proj, vals, ranges, T, nc,
                                   grad_image.contiguous(), bg=s.bg)
        return dparams, None


def rasterize(params, setup: RenderSetup):
    return GaussianRasterize.apply(params, setup)


def check_status(setup: RenderSetup) -> None:
    """Raise if a kernel recorded an error (for example a key capacity that
    was too small for the current model)."""
    code, detail = setup.ctx.status()
    if code != _lib.GS_OK:
        raise _lib.GsError(f"device status (detail {detail})", code)


class L1DSSIMLoss(torch.autograd.Function):
    """loss = L1DSSIMLoss.apply(image, target, setup, H, W, w_l1, w_ssim):
    w_l1 mean|x - y| + w_ssim (1 - mean SSIM) over equal-size views, with the
    image gradient computed by the same call (gs_loss)."""

    @staticmethod
    def forward(ctx, image, target, setup: RenderSetup, H: int, W: int, w_l1: float = 0.8, w_ssim: float = 0.2):
        from . import gs_loss
        d_loss, dimage = gs_loss(setup.ctx, image.contiguous(), target.contiguous(), setup.V, H, W, w_l1, w_ssim)
        ctx.save_for_backward(dimage)
        return d_loss[0]

    @staticmethod
    def backward(ctx, grad_out):
        (dimage,) = ctx.saved_tensors
        return dimage * grad_out, None, None, None, None, None, None
