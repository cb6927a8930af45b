"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and convert its outputs into the oracle's layouts (no arithmetic of the
method here; only reinterpretation of bits and layouts)."""
from __future__ import annotations

import numpy as np

import gs_inputs as gi


def cams32(cams: dict) -> dict:
    """The camera set as the GPU sees it (float32-rounded), for the oracle."""
    out = dict(cams)
    for k in ("R", "t", "fx", "fy", "cx", "cy", "near"):
        out[k] = np.asarray(cams[k], dtype=np.float32).astype(np.float64)
    return out


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def gpu_proj_to_oracle(proj_gpu: np.ndarray) -> np.ndarray:
    """float32 [V][n][16] GPU records -> oracle proj layout (float64)."""
    p = np.ascontiguousarray(proj_gpu, dtype=np.float32)
    bits = p.view(np.uint32)
    out = p.astype(np.float64)
    out[..., 11] = bits[..., 11]
    lo, hi = bits[..., 12], bits[..., 13]
    out[..., 12] = lo & 0xFFFF
    out[..., 13] = lo >> 16
    out[..., 14] = hi & 0xFFFF
    out[..., 15] = hi >> 16
    return out


def oracle_grad2d_to_gpu_order(g9: np.ndarray) -> np.ndarray:
    """Oracle [V][n][9] -> [V][n][12] with zero padding, as the GPU stores it."""
    V, n = g9.shape[:2]
    out = np.zeros((V, n, 12))
    out[..., :9] = g9
    return out


# |x - y| below which the sign of the L1 term is not fixed by a float32
# render: the compositing error of one pixel is ~1e-7..1e-6 (image rel-L2
# ~6e-7 at these sizes), so 1e-5 leaves a margin of ten.
L1_TIE_TAU = 1e-5


def l1_sign_expected(O, planes, sh, cams, r, target, image_gpu, w_l1=0.8, tau=L1_TIE_TAU, dyn=None):
    """The oracle's parameter gradient with the L1 sign taken as the float32
    render takes it, where that choice is one of the correct ones.

    The L1 term's derivative is w_l1 sign(x - y) / M.  Where the FP64 image
    lies within `tau` of the target (and is not equal to it), a float32
    render may land on either side of the target or on it, so sign -1, 0 and
    +1 are all correct results of the method there.  The float32 decision
    sign(x32 - y32) is exact given the float32 image; it must agree with the
    oracle's everywhere else (asserted).  The adjoint is linear in dL/dimage
    for a fixed forward pass, so the oracle's gradient for the float32 signs
    is its own gradient plus its adjoint of the sign changes at the ties.
    Returns (expected dparams, number of tie elements whose sign differs)."""
    img = np.asarray(r["image"], dtype=np.float64).ravel()
    tgt32 = np.asarray(target, dtype=np.float32).ravel()
    tgt = tgt32.astype(np.float64)
    s_o = np.sign(img - tgt)
    s_g = np.sign(np.asarray(image_gpu, dtype=np.float32).ravel() - tgt32).astype(np.float64)
    differ = s_o != s_g
    if not differ.any():
        return r["dparams"], 0
    gap = np.abs(img - tgt)[differ]
    assert np.all(gap <= tau), f"L1 sign differs at |x - y| = {gap.max():.3g}, above the tie band {tau}"
    c = np.zeros(img.size)
    c[differ] = (s_g - s_o)[differ] * w_l1 / img.size
    g2 = O.render_bwd(cams, r["proj"], r["vals"], r["ranges"], c)
    return r["dparams"] + O.project_bwd(planes, sh, cams, g2, dyn=dyn), int(differ.sum())


class GpuRun:
    """One pass of the whole CUDA path on a small case, all intermediates kept."""

    def __init__(self, planes, sh_degree, cams, target=None, keys_cap=None, bg=(0.0, 0.0, 0.0),
                 tile=16, sort_bits=8, w_l1=0.8, w_ssim=0.2, dyn=None, raster_threads=4, lighting=None,
                 raster_bwd_threads=None):
        import torch
        import paper_2604_02851_b300 as gs
        self.gs = gs
        self.torch = torch
        self.cams = cams
        self.V = V = len(cams["fx"])
        self.n = n = planes.shape[1]
        self.sh = sh_degree
        self.bg = bg
        self.ctx = gs.Context(0, 0, tile=tile, sort_bits=sort_bits, raster_threads=raster_threads,
                              raster_bwd_threads=raster_bwd_threads)
        self.params = torch.from_numpy(np.ascontiguousarray(planes, dtype=np.float32)).cuda()
        self.d_cams = gs.cameras_to_device(cams)
        self.tt = self.ctx.total_tiles(cams)
        self.npix = gs.total_pixels(cams)
        if keys_cap is None:
            keys_cap = 1 << 16
        self.ctx.reserve(self.ctx.workspace_size(cams, n, keys_cap))
        self.dyn = dyn
        self.lighting = lighting
        self.proj = gs.gs_project(self.ctx, self.params, sh_degree, self.d_cams, V, dyn=dyn, lighting=lighting)
        self.keys, self.vals, self.ranges, self.nk = gs.gs_bin_sort(
            self.ctx, self.proj, self.d_cams, V, n, self.tt, keys_cap)
        torch.cuda.synchronize()
        code, detail = self.ctx.status()
        if code == 2:  # capacity: grow and redo, as a caller would
            keys_cap = int(detail) + 1024
            self.ctx.reserve(self.ctx.workspace_size(cams, n, keys_cap))
            self.keys, self.vals, self.ranges, self.nk = gs.gs_bin_sort(
                self.ctx, self.proj, self.d_cams, V, n, self.tt, keys_cap)
            torch.cuda.synchronize()
            code, detail = self.ctx.status()
        assert code == 0, (code, detail)
        self.K = int(self.nk.item())
        self.image, self.T, self.nc = gs.gs_render_fwd(self.ctx, self.proj, self.d_cams, V, n, self.tt,
                                                       self.vals, self.ranges, self.npix, bg=bg)
        if target is not None:
            H, W = int(cams["height"][0]), int(cams["width"][0])
            self.target = torch.from_numpy(np.ascontiguousarray(target, dtype=np.float32)).cuda()
            self.loss, self.dimage = gs.gs_loss(self.ctx, self.image, self.target, V, H, W, w_l1, w_ssim)
            self.grad2d, self.dparams = gs.gs_render_bwd(
                self.ctx, self.params, sh_degree, self.d_cams, V, self.tt, self.proj, self.vals, self.ranges,
                self.T, self.nc, self.dimage, bg=bg, dyn=dyn, lighting=lighting)
        torch.cuda.synchronize()
        code, detail = self.ctx.status()
        assert code == 0, (code, detail)

    def np(self, name):
        return getattr(self, name).cpu().numpy()

    def oracle_proj(self):
        return gpu_proj_to_oracle(self.np("proj"))

    def sorted_vals(self):
        return self.np("vals")[:self.K].view(np.uint32)

    def sorted_keys(self):
        return self.np("keys")[:self.K].view(np.uint32)

    def ranges_np(self):
        return self.np("ranges").view(np.uint32)

    def close(self):
        self.ctx.close()


def scene(n, sh_degree, seed=0, scale_shift=0.0):
    p = gi.make_scene(n, sh_degree, seed)
    if scale_shift:
        p[1, :, :3] += scale_shift
    return p
