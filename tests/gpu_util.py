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


def oracle_proj_to_gpu(og: np.ndarray) -> np.ndarray:
    """Oracle proj [V][n][16] (float64) -> the GPU's float32 record layout
    [V][n][16]: float fields rounded to float32, the clamp mask and the tile
    rectangle as bits, the rectangle's tile count in field 14.  The inverse of
    gpu_proj_to_oracle on the fields both keep."""
    og = np.asarray(og, dtype=np.float64)
    out = og.astype(np.float32)
    bits = out.view(np.uint32)
    x0, y0, x1, y1 = (og[..., 12 + i].astype(np.uint32) for i in range(4))
    bits[..., 11] = og[..., 11].astype(np.uint32)
    bits[..., 12] = x0 | (y0 << np.uint32(16))
    bits[..., 13] = x1 | (y1 << np.uint32(16))
    bits[..., 14] = (x1 - x0) * (y1 - y0)
    bits[..., 15] = 0
    return np.ascontiguousarray(out)


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


def l1_sign_expected(O, planes, sh, cams, r, target, grad_gpu, w_l1=0.8, tau=L1_TIE_TAU, dyn=None, keep=None):
    """The oracle's parameter gradient for the L1 signs the float32 render
    took where each sign is correct, found without feeding the oracle any
    GPU value.

    The L1 term's derivative is w_l1 sign(x - y) / M.  Where the FP64 image
    lies within `tau` of the target (and is not equal to it), a float32
    render may land on either side of the target, so the derivative at such a
    tie element e may be anything in w_l1 / M [-1, 1].  The oracle's adjoint
    is linear in dL/dimage: the correct gradients form the family
    base + A s, base the oracle's gradient without the tie elements' L1
    terms, A[:, e] the oracle's adjoint of w_l1 / M at element e, |s_e| <= 1.
    The member closest (least squares over the Gaussians in `keep`) to the
    GPU gradient is returned; the caller compares the GPU gradient with it.
    Returns (expected dparams, number of tie elements)."""
    img = np.asarray(r["image"], dtype=np.float64).ravel()
    tgt = np.asarray(target, dtype=np.float32).ravel().astype(np.float64)
    d = img - tgt
    ties = np.nonzero((np.abs(d) <= tau) & (d != 0.0))[0]
    if len(ties) == 0:
        return r["dparams"], 0
    shape = r["dparams"].shape
    sel = np.ones(shape, dtype=bool) if keep is None else np.broadcast_to(np.asarray(keep)[None, :, None], shape)
    sel = sel.ravel()
    gg = np.asarray(grad_gpu, dtype=np.float64).ravel()
    od = r["dparams"].ravel()
    # the oracle's own signs are one member of the family: when they already
    # match closely, the per-element adjoints are not needed
    if np.linalg.norm((gg - od)[sel]) <= 0.25 * 1e-4 * np.linalg.norm(od[sel]):
        return r["dparams"], len(ties)
    M = img.size
    cols = []
    for e in ties:
        c = np.zeros(M)
        c[e] = w_l1 / M
        g2 = O.render_bwd(cams, r["proj"], r["vals"], r["ranges"], c)
        cols.append(O.project_bwd(planes, sh, cams, g2, dyn=dyn).ravel())
    A = np.stack(cols, 1)
    base = od - A @ np.sign(d[ties])
    s, *_ = np.linalg.lstsq(A[sel], (gg - base)[sel], rcond=None)
    s = np.clip(s, -1.0, 1.0)
    return (base + A @ s).reshape(shape), len(ties)


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


class OracleStages:
    """The oracle's own chain on one case, each intermediate rounded to
    float32 as the GPU stages take it, and each GPU stage run through the C
    ABI on those oracle inputs.  Nothing the CUDA path computes flows into the
    oracle: the GPU stage's inputs come from the oracle, and its output is
    compared with the oracle stage on the same (float32) inputs."""

    def __init__(self, O, planes, sh_degree, cams, target, dyn=None, gpu_dyn=None, gpu_lighting=None, tile=16):
        """dyn: the oracle's dynamics / lighting dict; gpu_dyn, gpu_lighting:
        the same inputs as the binding's Dynamics / Lighting objects."""
        import torch
        import paper_2604_02851_b300 as gs
        self.O, self.gs, self.torch = O, gs, torch
        self.planes, self.sh, self.cams, self.dyn = planes, sh_degree, cams, dyn
        self.gpu_dyn, self.gpu_lighting = gpu_dyn, gpu_lighting
        self.V = len(cams["fx"])
        self.n = planes.shape[1]
        self.H, self.W = int(cams["height"][0]), int(cams["width"][0])
        # oracle chain; the projection records rounded to float32 are the
        # shared input of every later stage on both sides
        og = O.project(planes, sh_degree, cams, tile, dyn)
        self.proj32 = oracle_proj_to_gpu(og)
        self.projd = gpu_proj_to_oracle(self.proj32)
        self.depth32 = self.proj32[..., 2].copy()
        self.rects = self.projd[..., 12:16].astype(np.int32)
        self.keys, self.vals, self.ranges = O.bin_sort(cams, self.rects, self.depth32, tile)
        img, T, nc = O.render(cams, self.projd, self.vals, self.ranges, tile=tile)
        self.image, self.T, self.nc = img, T, nc
        self.target = np.asarray(target, dtype=np.float32)
        self.image32 = img.astype(np.float32)
        self.loss, dimg = O.loss(self.image32.astype(np.float64), self.target.astype(np.float64), self.V, self.H, self.W)
        self.dimage32 = dimg.astype(np.float32)
        self.grad2d = O.render_bwd(cams, self.projd, self.vals, self.ranges, self.dimage32.astype(np.float64), tile=tile)
        self.grad2d32 = self.grad2d.astype(np.float32)
        self.dparams = O.project_bwd(planes, sh_degree, cams, self.grad2d32.astype(np.float64), tile, dyn)
        # device copies of the oracle's inputs
        self.ctx = gs.Context(0, 0, tile=tile)
        self.d_cams = gs.cameras_to_device(cams)
        self.tt = self.ctx.total_tiles(cams)
        self.npix = gs.total_pixels(cams)
        self.K = len(self.vals)
        self.ctx.reserve(self.ctx.workspace_size(cams, self.n, max(self.K, 1)))
        self.t_proj = torch.from_numpy(self.proj32).cuda()
        self.t_vals = torch.from_numpy(np.ascontiguousarray(self.vals.view(np.int32))).cuda()
        self.t_ranges = torch.from_numpy(np.ascontiguousarray(self.ranges.view(np.int32))).cuda()
        self.t_params = torch.from_numpy(np.ascontiguousarray(planes, dtype=np.float32)).cuda()

    def gpu_bin_sort(self):
        gs, torch = self.gs, self.torch
        keys, vals, ranges, nk = gs.gs_bin_sort(self.ctx, self.t_proj, self.d_cams, self.V, self.n, self.tt,
                                                max(self.K, 1))
        torch.cuda.synchronize()
        K = int(nk.item())
        return (keys.cpu().numpy()[:K].view(np.uint32), vals.cpu().numpy()[:K].view(np.uint32),
                ranges.cpu().numpy().view(np.uint32))

    def gpu_render_fwd(self):
        gs, torch = self.gs, self.torch
        img, T, nc = gs.gs_render_fwd(self.ctx, self.t_proj, self.d_cams, self.V, self.n, self.tt, self.t_vals,
                                      self.t_ranges, self.npix)
        torch.cuda.synchronize()
        return img, T, nc

    def gpu_loss(self):
        gs, torch = self.gs, self.torch
        img = torch.from_numpy(self.image32).cuda()
        tgt = torch.from_numpy(self.target).cuda()
        loss, dimg = gs.gs_loss(self.ctx, img, tgt, self.V, self.H, self.W)
        torch.cuda.synchronize()
        return float(loss.item()), dimg.cpu().numpy()

    def gpu_raster_bwd(self):
        """The GPU adjoint on the oracle's records, lists and image gradient;
        its transmittance and contributor counts come from the GPU's own
        compositing of the same records (a GPU stage feeding a GPU stage)."""
        gs, torch = self.gs, self.torch
        _, T, nc = self.gpu_render_fwd()
        dimg = torch.from_numpy(self.dimage32).cuda()
        g2 = gs.gs_raster_bwd(self.ctx, self.t_proj, self.d_cams, self.V, self.n, self.tt, self.t_vals,
                              self.t_ranges, T, nc, dimg)
        torch.cuda.synchronize()
        return g2.cpu().numpy()

    def gpu_project_bwd(self):
        gs, torch = self.gs, self.torch
        g12 = np.zeros((self.V, self.n, 12), dtype=np.float32)
        g12[..., :9] = self.grad2d32
        g2 = torch.from_numpy(g12).cuda()
        dp = gs.gs_project_bwd(self.ctx, self.t_params, self.sh, self.d_cams, self.V, self.t_proj, g2,
                               dyn=self.gpu_dyn, lighting=self.gpu_lighting)
        torch.cuda.synchronize()
        return dp.cpu().numpy()

    def close(self):
        self.ctx.raise_status()
        self.ctx.close()
