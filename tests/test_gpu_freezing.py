"""Gaussian freezing (Sec. 3.3): a frozen pool is rendered with the active
one but gets no gradient, no Adam update and no delta.  The fused step with a
frozen pool must equal the step over the union through the separate entry
points with the frozen rows' update dropped, and the active gradient must
match the oracle's gradient of the union."""
import numpy as np
import pytest

import gs_inputs as gi
import oracle as O
from flips import decision_flips
from gpu_util import cams32, gpu_proj_to_oracle, l1_sign_expected, rel_l2, scene

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bwd_threads", [4, 2])
def test_frozen_pool_step_equals_union_step_with_frozen_rows_fixed(bwd_threads):
    """bwd_threads: the compositing adjoint's layout in the fused step."""
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import OnlineTrainer, estimate_keys
    na, nf, sh = 12_000, 8_000, 2
    cams = gi.ring_cameras(3, 176, 112)
    union = scene(na + nf, sh, 80)
    active = np.ascontiguousarray(union[:, :na])
    frozen = np.ascontiguousarray(union[:, na:])
    target = O.forward(scene(na + nf, sh, 81), sh, cams32(cams))["image"].astype(np.float32)

    # fused step with the frozen pool
    ctx = gs.Context(0, 0, raster_bwd_threads=bwd_threads)
    t_union = torch.from_numpy(union).cuda()
    keys = estimate_keys(ctx, t_union, sh, cams, slack=1.5)
    t_active = torch.from_numpy(active).cuda()
    t_frozen = torch.from_numpy(frozen).cuda()
    tr = OnlineTrainer(t_active, sh, cams, keys, ctx=ctx, frozen=t_frozen)
    tr.targets.copy_(torch.from_numpy(target.ravel()))
    tr.step_eager()
    torch.cuda.synchronize()
    tr.raise_status()

    # the same over the union, separate entry points, Adam on the active rows only
    c2 = gs.Context(0, 0)
    c2.reserve(c2.workspace_size(cams, na + nf, keys))
    d_cams = gs.cameras_to_device(cams)
    tt = c2.total_tiles(cams)
    npix = gs.total_pixels(cams)
    proj = gs.gs_project(c2, t_union, sh, d_cams, 3)
    _, vals, ranges, nk = gs.gs_bin_sort(c2, proj, d_cams, 3, na + nf, tt, keys, want_keys=False)
    image, T, nc = gs.gs_render_fwd(c2, proj, d_cams, 3, na + nf, tt, vals, ranges, npix)
    tgt = torch.from_numpy(target.ravel()).cuda()
    loss, dimg = gs.gs_loss(c2, image, tgt, 3, 112, 176)
    _, dpar = gs.gs_render_bwd(c2, t_union, sh, d_cams, 3, tt, proj, vals, ranges, T, nc, dimg)
    ga = dpar[:, :na].contiguous()
    th = torch.from_numpy(active).cuda()
    m = torch.zeros_like(th); v = torch.zeros_like(th)
    gs.gs_adam_step(c2, th, ga, m, v, gs.adam_cfg(lr=1e-3, step=1))
    torch.cuda.synchronize()
    assert c2.status()[0] == 0

    np.testing.assert_array_equal(tr.image.cpu().numpy(), image.cpu().numpy())
    assert abs(tr.loss() - float(loss.item())) <= 1e-6 * abs(float(loss.item()))
    assert rel_l2(tr.grads.cpu().numpy(), ga.cpu().numpy()) <= 1e-5
    assert rel_l2(t_active.cpu().numpy() - active, th.cpu().numpy() - active) <= 1e-4
    np.testing.assert_array_equal(t_frozen.cpu().numpy(), frozen)       # never written
    idx = tr.d_idx[:tr.delta_count()].cpu().numpy()
    assert tr.delta_count() == 0 or idx.max() < na                       # deltas cover the active pool

    # active gradient against the oracle's gradient of the union
    c32 = cams32(cams)
    r = O.loss_and_grad(union, sh, c32, target)
    gp = gpu_proj_to_oracle(proj.cpu().numpy())
    K = int(nk.item())
    flips, _ = decision_flips(c32, r["proj"], r["vals"], r["ranges"], gp,
                                vals.cpu().numpy()[:K].view(np.uint32), ranges.cpu().numpy().view(np.uint32))
    support = np.any(r["proj"][..., [7, 12, 13, 14, 15]] != gp[..., [7, 12, 13, 14, 15]], axis=(0, 2))
    odd = (flips.any(axis=0) | support)[:na]
    assert odd.mean() <= 1e-3
    g = tr.grads.cpu().numpy()
    gu = np.zeros_like(r["dparams"])
    gu[:, :na] = g
    keep_u = np.zeros(na + nf, dtype=bool)
    keep_u[:na] = ~odd
    od, _ = l1_sign_expected(O, union, sh, c32, r, target, gu, keep=keep_u)
    assert rel_l2(g[:, ~odd], od[:, :na][:, ~odd]) <= 1e-4
    for c in (ctx, c2):
        c.close()
