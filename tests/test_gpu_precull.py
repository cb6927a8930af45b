"""Preculling (Sec. 3.3): cell visibility by the conservative hierarchical
depth test bit-exact against the oracle; a train step with preculling renders
and updates only the Gaussians of kept cells."""
import numpy as np
import pytest

import gs_inputs as gi
import oracle as O
from gpu_util import cams32, rel_l2, scene

pytestmark = pytest.mark.gpu


def _depths(cams, seed, walls=6):
    rng = np.random.default_rng(seed)
    out = []
    for w, h in zip(cams["width"], cams["height"]):
        d = np.full((int(h), int(w)), np.inf, np.float32)
        for _ in range(walls):
            y0, x0 = rng.integers(0, h), rng.integers(0, w)
            d[y0:y0 + rng.integers(4, h), x0:x0 + rng.integers(4, w)] = rng.uniform(1.0, 7.0)
        out.append(d)
    return out


@pytest.mark.parametrize("case", ["ring", "inside", "mixed_sizes"])
def test_cell_visibility_bit_exact(case):
    import torch
    import paper_2604_02851_b300 as gs
    if case == "ring":
        cams = gi.ring_cameras(4, 160, 96, radius=4.0)
        origin, size, dims = (-4.0, -2.0, -4.0), 0.5, (16, 8, 16)
    elif case == "inside":   # grid around the cameras: cells straddle the near plane
        cams = gi.ring_cameras(3, 120, 80, radius=1.0)
        origin, size, dims = (-2.0, -1.0, -2.0), 0.25, (16, 8, 16)
    else:
        cams = gi.cameras_from_eyes([(0.0, 0.5, 5.0), (3.0, 0.0, -4.0)], [200, 61], [113, 47])
        origin, size, dims = (-3.0, -3.0, -3.0), 0.37, (17, 17, 17)
    depths = _depths(cams, 3)
    ref = O.cell_visible(cams32(cams), depths, origin, size, dims)
    pc = gs.Precull(origin, size, dims)
    ctx = gs.Context(0, 0)
    dep = torch.from_numpy(np.concatenate([d.ravel() for d in depths])).cuda()
    pc.update(ctx, cams, dep)
    torch.cuda.synchronize()
    got = pc.visible.cpu().numpy()
    assert 0 < ref.sum() < ref.size
    np.testing.assert_array_equal(got, ref)
    ctx.close()


def test_train_step_with_preculling_updates_only_kept_gaussians():
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import OnlineTrainer, estimate_keys
    n, sh = 20_000, 1
    cams = gi.ring_cameras(3, 160, 112)
    planes = scene(n, sh, 90)
    target = O.forward(scene(n, sh, 91), sh, cams32(cams))["image"].astype(np.float32)
    origin, size, dims = (-1.0, -1.0, -1.0), 0.25, (8, 8, 8)
    pc = gs.Precull(origin, size, dims)
    rng = np.random.default_rng(4)
    vis = (rng.random(dims[::-1]) < 0.6).astype(np.uint8)
    pc.visible.copy_(torch.from_numpy(vis))
    cell = O.cell_of(gi.planes_to_rows(planes)[:, :3], origin, size, dims)
    kept = vis.ravel()[cell].astype(bool)
    assert 0.3 < kept.mean() < 0.9

    ctx = gs.Context(0, 0)
    t_all = torch.from_numpy(planes).cuda()
    keys = estimate_keys(ctx, t_all, sh, cams, slack=1.5)
    p_a = torch.from_numpy(planes).cuda()
    tr = OnlineTrainer(p_a, sh, cams, keys, ctx=ctx, precull=pc)
    tr.targets.copy_(torch.from_numpy(target.ravel()))
    tr.step()
    torch.cuda.synchronize()
    tr.raise_status()

    # reference: the culled Gaussians made transparent (they never pass the
    # 1/255 cut-off, so they contribute nothing and get zero gradient)
    ref_planes = planes.copy()
    ref_planes[0, ~kept, 3] = -60.0
    p_b = torch.from_numpy(ref_planes).cuda()
    ctx2 = gs.Context(0, 0)
    tr2 = OnlineTrainer(p_b, sh, cams, keys, ctx=ctx2)
    tr2.targets.copy_(torch.from_numpy(target.ravel()))
    tr2.step()
    torch.cuda.synchronize()
    tr2.raise_status()

    np.testing.assert_array_equal(tr.image.cpu().numpy(), tr2.image.cpu().numpy())
    assert abs(tr.loss() - tr2.loss()) <= 1e-6 * abs(tr2.loss())
    pa, pb = p_a.cpu().numpy(), p_b.cpu().numpy()
    # culled: parameters and Adam moments untouched
    np.testing.assert_array_equal(pa[:, ~kept], planes[:, ~kept])
    assert not tr.m.cpu().numpy()[:, ~kept].any() and not tr.v.cpu().numpy()[:, ~kept].any()
    # kept: the same update as the reference
    assert rel_l2(pa[:, kept] - planes[:, kept], pb[:, kept] - planes[:, kept]) <= 1e-4
    for c in (ctx, ctx2):
        c.close()


def test_render_with_all_cells_kept_equals_plain_render():
    """Kept cells everywhere: the depth items of Gaussians culled by the
    frustum are compacted away before the sort, and the image is unchanged."""
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import estimate_keys
    n, sh = 30_000, 2
    planes = scene(n, sh, 95)
    rows = gi.planes_to_rows(planes)
    rows[: n // 2, 2] += 6.0    # half the model behind view 0 / outside several frusta
    planes = gi.rows_to_planes(rows)
    cams = gi.ring_cameras(4, 144, 96)
    params = torch.from_numpy(planes).cuda()
    ctx = gs.Context(0, 0)
    keys = estimate_keys(ctx, params, sh, cams, slack=1.5)
    ctx.reserve(ctx.workspace_size(cams, n, keys))
    d_cams = gs.cameras_to_device(cams)
    tt = ctx.total_tiles(cams)
    npix = gs.total_pixels(cams)
    a = gs.gs_render_batch(ctx, params, sh, d_cams, 4, tt, keys, npix)
    pc = gs.Precull((-4.0, -4.0, -4.0), 1.0, (8, 8, 12))
    b = gs.gs_render_batch(ctx, params, sh, d_cams, 4, tt, keys, npix, precull=pc)
    torch.cuda.synchronize()
    assert ctx.status()[0] == 0
    np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    ctx.close()
