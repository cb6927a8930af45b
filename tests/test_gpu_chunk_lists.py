"""Per-tile lists in chunk-bitmap form against the expanded lists.

With two-level binning, gs_train_step and gs_render_batch do not expand the
super-tile lists into per-tile arrays: both raster kernels walk each tile's
entries through the bitmaps of its super-tile's 256-item chunks (forward in
list order, the adjoint back to front from the chunk of the last
contributor).  With direct binning they read the expanded lists.  Both forms
visit the same fragments in the same order, so the first step's rendered
image and loss are bit-identical; the gradients differ only in the order of
the float atomics, and so do the parameters (and the next step's image) by
rounding.  Cases: one super-tile holding many chunks, ragged image edges, big
splats spanning many super-tiles, both raster layouts, 8-pixel tiles, an
opaque scene whose pixels stop early, a tiny scene over many views (more
chunks than keys_cap / 256), 320 or 512 super-tiles, whose 9-bit key the
fused step sorts in one wide pass (the direct binning sorts tile keys), and
2304 super-tiles, more than the longest-list-first order ranks (the raster
kernels then take them in index order).
"""
import numpy as np
import pytest

import gs_inputs as gi
import oracle as O
from gpu_util import cams32, rel_l2, scene

pytestmark = pytest.mark.gpu

CASES = {
    # name: (n, sh, views, width, height, log-scale shift, logit shift, tile, fwd layout, bwd layout)
    "one_supertile_chunks": (60_000, 1, 1, 128, 128, 0.5, 0.0, 16, 4, 2),
    "ragged_edges": (20_000, 2, 3, 200, 136, 0.0, 0.0, 16, 2, 4),
    "big_splats": (3_000, 0, 2, 333, 250, 1.5, 0.0, 16, 4, 4),
    "opaque_early_stop": (30_000, 1, 2, 176, 112, 0.8, 4.0, 16, 4, 2),
    "tile8": (8_000, 0, 2, 150, 90, 0.5, 0.0, 8, 4, 4),
    # a handful of Gaussians over many views: more chunks (one per non-empty
    # super-tile) than keys_cap / 256, the bitmaps still fit
    "tiny_many_views": (12, 0, 16, 256, 160, 1.0, 2.0, 16, 4, 2),
    # 320 and 512 super-tiles (8-pixel tiles, 8 x 8 of them a super-tile):
    # the fused step sorts the 9-bit super-tile key in one wide pass
    "wide_key_320": (6_000, 0, 16, 320, 256, 0.3, 0.0, 8, 4, 4),
    "wide_key_512": (6_000, 0, 16, 512, 256, 0.3, 0.0, 8, 4, 4),
    # 2304 super-tiles, more than the raster order ranks: the identity order
    "many_supertiles": (3_000, 0, 16, 1536, 1536, 1.0, 0.0, 16, 4, 2),
}


def _trainer(mode, planes, sh, cams, target, tile, tpr, btpr):
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import OnlineTrainer, estimate_keys
    ctx = gs.Context(0, 0, tile=tile, binning=mode, raster_threads=tpr, raster_bwd_threads=btpr)
    params = torch.from_numpy(np.ascontiguousarray(planes)).cuda()
    cap = estimate_keys(ctx, params, sh, cams, slack=1.5)
    tr = OnlineTrainer(params, sh, cams, cap, ctx=ctx)
    tr.targets.copy_(target)
    return tr


@pytest.mark.parametrize("name", list(CASES))
def test_train_step_chunk_lists_match_expanded_lists(name):
    import torch
    n, sh, V, W, H, sshift, lshift, tile, tpr, btpr = CASES[name]
    planes = scene(n, sh, 21, sshift)
    planes[0, :, 3] += lshift
    cams = gi.ring_cameras(V, W, H)
    tgt = O.forward(scene(n, sh, 22, sshift), sh, cams32(cams))["image"].astype(np.float32)
    target = torch.from_numpy(np.ascontiguousarray(tgt.reshape(-1))).cuda()
    a = _trainer("two_level", planes, sh, cams, target, tile, tpr, btpr)
    b = _trainer("direct", planes, sh, cams, target, tile, tpr, btpr)
    for step in (1, 2):
        a.step()
        b.step()
        torch.cuda.synchronize()
        assert a.ctx.status()[0] == 0 and b.ctx.status()[0] == 0
        if step == 1:  # same parameters: same image and loss, bit for bit
            np.testing.assert_array_equal(a.image.cpu().numpy(), b.image.cpu().numpy())
            assert a.loss() == b.loss()
        else:
            # the second image differs by the rounding of the first update
            # (float atomics order); splats that each cover thousands of
            # pixels carry it into more of the image
            tol = 1e-5 if name == "many_supertiles" else 1e-6
            assert rel_l2(a.image.cpu().numpy(), b.image.cpu().numpy()) <= tol
            assert abs(a.loss() - b.loss()) <= tol * b.loss()
        assert rel_l2(a.grads.cpu().numpy(), b.grads.cpu().numpy()) <= 1e-5
        upd = np.linalg.norm(b.params.cpu().numpy() - planes)
        assert np.linalg.norm(a.params.cpu().numpy() - b.params.cpu().numpy()) <= 1e-3 * upd
    if name == "one_supertile_chunks":
        # the super-tile's list spans many 256-item chunks
        K = int(np.count_nonzero(O.project(planes, sh, cams32(cams))[..., 14] > 0))
        assert K > 20 * 256
    if name.startswith("wide_key"):
        st = tile * 8
        n_super = V * ((W + st - 1) // st) * ((H + st - 1) // st)
        assert 256 < n_super <= 512 and n_super == int(name.split("_")[-1])
    if name == "many_supertiles":
        n_super = V * ((W + 127) // 128) * ((H + 127) // 128)
        assert n_super > 2048
    if name == "tiny_many_views":
        # every non-empty super-tile takes a chunk: more than keys_cap / 256
        rect = O.project(planes, sh, cams32(cams))[..., 12:16].astype(np.int64)
        sup = {(v, sy, sx) for v in range(V) for g in range(n)
               for x0, x1, y0, y1 in [rect[v, g]] if x1 > x0 and y1 > y0
               for sy in range(y0 >> 3, ((y1 - 1) >> 3) + 1) for sx in range(x0 >> 3, ((x1 - 1) >> 3) + 1)}
        assert len(sup) > a.keys_cap // 256
    a.ctx.close()
    b.ctx.close()


@pytest.mark.parametrize("name", ["one_supertile_chunks", "ragged_edges", "opaque_early_stop", "tile8",
                                  "wide_key_320", "many_supertiles"])
def test_render_batch_chunk_lists_match_expanded_lists(name):
    """gs_render_batch with chunk-bitmap and expanded lists, and
    gs_render_batch_sized (exact super-tile count: a 9-bit key in one pass for
    wide_key_320, longest lists first up to 2048 super-tiles): the same image,
    bit for bit."""
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import estimate_keys
    n, sh, V, W, H, sshift, lshift, tile, tpr, _ = CASES[name]
    planes = scene(n, sh, 23, sshift)
    planes[0, :, 3] += lshift
    cams = gi.ring_cameras(V, W, H)
    params = torch.from_numpy(np.ascontiguousarray(planes)).cuda()
    imgs = []
    for mode, sized in (("two_level", False), ("direct", False), ("two_level", True)):
        ctx = gs.Context(0, 0, tile=tile, binning=mode, raster_threads=tpr)
        cap = max(1 << 22, estimate_keys(ctx, params, sh, cams, slack=1.5))
        ctx.reserve(ctx.workspace_size(cams, n, cap))
        d_cams = gs.cameras_to_device(cams)
        img = gs.gs_render_batch(ctx, params, sh, d_cams, V, ctx.total_tiles(cams), cap, gs.total_pixels(cams),
                                 host_cams=cams if sized else None)
        torch.cuda.synchronize()
        assert ctx.status()[0] == 0
        imgs.append(img.cpu().numpy())
        ctx.close()
    np.testing.assert_array_equal(imgs[0], imgs[1])
    np.testing.assert_array_equal(imgs[2], imgs[1])


@pytest.mark.parametrize("case", ["all_culled", "one_gaussian"])
def test_train_step_chunk_lists_degenerate(case):
    """Degenerate scenes through the fused step with chunk-bitmap lists: every
    Gaussian outside every view (no list entry at all: the image is the
    background, no gradient, Adam leaves the parameters), and a single
    Gaussian; both as with the expanded lists."""
    import torch
    n, sh, V, W, H = (64, 0, 2, 96, 80) if case == "all_culled" else (1, 1, 3, 96, 80)
    planes = scene(n, sh, 31, 2.0)
    if case == "all_culled":
        planes[0, :, 0:3] = np.array([0.0, 40.0, 0.0], dtype=np.float32)  # far above every ring camera's view
    cams = gi.ring_cameras(V, W, H)
    target = torch.full((3 * V * W * H,), 0.25, dtype=torch.float32, device="cuda")
    a = _trainer("two_level", planes, sh, cams, target, 16, 4, 2)
    b = _trainer("direct", planes, sh, cams, target, 16, 4, 2)
    for tr in (a, b):
        tr.step()
    torch.cuda.synchronize()
    assert a.ctx.status()[0] == 0 and b.ctx.status()[0] == 0
    np.testing.assert_array_equal(a.image.cpu().numpy(), b.image.cpu().numpy())
    assert a.loss() == b.loss()
    if case == "all_culled":
        np.testing.assert_array_equal(a.image.cpu().numpy(), np.zeros(3 * V * W * H, np.float32))
        assert not np.any(a.grads.cpu().numpy())
        np.testing.assert_array_equal(a.params.cpu().numpy(), planes)
    else:
        assert np.any(a.image.cpu().numpy() > 0)
        assert rel_l2(a.grads.cpu().numpy(), b.grads.cpu().numpy()) <= 1e-5
    a.ctx.close()
    b.ctx.close()
