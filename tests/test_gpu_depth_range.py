"""The depth sort's two key forms against the oracle.

The depth sort orders the float bits of each visible Gaussian's view depth
(positive floats order as their bit patterns).  When the visible keys span
fewer than 2^24 - 1 values it orders key - smallest visible key instead, so
three 8-bit passes settle the order and the fourth is skipped; otherwise it
runs all four passes on the raw bits.  Either way the (tile, depth, index)
order is unique, so the sorted lists must equal the oracle's bit for bit.

Two scenes: the default one (view depths 2 to 4, a span under 2^24) and
a deep one whose Gaussians sit between depth 0.3 and 40 in front of view
0 (a span of about 6e7).  The tests first check on the oracle's records
that each scene falls on the side it is meant to.
"""
import numpy as np
import pytest

import gs_inputs as gi
import oracle as O
from gpu_util import cams32, gpu_proj_to_oracle, oracle_proj_to_gpu, rel_l2, scene

pytestmark = pytest.mark.gpu

NARROW = 0xFFFFFF
W, H, V = 256, 160, 2


def _deep_scene(n, seed):
    """Default Gaussians moved so view 0 (at (0, 0, 3), looking down -z)
    sees them at log-uniform depths in [0.3, 40], inside its frustum."""
    p = scene(n, 0, seed)
    rng = np.random.default_rng(seed + 1000)
    d = np.exp(rng.uniform(np.log(0.3), np.log(40.0), n))
    tx = np.tan(np.radians(30.0))
    ty = tx * H / W
    p[0, :, 0] = (rng.uniform(-0.45, 0.45, n) * d * tx).astype(np.float32)
    p[0, :, 1] = (rng.uniform(-0.45, 0.45, n) * d * ty).astype(np.float32)
    p[0, :, 2] = (3.0 - d).astype(np.float32)
    return p


SCENES = {"narrow": lambda: scene(20_000, 0, 31), "wide": lambda: _deep_scene(20_000, 31)}


def _oracle_lists(planes, cams):
    og32 = oracle_proj_to_gpu(O.project(planes, 0, cams32(cams)))
    ogd = gpu_proj_to_oracle(og32)
    rect = ogd[..., 12:16].astype(np.int32)
    vis = (rect[..., 2] > rect[..., 0]) & (rect[..., 3] > rect[..., 1])
    bits = og32[..., 2].copy().view(np.uint32)[vis]
    span = int(bits.max()) - int(bits.min())
    keys, vals, ranges = O.bin_sort(cams32(cams), rect, og32[..., 2].copy())
    return og32, span, keys, vals, ranges


def _check_side(name, span):
    if name == "narrow":
        assert span < NARROW, span
    else:
        assert span > 2 * NARROW, span


@pytest.mark.parametrize("mode", ["two_level", "direct"])
@pytest.mark.parametrize("name", list(SCENES))
def test_depth_sort_either_key_form_matches_oracle(name, mode):
    """gs_bin_sort of the oracle's float32 records gives the oracle's lists."""
    import torch
    import paper_2604_02851_b300 as gs
    planes = SCENES[name]()
    cams = gi.ring_cameras(V, W, H)
    og32, span, keys, vals, ranges = _oracle_lists(planes, cams)
    _check_side(name, span)
    n = planes.shape[1]
    ctx = gs.Context(0, 0, binning=mode)
    cap = max(1 << 20, 2 * len(vals))
    ctx.reserve(ctx.workspace_size(cams, n, cap))
    d_cams = gs.cameras_to_device(cams)
    proj = torch.from_numpy(np.ascontiguousarray(og32)).cuda()
    k, v, r, nk = gs.gs_bin_sort(ctx, proj, d_cams, V, n, ctx.total_tiles(cams), cap)
    torch.cuda.synchronize()
    assert ctx.status()[0] == 0
    K = int(nk.item())
    assert K == len(vals) > 0
    np.testing.assert_array_equal(v.cpu().numpy()[:K].view(np.uint32), vals)
    np.testing.assert_array_equal(k.cpu().numpy()[:K].view(np.uint32), (keys >> np.uint64(32)).astype(np.uint32))
    np.testing.assert_array_equal(r.cpu().numpy().view(np.uint32), ranges)
    ctx.close()


@pytest.mark.parametrize("mode", ["two_level", "direct"])
@pytest.mark.parametrize("name", list(SCENES))
def test_fused_paths_either_key_form_match_oracle_image(name, mode):
    """The fused training step (projection ranges the keys itself) and the
    batch render give the oracle's image of the scene."""
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import OnlineTrainer, estimate_keys
    planes = SCENES[name]()
    cams = gi.ring_cameras(V, W, H)
    _, span, _, _, _ = _oracle_lists(planes, cams)
    _check_side(name, span)
    ref = O.forward(planes, 0, cams32(cams))["image"].astype(np.float32)
    ctx = gs.Context(0, 0, binning=mode)
    params = torch.from_numpy(np.ascontiguousarray(planes)).cuda()
    cap = estimate_keys(ctx, params, 0, cams, slack=1.5)
    tr = OnlineTrainer(params.clone(), 0, cams, cap, ctx=ctx)
    tr.targets.copy_(torch.from_numpy(np.ascontiguousarray(ref.reshape(-1))).cuda())
    tr.step()
    torch.cuda.synchronize()
    assert ctx.status()[0] == 0
    assert rel_l2(tr.image.cpu().numpy().reshape(ref.shape), ref) <= 1e-4
    rctx = gs.Context(0, 0, binning=mode)
    rctx.reserve(rctx.workspace_size(cams, planes.shape[1], cap))
    d_cams = gs.cameras_to_device(cams)
    img = gs.gs_render_batch(rctx, params, 0, d_cams, V, rctx.total_tiles(cams), cap, gs.total_pixels(cams),
                             host_cams=cams)
    torch.cuda.synchronize()
    assert rctx.status()[0] == 0
    assert rel_l2(img.cpu().numpy().reshape(ref.shape), ref) <= 1e-4
    rctx.close()


@pytest.mark.parametrize("span", [NARROW - 1, NARROW])
def test_depth_sort_at_the_narrow_limit(span):
    """One visible Gaussian's depth moved so that the visible keys span
    exactly 2^24 - 2 values (the largest narrow span: the culled key
    2^24 - 1 still sorts after every visible one) or 2^24 - 1 (the smallest
    wide span): gs_bin_sort gives the oracle's lists either way."""
    import torch
    import paper_2604_02851_b300 as gs
    planes = SCENES["narrow"]()
    cams = gi.ring_cameras(V, W, H)
    og32 = oracle_proj_to_gpu(O.project(planes, 0, cams32(cams)))
    rect = gpu_proj_to_oracle(og32)[..., 12:16].astype(np.int32)
    vis = (rect[..., 2] > rect[..., 0]) & (rect[..., 3] > rect[..., 1])
    bits = og32[..., 2].copy().view(np.uint32)
    lo = int(bits[vis].min())
    far = np.flatnonzero(vis.reshape(-1))[-1]  # some visible record other than the nearest
    depth = og32[..., 2].copy().reshape(-1)
    depth.view(np.uint32)[far] = lo + span
    og32[..., 2] = depth.reshape(og32.shape[:-1])
    b2 = og32[..., 2].copy().view(np.uint32)[vis]
    assert int(b2.max()) - int(b2.min()) == span
    keys, vals, ranges = O.bin_sort(cams32(cams), rect, og32[..., 2].copy())
    n = planes.shape[1]
    for mode in ("two_level", "direct"):
        ctx = gs.Context(0, 0, binning=mode)
        cap = max(1 << 20, 2 * len(vals))
        ctx.reserve(ctx.workspace_size(cams, n, cap))
        d_cams = gs.cameras_to_device(cams)
        proj = torch.from_numpy(np.ascontiguousarray(og32)).cuda()
        k, v, r, nk = gs.gs_bin_sort(ctx, proj, d_cams, V, n, ctx.total_tiles(cams), cap)
        torch.cuda.synchronize()
        assert ctx.status()[0] == 0
        K = int(nk.item())
        assert K == len(vals) > 0
        np.testing.assert_array_equal(v.cpu().numpy()[:K].view(np.uint32), vals)
        np.testing.assert_array_equal(r.cpu().numpy().view(np.uint32), ranges)
        ctx.close()
