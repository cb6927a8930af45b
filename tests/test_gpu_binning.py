"""Two-level binning (super-tile lists expanded into tile lists) against the
direct tile-key sort and the oracle.

Both modes must give the identical sorted values, keys, per-tile ranges and
entry counts: the (tile, depth, Gaussian index) order is unique.  The cases
cover one super-tile holding several expansion chunks, super-tiles cut by the
image edge, Gaussians spanning many super-tiles, many views, small digit
widths and 8-pixel tiles.
"""
import numpy as np
import pytest

import gs_inputs as gi
import oracle as O
from gpu_util import cams32, gpu_proj_to_oracle, oracle_proj_to_gpu, scene

pytestmark = pytest.mark.gpu

CASES = {
    # name: (n, sh_degree, views, width, height, log-scale shift, tile, sort_bits, sort_items)
    "one_supertile_chunks": (10_000, 0, 1, 128, 128, 0.0, 16, 8, 16),
    "ragged_edges": (20_000, 1, 3, 200, 136, 0.0, 16, 8, 12),
    "big_splats": (3_000, 0, 2, 333, 250, 1.5, 16, 5, 8),
    "many_views": (40_000, 0, 16, 256, 160, 0.0, 16, 8, 16),
    "tile8": (8_000, 0, 2, 150, 90, 0.5, 8, 6, 16),
}


def _bin(mode, planes, sh, cams, tile, bits, items, keys_cap, proj32=None):
    """GPU projection + binning, or binning alone of given float32 records."""
    import torch
    import paper_2604_02851_b300 as gs
    n, V = planes.shape[1], len(cams["fx"])
    ctx = gs.Context(0, 0, tile=tile, sort_bits=bits, sort_items=items, binning=mode)
    ctx.reserve(ctx.workspace_size(cams, n, keys_cap))
    params = torch.from_numpy(np.ascontiguousarray(planes)).cuda()
    d_cams = gs.cameras_to_device(cams)
    tt = ctx.total_tiles(cams)
    if proj32 is None:
        proj = gs.gs_project(ctx, params, sh, d_cams, V)
    else:
        proj = torch.from_numpy(np.ascontiguousarray(proj32)).cuda()
    keys, vals, ranges, nk = gs.gs_bin_sort(ctx, proj, d_cams, V, n, tt, keys_cap)
    torch.cuda.synchronize()
    code, detail = ctx.status()
    K = int(nk.item())
    out = {"code": code, "detail": detail, "K": K, "proj": proj.cpu().numpy(),
           "keys": keys.cpu().numpy()[:min(K, keys_cap)].view(np.uint32),
           "vals": vals.cpu().numpy()[:min(K, keys_cap)].view(np.uint32),
           "ranges": ranges.cpu().numpy().view(np.uint32)}
    ctx.close()
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_two_level_matches_direct_and_oracle(name):
    n, sh, V, W, H, shift, tile, bits, items = CASES[name]
    planes = scene(n, sh, 7, shift)
    cams = gi.ring_cameras(V, W, H)
    cap = 1 << 22
    a = _bin("two_level", planes, sh, cams, tile, bits, items, cap)
    b = _bin("direct", planes, sh, cams, tile, bits, items, cap)
    assert a["code"] == 0 and b["code"] == 0, (a["code"], a["detail"], b["code"], b["detail"])
    np.testing.assert_array_equal(a["proj"], b["proj"])
    assert a["K"] == b["K"] > 0
    np.testing.assert_array_equal(a["keys"], b["keys"])
    np.testing.assert_array_equal(a["vals"], b["vals"])
    np.testing.assert_array_equal(a["ranges"], b["ranges"])
    # both modes on the oracle's own records (rounded to float32) against
    # the oracle's sort of them
    og32 = oracle_proj_to_gpu(O.project(planes, sh, cams32(cams), tile))
    ogd = gpu_proj_to_oracle(og32)
    keys, vals, ranges = O.bin_sort(cams32(cams), ogd[..., 12:16].astype(np.int32), og32[..., 2].copy(), tile=tile)
    for mode in ("two_level", "direct"):
        c = _bin(mode, planes, sh, cams, tile, bits, items, cap, proj32=og32)
        assert c["code"] == 0 and c["K"] == len(vals)
        np.testing.assert_array_equal(c["vals"], vals)
        np.testing.assert_array_equal(c["keys"], (keys >> np.uint64(32)).astype(np.uint32))
        np.testing.assert_array_equal(c["ranges"], ranges)


def test_two_level_chunks_span_super_tiles():
    """A super-tile list several times the expansion chunk: every chunk's
    entries land after the previous chunk's in each tile list."""
    n, sh = 60_000, 0
    planes = scene(n, sh, 11, 0.5)
    cams = gi.ring_cameras(1, 128, 128)  # one super-tile
    a = _bin("two_level", planes, sh, cams, 16, 8, 16, 1 << 23)
    b = _bin("direct", planes, sh, cams, 16, 8, 16, 1 << 23)
    assert a["code"] == 0 and a["K"] == b["K"]
    np.testing.assert_array_equal(a["vals"], b["vals"])
    np.testing.assert_array_equal(a["ranges"], b["ranges"])
    # the list is much longer than one chunk (2048 entries)
    visible = int((gpu_proj_to_oracle(a["proj"])[..., 14] > 0).sum())
    assert visible > 10 * 2048


@pytest.mark.parametrize("mode", ["two_level", "direct"])
def test_capacity_overflow_reports_exact_count(mode):
    n, sh = 4000, 0
    planes = scene(n, sh, 2, 1.0)
    cams = gi.ring_cameras(2, 64, 64)
    full = _bin(mode, planes, sh, cams, 16, 8, 16, 1 << 20)
    assert full["code"] == 0
    small = _bin(mode, planes, sh, cams, 16, 8, 16, 100)
    assert small["code"] == 2
    assert small["detail"] == small["K"] == full["K"] > 100


@pytest.mark.parametrize("mode", ["two_level", "direct"])
def test_render_after_overflow_reads_stored_entries_only(mode):
    """After a capacity overflow the ranges stay inside the stored prefix, so
    compositing the truncated lists is safe; the status reports the count."""
    import torch
    import paper_2604_02851_b300 as gs
    n, sh = 4000, 0
    planes = scene(n, sh, 2, 1.0)
    cams = gi.ring_cameras(2, 64, 64)
    ctx = gs.Context(0, 0, binning=mode)
    cap = 500
    ctx.reserve(ctx.workspace_size(cams, n, cap))
    params = torch.from_numpy(planes).cuda()
    d_cams = gs.cameras_to_device(cams)
    tt = ctx.total_tiles(cams)
    proj = gs.gs_project(ctx, params, sh, d_cams, 2)
    _, vals, ranges, nk = gs.gs_bin_sort(ctx, proj, d_cams, 2, n, tt, cap, want_keys=False)
    r = ranges.cpu().numpy().view(np.uint32)
    assert r.max() <= cap
    gs.gs_render_fwd(ctx, proj, d_cams, 2, n, tt, vals, ranges, gs.total_pixels(cams))
    torch.cuda.synchronize()
    code, detail = ctx.status()
    assert code == 2 and detail == int(nk.item()) > cap
    ctx.close()


def test_autotune_times_every_configuration_and_keeps_results_exact():
    """gs_autotune tries 2 binnings x 3 digit widths x 3 item counts x 2 raster
    layouts.  Per binning (whose raster kernels read different list forms) it
    takes the sort settings with the least time outside compositing and the
    fastest compositing and adjoint layouts; it keeps the binning whose sum of
    the three is smaller.  The sort it then produces is still the oracle's."""
    import torch
    import paper_2604_02851_b300 as gs
    n, sh = 30_000, 1
    planes = scene(n, sh, 13)
    cams = gi.ring_cameras(3, 256, 160)
    ctx = gs.Context(0, 0)
    cap = 1 << 22
    ctx.reserve(ctx.workspace_size(cams, n, cap))
    params = torch.from_numpy(planes).cuda()
    best, entries = gs.gs_autotune(ctx, params, sh, cams, cap, reps=2)
    assert len(entries) == 36
    assert {(e["binning"], e["sort_bits"], e["sort_items"], e["raster_threads"]) for e in entries} == {
        (b, bits, it, t) for b in ("two_level", "direct") for bits in (8, 7, 6) for it in (16, 12, 8) for t in (4, 2)}
    assert all(e["ms"] > 0 and 0 < e["ms_render_fwd"] and 0 < e["ms_render_bwd"] for e in entries)
    assert all(e["ms_render_fwd"] + e["ms_render_bwd"] < e["ms"] for e in entries)
    def pre(e):
        return e["ms"] - e["ms_render_fwd"] - e["ms_render_bwd"]

    total = {}
    for b in ("two_level", "direct"):
        es = [e for e in entries if e["binning"] == b]
        fwd = {t: min(e["ms_render_fwd"] for e in es if e["raster_threads"] == t) for t in (4, 2)}
        bwd = {t: min(e["ms_render_bwd"] for e in es if e["raster_threads"] == t) for t in (4, 2)}
        total[b] = min(pre(e) for e in es) + min(fwd.values()) + min(bwd.values())
        if b == best["binning"]:
            low = min(pre(e) for e in es)
            chosen = [pre(e) for e in es if (e["sort_bits"], e["sort_items"]) == (best["sort_bits"], best["sort_items"])]
            assert min(chosen) <= low * (1 + 1e-5) + 1e-6
            assert fwd[best["raster_threads"]] <= min(fwd.values()) * (1 + 1e-5)
            assert bwd[best["raster_bwd_threads"]] <= min(bwd.values()) * (1 + 1e-5)
    assert total[best["binning"]] <= min(total.values()) * (1 + 1e-5) + 1e-6
    assert ctx.status()[0] == 0
    d_cams = gs.cameras_to_device(cams)
    tt = ctx.total_tiles(cams)
    # the tuned context bins the oracle's own records (rounded to float32) as the oracle does
    og32 = oracle_proj_to_gpu(O.project(planes, sh, cams32(cams)))
    ogd = gpu_proj_to_oracle(og32)
    proj = torch.from_numpy(og32).cuda()
    keys, vals, ranges, nk = gs.gs_bin_sort(ctx, proj, d_cams, 3, n, tt, cap)
    torch.cuda.synchronize()
    K = int(nk.item())
    okeys, ovals, oranges = O.bin_sort(cams32(cams), ogd[..., 12:16].astype(np.int32), og32[..., 2].copy())
    np.testing.assert_array_equal(vals.cpu().numpy()[:K].view(np.uint32), ovals)
    np.testing.assert_array_equal(ranges.cpu().numpy().view(np.uint32), oranges)
    ctx.close()
