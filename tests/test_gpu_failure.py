"""Failure detection without a GPU fault: a bounded inter-block wait that
runs out.

The onesweep sort's look-back waits for the digit counts of the tiles before
it.  The context's test hook (gs_ctx_set_wait_test) makes one tile of the
last pass of the direct binning's tile-key sort withhold them -- a flag that
nothing else sets -- and a lowered wait limit (gs_ctx_set_wait_limit) makes
the waits of the tiles after it end within microseconds.  The call must
return, the status word must read GS_ERR_TIMEOUT, and the context must stay
usable: the next sort without the hook gives the oracle's keys, order and
ranges again.  Nothing here faults, traps or hangs the GPU: every wait is
bounded and the withheld pass writes only the caller's arrays, which no later
kernel of the call reads."""
import ctypes as C
import time

import numpy as np
import pytest

import gs_inputs as gi
import oracle as O
from gpu_util import cams32, oracle_proj_to_gpu, gpu_proj_to_oracle, scene

pytestmark = pytest.mark.gpu


def _case():
    """2 views of 128 x 96 (96 tiles: one 8-bit pass of the tile-key sort)
    and the oracle's float32 records, keys and ranges."""
    cams = cams32(gi.ring_cameras(2, 128, 96))
    planes = scene(20_000, 1, 3)
    proj32 = oracle_proj_to_gpu(O.project(planes, 1, cams))
    projd = gpu_proj_to_oracle(proj32)
    keys, vals, ranges = O.bin_sort(cams, projd[..., 12:16].astype(np.int32), proj32[..., 2].copy())
    return cams, planes.shape[1], proj32, keys, vals, ranges


def _sort(gs, torch, ctx, t_proj, d_cams, n, tt, cap):
    keys, vals, ranges, nk = gs.gs_bin_sort(ctx, t_proj, d_cams, 2, n, tt, cap)
    torch.cuda.synchronize()
    return keys, vals, ranges, nk


def test_withheld_lookback_times_out_and_the_context_recovers():
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300 import _lib
    cams, n, proj32, okeys, ovals, oranges = _case()
    K = len(ovals)
    # the pass has several onesweep tiles (2048 keys each at 8 items a thread)
    assert K > 4 * 2048, K
    ctx = gs.Context(0, 0, binning="direct", sort_items=8)
    ctx.reserve(ctx.workspace_size(cams, n, K))
    d_cams = gs.cameras_to_device(cams)
    tt = ctx.total_tiles(cams)
    t_proj = torch.from_numpy(proj32).cuda()

    def check_exact():
        keys, vals, ranges, nk = _sort(gs, torch, ctx, t_proj, d_cams, n, tt, K)
        assert ctx.status() == (0, 0)
        assert int(nk.item()) == K
        np.testing.assert_array_equal(vals.cpu().numpy()[:K].view(np.uint32), ovals)
        np.testing.assert_array_equal(keys.cpu().numpy()[:K].view(np.uint32),
                                      (okeys >> np.uint64(32)).astype(np.uint32))
        np.testing.assert_array_equal(ranges.cpu().numpy().view(np.uint32), oranges)

    check_exact()
    # tile 1 withholds its counts; the tiles after it give up after 2e5 cycles
    ctx.set_wait_limit(200_000)
    ctx.set_wait_test(1)
    t0 = time.perf_counter()
    _sort(gs, torch, ctx, t_proj, d_cams, n, tt, K)
    wall = time.perf_counter() - t0
    code, detail = ctx.status()
    assert code == _lib.GS_ERR_TIMEOUT, (code, detail)
    assert detail >= 2  # the slot of a tile after the withheld one
    assert wall < 10.0
    # a second read of the status word is clear
    assert ctx.status() == (0, 0)
    # hook off, default limit: the context sorts exactly again
    ctx.set_wait_test(-1)
    ctx.set_wait_limit(0)
    check_exact()
    # two-level binning ignores the hook (its sort feeds the expansion)
    check = _lib.lib().gs_ctx_set_binning(ctx.ptr, 0)
    assert check == 0
    ctx.set_wait_test(1)
    check_exact()
    ctx.set_wait_test(-1)
    ctx.close()


def test_wait_settings_are_checked_on_the_host():
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300 import _lib
    ctx = gs.Context(0, 0)
    assert _lib.lib().gs_ctx_set_wait_limit(ctx.ptr, -1) == _lib.GS_ERR_ARG
    assert _lib.lib().gs_ctx_set_wait_test(ctx.ptr, -2) == _lib.GS_ERR_ARG
    assert _lib.lib().gs_ctx_set_wait_limit(None, 10) == _lib.GS_ERR_ARG
    assert _lib.lib().gs_ctx_set_wait_test(C.c_void_p(), 1) == _lib.GS_ERR_ARG
    ctx.close()
