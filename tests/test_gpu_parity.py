"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: keys, sort order, tile ranges and delta indices/records bit-exact
(stage-wise: each GPU stage runs on the oracle's own upstream results rounded
to float32 and is compared with the oracle stage on the same inputs);
images, losses and gradients within 1e-4 relative L2.  Integer decisions taken
by floating point (radius, tile rectangle, termination) are compared where
both sides decide them in the same precision, and otherwise counted and
bounded.
"""
import math

import numpy as np
import pytest

import gs_inputs as gi
import oracle as O
from flips import decision_flips, decision_margins
from gpu_util import GpuRun, OracleStages, cams32, gpu_proj_to_oracle, l1_sign_expected, rel_l2, scene

pytestmark = pytest.mark.gpu

TOL = 1e-4
# relative distance from a threshold within which float32 and float64 walks
# of the same records may take a compositing decision differently (float32
# transmittance over a few hundred fragments drifts by ~1e-5 relative)
NEAR_DECISION = 1e-4

CASES = {
    # name: (n, sh_degree, views, width, height, scale shift)
    "c1_128": (10_000, 0, 1, 128, 128, 0.0),
    "ragged_sh3": (20_000, 3, 2, 200, 136, 0.0),
    "big_splats_sh1": (3_000, 1, 3, 97, 61, 1.0),
}


def _setup(name, seed=0, with_target=True):
    n, sh, V, W, H, shift = CASES[name]
    planes = scene(n, sh, seed, shift)
    cams = gi.ring_cameras(V, W, H)
    target = None
    if with_target:
        tp = scene(n, sh, seed + 1, shift)
        target = O.forward(tp, sh, cams32(cams))["image"]
    run = GpuRun(planes, sh, cams, target)
    return planes, sh, cams32(cams), run


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    planes, sh, cams, run = _setup(request.param)
    yield request.param, planes, sh, cams, run
    run.close()


def test_projection_matches_oracle(case):
    name, planes, sh, cams, run = case
    og = O.project(planes, sh, cams)
    gp = run.oracle_proj()
    vis_o = og[..., 14] > og[..., 12]
    vis_g = gp[..., 14] > gp[..., 12]
    both = vis_o & vis_g
    # visibility differs only where the FP64 radius / rectangle sits on an integer boundary
    diff = np.argwhere(vis_o != vis_g)
    assert len(diff) <= max(2, 1e-4 * both.sum()), len(diff)
    for f in (0, 1, 2, 3, 4, 5, 6, 8, 9, 10):
        assert rel_l2(gp[..., f][both], og[..., f][both]) <= TOL, (name, f)
    # radius: equal unless 3 sqrt(lambda) is within 1e-5 (relative) of an integer
    r_o, r_g = og[..., 7][both], gp[..., 7][both]
    bad = np.nonzero(r_o != r_g)[0]
    assert len(bad) <= max(2, 1e-4 * both.sum())
    np.testing.assert_array_equal(gp[..., 11][both], og[..., 11][both])


@pytest.fixture(scope="module", params=list(CASES))
def stages(request):
    """The oracle's chain on the case, and the GPU stages run on its float32
    intermediates (see OracleStages)."""
    n, sh, V, W, H, shift = CASES[request.param]
    planes = scene(n, sh, 0, shift)
    cams = cams32(gi.ring_cameras(V, W, H))
    target = O.forward(scene(n, sh, 1, shift), sh, cams)["image"]
    st = OracleStages(O, planes, sh, cams, target)
    yield request.param, st
    st.close()


def test_bin_sort_bit_exact_stagewise(stages):
    """The GPU's binning and sort of the oracle's float32 records must give
    the oracle's keys, order and ranges exactly."""
    name, st = stages
    keys, vals, ranges = st.gpu_bin_sort()
    assert len(vals) == st.K
    np.testing.assert_array_equal(vals, st.vals)
    np.testing.assert_array_equal(keys, (st.keys >> np.uint64(32)).astype(np.uint32))
    np.testing.assert_array_equal(ranges, st.ranges)


def test_render_fwd_stagewise(stages):
    """Both sides composite the same float32 records and lists, so a
    contributor count may differ only at a pixel where a decision of the walk
    (the alpha cut-off, the termination test, the sign of P) lies within
    rounding of its threshold: every mismatch must be such a pixel."""
    name, st = stages
    img, T, nc = st.gpu_render_fwd()
    assert rel_l2(img.cpu().numpy(), st.image) <= TOL
    assert rel_l2(T.cpu().numpy(), st.T) <= TOL
    mism = nc.cpu().numpy().view(np.uint32) != st.nc
    near = decision_margins(st.cams, st.projd, st.vals, st.ranges) <= NEAR_DECISION
    print("render stage-wise", name, "count mismatches", int(mism.sum()), "near-threshold pixels", int(near.sum()))
    assert not np.any(mism & ~near), np.nonzero(mism & ~near)[0][:10]


def test_render_end_to_end(case):
    name, planes, sh, cams, run = case
    f = O.forward(planes, sh, cams)
    assert rel_l2(run.np("image"), f["image"]) <= TOL


def test_loss_matches_oracle(stages):
    name, st = stages
    L, dimg = st.gpu_loss()
    assert abs(L - st.loss) <= TOL * abs(st.loss)
    assert rel_l2(dimg, st.dimage32) <= TOL


def test_raster_bwd_stagewise(stages):
    name, st = stages
    gg = st.gpu_raster_bwd()
    assert np.all(gg[..., 9:] == 0)
    for k in range(9):
        assert rel_l2(gg[..., k], st.grad2d[..., k]) <= TOL, k


def test_project_bwd_stagewise(stages):
    name, st = stages
    gd, dp = st.gpu_project_bwd(), st.dparams
    sh = st.sh
    nb = (sh + 1) ** 2
    groups = {"mean": (0, slice(0, 3)), "logit": (0, slice(3, 4)), "scale": (1, slice(0, 3)),
              "quat": (2, slice(0, 4))}
    for gname, (pl, sl) in groups.items():
        assert rel_l2(gd[pl, :, sl], dp[pl, :, sl]) <= TOL, gname
    sh_g = gi.planes_to_rows(gd)[:, 12:12 + 3 * nb]
    sh_o = gi.planes_to_rows(dp)[:, 12:12 + 3 * nb]
    assert rel_l2(sh_g, sh_o) <= TOL
    assert np.all(gi.planes_to_rows(gd)[:, 12 + 3 * nb:] == 0)
    assert np.all(gd[1, :, 3] == 0)


def test_gradient_end_to_end(case):
    """Float32 GPU chain vs the FP64 oracle chain from the same parameters.

    The alpha cut-off (1/255) and the termination test are decisions taken by
    floating point: a fragment within rounding of a threshold is kept by one
    precision and dropped by the other, which moves one pixel's share of that
    Gaussian's gradient.  Those Gaussians are found exactly (the oracle walks
    every pixel under both projections and compares the kept sets), must be
    rare, and are left out; every other Gaussian must match to 1e-4.
    Gaussians whose integer support (radius, rectangle) differs likewise.
    The sign of the L1 term is a decision too: where the image meets the
    target within float32 rendering error, each sign is a correct result,
    and the oracle's gradient is taken with the float32 render's choice there."""
    name, planes, sh, cams, run = case
    target = run.np("target")
    r = O.loss_and_grad(planes, sh, cams, target)
    assert abs(float(run.loss.item()) - r["loss"]) <= TOL * abs(r["loss"])
    gd, od = run.np("dparams"), r["dparams"]
    og, gp = r["proj"], run.oracle_proj()
    fields = [7, 12, 13, 14, 15]
    support = np.any(og[..., fields] != gp[..., fields], axis=(0, 2))
    flips, npix = decision_flips(cams, og, r["vals"], r["ranges"], gp, run.sorted_vals(), run.ranges_np())
    odd = support | flips.any(axis=0)
    keep = ~odd
    od, ties = l1_sign_expected(O, planes, sh, cams, r, target, gd, keep=keep)
    e_all, e_keep = rel_l2(gd, od), rel_l2(gd[:, keep], od[:, keep])
    print("gradient end-to-end", name, "all", e_all, "kept", e_keep, "threshold flips", int(odd.sum()),
          "pixels", npix, "L1 sign ties", ties)
    assert odd.mean() <= 1e-3, int(odd.sum())
    # the L1 tie family must stay small, or its fit could absorb a real error
    assert ties <= 1e-4 * target.size, ties
    assert e_keep <= TOL, (e_all, e_keep)


# ---------------------------------------------------------------- Adam, delta
def test_adam_matches_oracle():
    import torch
    import paper_2604_02851_b300 as gs
    n = 5000
    rng = np.random.default_rng(5)
    theta = gi.make_scene(n, 3, 3)
    ctx = gs.Context(0, 1 << 20)
    th = torch.from_numpy(theta).cuda()
    m = torch.zeros_like(th); v = torch.zeros_like(th)
    lr = rng.uniform(1e-4, 1e-2, 60).astype(np.float32)
    th_o = gi.planes_to_rows(theta).astype(np.float64)
    m_o = np.zeros_like(th_o); v_o = np.zeros_like(th_o)
    d_step = torch.ones(1, dtype=torch.int32, device="cuda")
    for step in range(1, 4):
        g = (rng.normal(size=theta.shape) * 10 ** rng.uniform(-5, 0, size=theta.shape)).astype(np.float32)
        g[1, :, 3] = 0
        gt = torch.from_numpy(g).cuda()
        use_dev = step == 2
        cfg = gs.adam_cfg(lr=lr, step=step, d_step=d_step if use_dev else None, increment=use_dev)
        if use_dev:
            d_step.fill_(2)
        gs.gs_adam_step(ctx, th, gt, m, v, cfg)
        torch.cuda.synchronize()
        O.adam(th_o, gi.planes_to_rows(g).astype(np.float64), m_o, v_o, np.tile(lr, (n, 1)).astype(np.float64), step)
        # each side carries its own state; the updates so far must agree
        upd_g = gi.planes_to_rows(th.cpu().numpy()).astype(np.float64) - gi.planes_to_rows(theta).astype(np.float64)
        upd_o = th_o - gi.planes_to_rows(theta).astype(np.float64)
        assert rel_l2(upd_g, upd_o) <= TOL
    assert int(d_step.item()) == 3
    ctx.close()


@pytest.mark.parametrize("n,frac", [(1, 1.0), (257, 0.3), (100_000, 0.05), (4096, 0.0)])
def test_delta_bit_exact(n, frac):
    import torch
    import paper_2604_02851_b300 as gs
    rng = np.random.default_rng(n)
    base = gi.make_scene(n, 3, 11)
    theta = base.copy()
    pick = np.nonzero(rng.random(n) < frac)[0]
    for i in pick:
        p = rng.integers(0, 15); c = rng.integers(0, 4)
        if p == 1 and c == 3:
            c = 0
        theta[p, i, c] += np.float32(rng.choice([1.1e-3, -2e-3, 9e-4, 1e-3]))
    ctx = gs.Context(0, 1 << 24)
    th = torch.from_numpy(theta).cuda()
    bs = torch.from_numpy(base).cuda()
    idx, rec, cnt = gs.gs_extract_delta(ctx, th, bs, 1e-3)
    torch.cuda.synchronize()
    M = int(cnt.item())
    oi, orec, obase = O.delta(theta, base, 1e-3)
    assert M == len(oi)
    np.testing.assert_array_equal(idx.cpu().numpy()[:M].view(np.uint32), oi)
    np.testing.assert_array_equal(rec.cpu().numpy()[:M], orec)
    np.testing.assert_array_equal(bs.cpu().numpy(), obase)
    ctx.close()


# ---------------------------------------------------------------- edge cases
def test_all_culled_and_empty_lists():
    planes = scene(500, 0, 3)
    planes[0, :, 2] = 10.0  # every mean behind the camera at z = 3
    cams = gi.ring_cameras(1, 48, 32)
    run = GpuRun(planes, 0, cams)
    assert run.K == 0
    assert np.all(run.np("image") == 0)
    assert np.all(run.np("T") == 1)
    assert np.all(run.ranges_np() == 0)
    run.close()


def test_capacity_overflow_is_reported():
    import torch
    import paper_2604_02851_b300 as gs
    planes = scene(4000, 0, 2, 1.0)
    cams = gi.ring_cameras(2, 64, 64)
    ctx = gs.Context(0, 0)
    params = torch.from_numpy(planes).cuda()
    d_cams = gs.cameras_to_device(cams)
    tt = ctx.total_tiles(cams)
    cap = 100
    ctx.reserve(ctx.workspace_size(cams, 4000, cap))
    proj = gs.gs_project(ctx, params, 0, d_cams, 2)
    _, vals, ranges, nk = gs.gs_bin_sort(ctx, proj, d_cams, 2, 4000, tt, cap)
    torch.cuda.synchronize()
    code, detail = ctx.status()
    r = gpu_proj_to_oracle(proj.cpu().numpy())[..., 12:16]
    K = int(((r[..., 2] - r[..., 0]) * (r[..., 3] - r[..., 1])).sum())
    assert code == 2
    assert detail == int(nk.item()) == K and K > cap
    # a second read is clear
    assert ctx.status()[0] == 0
    ctx.close()


def test_bad_arguments_rejected_on_host():
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300._lib import GsError
    ctx = gs.Context(0, 1 << 20)
    params = torch.zeros((15, 10, 4), device="cuda")
    d_cams = gs.cameras_to_device(gi.ring_cameras(1, 16, 16))
    with pytest.raises(GsError):
        gs.gs_project(ctx, params, 4, d_cams, 1)  # SH degree out of range
    with pytest.raises(GsError):
        gs.gs_project(ctx, params, 0, d_cams, 0)  # no views
    with pytest.raises(GsError):
        ctx2 = gs.Context(0, 0)
        gs.gs_loss(ctx2, params.view(-1), params.view(-1), 1, 10, 20)  # no workspace
    ctx.close()


def test_tile_size_8_matches_16():
    planes = scene(3000, 1, 4)
    cams = gi.ring_cameras(2, 72, 40)
    tp = scene(3000, 1, 5)
    target = O.forward(tp, 1, cams32(cams))["image"]
    a = GpuRun(planes, 1, cams, target, tile=16)
    b = GpuRun(planes, 1, cams, target, tile=8, sort_bits=5)
    f8 = O.forward(planes, 1, cams32(cams), tile=8)
    assert rel_l2(b.np("image"), f8["image"]) <= TOL
    # tile size changes the (P, rect) support: the 8-px binning of the
    # oracle's own records must be the oracle's
    st = OracleStages(O, planes, 1, cams32(cams), target, tile=8)
    _, vals, ranges = st.gpu_bin_sort()
    np.testing.assert_array_equal(vals, st.vals)
    np.testing.assert_array_equal(ranges, st.ranges)
    st.close()
    a.close(); b.close()


def test_raster_threads_per_row_2_matches_4():
    """Two or four threads per pixel row change only which thread owns which
    pixels: the images, transmittances and contributor counts are identical
    and the 2D gradients agree up to the order of the float32 sums."""
    planes = scene(20_000, 2, 6)
    cams = gi.ring_cameras(2, 200, 136)
    target = O.forward(scene(20_000, 2, 7), 2, cams32(cams))["image"]
    a = GpuRun(planes, 2, cams, target, raster_threads=4)
    b = GpuRun(planes, 2, cams, target, raster_threads=2)
    np.testing.assert_array_equal(a.np("image"), b.np("image"))
    np.testing.assert_array_equal(a.np("T"), b.np("T"))
    np.testing.assert_array_equal(a.np("nc"), b.np("nc"))
    assert rel_l2(b.np("grad2d"), a.np("grad2d")) <= 1e-5
    assert rel_l2(b.np("dparams"), a.np("dparams")) <= 1e-5
    a.close(); b.close()
