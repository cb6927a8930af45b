"""Parity at the benchmarked sizes, through the autotuned path bench.py times.

* 1M Gaussians, SH3, 8 views of 1280x720 (the headline step).
* 3M Gaussians in 16 rigid objects with the Lambertian DC factor, 8 views
  of 1920x1080 (ragged last tile row).

The FP64 oracle cannot redo whole steps of this size in a test's time.  It
checks three sampled 16-row bands in each of three views (at 1080 rows they
include the ragged last band), plus everything that is cheap at full size.

Stage-wise (each GPU stage runs on the oracle's own float32 upstream results):
  * binning and sort of all 8 views: the entry count and the [start, end)
    range of EVERY tile bit-exact; the sorted lists of the band tiles
    bit-exact;
  * compositing: band image and transmittance within 1e-4 relative L2.
    Contributor counts are equal except at pixels where a decision of the
    walk lies within rounding of its threshold;
  * raster adjoint, with an image gradient that is zero outside the bands:
    every Gaussian's 2D gradient within 1e-4;
  * projection adjoint of the oracle's 2D gradient within 1e-4;
  * the loss at full size (at 3M x 1080p: two views) on seeded images; Adam and
    the delta extraction at the full parameter count on seeded inputs.

End to end (the float32 GPU chain from the parameters against the FP64
oracle chain, three views): at the band pixels whose walks keep the same
fragments in the same order on both sides (at least 98 %), the image within
1e-4, and the whole parameter gradient of an image gradient on those pixels
within 1e-4.

The timed path itself (gs_train_step with chunk-bitmap lists, all 8 views in
one graph launch), against the separate calls on the same inputs:
  * image bit-identical to the expanded-list compositing of the same
    projection;
  * loss equal to gs_loss on that image;
  * gradient within 1e-5 (float atomics);
  * Adam update and delta records bit-identical to gs_adam_step and
    gs_extract_delta on that gradient.

Each oracle stage gets seeded inputs or the oracle's own outputs; GPU values
are only compared, never fed to it.  Where only some Gaussians can have a
nonzero result (the band-masked adjoints), the oracle runs on those
Gaussians' records, a relabelling of indices and no arithmetic."""
import numpy as np
import pytest

import gs_inputs as gi
import oracle as O
from flips import decision_margins, same_sequences
from gpu_util import cams32, gpu_proj_to_oracle, oracle_proj_to_gpu, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-4
NEAR_DECISION = 1e-4
B = 16

CONFIGS = {
    # name: Gaussians, views, width, height, dynamic, checked views, 16-row bands
    "c3_1M_8x720p": (1_000_000, 8, 1280, 720, False, (0, 3, 6), (5, 22, 44)),
    "c5_3M_8x1080p_dynamic": (3_000_000, 8, 1920, 1080, True, (1, 4, 7), (8, 33, 67)),
}
SH = 3


# ---------------------------------------------------------------- inputs
class Case:
    """Seeded inputs of one benchmarked configuration (bench.py's generators)."""

    def __init__(self, name):
        n, V, W, H, dynamic, views, bands = CONFIGS[name]
        self.name, self.n, self.V, self.W, self.H = name, n, V, W, H
        self.views, self.bands = views, bands
        self.planes = gi.make_scene(n, SH, gi.SEED_MODEL)
        self.rows = gi.planes_to_rows(self.planes).astype(np.float64)
        self.cams = cams32(gi.ring_cameras(V, W, H))
        self.TX, self.TY = (W + B - 1) // B, (H + B - 1) // B
        self.dyn = None
        if dynamic:
            # frame 1 of the dynamic workload: 16 rigid objects, Lambertian DC
            self.dyn = {"group": gi.rigid_groups(n, 16), "poses": gi.frame_poses(2, 16)[1],
                        "normals": gi.unit_normals(n), "light": gi.light_directions(2)[1],
                        "ambient": 0.3, "diffuse": 0.7}

    def band_tiles(self, views=None):
        """Global indices of the band tiles (8-view tile numbering), views in order."""
        views = self.views if views is None else views
        out = []
        for v in views:
            for b in self.bands:
                out.extend(v * self.TX * self.TY + b * self.TX + np.arange(self.TX))
        return np.asarray(out, dtype=np.int64)

    def band_pixel_mask(self, views):
        """Pixels of the bands of `views`, for an image of those views concatenated."""
        m = np.zeros((len(views), self.H, self.W), dtype=bool)
        for i, _ in enumerate(views):
            for b in self.bands:
                m[i, b * B:min((b + 1) * B, self.H)] = True
        return m.ravel()

    def gpu_dyn(self, device="cuda"):
        import paper_2604_02851_b300 as gs
        if self.dyn is None:
            return None
        d = self.dyn
        return gs.Dynamics(d["group"], d["poses"], d["normals"], d["light"], d["ambient"], d["diffuse"],
                           device=device)

    def sub_dyn(self, U):
        """The dynamics inputs of the Gaussians U (relabelled)."""
        if self.dyn is None:
            return None
        d = dict(self.dyn)
        d["group"] = self.dyn["group"][U]
        d["normals"] = self.dyn["normals"][U]
        return d


def oracle_records(case, cams, views_idx):
    """The oracle's projection of all Gaussians for the given views, rounded
    to the GPU's float32 record layout [len(views)][n][16] (one view at a
    time, to bound the float64 working set)."""
    out = np.zeros((len(views_idx), case.n, 16), dtype=np.float32)
    for i, v in enumerate(views_idx):
        og = O.project(case.rows, SH, gi.subset_cameras(cams, [v]), B, case.dyn)
        out[i] = oracle_proj_to_gpu(og)[0]
        del og
    return out


def band_lists(cams, rects, depth32, tiles):
    """Band-only list arrays for the oracle: the given tiles' sorted lists
    (bin_tiles), every other tile empty; plus the per-tile runs."""
    vals, start = O.bin_tiles(cams, rects, depth32, tiles, B)
    ranges = np.zeros((O.n_tiles(cams, B), 2), dtype=np.uint32)
    ranges[tiles, 0] = start[:-1]
    ranges[tiles, 1] = start[1:]
    return vals, start, ranges


def compact(U, vals):
    """Relabel list entries (Gaussian indices) to positions in the sorted set U."""
    return np.searchsorted(U, vals).astype(np.uint32)


# ---------------------------------------------------------------- fixtures
@pytest.fixture(scope="module", params=list(CONFIGS))
def case(request):
    import torch
    c = Case(request.param)
    yield c
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def tuned(case):
    """A context set by gs_autotune for the configuration (as bench.py runs it)."""
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import estimate_keys
    params = torch.from_numpy(case.planes).cuda()
    dyn = case.gpu_dyn()
    ctx = gs.Context(0, 0)
    keys_cap = estimate_keys(ctx, params, SH, case.cams, slack=1.05, dyn=dyn)
    ctx.reserve(ctx.workspace_size(case.cams, case.n, keys_cap))
    chosen, _ = gs.gs_autotune(ctx, params, SH, case.cams, keys_cap, reps=1, dyn=dyn)
    print("autotuned", case.name, chosen)
    yield ctx, params, dyn, keys_cap
    ctx.close()
    del params
    torch.cuda.empty_cache()


# ---------------------------------------------------------------- stage-wise
def test_stagewise_binning_compositing_and_adjoints(case, tuned):
    import torch
    import paper_2604_02851_b300 as gs
    ctx, params, dyn, _ = tuned
    cams, V = case.cams, case.V
    proj32 = oracle_records(case, cams, range(V))
    bits = proj32.view(np.uint32)
    rects = np.stack([bits[..., 12] & 0xFFFF, bits[..., 12] >> 16, bits[..., 13] & 0xFFFF, bits[..., 13] >> 16],
                     -1).astype(np.int32)
    depth32 = np.ascontiguousarray(proj32[..., 2])
    o_ranges, K = O.bin_ranges(cams, rects, B)
    tiles = case.band_tiles()
    b_vals, b_start, b_ranges = band_lists(cams, rects, depth32, tiles)

    # ---- GPU binning and sort of all 8 views (the tuned binning)
    d_cams = gs.cameras_to_device(cams)
    tt = ctx.total_tiles(cams)
    t_proj = torch.from_numpy(proj32).cuda()
    keys, vals, ranges, nk = gs.gs_bin_sort(ctx, t_proj, d_cams, V, case.n, tt, K)
    torch.cuda.synchronize()
    assert ctx.status() == (0, 0)
    assert int(nk.item()) == K
    g_ranges = ranges.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(g_ranges, o_ranges)
    for i, t in enumerate(tiles):
        s, e = g_ranges[t]
        np.testing.assert_array_equal(vals[int(s):int(e)].cpu().numpy().view(np.uint32),
                                      b_vals[b_start[i]:b_start[i + 1]])
        assert np.all(keys[int(s):int(e)].cpu().numpy().view(np.uint32) == t)
    print(case.name, "entries", K, "band tiles", len(tiles), "band entries", len(b_vals))

    # ---- compositing of the band pixels on the same records and lists
    npix = gs.total_pixels(cams)
    img, T, nc = gs.gs_render_fwd(ctx, t_proj, d_cams, V, case.n, tt, vals, ranges, npix)
    torch.cuda.synchronize()
    U = np.unique(b_vals)
    proj_c = gpu_proj_to_oracle(proj32[:, U])
    cvals = compact(U, b_vals)
    o_img, o_T, o_nc = O.render(cams, proj_c, cvals, b_ranges, tile=B)
    pm = case.band_pixel_mask(range(V))
    views_mask = np.zeros((V, case.H, case.W), dtype=bool)
    views_mask[list(case.views)] = True
    pm &= views_mask.ravel()
    pm3 = np.repeat(pm.reshape(V, 1, -1), 3, axis=1).ravel()
    g_img, g_T = img.cpu().numpy(), T.cpu().numpy()
    g_nc = nc.cpu().numpy().view(np.uint32)
    assert rel_l2(g_img[pm3], o_img[pm3]) <= TOL
    assert rel_l2(g_T[pm], o_T[pm]) <= TOL
    margin = decision_margins(cams, proj_c, cvals, b_ranges, B)
    mism = (g_nc != o_nc) & pm
    near = margin <= NEAR_DECISION
    print(case.name, "band pixels", int(pm.sum()), "count mismatches", int(mism.sum()),
          "near-threshold pixels", int((near & pm).sum()))
    assert not np.any(mism & ~near), np.nonzero(mism & ~near)[0][:10]

    # ---- raster adjoint: image gradient on the band pixels only (and not
    #      where the two walks end differently)
    rng = np.random.default_rng(31)
    dimg = rng.normal(0.0, 1e-6, 3 * npix).astype(np.float32)
    keep_px = pm & ~mism
    dimg[~np.repeat(keep_px.reshape(V, 1, -1), 3, axis=1).ravel()] = 0.0
    t_dimg = torch.from_numpy(dimg).cuda()
    g2 = gs.gs_raster_bwd(ctx, t_proj, d_cams, V, case.n, tt, vals, ranges, T, nc, t_dimg)
    torch.cuda.synchronize()
    assert ctx.status() == (0, 0)
    g2 = g2.cpu().numpy()
    o_g2c = O.render_bwd(cams, proj_c, cvals, b_ranges, dimg.astype(np.float64), tile=B)
    others = np.ones(case.n, dtype=bool)
    others[U] = False
    assert np.all(g2[:, others] == 0)
    assert np.all(g2[..., 9:] == 0)
    for k in range(9):
        assert rel_l2(g2[:, U, k], o_g2c[..., k]) <= TOL, k
    del g2, img, T, nc, vals, keys, ranges
    torch.cuda.empty_cache()

    # ---- projection adjoint of the oracle's 2D gradient (float32)
    g12 = np.zeros((V, case.n, 12), dtype=np.float32)
    g12[:, U, :9] = o_g2c.astype(np.float32)
    dp = gs.gs_project_bwd(ctx, params, SH, d_cams, V, t_proj, torch.from_numpy(g12).cuda(), dyn=dyn)
    torch.cuda.synchronize()
    dp = gi.planes_to_rows(dp.cpu().numpy())
    o_dp = gi.planes_to_rows(O.project_bwd(case.rows[U], SH, cams, g12[:, U, :9].astype(np.float64), B,
                                           case.sub_dyn(U)))
    assert np.all(dp[others] == 0)
    assert rel_l2(dp[U], o_dp) <= TOL
    del t_proj, g12
    torch.cuda.empty_cache()


def test_end_to_end_bands(case, tuned):
    """Float32 GPU chain from the parameters against the FP64 oracle chain,
    on three views, the image gradient zero outside the bands.

    At this size a tile's list holds thousands of Gaussians, and pairs whose
    depths lie within one float32 rounding of each other are common: the two
    precisions may sort such a pair either way, and where both fragments
    reach a pixel, either order is a correct result.  Pixels whose walks keep
    different fragments, or the same ones in another order, are found
    exactly (tests/flips.c: same_sequences) and left out of both sides'
    image gradient; they must be rare (at most 2 % of the band pixels).  At
    every other band pixel both chains composite the same fragments in the
    same order, so the image and the whole parameter gradient must agree to
    1e-4 with no Gaussian left out."""
    import torch
    import paper_2604_02851_b300 as gs
    ctx, params, dyn, keys_cap = tuned
    views = list(case.views)
    cams = gi.subset_cameras(case.cams, views)
    V3 = len(views)
    # oracle: FP64 projection, band lists of the three views
    og = np.zeros((V3, case.n, 16))
    for i, v in enumerate(views):
        og[i] = O.project(case.rows, SH, gi.subset_cameras(case.cams, [v]), B, case.dyn)[0]
    TX, TY = case.TX, case.TY
    tiles3 = np.asarray([i * TX * TY + b * TX + x for i in range(V3) for b in case.bands for x in range(TX)],
                        dtype=np.int64)
    o_vals, _, o_ranges = band_lists(cams, og[..., 12:16].astype(np.int32), og[..., 2].astype(np.float32),
                                     tiles3)
    # GPU: projection, binning and compositing of the same three views
    d_cams = gs.cameras_to_device(cams)
    tt = ctx.total_tiles(cams)
    npix = gs.total_pixels(cams)
    proj = gs.gs_project(ctx, params, SH, d_cams, V3, dyn=dyn)
    _, vals, ranges, nk = gs.gs_bin_sort(ctx, proj, d_cams, V3, case.n, tt, keys_cap, want_keys=False)
    img, T, nc = gs.gs_render_fwd(ctx, proj, d_cams, V3, case.n, tt, vals, ranges, npix)
    torch.cuda.synchronize()
    assert ctx.status() == (0, 0)
    gp = gpu_proj_to_oracle(proj.cpu().numpy())
    g_full = ranges.cpu().numpy().view(np.uint32)
    g_vals = np.concatenate([vals[int(g_full[t, 0]):int(g_full[t, 1])].cpu().numpy()
                             for t in tiles3]).view(np.uint32)
    g_start = np.concatenate([[0], np.cumsum(g_full[tiles3, 1].astype(np.int64) - g_full[tiles3, 0])])
    g_ranges = np.zeros_like(o_ranges)
    g_ranges[tiles3, 0] = g_start[:-1]
    g_ranges[tiles3, 1] = g_start[1:]
    U = np.union1d(np.unique(o_vals), np.unique(g_vals))
    og_c, gp_c = og[:, U], gp[:, U]
    del og, gp
    o_cv, g_cv = compact(U, o_vals), compact(U, g_vals)
    pm = case.band_pixel_mask(views)
    same = same_sequences(cams, og_c, o_cv, o_ranges, gp_c, g_cv, g_ranges, B)
    use = pm & same
    print(case.name, "end-to-end: band pixels", int(pm.sum()), "with another kept sequence", int((pm & ~same).sum()))
    assert (pm & ~same).sum() <= 0.02 * pm.sum()
    use3 = np.repeat(use.reshape(V3, 1, -1), 3, axis=1).ravel()
    o_img, _, _ = O.render(cams, og_c, o_cv, o_ranges, tile=B)
    e_img = rel_l2(img.cpu().numpy()[use3], o_img[use3])
    print(case.name, "end-to-end band image rel-L2", e_img)
    assert e_img <= TOL
    # the parameter gradient of an image gradient on those pixels only
    rng = np.random.default_rng(32)
    dimg = rng.normal(0.0, 1e-6, 3 * npix).astype(np.float32)
    dimg[~use3] = 0.0
    _, dparams = gs.gs_render_bwd(ctx, params, SH, d_cams, V3, tt, proj, vals, ranges, T, nc,
                                  torch.from_numpy(dimg).cuda(), dyn=dyn)
    torch.cuda.synchronize()
    assert ctx.status() == (0, 0)
    gd = gi.planes_to_rows(dparams.cpu().numpy())
    o_g2 = O.render_bwd(cams, og_c, o_cv, o_ranges, dimg.astype(np.float64), tile=B)
    od = gi.planes_to_rows(O.project_bwd(case.rows[U], SH, cams, o_g2, B, case.sub_dyn(U)))
    others = np.ones(case.n, dtype=bool)
    others[U] = False
    assert np.all(gd[others] == 0)
    e_grad = rel_l2(gd[U], od)
    print(case.name, "end-to-end gradient rel-L2", e_grad, "over", len(U), "Gaussians")
    assert e_grad <= TOL
    del proj, vals, ranges, img, T, nc, dparams
    torch.cuda.empty_cache()


def test_loss_adam_delta_full_size(case, tuned):
    import torch
    import paper_2604_02851_b300 as gs
    ctx = tuned[0]
    rng = np.random.default_rng(33)
    # loss on seeded images at full size (at 3M x 1080p: two of its views)
    V = case.V if case.n <= 1_000_000 else 2
    m = V * 3 * case.H * case.W
    x = rng.uniform(0.0, 1.0, m).astype(np.float32)
    y = np.clip(x + rng.normal(0.0, 0.05, m), 0.0, 1.0).astype(np.float32)
    L, dimg = gs.gs_loss(ctx, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), V, case.H, case.W)
    torch.cuda.synchronize()
    oL, odimg = O.loss(x.astype(np.float64), y.astype(np.float64), V, case.H, case.W)
    assert abs(float(L.item()) - oL) <= TOL * abs(oL)
    assert rel_l2(dimg.cpu().numpy(), odimg) <= TOL
    del x, y, dimg, odimg
    # Adam at the full parameter count, seeded gradient
    n = case.n
    theta = case.planes
    g = (rng.standard_normal(theta.shape, dtype=np.float32)
         * (10.0 ** rng.uniform(-5, 0, theta.shape)).astype(np.float32))
    g[1, :, 3] = 0.0
    th = torch.from_numpy(theta).cuda()
    mm = torch.zeros_like(th)
    vv = torch.zeros_like(th)
    lr = rng.uniform(1e-4, 1e-2, 60).astype(np.float32)
    gs.gs_adam_step(ctx, th, torch.from_numpy(g).cuda(), mm, vv, gs.adam_cfg(lr=lr, step=1))
    torch.cuda.synchronize()
    upd_g = gi.planes_to_rows(th.cpu().numpy()).astype(np.float64) - case.rows
    num = den = 0.0
    grow = gi.planes_to_rows(g)
    for a in range(0, n, 250_000):  # elementwise: the oracle runs on slices
        sl = slice(a, min(n, a + 250_000))
        t_o = case.rows[sl].copy()
        m_o = np.zeros_like(t_o)
        v_o = np.zeros_like(t_o)
        O.adam(t_o, grow[sl].astype(np.float64), m_o, v_o, np.tile(lr, (t_o.shape[0], 1)).astype(np.float64), 1)
        d = t_o - case.rows[sl]
        num += float(np.sum((upd_g[sl] - d) ** 2))
        den += float(np.sum(d ** 2))
    assert (num / den) ** 0.5 <= TOL
    del th, mm, vv, upd_g, grow
    # delta extraction at the full parameter count
    base = case.planes
    pert = base.copy()
    pick = rng.choice(n, n // 20, replace=False)
    pert[rng.integers(0, 15, pick.size), pick, rng.integers(0, 3, pick.size)] += np.float32(2e-3)
    t_th = torch.from_numpy(pert).cuda()
    t_b = torch.from_numpy(base).cuda()
    idx, rec, cnt = gs.gs_extract_delta(ctx, t_th, t_b, 1e-3)
    torch.cuda.synchronize()
    M = int(cnt.item())
    oi, orec, obase = O.delta(pert, base, 1e-3)
    assert M == len(oi) == pick.size
    np.testing.assert_array_equal(idx[:M].cpu().numpy().view(np.uint32), oi)
    np.testing.assert_array_equal(rec[:M].cpu().numpy(), orec)
    np.testing.assert_array_equal(t_b.cpu().numpy(), obase)
    del t_th, t_b, idx, rec
    torch.cuda.empty_cache()


# ---------------------------------------------------------------- the timed path
def test_train_step_equals_separate_calls(case, tuned):
    """gs_train_step (chunk-bitmap lists, graph launch) against the separate
    entry points on the same parameters and targets."""
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import OnlineTrainer
    ctx, params0, dyn, keys_cap = tuned
    cams, V, n = case.cams, case.V, case.n
    tune = ctx.tuning()
    mk = lambda: gs.Context(0, 0, sort_bits=tune["sort_bits"], sort_items=tune["sort_items"],  # noqa: E731
                            binning=tune["binning"], raster_threads=tune["raster_threads"],
                            raster_bwd_threads=tune["raster_bwd_threads"])
    params = params0.clone()
    # one Adam step moves a parameter by just under lr = 1e-3: a lower delta
    # threshold makes the first step's changed set large
    tr = OnlineTrainer(params, SH, cams, keys_cap, ctx=mk(), dyn=dyn, delta_thr=5e-4)
    # targets: the seed-1 model rendered by the serving path
    tparams = torch.from_numpy(gi.make_scene(n, SH, gi.SEED_TARGET)).cuda()
    gs.gs_render_batch(tr.ctx, tparams, SH, tr.d_cams, V, tr.total_tiles, keys_cap, tr.npix, image=tr.targets,
                       dyn=dyn)
    del tparams
    base0 = tr.baseline.clone()
    tr.step()
    torch.cuda.synchronize()
    tr.raise_status()
    # the separate calls
    sep = mk()
    sep.reserve(sep.workspace_size(cams, n, keys_cap))
    proj = gs.gs_project(sep, params0, SH, tr.d_cams, V, dyn=dyn)
    _, vals, ranges, nk = gs.gs_bin_sort(sep, proj, tr.d_cams, V, n, tr.total_tiles, keys_cap, want_keys=False)
    img, T, nc = gs.gs_render_fwd(sep, proj, tr.d_cams, V, n, tr.total_tiles, vals, ranges, tr.npix)
    loss, dimg = gs.gs_loss(sep, img, tr.targets, V, case.H, case.W)
    _, dparams = gs.gs_render_bwd(sep, params0, SH, tr.d_cams, V, tr.total_tiles, proj, vals, ranges, T, nc, dimg,
                                  dyn=dyn)
    torch.cuda.synchronize()
    sep.raise_status()
    assert torch.equal(tr.image, img)
    assert float(tr.d_loss.item()) == float(loss.item())
    e_grad = rel_l2(tr.grads.cpu().numpy(), dparams.cpu().numpy())
    print(case.name, "train step vs separate calls: gradient rel-L2", e_grad)
    assert e_grad <= 1e-5
    del proj, vals, ranges, img, T, nc, dimg, dparams
    # Adam and the delta on the step's own gradient: bit-identical
    th = params0.clone()
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    gs.gs_adam_step(sep, th, tr.grads, m, v, gs.adam_cfg(lr=tr.lr, step=1))
    idx, rec, cnt = gs.gs_extract_delta(sep, th, base0, tr.delta_thr)
    torch.cuda.synchronize()
    assert torch.equal(th, params)
    assert torch.equal(m, tr.m) and torch.equal(v, tr.v)
    M = int(cnt.item())
    assert M == tr.delta_count() > 0
    assert torch.equal(idx[:M], tr.d_idx[:M]) and torch.equal(rec[:M], tr.d_records[:M])
    assert torch.equal(base0, tr.baseline)
    sep.close()
    tr.ctx.close()
    del tr, th, m, v, base0, params
    torch.cuda.empty_cache()


# ---------------------------------------------------------------- serving renders
def test_serving_render_bands_2M_mixed_resolutions():
    """Serving renders (2M Gaussians, SH3, the three request resolutions in one
    batch): gs_render_batch (chunk-bitmap lists) equals the expanded-list
    compositing of the same projection bit for bit, and three 16-row bands of
    every request match the FP64 oracle's render within 1e-4, at the pixels
    whose walks keep the same fragments in the same order on both sides."""
    import torch
    import paper_2604_02851_b300 as gs
    n = 2_000_000
    planes = gi.make_scene(n, SH, gi.SEED_SERVING)
    rows = gi.planes_to_rows(planes).astype(np.float64)
    reqs = gi.serving_requests(40, rate_hz=100.0, seed=gi.SEED_SERVING + 60)
    pick = []
    for r in reqs:  # one request of each resolution class
        if all((r["width"], r["height"]) != (p["width"], p["height"]) for p in pick):
            pick.append(r)
    assert len(pick) == 3
    cams = cams32(gi.cameras_from_eyes([p["eye"] for p in pick], [p["width"] for p in pick],
                                       [p["height"] for p in pick]))
    V = 3
    params = torch.from_numpy(planes).cuda()
    ctx = gs.Context(0, 0)
    from paper_2604_02851_b300.train import estimate_keys
    keys_cap = estimate_keys(ctx, params, SH, cams, slack=1.05)
    ctx.reserve(ctx.workspace_size(cams, n, keys_cap))
    d_cams = gs.cameras_to_device(cams)
    tt = ctx.total_tiles(cams)
    npix = gs.total_pixels(cams)
    img_b = gs.gs_render_batch(ctx, params, SH, d_cams, V, tt, keys_cap, npix)
    proj = gs.gs_project(ctx, params, SH, d_cams, V)
    _, vals, ranges, nk = gs.gs_bin_sort(ctx, proj, d_cams, V, n, tt, keys_cap, want_keys=False)
    img, _, _ = gs.gs_render_fwd(ctx, proj, d_cams, V, n, tt, vals, ranges, npix)
    torch.cuda.synchronize()
    assert ctx.status() == (0, 0)
    assert torch.equal(img_b, img)
    # bands: rows 4, the middle and the last of every request (ragged where H % 16 != 0)
    TXs = [(int(w) + B - 1) // B for w in cams["width"]]
    TYs = [(int(h) + B - 1) // B for h in cams["height"]]
    toff = np.concatenate([[0], np.cumsum([a * b for a, b in zip(TXs, TYs)])])
    tiles, pm = [], []
    for v in range(V):
        m = np.zeros((int(cams["height"][v]), int(cams["width"][v])), dtype=bool)
        for b in (4, TYs[v] // 2, TYs[v] - 1):
            tiles.extend(toff[v] + b * TXs[v] + np.arange(TXs[v]))
            m[b * B:(b + 1) * B] = True
        pm.append(m.ravel())
    tiles = np.asarray(tiles, dtype=np.int64)
    pm = np.concatenate(pm)
    og = np.zeros((V, n, 16))
    for v in range(V):
        og[v] = O.project(rows, SH, gi.subset_cameras(cams, [v]), B)[0]
    o_vals, _, o_ranges = band_lists(cams, og[..., 12:16].astype(np.int32), og[..., 2].astype(np.float32),
                                     tiles)
    gp = gpu_proj_to_oracle(proj.cpu().numpy())
    g_full = ranges.cpu().numpy().view(np.uint32)
    g_vals = np.concatenate([vals[int(g_full[t, 0]):int(g_full[t, 1])].cpu().numpy() for t in tiles]).view(np.uint32)
    g_start = np.concatenate([[0], np.cumsum(g_full[tiles, 1].astype(np.int64) - g_full[tiles, 0])])
    g_ranges = np.zeros_like(o_ranges)
    g_ranges[tiles, 0] = g_start[:-1]
    g_ranges[tiles, 1] = g_start[1:]
    U = np.union1d(np.unique(o_vals), np.unique(g_vals))
    og_c, gp_c = og[:, U], gp[:, U]
    del og, gp
    o_cv, g_cv = compact(U, o_vals), compact(U, g_vals)
    same = same_sequences(cams, og_c, o_cv, o_ranges, gp_c, g_cv, g_ranges, B)
    use = pm & same
    print("serving: band pixels", int(pm.sum()), "with another kept sequence", int((pm & ~same).sum()))
    assert (pm & ~same).sum() <= 0.02 * pm.sum()
    o_img, _, _ = O.render(cams, og_c, o_cv, o_ranges, tile=B)
    use3 = np.concatenate([np.repeat(u.reshape(1, -1), 3, axis=0).ravel()
                           for u in np.split(use, np.cumsum([int(w) * int(h) for w, h in
                                                             zip(cams["width"], cams["height"])])[:-1])])
    e = rel_l2(img.cpu().numpy()[use3], o_img[use3])
    print("serving: band image rel-L2", e)
    assert e <= TOL
    ctx.close()
