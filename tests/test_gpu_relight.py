"""SH relighting and light visibility (Sec. 3.4.1) on the GPU against the
FP64 oracle: the relit colour and its adjoint (static and rigid objects), the
fused training step with lighting, and the light-space depth map and
per-Gaussian visibility test."""
import numpy as np
import pytest

import gs_inputs as gi
import oracle as O
from flips import decision_flips
from gpu_util import GpuRun, OracleStages, cams32, l1_sign_expected, rel_l2, scene

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _poses(G, seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(G, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    poses = np.zeros((G, 8)); poses[:, :4] = q; poses[:, 4:7] = rng.uniform(-0.2, 0.2, (G, 3))
    return poses.astype(np.float32).astype(np.float64)


def _lighting(n, seed, vis=True):
    import paper_2604_02851_b300 as gs
    rng = np.random.default_rng(seed)
    env = rng.normal(0.0, 0.3, (16, 3))
    env[0] = 1.2  # a positive ambient term
    d = np.array([0.35, 0.8, -0.3]); d /= np.linalg.norm(d)
    lt = gs.Lighting(n, env, d, (0.9, 0.8, 0.6), with_visibility=vis)
    v = None
    if vis:
        v = rng.integers(0, 256, n).astype(np.uint8)
        v[rng.random(n) < 0.3] = 0
        v[rng.random(n) < 0.3] = 255
        import torch
        lt.visibility[:n].copy_(torch.from_numpy(v))
    return lt, v


def _oracle_dyn(lt, vis, group=None, poses=None):
    # the lighting buffer as the GPU holds it (an input, written from the host)
    d = {"sh_light": lt.light.cpu().numpy().astype(np.float64)}
    if vis is not None:
        d["visibility"] = vis
    if group is not None:
        d["group"], d["poses"] = group, poses
    return d


@pytest.fixture(scope="module", params=[False, True], ids=["static", "rigid"])
def rcase(request):
    import paper_2604_02851_b300 as gs
    n, sh = 20_000, 3
    planes = scene(n, sh, 51)
    cams = gi.ring_cameras(2, 200, 136)
    lt, vis = _lighting(n, 52)
    group = poses = dyn = None
    if request.param:
        group = (np.arange(n) % 8).astype(np.int32)
        poses = _poses(8, 53)
        dyn = gs.Dynamics(group, poses)
    d = _oracle_dyn(lt, vis, group, poses)
    target = O.forward(scene(n, sh, 54), sh, cams32(cams), dyn=d)["image"]
    run = GpuRun(planes, sh, cams, target, dyn=dyn, lighting=lt)
    yield planes, sh, cams32(cams), d, run
    run.close()


def test_relit_projection_matches_oracle(rcase):
    planes, sh, cams, d, run = rcase
    og = O.project(planes, sh, cams, dyn=d)
    gp = run.oracle_proj()
    both = (og[..., 14] > og[..., 12]) & (gp[..., 14] > gp[..., 12])
    assert np.sum((og[..., 14] > og[..., 12]) != (gp[..., 14] > gp[..., 12])) <= max(2, 1e-4 * both.sum())
    for f in (0, 1, 2, 3, 4, 5, 6, 8, 9, 10):
        assert rel_l2(gp[..., f][both], og[..., f][both]) <= TOL, f
    # clamp masks agree wherever the colour is not within rounding of zero
    mo = og[..., 11].astype(np.int64)
    mg = gp[..., 11].astype(np.int64)
    for ch in range(3):
        assert not np.any(both & (og[..., 8 + ch] > 1e-5) & (((mg >> ch) & 1) == 1))
        assert not np.any(both & (gp[..., 8 + ch] > 1e-5) & (((mo >> ch) & 1) == 1))
    # the lighting changes the colours: not the view-dependent ones
    plain = O.project(planes, sh, cams)
    assert rel_l2(plain[..., 8:11][both], og[..., 8:11][both]) > 0.05


def test_relit_gradients_match_oracle(rcase):
    planes, sh, cams, d, run = rcase
    gp = run.oracle_proj()
    # stage-wise: the GPU projection adjoint on the oracle's 2D gradients
    st = OracleStages(O, planes, sh, cams, run.np("target"), dyn=d, gpu_dyn=run.dyn, gpu_lighting=run.lighting)
    gd = st.gpu_project_bwd()
    assert rel_l2(gd, st.dparams) <= TOL
    assert rel_l2(gd[3:], st.dparams[3:]) <= TOL  # the SH (transfer) part alone
    st.close()
    r = O.loss_and_grad(planes, sh, cams, run.np("target"), dyn=d)  # end to end
    flips, _ = decision_flips(cams, r["proj"], r["vals"], r["ranges"], gp, run.sorted_vals(), run.ranges_np())
    support = np.any(r["proj"][..., [7, 12, 13, 14, 15]] != gp[..., [7, 12, 13, 14, 15]], axis=(0, 2))
    odd = flips.any(axis=0) | support
    assert odd.mean() <= 1e-3
    od, _ = l1_sign_expected(O, planes, sh, cams, r, run.np("target"), run.np("dparams"), dyn=d, keep=~odd)
    assert rel_l2(run.np("dparams")[:, ~odd], od[:, ~odd]) <= TOL
    assert abs(float(run.loss.item()) - r["loss"]) <= TOL * r["loss"]


def test_relit_fused_train_step_equals_separate_calls():
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import OnlineTrainer, estimate_keys
    n, sh, V, W, H = 30_000, 3, 3, 160, 112
    planes = scene(n, sh, 55)
    cams = gi.ring_cameras(V, W, H)
    group = (np.arange(n) % 4).astype(np.int32)
    dyn = gs.Dynamics(group, _poses(4, 56))
    lt, vis = _lighting(n, 57)
    d = _oracle_dyn(lt, vis, group, _poses(4, 56))
    target = torch.from_numpy(O.forward(scene(n, sh, 58), sh, cams32(cams), dyn=d)["image"].astype(np.float32)).cuda()
    p_fused = torch.from_numpy(planes).cuda()
    p_sep = torch.from_numpy(planes).cuda()
    ctx = gs.Context(0, 0)
    cap = estimate_keys(ctx, p_fused, sh, cams, slack=1.5)
    tr = OnlineTrainer(p_fused, sh, cams, cap, ctx=ctx, dyn=dyn, lighting=lt)
    tr.targets.copy_(target)
    c2 = gs.Context(0, 0)
    c2.reserve(c2.workspace_size(cams, n, cap))
    d_cams = gs.cameras_to_device(cams)
    tt = c2.total_tiles(cams)
    npix = V * W * H
    m = torch.zeros_like(p_sep); v = torch.zeros_like(p_sep); base = p_sep.clone()
    for step in (1, 2):
        tr.step()
        proj = gs.gs_project(c2, p_sep, sh, d_cams, V, dyn=dyn, lighting=lt)
        _, vals, ranges, nk = gs.gs_bin_sort(c2, proj, d_cams, V, n, tt, cap, want_keys=False)
        img, T, nc = gs.gs_render_fwd(c2, proj, d_cams, V, n, tt, vals, ranges, npix)
        loss, dimg = gs.gs_loss(c2, img, target, V, H, W)
        _, dpar = gs.gs_render_bwd(c2, p_sep, sh, d_cams, V, tt, proj, vals, ranges, T, nc, dimg, dyn=dyn,
                                   lighting=lt)
        gs.gs_adam_step(c2, p_sep, dpar, m, v, gs.adam_cfg(1e-3, step=step))
        gs.gs_extract_delta(c2, p_sep, base, 1e-3)
        torch.cuda.synchronize()
        assert abs(tr.loss() - float(loss.item())) <= 1e-6 * abs(float(loss.item()))
        assert rel_l2(tr.grads.cpu().numpy(), dpar.cpu().numpy()) <= 1e-5
        upd = np.linalg.norm((p_sep - torch.from_numpy(planes).cuda()).cpu().numpy())
        assert np.linalg.norm((p_fused - p_sep).cpu().numpy()) <= 1e-3 * upd
    tr.raise_status()
    c2.raise_status()


def test_relit_serving_matches_projection_path():
    """gs_render_batch with lighting renders what project + sort + compose do."""
    import torch
    import paper_2604_02851_b300 as gs
    n, sh = 20_000, 2
    planes = scene(n, sh, 59)
    cams = gi.ring_cameras(3, 128, 96)
    lt, vis = _lighting(n, 60)
    run = GpuRun(planes, sh, cams, lighting=lt)
    img = gs.gs_render_batch(run.ctx, run.params, sh, run.d_cams, 3, run.tt, 1 << 18, run.npix, lighting=lt)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(img.cpu().numpy(), run.np("image"))
    f = O.forward(planes, sh, cams32(cams), dyn=_oracle_dyn(lt, vis))
    assert rel_l2(img.cpu().numpy(), f["image"]) <= TOL
    run.close()


# ---------------------------------------------------------------- light-space depth map and visibility
def _light_case(n, seed, W=512, H=384, dynamic=True):
    import paper_2604_02851_b300 as gs
    planes = scene(n, 0, seed)
    planes[1, :, :3] += 0.8  # larger splats: footprints of tens of texels
    d = np.array([0.5, 0.75, 0.3]); d /= np.linalg.norm(d)
    lc = gs.light_camera(direction=d, width=W, height=H, extent=3.2, alpha_min=0.5, bias=0.02)
    lcd = gs.light_camera_dict(lc)  # the float32 fields the GPU receives
    group = poses = dyn = None
    if dynamic:
        group = (np.arange(n) % 16).astype(np.int32)
        poses = _poses(16, seed + 1)
        dyn = gs.Dynamics(group, poses)
    od = None if group is None else {"group": group, "poses": poses}
    return planes, lc, lcd, dyn, od


SLACK = 1e-3


def _atol(D):
    return 1e-5 * (1.0 + np.abs(np.where(np.isfinite(D), D, 0.0)))


@pytest.mark.parametrize("dynamic", [False, True])
def test_light_depth_map_is_bracketed_by_the_oracle(dynamic):
    """Where float32 may decide a footprint test either way (q within SLACK of
    tau), either depth is correct: the GPU map lies between the oracle maps
    with the bound moved by +-SLACK; elsewhere it equals the oracle's."""
    import torch
    import paper_2604_02851_b300 as gs
    n = 20_000
    planes, lc, lcd, dyn, od = _light_case(n, 61, dynamic=dynamic)
    ctx = gs.Context(0, 0)
    p = torch.from_numpy(planes).cuda()
    D = gs.gs_light_depth_map(ctx, p, lc, dyn=dyn).cpu().numpy().astype(np.float64)
    ctx.raise_status()
    lo = O.light_depth(planes, lcd, dyn=od, slack=SLACK)
    hi = O.light_depth(planes, lcd, dyn=od, slack=-SLACK)
    ex = O.light_depth(planes, lcd, dyn=od)
    assert np.isfinite(ex).mean() > 0.2
    # finite exactly where some Gaussian may cover the texel
    assert np.all(np.isinf(D) <= np.isinf(hi)) and np.all(np.isfinite(D) <= np.isfinite(lo))
    fin = np.isfinite(D)
    assert np.all(D[fin] >= lo[fin] - _atol(lo)[fin])
    hf = fin & np.isfinite(hi)
    assert np.all(D[hf] <= hi[hf] + _atol(hi)[hf])
    same = (np.isinf(D) & np.isinf(ex)) | (np.abs(D - np.where(np.isfinite(ex), ex, 0)) <= _atol(ex))
    assert same.mean() >= 0.999


def test_light_depth_map_accumulates_bit_exactly():
    """The atomic min does not depend on order: two pools splatted into one map
    give the map of their union, bit for bit."""
    import torch
    import paper_2604_02851_b300 as gs
    n = 20_000
    planes, lc, _, _, _ = _light_case(n, 62, dynamic=False)
    ctx = gs.Context(0, 0)
    p = torch.from_numpy(planes).cuda()
    full = gs.gs_light_depth_map(ctx, p, lc)
    a = torch.from_numpy(np.ascontiguousarray(planes[:, : n // 3])).cuda()
    b = torch.from_numpy(np.ascontiguousarray(planes[:, n // 3:])).cuda()
    part = gs.gs_light_depth_map(ctx, b, lc)
    gs.gs_light_depth_map(ctx, a, lc, part, accumulate=True)
    torch.cuda.synchronize()
    assert torch.equal(full.view(torch.int32), part.view(torch.int32))
    ctx.raise_status()


@pytest.mark.parametrize("dynamic", [False, True])
def test_light_visibility_matches_oracle(dynamic):
    """Visibility equals the oracle's wherever the decision is not within
    rounding of a texel edge or of the depth test; the map is the oracle's
    own (no GPU value is fed to the oracle)."""
    import torch
    import paper_2604_02851_b300 as gs
    n = 20_000
    planes, lc, lcd, dyn, od = _light_case(n, 63, dynamic=dynamic)
    ctx = gs.Context(0, 0)
    p = torch.from_numpy(planes).cuda()
    D = gs.gs_light_depth_map(ctx, p, lc, dyn=dyn)
    vis = gs.gs_light_visibility(ctx, p, lc, D, dyn=dyn).cpu().numpy()
    ctx.raise_status()
    ex = O.light_depth(planes, lcd, dyn=od)
    lo = O.light_depth(planes, lcd, dyn=od, slack=SLACK)
    hi = O.light_depth(planes, lcd, dyn=od, slack=-SLACK)
    ov, uvz = O.light_visibility(planes, lcd, ex, dyn=od)
    W, H = lcd["width"], lcd["height"]
    u, v, z = uvz[:, 0], uvz[:, 1], uvz[:, 2]
    edge = (np.abs(u - np.round(u)) < 2e-3) | (np.abs(v - np.round(v)) < 2e-3)
    inside = (u >= 0) & (u < W) & (v >= 0) & (v < H)
    ti = np.clip(np.floor(u), 0, W - 1).astype(np.int64)
    tj = np.clip(np.floor(v), 0, H - 1).astype(np.int64)
    zb = z - lcd["bias"]
    Dlo, Dhi, Dex = lo[tj, ti], hi[tj, ti], ex[tj, ti]
    near_test = np.isfinite(Dex) & (np.abs(zb - Dex) <= 1e-4 * (1 + np.abs(z)))
    in_bracket = (zb >= Dlo - 1e-4) & ((zb <= Dhi + 1e-4) | np.isinf(Dhi)) & (Dlo < Dhi)
    ambiguous = inside & (edge | near_test | in_bracket)
    mism = vis != ov
    assert not np.any(mism & ~ambiguous), np.nonzero(mism & ~ambiguous)[0][:10]
    assert ambiguous.mean() <= 0.01
    shadowed = (ov == 0).mean()
    assert 0.05 < shadowed < 0.95
    assert np.all(vis[~inside] == 255)


def test_light_map_edge_cases():
    import torch
    import paper_2604_02851_b300 as gs
    ctx = gs.Context(0, 0)
    empty = torch.zeros((15, 0, 4), dtype=torch.float32, device="cuda")
    lc = gs.light_camera(direction=(0.0, 1.0, 0.0), width=7, height=5, extent=2.0)
    D = gs.gs_light_depth_map(ctx, empty, lc)
    assert torch.isinf(D).all() and D.shape == (5, 7)
    # a 1x1 map, a Gaussian outside it and one inside
    planes = scene(2, 0, 64)
    planes[0, 0, :3] = (5.0, 0.0, 5.0)
    planes[0, 1, :3] = (0.0, 0.0, 0.0)
    planes[0, :, 3] = 4.0
    lc1 = gs.light_camera(direction=(0.0, 1.0, 0.0), width=1, height=1, extent=0.5)
    p = torch.from_numpy(planes).cuda()
    D1 = gs.gs_light_depth_map(ctx, p, lc1)
    v1 = gs.gs_light_visibility(ctx, p, lc1, D1).cpu().numpy()
    assert list(v1) == [255, 255]
    ex = O.light_depth(planes, gs.light_camera_dict(lc1))
    assert np.isfinite(D1.cpu().numpy()).all() == np.isfinite(ex).all()
    for bad in (dict(alpha_min=1.0), dict(alpha_min=0.0), dict(width=0), dict(width=20000), dict(bias=-1.0)):
        kw = dict(direction=(0.0, 1.0, 0.0), width=8, height=8, extent=1.0)
        kw.update(bad)
        with pytest.raises(gs.GsError):
            gs.gs_light_depth_map(ctx, p, gs.light_camera(**kw))
    # SH lighting together with the Lambertian factor is refused
    lt = gs.Lighting(2)
    dyn = gs.Dynamics(np.zeros(2, np.int32), _poses(1, 65), normals=np.ones((2, 3)) / np.sqrt(3))
    d_cams = gs.cameras_to_device(gi.ring_cameras(1, 32, 32))
    with pytest.raises(gs.GsError):
        gs.gs_project(ctx, p, 0, d_cams, 1, dyn=dyn, lighting=lt)
    ctx.raise_status()
