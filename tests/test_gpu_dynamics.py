"""Scene dynamics (rigid-object poses and Lambertian relighting, Sec. 3.4) on
the GPU against the FP64 oracle, and the fused graph-captured training step
against the same step through the separate C entry points."""
import numpy as np
import pytest

import gs_inputs as gi
import oracle as O
from flips import decision_flips
from gpu_util import GpuRun, OracleStages, cams32, gpu_proj_to_oracle, l1_sign_expected, rel_l2, scene

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _dyn_np(n, G, seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(G, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    poses = np.zeros((G, 8)); poses[:, :4] = q; poses[:, 4:7] = rng.uniform(-0.2, 0.2, (G, 3))
    nn = rng.normal(size=(n, 3)); nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    light = np.array([0.4, 0.8, 0.45]); light /= np.linalg.norm(light)
    return {"group": (np.arange(n) % G).astype(np.int32), "poses": poses.astype(np.float32).astype(np.float64),
            "normals": nn.astype(np.float32).astype(np.float64),
            "light": light.astype(np.float32).astype(np.float64), "ambient": 0.3, "diffuse": 0.7}


def _dyn_gpu(d):
    import paper_2604_02851_b300 as gs
    return gs.Dynamics(d["group"], d["poses"], d["normals"], d["light"], d["ambient"], d["diffuse"])


@pytest.fixture(scope="module")
def dcase():
    n, sh = 20_000, 3
    planes = scene(n, sh, 31)
    cams = gi.ring_cameras(2, 200, 136)
    d = _dyn_np(n, 8, 3)
    target = O.forward(scene(n, sh, 32), sh, cams32(cams), dyn=d)["image"]
    run = GpuRun(planes, sh, cams, target, dyn=_dyn_gpu(d))
    yield planes, sh, cams32(cams), d, run
    run.close()


def test_dynamic_projection_matches_oracle(dcase):
    planes, sh, cams, d, run = dcase
    og = O.project(planes, sh, cams, dyn=d)
    gp = run.oracle_proj()
    both = (og[..., 14] > og[..., 12]) & (gp[..., 14] > gp[..., 12])
    assert np.sum((og[..., 14] > og[..., 12]) != (gp[..., 14] > gp[..., 12])) <= max(2, 1e-4 * both.sum())
    for f in (0, 1, 2, 3, 4, 5, 6, 8, 9, 10):
        assert rel_l2(gp[..., f][both], og[..., f][both]) <= TOL, f


def test_dynamic_gradients_match_oracle(dcase):
    planes, sh, cams, d, run = dcase
    gp = run.oracle_proj()
    # stage-wise: the GPU projection adjoint on the oracle's 2D gradients
    st = OracleStages(O, planes, sh, cams, run.np("target"), dyn=d, gpu_dyn=run.dyn)
    assert rel_l2(st.gpu_project_bwd(), st.dparams) <= TOL
    st.close()
    r = O.loss_and_grad(planes, sh, cams, run.np("target"), dyn=d)  # end to end
    flips, _ = decision_flips(cams, r["proj"], r["vals"], r["ranges"], gp, run.sorted_vals(), run.ranges_np())
    support = np.any(r["proj"][..., [7, 12, 13, 14, 15]] != gp[..., [7, 12, 13, 14, 15]], axis=(0, 2))
    odd = flips.any(axis=0) | support
    assert odd.mean() <= 1e-3
    od, _ = l1_sign_expected(O, planes, sh, cams, r, run.np("target"), run.np("dparams"), dyn=d, keep=~odd)
    assert rel_l2(run.np("dparams")[:, ~odd], od[:, ~odd]) <= TOL
    assert abs(float(run.loss.item()) - r["loss"]) <= TOL * r["loss"]


@pytest.mark.parametrize("dynamic", [False, True])
def test_fused_train_step_equals_separate_calls(dynamic):
    """Two graph launches of gs_train_step against the same two steps through
    gs_project ... gs_extract_delta: parameters, Adam moments, delta sets."""
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import OnlineTrainer, estimate_keys
    n, sh, V, W, H = 30_000, 3, 3, 160, 112
    planes = scene(n, sh, 41)
    cams = gi.ring_cameras(V, W, H)
    d = _dyn_np(n, 4, 9) if dynamic else None
    dyn = _dyn_gpu(d) if dynamic else None
    target = torch.from_numpy(O.forward(scene(n, sh, 42), sh, cams32(cams), dyn=d)["image"].astype(np.float32)).cuda()
    p_fused = torch.from_numpy(planes).cuda()
    p_sep = torch.from_numpy(planes).cuda()
    ctx = gs.Context(0, 0)
    cap = estimate_keys(ctx, p_fused, sh, cams, slack=1.5)
    tr = OnlineTrainer(p_fused, sh, cams, cap, ctx=ctx, dyn=dyn)
    tr.targets.copy_(target)
    c2 = gs.Context(0, 0)
    c2.reserve(c2.workspace_size(cams, n, cap))
    d_cams = gs.cameras_to_device(cams)
    tt = c2.total_tiles(cams)
    npix = V * W * H
    m = torch.zeros_like(p_sep); v = torch.zeros_like(p_sep); base = p_sep.clone()
    for step in (1, 2):
        tr.step()
        proj = gs.gs_project(c2, p_sep, sh, d_cams, V, dyn=dyn)
        _, vals, ranges, nk = gs.gs_bin_sort(c2, proj, d_cams, V, n, tt, cap, want_keys=False)
        img, T, nc = gs.gs_render_fwd(c2, proj, d_cams, V, n, tt, vals, ranges, npix)
        loss, dimg = gs.gs_loss(c2, img, target, V, H, W)
        _, dpar = gs.gs_render_bwd(c2, p_sep, sh, d_cams, V, tt, proj, vals, ranges, T, nc, dimg, dyn=dyn)
        gs.gs_adam_step(c2, p_sep, dpar, m, v, gs.adam_cfg(1e-3, step=step))
        idx, rec, cnt = gs.gs_extract_delta(c2, p_sep, base, 1e-3)
        torch.cuda.synchronize()
        assert abs(tr.loss() - float(loss.item())) <= 1e-6 * abs(float(loss.item()))
        # gradients differ only in the order of float atomics
        assert rel_l2(tr.grads.cpu().numpy(), dpar.cpu().numpy()) <= 1e-5
        upd = np.linalg.norm((p_sep - torch.from_numpy(planes).cuda()).cpu().numpy())
        assert np.linalg.norm((p_fused - p_sep).cpu().numpy()) <= 1e-3 * upd
    tr.raise_status()
    c2.raise_status()
