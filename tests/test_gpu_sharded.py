"""The training step split into its gradient and update parts
(gs_train_cfg.phases), as the view-sharded step across GPUs runs it.

One GPU stands in for two ranks, one after the other (nothing waits on
another launch): each rank's gradient part renders its views with its loss
share; the test sums the two gradients, as the all-reduce would, and runs the
update part on the sum.  The sum must be the gradient of the unsplit step
(within float atomics order), the loss shares must add up to its loss, the
update must equal gs_adam_step and gs_extract_delta on that gradient bit for
bit, and the gradient part must leave the model and the optimiser state
alone."""
import numpy as np
import pytest

import gs_inputs as gi
from gpu_util import rel_l2

pytestmark = pytest.mark.gpu

N, SH, V, W, H = 20_000, 2, 4, 128, 96


def _views(images, views):
    per = 3 * H * W
    import torch
    return torch.cat([images[v * per:(v + 1) * per] for v in views])


def test_gradient_and_update_parts_compose_to_the_step():
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300 import parallel
    from paper_2604_02851_b300.train import OnlineTrainer, estimate_keys
    cams = gi.ring_cameras(V, W, H)
    planes = gi.make_scene(N, SH, 41)
    p0 = torch.from_numpy(planes).cuda()
    ctx = gs.Context(0, 0)
    keys_cap = estimate_keys(ctx, p0, SH, cams, slack=1.3)
    full = OnlineTrainer(p0.clone(), SH, cams, keys_cap, ctx=ctx)
    tparams = torch.from_numpy(gi.make_scene(N, SH, 42)).cuda()
    gs.gs_render_batch(full.ctx, tparams, SH, full.d_cams, V, full.total_tiles, keys_cap, full.npix,
                       image=full.targets)
    shards = []
    for r in range(2):
        t = parallel.ViewShardedTrainer(p0.clone(), SH, cams, keys_cap, rank=r, world=2)
        t.targets.copy_(_views(full.targets, t.views))
        shards.append(t)
    full.step()
    for t in shards:
        t.trainer.step()  # the gradient part only
    torch.cuda.synchronize()
    full.raise_status()
    # the gradient part leaves the model, the optimiser state and the step alone
    for t in shards:
        tr = t.trainer
        assert torch.equal(tr.params, p0) and torch.equal(tr.baseline, p0)
        assert not tr.m.any() and not tr.v.any()
        assert int(tr.d_step.item()) == 1 and tr.delta_count() == 0
        tr.raise_status()
    gsum = shards[0].trainer.grads + shards[1].trainer.grads  # what the all-reduce sums
    e = rel_l2(gsum.cpu().numpy(), full.grads.cpu().numpy())
    lsum = float(shards[0].trainer.d_loss.item()) + float(shards[1].trainer.d_loss.item())
    print("sharded gradient rel-L2", e, "loss", lsum, float(full.d_loss.item()))
    assert e <= 1e-5
    assert abs(lsum - float(full.d_loss.item())) <= 1e-6 * abs(float(full.d_loss.item()))
    # the update part on the summed gradient: gs_adam_step + gs_extract_delta
    t0 = shards[0].trainer
    t0.grads.copy_(gsum)
    t0.step_update()
    th = p0.clone()
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    base = p0.clone()
    gs.gs_adam_step(ctx, th, gsum, m, v, gs.adam_cfg(lr=t0.lr, step=1))
    idx, rec, cnt = gs.gs_extract_delta(ctx, th, base, t0.delta_thr)
    torch.cuda.synchronize()
    t0.raise_status()
    assert torch.equal(t0.params, th) and torch.equal(t0.m, m) and torch.equal(t0.v, v)
    M = int(cnt.item())
    assert t0.delta_count() == M
    assert torch.equal(t0.d_idx[:M], idx[:M]) and torch.equal(t0.d_records[:M], rec[:M])
    assert torch.equal(t0.baseline, base)
    assert int(t0.d_step.item()) == 2
    for t in shards:
        t.trainer.ctx.close()
    ctx.close()


def test_phases_out_of_range_are_rejected():
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300 import _lib
    from paper_2604_02851_b300.train import OnlineTrainer
    cams = gi.ring_cameras(1, 32, 32)
    p = torch.from_numpy(gi.make_scene(100, 0, 1)).cuda()
    tr = OnlineTrainer(p, 0, cams, 4096)
    tr.cfg.phases = 4
    with pytest.raises(gs.GsError):
        tr.step_eager()
    tr.cfg.phases = -1
    with pytest.raises(gs.GsError):
        tr.step_eager()
    tr.cfg.phases = _lib.TRAIN_ALL
    tr.step_eager()
    torch.cuda.synchronize()
    tr.raise_status()
    tr.ctx.close()


def test_update_part_with_preculling_matches_the_full_step():
    """The update part alone, given the full step's gradient, reproduces the
    full step's update bit for bit with a preculling grid: it finds the kept
    Gaussians itself (Adam leaves the culled ones and their moments alone)."""
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import OnlineTrainer, estimate_keys
    n, sh = 20_000, 1
    cams = gi.ring_cameras(3, 160, 112)
    planes = gi.make_scene(n, sh, 93)
    origin, size, dims = (-1.0, -1.0, -1.0), 0.25, (8, 8, 8)
    pc = gs.Precull(origin, size, dims)
    vis = (np.random.default_rng(6).random(dims[::-1]) < 0.6).astype(np.uint8)
    pc.visible.copy_(torch.from_numpy(vis))
    ctx = gs.Context(0, 0)
    p0 = torch.from_numpy(planes).cuda()
    keys = estimate_keys(ctx, p0, sh, cams, slack=1.5)
    full = OnlineTrainer(p0.clone(), sh, cams, keys, ctx=ctx, precull=pc)
    tparams = torch.from_numpy(gi.make_scene(n, sh, 94)).cuda()
    gs.gs_render_batch(full.ctx, tparams, sh, full.d_cams, 3, full.total_tiles, keys, full.npix, image=full.targets)
    full.step()
    torch.cuda.synchronize()
    full.raise_status()
    upd = OnlineTrainer(p0.clone(), sh, cams, keys, ctx=gs.Context(0, 0), precull=pc)
    upd.grads.copy_(full.grads)
    upd.step_update()
    torch.cuda.synchronize()
    upd.raise_status()
    assert torch.equal(upd.params, full.params)
    assert torch.equal(upd.m, full.m) and torch.equal(upd.v, full.v)
    assert torch.equal(upd.baseline, full.baseline)
    M = full.delta_count()
    assert upd.delta_count() == M and torch.equal(upd.d_records[:M], full.d_records[:M])
    # some Gaussians are culled, and those keep their parameters
    changed = (upd.params != p0).any(dim=2).any(dim=0).cpu().numpy()
    assert 0.2 < changed.mean() < 0.95
    upd.ctx.close()
    ctx.close()
