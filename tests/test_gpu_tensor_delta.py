"""Tensor deltas per attribute group and their client-side replay (Sec. 3.5)
against the oracle: indices, records, baselines and replayed parameters
bit-exact."""
import numpy as np
import pytest

import gs_inputs as gi
import oracle as O

pytestmark = pytest.mark.gpu

GROUPS = ["mean", "opacity", "scale", "rotation", "dc", "sh_rest"]


def _perturb(n, seed, frac):
    th = gi.make_scene(n, 3, seed)
    base = th.copy()
    rows = gi.planes_to_rows(th).astype(np.float32)
    rng = np.random.default_rng(seed)
    for lo, hi in [(0, 3), (3, 4), (4, 7), (8, 12), (12, 15), (15, 60)]:
        pick = np.nonzero(rng.random(n) < frac)[0]
        col = rng.integers(lo, hi, len(pick))
        rows[pick, col] += rng.choice([2e-3, -5e-3, 9e-4, 1e-3], len(pick)).astype(np.float32)
    return gi.rows_to_planes(rows), base


@pytest.mark.parametrize("name", GROUPS)
@pytest.mark.parametrize("n", [1, 1000, 70_001])
def test_tensor_delta_bit_exact(name, n):
    import torch
    import paper_2604_02851_b300 as gs
    th, base = _perturb(n, 50 + n % 7, 0.15)
    ctx = gs.Context(0, 1 << 24)
    t_th = torch.from_numpy(th).cuda()
    t_base = torch.from_numpy(base).cuda()
    idx, vals, cnt = gs.gs_extract_tensor_delta(ctx, t_th, t_base, name, 1e-3)
    torch.cuda.synchronize()
    m = int(cnt.item())
    oidx, ovals, obase = O.tensor_delta(th, base, O.ATTR_GROUPS[name], 1e-3)
    assert m == len(oidx)
    np.testing.assert_array_equal(idx.cpu().numpy()[:m].view(np.uint32), oidx)
    np.testing.assert_array_equal(vals.cpu().numpy()[:m], ovals)
    np.testing.assert_array_equal(t_base.cpu().numpy(), obase)
    # replay into a client that holds the old baseline
    client = torch.from_numpy(base).cuda()
    gs.gs_apply_tensor_delta(ctx, client, name, idx, vals, cnt)
    torch.cuda.synchronize()
    assert ctx.status()[0] == 0
    np.testing.assert_array_equal(client.cpu().numpy(), O.apply_tensor_delta(base, O.ATTR_GROUPS[name], oidx, ovals))
    ctx.close()


def test_full_record_replay_bit_exact():
    import torch
    import paper_2604_02851_b300 as gs
    n = 50_000
    th, base = _perturb(n, 61, 0.2)
    ctx = gs.Context(0, 1 << 24)
    t_base = torch.from_numpy(base).cuda()
    idx, rec, cnt = gs.gs_extract_delta(ctx, torch.from_numpy(th).cuda(), t_base, 1e-3)
    torch.cuda.synchronize()
    m = int(cnt.item())
    oi, orec, _ = O.delta(th, base, 1e-3)
    assert m == len(oi) > 0
    np.testing.assert_array_equal(rec.cpu().numpy()[:m], orec)
    # the client replays the oracle's records; the oracle replays the same
    client = torch.from_numpy(base).cuda()
    d_rec = torch.from_numpy(np.ascontiguousarray(orec)).cuda()
    d_cnt = torch.tensor([len(oi)], dtype=torch.int32, device="cuda")
    gs.gs_apply_delta(ctx, client, d_rec, d_cnt)
    torch.cuda.synchronize()
    assert ctx.status()[0] == 0
    np.testing.assert_array_equal(client.cpu().numpy(), O.apply_delta(base, orec))
    ctx.close()


def test_replay_rejects_out_of_range_index_without_writing():
    import torch
    import paper_2604_02851_b300 as gs
    n = 64
    ctx = gs.Context(0, 1 << 20)
    params = torch.zeros((15, n, 4), device="cuda")
    idx = torch.tensor([3, n + 5], dtype=torch.int32, device="cuda")
    vals = torch.zeros((2, 2), dtype=torch.uint8, device="cuda")
    vals[:, 1] = 0x3C  # float16 1.0
    cnt = torch.tensor([2], dtype=torch.int32, device="cuda")
    gs.gs_apply_tensor_delta(ctx, params, "opacity", idx, vals, cnt)
    torch.cuda.synchronize()
    code, detail = ctx.status()
    assert code == 1 and detail == n + 5
    p = params.cpu().numpy()
    assert p[0, 3, 3] == 1.0 and np.count_nonzero(p) == 1
    from paper_2604_02851_b300._lib import GsError
    with pytest.raises(GsError):
        gs.gs_extract_tensor_delta(ctx, params, params.clone(), 64, 1e-3)  # not one group
    ctx.close()


def test_scheduled_stream_keeps_the_client_close_to_the_server():
    """Server: a few optimisation steps; each step sends opacity and DC, every
    third step all groups.  Client: replays.  After a step that sent every
    group, every client float is within the threshold (plus the float16 step)
    of the server's; after the others, opacity and DC are."""
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import OnlineTrainer, estimate_keys
    n, sh = 20_000, 3
    cams = gi.ring_cameras(4, 128, 96)
    planes = gi.make_scene(n, sh, 70)
    params = torch.from_numpy(planes).cuda()
    ctx = gs.Context(0, 0)
    keys = estimate_keys(ctx, params, sh, cams, slack=2.0)
    tr = OnlineTrainer(params, sh, cams, keys, ctx=ctx, lr=3e-3)
    tgt = torch.from_numpy(gi.make_scene(n, sh, 71)).cuda()
    tctx = gs.Context(0, 0)
    tk = estimate_keys(tctx, tgt, sh, cams, slack=1.5)
    tctx.reserve(tctx.workspace_size(cams, n, tk))
    gs.gs_render_batch(tctx, tgt, sh, tr.d_cams, 4, tr.total_tiles, tk, tr.npix, image=tr.targets)
    client = params.clone()
    sent = params.clone()         # the server's per-group transmitted state
    dctx = gs.Context(0, 1 << 24)
    thr = 1e-3
    for k in range(6):
        tr.step()
        groups = ["opacity", "dc"] + (["mean", "scale", "rotation", "sh_rest"] if k % 3 == 2 else [])
        for name in groups:
            idx, vals, cnt = gs.gs_extract_tensor_delta(dctx, params, sent, name, thr)
            gs.gs_apply_tensor_delta(dctx, client, name, idx, vals, cnt)
        torch.cuda.synchronize()
        sr = gi.planes_to_rows(params.cpu().numpy())
        cr = gi.planes_to_rows(client.cpu().numpy())
        tol = thr + np.abs(sr) * 2.0 ** -11 + 1e-7
        check = [3, 12, 13, 14] if k % 3 != 2 else [c for c in range(60) if c != 7]
        assert np.all(np.abs(cr[:, check] - sr[:, check]) <= tol[:, check]), k
    assert dctx.status()[0] == 0
    tr.raise_status()
    for c in (ctx, tctx, dctx):
        c.close()
