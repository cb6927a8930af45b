"""StreamingTrainer: host uploads and read-backs overlapped with compute over
two graph slots must give the same steps as the one-slot loop."""
import numpy as np
import pytest

import gs_inputs as gi
from gpu_util import rel_l2, scene

pytestmark = pytest.mark.gpu


def test_streaming_matches_sequential_steps():
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import OnlineTrainer, StreamingTrainer, estimate_keys
    n, sh = 20_000, 1
    cams = gi.ring_cameras(4, 128, 96)
    planes = scene(n, sh, 21)
    # two target sets, alternating, rendered by the GPU forward from other scenes
    ctx = gs.Context(0, 0)
    targets = []
    for seed in (22, 23):
        tp = torch.from_numpy(scene(n, sh, seed)).cuda()
        d_cams = gs.cameras_to_device(cams)
        k = estimate_keys(ctx, tp, sh, cams, slack=1.3)
        ctx.reserve(ctx.workspace_size(cams, n, k))
        img = gs.gs_render_batch(ctx, tp, sh, d_cams, 4, ctx.total_tiles(cams), k, gs.total_pixels(cams))
        targets.append(img.cpu().pin_memory())
    keys = estimate_keys(ctx, torch.from_numpy(planes).cuda(), sh, cams, slack=2.0)
    steps = 6

    seq_params = torch.from_numpy(planes).cuda()
    seq = OnlineTrainer(seq_params, sh, cams, keys)
    seq_out = []
    for k in range(steps):
        seq.targets.copy_(targets[k % 2])
        seq.step()
        torch.cuda.synchronize()
        m = seq.delta_count()
        seq_out.append((seq.loss(), m, seq.d_records[:m].cpu().numpy().copy()))
    seq.raise_status()

    st_params = torch.from_numpy(planes).cuda()
    st = StreamingTrainer(st_params, sh, cams, keys, lambda: gs.Context(0, 0))
    got = []
    st.run(lambda k: targets[k % 2], steps, on_delta=lambda k, loss, m, rec: got.append((k, loss, m, rec.numpy().copy())))
    torch.cuda.synchronize()
    st.raise_status()

    assert [g[0] for g in got] == list(range(steps))
    for (k, loss, m, rec), (sl, sm, srec) in zip(got, seq_out):
        assert abs(loss - sl) <= 1e-5 * abs(sl), k
        # float atomics in the adjoint may order sums differently, so a
        # parameter within rounding of the 1e-3 delta threshold may flip
        assert abs(m - sm) <= max(2, 0.002 * sm), (k, m, sm)
        if m == sm:
            idx = rec[:, :4].view(np.uint32).ravel()
            sidx = srec[:, :4].view(np.uint32).ravel()
            assert np.mean(idx == sidx) > 0.99
    assert rel_l2(st_params.cpu().numpy(), seq_params.cpu().numpy()) <= 1e-5
    assert st.h2d_bytes == steps * targets[0].numel() * 4
    for t in st.slots:
        t.ctx.close()
    seq.ctx.close()
    ctx.close()
