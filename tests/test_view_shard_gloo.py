"""The view-sharded step's host logic on CPU: two gloo ranks (127.0.0.1).

Each rank takes its views (paper_2604_02851_b300.parallel.shard_views), the
oracle's gradient of its loss share (weights scaled by view_share) over them,
and the same reduction the GPU path uses (parallel.reduce_gradients, an
all-reduce sum).  The reduced gradient must be the oracle's gradient of the
mean loss over all views, the ranks' loss shares must sum to that loss, and
Adam on the reduced gradient must give both ranks the one-rank update."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import gs_inputs as gi


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


N, SH, V, W, H = 1500, 1, 4, 48, 40


def _inputs():
    import oracle as O
    cams = gi.ring_cameras(V, W, H)
    planes = gi.make_scene(N, SH, 21)
    target = O.forward(gi.make_scene(N, SH, 22), SH, cams)["image"]
    return planes, cams, target


def _view_slice(target, views):
    per = 3 * H * W
    return np.concatenate([target[v * per:(v + 1) * per] for v in views])


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    import oracle as O
    from paper_2604_02851_b300 import parallel
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        planes, cams, target = _inputs()
        views = parallel.shard_views(V, world, rank)
        share = parallel.view_share(V, world, rank)
        sub = parallel.subset_cameras(cams, views)
        r = O.loss_and_grad(planes, SH, sub, _view_slice(target, views), w_l1=0.8 * share, w_ssim=0.2 * share)
        g = torch.from_numpy(np.ascontiguousarray(r["dparams"]))
        parallel.reduce_gradients(g)
        loss = torch.tensor([r["loss"]], dtype=torch.float64)
        parallel.reduce_gradients(loss)
        # Adam on the reduced gradient, on every rank
        th = gi.planes_to_rows(planes).astype(np.float64)
        m = np.zeros_like(th)
        v = np.zeros_like(th)
        O.adam(th, gi.planes_to_rows(g.numpy()), m, v, 1e-3, 1)
        out[rank] = (views, g.numpy(), float(loss.item()), th)
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_to_the_full_view_gradient_and_update():
    import oracle as O
    from paper_2604_02851_b300 import parallel
    port = _free_port()
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    planes, cams, target = _inputs()
    full = O.loss_and_grad(planes, SH, cams, target)
    assert res[0][0] == [0, 2] and res[1][0] == [1, 3]
    g0, g1 = res[0][1], res[1][1]
    np.testing.assert_array_equal(g0, g1)
    ref = full["dparams"]
    assert np.linalg.norm(g0 - ref) <= 1e-12 * np.linalg.norm(ref)
    assert abs(res[0][2] - full["loss"]) <= 1e-12 * abs(full["loss"])
    th = gi.planes_to_rows(planes).astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    O.adam(th, gi.planes_to_rows(ref), m, v, 1e-3, 1)
    np.testing.assert_array_equal(res[0][3], res[1][3])
    assert np.max(np.abs(res[0][3] - th)) <= 1e-12
    assert parallel.view_share(V, world, 0) == 0.5


def test_shard_views_cover_every_view_once():
    from paper_2604_02851_b300 import parallel
    for V_, world in [(8, 1), (8, 2), (8, 3), (8, 8), (5, 4)]:
        got = sorted(v for r in range(world) for v in parallel.shard_views(V_, world, r))
        assert got == list(range(V_))
        assert abs(sum(parallel.view_share(V_, world, r) for r in range(world)) - 1.0) < 1e-12
    try:
        parallel.shard_views(4, 8, 0)
    except ValueError:
        pass
    else:
        raise AssertionError("more ranks than views must be refused")
