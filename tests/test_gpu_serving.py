"""Continuous-batching render server: a request's image is the same rendered
alone, inside a mixed-resolution batch, and under continuous batching with
overlapping slots (bit-identical: the forward path has no atomics and each
view's lists and pixels are computed independently of the other views), and
a single render matches the FP64 oracle."""
import numpy as np
import pytest

import gs_inputs as gi
import oracle as O
from gpu_util import cams32, rel_l2

pytestmark = pytest.mark.gpu


def _requests(specs):
    from paper_2604_02851_b300 import pack_cameras
    from paper_2604_02851_b300.serve import Request
    out = []
    for i, sp in enumerate(specs):
        cams = gi.cameras_from_eyes([sp["eye"]], [sp["width"]], [sp["height"]])
        out.append(Request(rid=i, width=sp["width"], height=sp["height"], cam=pack_cameras(cams),
                           t_arrival=float(sp.get("t_arrival", 0.0))))
    return out, [gi.cameras_from_eyes([sp["eye"]], [sp["width"]], [sp["height"]]) for sp in specs]


@pytest.fixture(scope="module")
def server():
    import torch
    from paper_2604_02851_b300.serve import RenderServer, measure_keys_per_pixel
    n, sh = 150_000, 3
    params = torch.from_numpy(gi.make_scene(n, sh, gi.SEED_SERVING)).cuda()
    kpp = measure_keys_per_pixel(params, sh, gi.ring_cameras(2, 640, 360))
    srv = RenderServer(params, sh, kpp, slots=3, max_batch=4, max_pixels_per_batch=3_000_000,
                       memory_budget=8 << 30, slack=2.0, keep_images=True)
    return srv, params, n, sh


def test_alone_equals_batched_equals_continuous(server):
    srv, params, n, sh = server
    specs = gi.serving_requests(10, rate_hz=400.0, seed=11)
    for sp in specs:  # smaller resolutions keep the test quick
        sp["width"], sp["height"] = sp["width"] // 2, sp["height"] // 2
    alone = [srv.render_now([r])[0].image for r in _requests(specs)[0]]
    mixed = [r.image for r in sorted(srv.render_now(_requests(specs)[0][:4]), key=lambda r: r.rid)]
    for a, b in zip(alone[:4], mixed):
        np.testing.assert_array_equal(a, b)
    reqs, _ = _requests(specs)
    done, _ = srv.run(reqs, realtime=True)
    srv.check()
    assert len(done) == len(specs)
    for r in done:
        np.testing.assert_array_equal(r.image, alone[r.rid])


def test_batches_overlap_and_admit_while_busy(server):
    srv, params, n, sh = server
    specs = gi.serving_requests(24, rate_hz=2000.0, seed=12)
    for sp in specs:
        sp["width"], sp["height"] = sp["width"] // 2, sp["height"] // 2
    srv.launch_while_busy = 0
    srv.max_busy = 0
    reqs, _ = _requests(specs)
    done, elapsed = srv.run(reqs, realtime=True)
    srv.check()
    assert len(done) == 24
    assert srv.max_busy >= 2 and srv.launch_while_busy >= 1
    assert all(r.t_done >= r.t_arrival for r in done)
    # the image is complete on the device before it reaches host memory
    assert all(r.t_arrival <= r.t_rendered <= r.t_done for r in done)


def test_single_render_matches_oracle(server):
    srv, params, n, sh = server
    specs = [{"width": 160, "height": 120, "eye": (0.4, 0.3, 2.9)}]
    reqs, cams = _requests(specs)
    img = srv.render_now(reqs)[0].image
    f = O.forward(gi.make_scene(n, sh, gi.SEED_SERVING), sh, cams32(cams[0]))
    assert rel_l2(img.ravel(), f["image"]) <= 1e-4
