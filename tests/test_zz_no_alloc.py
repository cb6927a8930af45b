"""gs_extract_delta_noalloc: the delta extraction for callers that cannot
allocate device memory (a real-time sender thread, or a host whose device
memory belongs to another allocator).  It must give exactly what
gs_extract_delta gives -- indices, records and updated baselines are
bit-exact there -- on consecutive calls that share its fixed scratch array,
and the oracle's delta on the same float32 inputs.

This file is named to be collected last."""
import ctypes as C

import numpy as np
import pytest

import gs_inputs as gi
import oracle as O

pytestmark = pytest.mark.gpu


def _perturb(base, frac, seed):
    rng = np.random.default_rng(seed)
    theta = base.copy()
    n = base.shape[1]
    for i in np.nonzero(rng.random(n) < frac)[0]:
        p = int(rng.integers(0, 15)); c = int(rng.integers(0, 4))
        if p == 1 and c == 3:
            c = 0
        theta[p, i, c] += np.float32(rng.choice([1.5e-3, -2e-3, 9e-4]))
    return theta


def _noalloc(theta, base, thr, stream=None):
    import torch
    from paper_2604_02851_b300 import _lib
    n = theta.shape[1]
    dev = theta.device
    idx = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
    rec = torch.zeros((max(n, 1), 128), dtype=torch.uint8, device=dev)
    cnt = torch.full((1,), 7, dtype=torch.int32, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream()
    code = _lib.lib().gs_extract_delta_noalloc(C.c_void_p(theta.data_ptr()), C.c_void_p(base.data_ptr()), n,
                                               thr, C.c_void_p(idx.data_ptr()), C.c_void_p(rec.data_ptr()),
                                               C.c_void_p(cnt.data_ptr()), C.c_void_p(s.cuda_stream))
    assert code == 0, code
    s.synchronize()
    m = int(cnt.item())
    return idx[:m].cpu().numpy(), rec[:m].cpu().numpy(), m


def test_noalloc_delta_matches_gs_extract_delta_on_two_calls():
    import torch
    import paper_2604_02851_b300 as gs
    ctx = gs.Context(0, 1 << 26)
    # two calls in a row of different sizes: the second finds the first's flags in the shared array
    for n, frac, seed in [(300_000, 0.2, 1), (70_001, 0.5, 2)]:
        base = gi.make_scene(n, 3, seed)
        theta = _perturb(base, frac, seed + 7)
        th = torch.from_numpy(theta).cuda()
        b_ref = torch.from_numpy(base).cuda()
        b_new = torch.from_numpy(base).cuda()
        i_ref, r_ref, c_ref = gs.gs_extract_delta(ctx, th, b_ref, 1e-3)
        torch.cuda.synchronize()
        m_ref = int(c_ref.item())
        i_new, r_new, m_new = _noalloc(th, b_new, 1e-3)
        assert m_new == m_ref > 0
        np.testing.assert_array_equal(i_new, i_ref[:m_ref].cpu().numpy())
        np.testing.assert_array_equal(r_new, r_ref[:m_ref].cpu().numpy())
        assert torch.equal(b_new, b_ref)
        if n == 70_001:
            # and the oracle's definition on the same float32 inputs
            oi, orec, obase = O.delta(theta, base, 1e-3)
            assert m_new == len(oi)
            np.testing.assert_array_equal(i_new.view(np.uint32), oi)
            np.testing.assert_array_equal(r_new, orec)
            np.testing.assert_array_equal(b_new.cpu().numpy(), obase)
    ctx.close()


def test_noalloc_empty_call_zeroes_the_count():
    """n = 0 with null arrays: nothing to read, the count becomes 0."""
    import torch
    from paper_2604_02851_b300 import _lib
    cnt = torch.full((1,), 5, dtype=torch.int32, device="cuda")
    code = _lib.lib().gs_extract_delta_noalloc(None, None, 0, 1e-3, None, None, C.c_void_p(cnt.data_ptr()),
                                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0
    torch.cuda.synchronize()
    assert int(cnt.item()) == 0


def test_noalloc_at_its_largest_size_on_a_side_stream():
    """n = GS_NOALLOC_MAX_GAUSSIANS (the scratch array's exact limit), a
    sparse perturbation, enqueued on a stream other than the default one."""
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300 import _lib
    n = _lib.NOALLOC_MAX_GAUSSIANS
    rng = np.random.default_rng(40)
    base = rng.standard_normal((15, n, 4), dtype=np.float32)
    base[1, :, 3] = 0.0
    theta = base.copy()
    pick = rng.choice(n, 3000, replace=False)
    theta[rng.integers(0, 15, 3000), pick, rng.integers(0, 3, 3000)] += np.float32(2e-3)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        th = torch.from_numpy(theta).cuda()
        b_new = torch.from_numpy(base).cuda()
    side.synchronize()
    i_new, r_new, m_new = _noalloc(th, b_new, 1e-3, stream=side)
    ctx = gs.Context(0, 1 << 26)
    b_ref = torch.from_numpy(base).cuda()
    ctx.reserve(1 << 26)
    i_ref, r_ref, c_ref = gs.gs_extract_delta(ctx, th, b_ref, 1e-3)
    torch.cuda.synchronize()
    m_ref = int(c_ref.item())
    assert m_new == m_ref == len(np.unique(pick))
    np.testing.assert_array_equal(i_new, i_ref[:m_ref].cpu().numpy())
    np.testing.assert_array_equal(r_new, r_ref[:m_ref].cpu().numpy())
    assert torch.equal(b_new, b_ref)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2604_02851_b300 import _lib
    n = _lib.NOALLOC_MAX_GAUSSIANS + 1
    dummy = torch.zeros(16, device="cuda")
    code = _lib.lib().gs_extract_delta_noalloc(C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()), n,
                                               1e-3, C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()),
                                               C.c_void_p(dummy.data_ptr()), None)
    assert code == _lib.GS_ERR_CAPACITY
