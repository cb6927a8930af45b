"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test checks the oracle against something other than itself: a library
routine of independent provenance (scipy spherical harmonics and rotations,
torch.optim.Adam, numpy float16), a closed form, a brute-force evaluation, an
invariant, or central finite differences.  A plausible slip in the oracle (a
dropped term, a wrong sign or index, a transposed operand) fails one of them.
"""
import math

import numpy as np
import pytest
import scipy.special as sp
from scipy.spatial.transform import Rotation

import gs_inputs as gi
import oracle as O

RNG = np.random.default_rng(1234)


def _real_sh_scipy(d):
    th = math.acos(max(-1.0, min(1.0, d[2])))
    ph = math.atan2(d[1], d[0])
    out = []
    for l in range(4):
        for m in range(-l, l + 1):
            if m == 0:
                out.append(sp.sph_harm_y(l, 0, th, ph).real)
            elif m > 0:
                out.append(math.sqrt(2) * sp.sph_harm_y(l, m, th, ph).real)
            else:
                out.append(math.sqrt(2) * sp.sph_harm_y(l, -m, th, ph).imag)
    return np.array(out)


# --------------------------------------------------------------- SH basis
def test_sh_basis_matches_scipy():
    for _ in range(50):
        d = RNG.normal(size=3); d /= np.linalg.norm(d)
        np.testing.assert_allclose(O.sh_basis(d), _real_sh_scipy(d), atol=1e-13, rtol=0)


def test_sh_basis_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6 exactly
    x, w = np.polynomial.legendre.leggauss(12)
    nphi = 16
    G = np.zeros((16, 16))
    for xi, wi in zip(x, w):
        s = math.sqrt(1 - xi * xi)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y = O.sh_basis(np.array([s * math.cos(ph), s * math.sin(ph), xi]))
            G += wi * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_basis_gradient_fd():
    for _ in range(10):
        d = RNG.normal(size=3)
        g = O.sh_basis_grad(d)
        h = 1e-6
        for i in range(3):
            e = np.zeros(3); e[i] = h
            fd = (O.sh_basis(d + e) - O.sh_basis(d - e)) / (2 * h)
            np.testing.assert_allclose(g[:, i], fd, atol=1e-8)


# --------------------------------------------------------------- projection
def _one_gaussian(mean, log_s, quat, logit, sh=None, sh_degree=0):
    planes = np.zeros((15, 1, 4), dtype=np.float64)
    planes[0, 0, :3] = mean; planes[0, 0, 3] = logit
    planes[1, 0, :3] = log_s
    planes[2, 0, :] = quat
    if sh is not None:
        flat = np.zeros(48); flat[:sh.size] = sh.ravel()
        planes[3:15, 0, :] = flat.reshape(12, 4)
    return planes


def _project_fn(cam, mean):
    R = np.asarray(cam["R"])[0]; t = np.asarray(cam["t"])[0]
    p = R @ mean + t
    return np.array([cam["fx"][0] * p[0] / p[2] + cam["cx"][0], cam["fy"][0] * p[1] / p[2] + cam["cy"][0]])


def test_projection_conic_from_fd_jacobian_and_scipy_rotation():
    cams = gi.cameras_from_eyes([(0.7, -0.4, 3.1)], [96], [80])
    for _ in range(20):
        mean = RNG.uniform(-0.4, 0.4, 3)
        log_s = RNG.normal(-2.5, 0.4, 3)
        q = RNG.normal(size=4)
        pl = _one_gaussian(mean, log_s, q, 0.3)
        pr = O.project(pl, 0, cams)[0, 0]
        assert pr[14] > pr[12]  # visible
        # Jacobian of the pinhole map by central differences (no J formula)
        M = np.zeros((2, 3))
        for i in range(3):
            e = np.zeros(3); e[i] = 1e-6
            M[:, i] = (_project_fn(cams, mean + e) - _project_fn(cams, mean - e)) / 2e-6
        Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy is (x, y, z, w)
        Sig = Rq @ np.diag(np.exp(2 * log_s)) @ Rq.T
        S2 = M @ Sig @ M.T + 0.3 * np.eye(2)
        inv = np.linalg.inv(S2)
        np.testing.assert_allclose([pr[4], pr[5], pr[6]], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=2e-6)
        np.testing.assert_allclose(pr[:2], _project_fn(cams, mean), rtol=1e-12)
        tz = (np.asarray(cams["R"])[0] @ mean + np.asarray(cams["t"])[0])[2]
        assert pr[2] == pytest.approx(tz, rel=1e-14)
        lam = np.linalg.eigvalsh(S2)
        mid = 0.5 * (S2[0, 0] + S2[1, 1])
        if mid * mid - np.linalg.det(S2) > 0.1:
            assert pr[7] == math.ceil(3 * math.sqrt(lam.max()))
        assert pr[3] == pytest.approx(1 / (1 + math.exp(-0.3)), rel=1e-14)


def test_projection_sh_colour_matches_scipy_basis():
    cams = gi.ring_cameras(3, 64, 64)
    sh = RNG.normal(0, 0.3, size=(16, 3))
    mean = np.array([0.1, -0.2, 0.15])
    pl = _one_gaussian(mean, [-2.0] * 3, [1, 0, 0, 0], 0.0, sh)
    pr = O.project(pl, 3, cams)
    for v in range(3):
        R = cams["R"][v]; t = cams["t"][v]
        centre = -R.T @ t
        d = mean - centre; d /= np.linalg.norm(d)
        rgb = _real_sh_scipy(d) @ sh + 0.5
        expect = np.maximum(rgb, 0.0)
        np.testing.assert_allclose(pr[v, 0, 8:11], expect, atol=1e-12)
        mask = sum(1 << c for c in range(3) if rgb[c] < 0)
        assert pr[v, 0, 11] == mask


def test_sh_degree0_colour_is_view_independent():
    cams = gi.ring_cameras(6, 64, 64)
    dc = np.array([[0.3, -0.7, 1.1]])
    pl = _one_gaussian([0.05, 0.0, -0.1], [-2.0] * 3, [1, 0, 0, 0], 0.0, dc)
    pr = O.project(pl, 0, cams)
    y00 = 0.5 / math.sqrt(math.pi)
    for v in range(6):
        np.testing.assert_allclose(pr[v, 0, 8:11], dc[0] * y00 + 0.5, atol=1e-14)


def test_projection_culls_behind_near_plane():
    cams = gi.cameras_from_eyes([(0, 0, 3.0)], [32], [32])
    # camera at z = 3 looking at -z: a point at z = 2.85 is 0.15 in front (< near 0.2)
    pl = _one_gaussian([0, 0, 2.85], [-2.0] * 3, [1, 0, 0, 0], 0.0)
    assert np.all(O.project(pl, 0, cams) == 0)
    pl = _one_gaussian([0, 0, 3.5], [-2.0] * 3, [1, 0, 0, 0], 0.0)  # behind the camera
    assert np.all(O.project(pl, 0, cams) == 0)


# --------------------------------------------------------------- compositing
def _iso_sigma2(cams, s, z):
    f = cams["fx"][0]
    return (f * s / z) ** 2 + 0.3


def test_single_gaussian_closed_form():
    """An isotropic Gaussian on the optical axis at depth z renders as
    rgb * min(0.99, o exp(-rho^2 / (2 sigma^2))) with sigma^2 = (f s / z)^2 + 0.3,
    or 0 where that alpha is below 1/255."""
    W = H = 32
    cams = gi.cameras_from_eyes([(0, 0, 3.0)], [W], [H])
    for log_s, logit in [(-3.0, 0.5), (-2.2, 2.0), (-3.5, -1.0), (-2.6, 5.0)]:
        s = math.exp(log_s)
        dc = np.array([[0.4, 0.1, -0.2]])
        pl = _one_gaussian([0, 0, 0], [log_s] * 3, [1, 0, 0, 0], logit, dc)
        f = O.forward(pl, 0, cams)
        sig2 = _iso_sigma2(cams, s, 3.0)
        o = 1 / (1 + math.exp(-logit))
        rgb = dc[0] * (0.5 / math.sqrt(math.pi)) + 0.5
        ys, xs = np.mgrid[0:H, 0:W]
        rho2 = (xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - H / 2) ** 2
        a = np.minimum(0.99, o * np.exp(-rho2 / (2 * sig2)))
        a[a < 1 / 255] = 0.0
        # the square support of half-side ceil(3 sqrt(lambda)) is wider than the image here
        assert f["proj"][0, 0, 7] >= 3 * math.sqrt(sig2)
        assert (f["proj"][0, 0, 12:16] == [0, 0, 2, 2]).all()
        img = f["image"].reshape(3, H, W)
        for c in range(3):
            np.testing.assert_allclose(img[c], rgb[c] * a, atol=1e-14)
        np.testing.assert_allclose(f["T_final"].reshape(H, W), 1 - a, atol=1e-14)


def test_two_gaussians_closed_form_and_order():
    W = H = 32
    cams = gi.cameras_from_eyes([(0, 0, 3.0)], [W], [H])
    y00 = 0.5 / math.sqrt(math.pi)
    c1 = np.array([0.9, 0.2, 0.1]); c2 = np.array([0.1, 0.3, 0.8])
    for z1, z2 in [(0.3, -0.3), (-0.3, 0.3)]:
        pl = np.concatenate([
            _one_gaussian([0, 0, z1], [-2.8] * 3, [1, 0, 0, 0], 0.4, ((c1 - 0.5) / y00)[None]),
            _one_gaussian([0, 0, z2], [-2.6] * 3, [1, 0, 0, 0], 1.0, ((c2 - 0.5) / y00)[None])], axis=1)
        f = O.forward(pl, 0, cams)
        ys, xs = np.mgrid[0:H, 0:W]
        rho2 = (xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - H / 2) ** 2
        alphas = []
        for z, ls, lg in [(z1, -2.8, 0.4), (z2, -2.6, 1.0)]:
            sig2 = _iso_sigma2(cams, math.exp(ls), 3.0 - z)
            a = np.minimum(0.99, np.exp(-rho2 / (2 * sig2)) / (1 + math.exp(-lg)))
            a[a < 1 / 255] = 0
            alphas.append(a)
        a1, a2 = alphas
        front_first = z1 > z2  # the camera sits at +z: larger z is nearer
        if front_first:
            expect = c1[:, None, None] * a1 + c2[:, None, None] * a2 * (1 - a1)
        else:
            expect = c2[:, None, None] * a2 + c1[:, None, None] * a1 * (1 - a2)
        np.testing.assert_allclose(f["image"].reshape(3, H, W), expect, atol=1e-14)


def _brute_force_render(cams, proj, tile=16, bg=(0, 0, 0)):
    """Per pixel: every Gaussian whose tile rectangle holds the pixel's tile,
    fully sorted by (float32 depth, index), composited front to back."""
    V, n = proj.shape[:2]
    outs = []
    for v in range(V):
        W, H = int(cams["width"][v]), int(cams["height"][v])
        img = np.zeros((3, H, W)); Tm = np.zeros((H, W))
        for y in range(H):
            for x in range(W):
                tx, ty = x // tile, y // tile
                cand = [g for g in range(n)
                        if proj[v, g, 12] <= tx < proj[v, g, 14] and proj[v, g, 13] <= ty < proj[v, g, 15]]
                cand.sort(key=lambda g: (np.float32(proj[v, g, 2]), g))
                T = 1.0; C = np.zeros(3)
                for g in cand:
                    o = proj[v, g]
                    dx, dy = o[0] - (x + 0.5), o[1] - (y + 0.5)
                    P = -0.5 * (o[4] * dx * dx + o[6] * dy * dy) - o[5] * dx * dy
                    if P > 0:
                        continue
                    a = min(0.99, o[3] * math.exp(P))
                    if a < 1 / 255:
                        continue
                    Tn = T * (1 - a)
                    if Tn < 1e-4:
                        break
                    C += o[8:11] * a * T
                    T = Tn
                img[:, y, x] = C + T * np.asarray(bg)
                Tm[y, x] = T
        outs.append((img, Tm))
    return outs


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiled_render_equals_brute_force_full_sort(seed):
    n = 48
    sc = gi.make_scene(n, 1, seed)
    sc[1, :, :3] += 1.5  # larger Gaussians so that lists overlap heavily
    cams = gi.ring_cameras(2, 32, 24)
    f = O.forward(sc, 1, cams, bg=(0.1, 0.2, 0.3))
    bf = _brute_force_render(cams, f["proj"], bg=(0.1, 0.2, 0.3))
    off = 0
    for v, (img, Tm) in enumerate(bf):
        P = img.shape[1] * img.shape[2]
        np.testing.assert_allclose(f["image"][3 * off:3 * (off + P)].reshape(img.shape), img, atol=1e-13)
        np.testing.assert_allclose(f["T_final"][off:off + P].reshape(Tm.shape), Tm, atol=1e-13)
        off += P


def test_bin_sort_matches_lexsort():
    V, n = 3, 400
    cams = gi.ring_cameras(V, 70, 50)
    rects = np.zeros((V, n, 4), dtype=np.int32)
    TX, TY = 5, 4
    x0 = RNG.integers(0, TX, (V, n)); y0 = RNG.integers(0, TY, (V, n))
    rects[..., 0] = x0; rects[..., 1] = y0
    rects[..., 2] = np.minimum(TX, x0 + RNG.integers(0, 3, (V, n)))
    rects[..., 3] = np.minimum(TY, y0 + RNG.integers(0, 3, (V, n)))
    depth = RNG.uniform(0.5, 5, (V, n)).astype(np.float32)
    depth[0, :50] = depth[0, 50:100]  # equal depths: ties broken by index
    keys, vals, ranges = O.bin_sort(cams, rects, depth)
    tl, dl, gl = [], [], []
    for v in range(V):
        for g in range(n):
            r = rects[v, g]
            for ty in range(r[1], r[3]):
                for tx in range(r[0], r[2]):
                    tl.append(v * TX * TY + ty * TX + tx)
                    dl.append(depth[v, g].view(np.uint32)); gl.append(g)
    tl, dl, gl = map(np.array, (tl, dl, gl))
    order = np.lexsort((gl, dl, tl))
    np.testing.assert_array_equal(vals, gl[order])
    np.testing.assert_array_equal(keys >> np.uint64(32), tl[order])
    for t in range(V * TX * TY):
        sel = np.nonzero(tl[order] == t)[0]
        if sel.size:
            assert tuple(ranges[t]) == (sel[0], sel[-1] + 1)
        else:
            assert ranges[t, 0] == ranges[t, 1]


def test_bin_ranges_and_tile_lists_match_numpy():
    """The ranges of every tile (without forming the entries) and the
    sorted lists of chosen tiles, against a numpy count per tile and a
    lexsort of each chosen tile's (depth bits, index) pairs, on ragged views
    of different sizes with equal depths."""
    cams = gi.cameras_from_eyes([(0, 0, 3), (3, 0, 0), (0, 0, -3)], [70, 33, 48], [50, 47, 16])
    TX = [(int(w) + 15) // 16 for w in cams["width"]]
    TY = [(int(h) + 15) // 16 for h in cams["height"]]
    V, n = 3, 500
    rects = np.zeros((V, n, 4), dtype=np.int32)
    for v in range(V):
        x0 = RNG.integers(0, TX[v], n); y0 = RNG.integers(0, TY[v], n)
        rects[v, :, 0] = x0; rects[v, :, 1] = y0
        rects[v, :, 2] = np.minimum(TX[v], x0 + RNG.integers(0, 3, n))
        rects[v, :, 3] = np.minimum(TY[v], y0 + RNG.integers(0, 3, n))
    depth = RNG.uniform(0.5, 5, (V, n)).astype(np.float32)
    depth[1, :80] = depth[1, 80:160]  # equal depths: ties broken by index
    off = np.concatenate([[0], np.cumsum([a * b for a, b in zip(TX, TY)])])
    count = np.zeros(off[-1], dtype=np.int64)
    members = [[] for _ in range(off[-1])]
    for v in range(V):
        for g in range(n):
            r = rects[v, g]
            for ty in range(r[1], r[3]):
                for tx in range(r[0], r[2]):
                    t = off[v] + ty * TX[v] + tx
                    count[t] += 1
                    members[t].append(g)
    ranges, K = O.bin_ranges(cams, rects)
    assert K == count.sum()
    start = np.concatenate([[0], np.cumsum(count)])[:-1]
    np.testing.assert_array_equal(ranges[:, 0], np.where(count > 0, start, 0))
    np.testing.assert_array_equal(ranges[:, 1], np.where(count > 0, start + count, 0))
    pick = np.array([0, 5, off[1], off[1] + 3, off[2] - 1, off[2], off[3] - 1, 7], dtype=np.int64)
    vals, st = O.bin_tiles(cams, rects, depth, pick)
    for i, t in enumerate(pick):
        v = int(np.searchsorted(off, t, side="right") - 1)
        g = np.array(members[t], dtype=np.int64)
        order = np.lexsort((g, depth[v, g].view(np.uint32))) if g.size else g
        np.testing.assert_array_equal(vals[st[i]:st[i + 1]], g[order])
    assert st[-1] == sum(len(members[t]) for t in pick)


def test_render_invariants():
    sc = gi.make_scene(3000, 2, 5)
    cams = gi.ring_cameras(2, 48, 40)
    f = O.forward(sc, 2, cams)
    T = f["T_final"]
    assert T.min() >= 1e-4 and T.max() <= 1.0
    rgbmax = f["proj"][..., 8:11].max()
    assert f["image"].min() >= 0 and f["image"].max() <= rgbmax + 1e-12
    # transmittance is non-increasing along each pixel's list: re-walk one tile
    vals, ranges, proj = f["vals"], f["ranges"], f["proj"]
    s, e = ranges[1]
    for x in range(16, 20):
        Tp = 1.0
        for j in range(s, e):
            o = proj[0, vals[j]]
            dx, dy = o[0] - (x + 0.5), o[1] - 0.5
            P = -0.5 * (o[4] * dx * dx + o[6] * dy * dy) - o[5] * dx * dy
            a = min(0.99, o[3] * math.exp(P)) if P <= 0 else 0.0
            if a >= 1 / 255:
                if Tp * (1 - a) < 1e-4:
                    break
                assert Tp * (1 - a) <= Tp
                Tp *= 1 - a
        assert Tp == pytest.approx(T[x], rel=1e-12)


# --------------------------------------------------------------- loss
def test_ssim_identity_and_zero_gradient():
    x = RNG.uniform(0, 1, size=(2, 3, 20, 24))
    L, g = O.loss(x.ravel(), x.ravel(), 2, 20, 24)
    assert L == pytest.approx(0.0, abs=1e-14)
    assert np.abs(g).max() < 1e-15
    s = O.ssim_map(x[0, 0], x[0, 0])
    np.testing.assert_allclose(s, 1.0, atol=1e-14)


def test_ssim_constant_images_closed_form():
    H, W = 30, 30
    for a, b in [(0.2, 0.7), (0.5, 0.5), (0.9, 0.05)]:
        s = O.ssim_map(np.full((H, W), a), np.full((H, W), b))
        c1 = 0.01 ** 2
        # interior pixels see the whole window: sigma terms vanish
        np.testing.assert_allclose(s[5:-5, 5:-5], (2 * a * b + c1) / (a * a + b * b + c1), rtol=1e-10)


def test_ssim_map_against_scipy_filtering():
    from scipy.ndimage import correlate
    x = RNG.uniform(0, 1, (25, 31)); y = np.clip(x + RNG.normal(0, 0.1, x.shape), 0, 1)
    g = np.exp(-((np.arange(11) - 5) ** 2) / (2 * 1.5 ** 2)); g /= g.sum()
    w = np.outer(g, g)
    f = lambda z: correlate(z, w, mode="constant", cval=0.0)
    mx, my = f(x), f(y)
    sxx, syy, sxy = f(x * x) - mx ** 2, f(y * y) - my ** 2, f(x * y) - mx * my
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    ref = (2 * mx * my + c1) * (2 * sxy + c2) / ((mx ** 2 + my ** 2 + c1) * (sxx + syy + c2))
    np.testing.assert_allclose(O.ssim_map(x, y), ref, atol=1e-13)


def test_loss_gradient_fd():
    V, H, W = 2, 14, 17
    x = RNG.uniform(0, 1, V * 3 * H * W); y = RNG.uniform(0, 1, x.size)
    L, g = O.loss(x, y, V, H, W, 0.8, 0.2)
    l1 = np.abs(x - y).mean(); assert L > 0.8 * l1
    for i in RNG.choice(x.size, 40, replace=False):
        h = 1e-7
        xp = x.copy(); xp[i] += h
        xm = x.copy(); xm[i] -= h
        fd = (O.loss(xp, y, V, H, W, 0.8, 0.2)[0] - O.loss(xm, y, V, H, W, 0.8, 0.2)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-11)


# --------------------------------------------------------------- gradients
def _discrete_state(planes, sh, cams):
    f = O.forward(planes, sh, cams)
    p = f["proj"]
    return (p[..., 12:16].copy(), p[..., 11].copy(), f["n_contrib"].copy())


def _same_state(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("sh_degree,seed", [(0, 0), (3, 1)])
def test_full_gradient_matches_central_differences(sh_degree, seed):
    """Analytic adjoint of render + loss vs central differences on 64 seeded
    parameters; a parameter whose +-h step changes any discrete state
    (tile rectangles, clamp flags, contributor counts) or shows a kink is
    resampled."""
    n = 60
    sc = gi.make_scene(n, sh_degree, seed).astype(np.float64)
    sc[1, :, :3] += 1.2
    sc[0, :, :3] *= 0.6
    cams = gi.ring_cameras(2, 40, 32)
    tgt_sc = gi.make_scene(n, sh_degree, seed + 10).astype(np.float64)
    tgt_sc[1, :, :3] += 1.2
    tgt_sc[0, :, :3] *= 0.6
    target = O.forward(tgt_sc, sh_degree, cams)["image"]
    r = O.loss_and_grad(sc, sh_degree, cams, target)
    g = r["dparams"]
    base_state = _discrete_state(sc, sh_degree, cams)
    nb = (sh_degree + 1) ** 2
    valid = [(p, i, c) for p in range(15) for i in range(n) for c in range(4)
             if not (p == 1 and c == 3) and not (p >= 3 and (4 * (p - 3) + c) >= 3 * nb)]
    rng = np.random.default_rng(seed + 99)
    checked, tries = 0, 0
    rel_errs = []
    while checked < 64 and tries < 400:
        tries += 1
        p, i, c = valid[rng.integers(len(valid))]
        if np.all(r["proj"][:, i, 14] == 0):
            continue  # never on screen: gradient is zero, nothing to check
        th = sc[p, i, c]
        h = 1e-6 * max(1.0, abs(th))
        sp_ = sc.copy(); sp_[p, i, c] = th + h
        sm_ = sc.copy(); sm_[p, i, c] = th - h
        if not (_same_state(_discrete_state(sp_, sh_degree, cams), base_state)
                and _same_state(_discrete_state(sm_, sh_degree, cams), base_state)):
            continue
        Lp = O.render_loss(sp_, sh_degree, cams, target)
        Lm = O.render_loss(sm_, sh_degree, cams, target)
        L0 = r["loss"]
        fwd, bwd = (Lp - L0) / h, (L0 - Lm) / h
        if abs(fwd - bwd) > 1e-3 * max(abs(fwd), abs(bwd), 1e-8):
            continue  # a skip threshold was crossed inside the step
        fd = (Lp - Lm) / (2 * h)
        an = g[p, i, c]
        # central differences carry a rounding error of about eps * |L| / h
        fd_noise = 100 * np.finfo(float).eps * abs(L0) / h
        rel_errs.append(max(abs(fd - an) - fd_noise, 0.0) / max(abs(fd), abs(an), 1e-12))
        checked += 1
    assert checked >= 48
    assert max(rel_errs) <= 1e-5, sorted(rel_errs)[-5:]


def test_render_bwd_matches_fd_in_screen_space():
    """Adjoint of compositing alone, w.r.t. the 2D quantities (u, v, A, B, C,
    opacity, rgb), against central differences through the oracle render."""
    sc = gi.make_scene(40, 0, 3)
    sc[1, :, :3] += 1.3
    cams = gi.ring_cameras(1, 32, 32)
    f = O.forward(sc, 0, cams)
    proj = f["proj"].copy()
    wimg = RNG.normal(size=f["image"].size)
    L = lambda pr: float(wimg @ O.render(cams, pr, f["vals"], f["ranges"])[0])
    g2 = O.render_bwd(cams, proj, f["vals"], f["ranges"], wimg)
    fields = [0, 1, 4, 5, 6, 3, 8, 9, 10]
    checked = 0
    for g in RNG.permutation(40):
        if proj[0, g, 14] == 0:
            continue
        for k, fld in enumerate(fields):
            h = 1e-7 * max(1.0, abs(proj[0, g, fld]))
            pp = proj.copy(); pp[0, g, fld] += h
            pm = proj.copy(); pm[0, g, fld] -= h
            if not np.array_equal(O.render(cams, pp, f["vals"], f["ranges"])[2], f["n_contrib"]) or \
               not np.array_equal(O.render(cams, pm, f["vals"], f["ranges"])[2], f["n_contrib"]):
                continue
            fd = (L(pp) - L(pm)) / (2 * h)
            assert fd == pytest.approx(g2[0, g, k], rel=2e-5, abs=1e-7), (g, fld)
            checked += 1
    assert checked > 100


# --------------------------------------------------------------- Adam, FP16, delta
def test_adam_equals_torch_adam_float64():
    import torch
    n = 257
    theta0 = RNG.normal(size=n)
    lr = 10 ** RNG.uniform(-4, -2, size=n)
    th = theta0.copy(); m = np.zeros(n); v = np.zeros(n)
    params = [torch.nn.Parameter(torch.tensor(theta0[i:i + 1], dtype=torch.float64)) for i in range(n)]
    opt = torch.optim.Adam([{"params": [p], "lr": float(lr[i])} for i, p in enumerate(params)],
                           betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 6):
        g = RNG.normal(size=n) * 10 ** RNG.uniform(-6, 0, size=n)
        O.adam(th, g, m, v, lr, step)
        for i, p in enumerate(params):
            p.grad = torch.tensor(g[i:i + 1], dtype=torch.float64)
        opt.step()
        ref = np.array([p.item() for p in params])
        np.testing.assert_allclose(th, ref, rtol=1e-12, atol=1e-15)


def test_f16_matches_numpy():
    vals = np.concatenate([
        RNG.normal(0, 1, 2000), RNG.normal(0, 1e-5, 500), RNG.normal(0, 3e4, 500),
        [0.0, -0.0, 65504.0, 65519.99, 65520.0, -70000.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26,
         2.0 ** -14, (1 + 2 ** -11) * 1.0, (1 + 3 * 2 ** -11), 6.1e-5, 1e-8]]).astype(np.float32)
    np.testing.assert_array_equal(O.f32_to_f16_bits(vals), vals.astype(np.float16).view(np.uint16))


def test_delta_against_numpy_definition():
    n = 500
    th = gi.make_scene(n, 3, 7)
    base = th.copy()
    rng = np.random.default_rng(3)
    pick = rng.random(n) < 0.3
    plane = rng.integers(0, 15, n); lane = rng.integers(0, 4, n)
    lane[(plane == 1) & (lane == 3)] = 0
    for i in np.nonzero(pick)[0]:
        th[plane[i], i, lane[i]] += np.float32(rng.choice([2e-3, -5e-3, 9e-4]))
    idx, rec, nb = O.delta(th, base, 1e-3)
    rows_t = gi.planes_to_rows(th).astype(np.float32)
    rows_b = gi.planes_to_rows(base).astype(np.float32)
    expect = np.nonzero((np.abs(rows_t - rows_b) > np.float32(1e-3)).any(axis=1))[0]
    np.testing.assert_array_equal(idx, expect)
    order = [4, 5, 6, 8, 9, 10, 11, 3] + list(range(12, 60))
    for k, g in enumerate(expect):
        r = rec[k]
        assert r[:4].view(np.uint32)[0] == g
        np.testing.assert_array_equal(r[4:16].view(np.float32), rows_t[g, :3])
        np.testing.assert_array_equal(r[16:128].view(np.float16), rows_t[g, order].astype(np.float16))
    nbr = gi.planes_to_rows(nb)
    np.testing.assert_array_equal(nbr[expect], rows_t[expect])
    keep = np.setdiff1d(np.arange(n), expect)
    np.testing.assert_array_equal(nbr[keep], rows_b[keep])


GROUP_FLOATS = {"mean": (0, 3), "opacity": (3, 4), "scale": (4, 7), "rotation": (8, 12), "dc": (12, 15),
                "sh_rest": (15, 60)}


def test_f16_decode_matches_numpy_for_every_bit_pattern():
    bits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    ref = bits.view(np.float16).astype(np.float32)
    got = O.f16_bits_to_f32(bits)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    np.testing.assert_array_equal(got[~nan].view(np.uint32), ref[~nan].view(np.uint32))


def _perturbed(n, seed, groups_hit):
    th = gi.make_scene(n, 3, seed)
    base = th.copy()
    rows = gi.planes_to_rows(th).astype(np.float32)
    rng = np.random.default_rng(seed)
    hit = {}
    for name, (lo, hi) in GROUP_FLOATS.items():
        pick = np.nonzero(rng.random(n) < groups_hit)[0]
        col = rng.integers(lo, hi, len(pick))
        rows[pick, col] += rng.choice([2e-3, -5e-3, 9e-4], len(pick)).astype(np.float32)
        hit[name] = pick
    return gi.rows_to_planes(rows), base, hit


@pytest.mark.parametrize("name", list(GROUP_FLOATS))
def test_tensor_delta_against_numpy_definition(name):
    n = 800
    th, base, _ = _perturbed(n, 31, 0.2)
    attr = O.ATTR_GROUPS[name]
    lo, hi = GROUP_FLOATS[name]
    idx, vals, nb = O.tensor_delta(th, base, attr, 1e-3)
    rt = gi.planes_to_rows(th).astype(np.float32)
    rb = gi.planes_to_rows(base).astype(np.float32)
    expect = np.nonzero((np.abs(rt[:, lo:hi] - rb[:, lo:hi]) > np.float32(1e-3)).any(axis=1))[0]
    np.testing.assert_array_equal(idx, expect)
    assert vals.shape[1] == (hi - lo) * (4 if name == "mean" else 2)
    if name == "mean":
        np.testing.assert_array_equal(vals.view(np.float32).reshape(-1, 3), rt[expect, lo:hi])
    else:
        np.testing.assert_array_equal(vals.view(np.float16).reshape(-1, hi - lo), rt[expect, lo:hi].astype(np.float16))
    nbr = gi.planes_to_rows(nb)
    # only the group's floats of the sent Gaussians move to theta
    want = rb.copy()
    want[np.ix_(expect, np.arange(lo, hi))] = rt[np.ix_(expect, np.arange(lo, hi))]
    np.testing.assert_array_equal(nbr, want)


def test_tensor_deltas_replay_on_the_client():
    """Client replay of every group's delta reproduces the server's values
    within the record encoding (float32 mean, float16 others); Gaussians that
    were not sent keep the client's values."""
    n = 600
    th, base, _ = _perturbed(n, 37, 0.3)
    client = base.copy()
    rt = gi.planes_to_rows(th).astype(np.float32)
    for name, attr in O.ATTR_GROUPS.items():
        idx, vals, base = O.tensor_delta(th, base, attr, 1e-3)
        client = O.apply_tensor_delta(client, attr, idx, vals)
        lo, hi = GROUP_FLOATS[name]
        cr = gi.planes_to_rows(client)
        enc = rt[idx, lo:hi] if name == "mean" else rt[idx, lo:hi].astype(np.float16).astype(np.float32)
        np.testing.assert_array_equal(cr[idx, lo:hi], enc)
    # every float of the client is within the threshold or the float16 step of the server
    cr = gi.planes_to_rows(client)
    err = np.abs(cr - rt)
    tol = np.float32(1e-3) + np.abs(rt) * np.float32(2.0 ** -11)
    assert np.all(err[:, :7] <= tol[:, :7]) and np.all(err[:, 8:] <= tol[:, 8:])


def test_full_record_replay_matches_record_fields():
    n = 400
    th, base, _ = _perturbed(n, 41, 0.25)
    idx, rec, _ = O.delta(th, base, 1e-3)
    client = O.apply_delta(base.copy(), rec)
    rt = gi.planes_to_rows(th).astype(np.float32)
    rb = gi.planes_to_rows(base).astype(np.float32)
    cr = gi.planes_to_rows(client)
    np.testing.assert_array_equal(cr[idx, :3], rt[idx, :3])
    cols = [3, 4, 5, 6] + list(range(8, 60))
    np.testing.assert_array_equal(cr[np.ix_(idx, cols)], rt[np.ix_(idx, cols)].astype(np.float16).astype(np.float32))
    keep = np.setdiff1d(np.arange(n), idx)
    np.testing.assert_array_equal(cr[keep], rb[keep])
    np.testing.assert_array_equal(cr[:, 7], rb[:, 7])


# --------------------------------------------------------------- dynamics (Sec. 3.4)
def _dyn(n, G, seed, normals=True, light=(0.3, 0.8, 0.52)):
    rng = np.random.default_rng(seed)
    poses = np.zeros((G, 8))
    q = rng.normal(size=(G, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    poses[:, :4] = q
    poses[:, 4:7] = rng.uniform(-0.2, 0.2, (G, 3))
    l = np.asarray(light, dtype=float); l /= np.linalg.norm(l)
    d = {"group": np.arange(n) % G, "poses": poses, "light": l, "ambient": 0.3, "diffuse": 0.7}
    if normals:
        nn = rng.normal(size=(n, 3)); d["normals"] = nn / np.linalg.norm(nn, axis=1, keepdims=True)
    return d


def test_dynamics_identity_pose_is_static():
    sc = gi.make_scene(300, 2, 21)
    cams = gi.ring_cameras(2, 64, 48)
    d = {"group": np.zeros(300, dtype=np.int32), "poses": np.array([[1, 0, 0, 0, 0, 0, 0, 0.0]])}
    np.testing.assert_array_equal(O.project(sc, 2, cams, dyn=d), O.project(sc, 2, cams))


def test_rigid_motion_equals_inverse_camera_motion():
    """Moving every Gaussian by (R_g, t_g) renders what the camera moved by the
    inverse motion sees: W' = W R_g, t' = W t_g + t (scipy builds R_g)."""
    sc = gi.make_scene(500, 1, 22)
    sc[1, :, :3] += 0.8
    cams = gi.ring_cameras(2, 64, 48)
    q = np.array([0.9, 0.2, -0.3, 0.25]); q /= np.linalg.norm(q)
    t = np.array([0.05, -0.1, 0.08])
    d = {"group": np.zeros(500, dtype=np.int32), "poses": np.array([[*q, *t, 0.0]])}
    Rg = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    cams2 = dict(cams)
    cams2["R"] = np.array([R @ Rg for R in cams["R"]])
    cams2["t"] = np.array([R @ t + tc for R, tc in zip(cams["R"], cams["t"])])
    a = O.forward(sc, 1, cams, dyn=d)["image"]
    b = O.forward(sc, 1, cams2)["image"]
    np.testing.assert_allclose(a, b, atol=1e-10)


def test_relight_factor_closed_form():
    n = 64
    sc = gi.make_scene(n, 0, 23)
    cams = gi.ring_cameras(1, 64, 64)
    d = _dyn(n, 4, 5)
    pr = O.project(sc, 0, cams, dyn=d)
    y00 = 0.5 / math.sqrt(math.pi)
    rows = gi.planes_to_rows(sc).astype(np.float64)
    for g in range(n):
        if pr[0, g, 14] == pr[0, g, 12]:
            continue
        q = d["poses"][d["group"][g], :4]
        Rg = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        L = 0.3 + 0.7 * max(0.0, float((Rg @ d["normals"][g]) @ d["light"]))
        expect = np.maximum(L * rows[g, 12:15] * y00 + 0.5, 0.0)
        np.testing.assert_allclose(pr[0, g, 8:11], expect, atol=1e-12)


def test_dynamic_gradient_matches_central_differences():
    n = 50
    sc = gi.make_scene(n, 1, 24).astype(np.float64)
    sc[1, :, :3] += 1.2
    sc[0, :, :3] *= 0.6
    cams = gi.ring_cameras(2, 40, 32)
    d = _dyn(n, 3, 6)
    tgt = gi.make_scene(n, 1, 25).astype(np.float64)
    tgt[1, :, :3] += 1.2
    tgt[0, :, :3] *= 0.6
    target = O.forward(tgt, 1, cams, dyn=d)["image"]
    r = O.loss_and_grad(sc, 1, cams, target, dyn=d)
    g = r["dparams"]
    rng = np.random.default_rng(77)
    errs, checked, tries = [], 0, 0
    while checked < 40 and tries < 400:
        tries += 1
        p, i, c = int(rng.integers(0, 4)), int(rng.integers(0, n)), int(rng.integers(0, 4))
        if (p == 1 and c == 3) or np.all(r["proj"][:, i, 14] == 0):
            continue
        th = sc[p, i, c]
        h = 1e-6 * max(1.0, abs(th))
        sp_ = sc.copy(); sp_[p, i, c] = th + h
        sm_ = sc.copy(); sm_[p, i, c] = th - h
        fp, fm = O.forward(sp_, 1, cams, dyn=d), O.forward(sm_, 1, cams, dyn=d)
        if not (np.array_equal(fp["n_contrib"], r["n_contrib"]) and np.array_equal(fm["n_contrib"], r["n_contrib"])
                and np.array_equal(fp["proj"][..., 12:16], r["proj"][..., 12:16])
                and np.array_equal(fm["proj"][..., 12:16], r["proj"][..., 12:16])):
            continue
        Lp = O.loss(fp["image"], target, 2, 32, 40)[0]
        Lm = O.loss(fm["image"], target, 2, 32, 40)[0]
        fwd, bwd = (Lp - r["loss"]) / h, (r["loss"] - Lm) / h
        if abs(fwd - bwd) > 1e-3 * max(abs(fwd), abs(bwd), 1e-8):
            continue
        fd = (Lp - Lm) / (2 * h)
        noise = 100 * np.finfo(float).eps * abs(r["loss"]) / h
        errs.append(max(abs(fd - g[p, i, c]) - noise, 0.0) / max(abs(fd), abs(g[p, i, c]), 1e-12))
        checked += 1
    assert checked >= 30
    assert max(errs) <= 1e-5, sorted(errs)[-3:]


# ---------------------------------------------------------------- preculling
def _maxpool_levels(a):
    levels = [a]
    while a.shape != (1, 1):
        h, w = a.shape
        h2, w2 = (h + 1) // 2, (w + 1) // 2
        p = np.full((2 * h2, 2 * w2), -np.inf, dtype=np.float32)
        p[:h, :w] = a
        a = p.reshape(h2, 2, w2, 2).max(axis=(1, 3))
        levels.append(a)
    return levels


def test_depth_pyramid_is_numpy_max_pooling():
    rng = np.random.default_rng(5)
    for H, W in [(1, 1), (3, 5), (17, 30), (64, 64), (45, 80)]:
        d = rng.random((H, W)).astype(np.float32)
        got = O.depth_mips(d)
        ref = _maxpool_levels(d)
        assert len(got) == len(ref)
        for g, r in zip(got, ref):
            np.testing.assert_array_equal(g, r)


def test_cell_of_matches_float32_floor_and_clamp():
    rng = np.random.default_rng(6)
    pts = rng.uniform(-3, 3, size=(500, 3)).astype(np.float32)
    origin = np.array([-2.0, -1.5, -2.5], dtype=np.float32)
    size, dims = np.float32(0.37), np.array([9, 11, 13])
    c = np.floor((pts - origin) / size).astype(np.int64)
    c = np.clip(c, 0, dims - 1)
    ref = (c[:, 2] * dims[1] + c[:, 1]) * dims[0] + c[:, 0]
    np.testing.assert_array_equal(O.cell_of(pts, origin, size, dims), ref)


def _grid_cams():
    cams = gi.ring_cameras(3, 96, 64, radius=4.0)
    return gi.subset_cameras(cams, [0, 1, 2])


def test_cell_visibility_against_a_constant_wall():
    """A depth buffer that is a wall at camera depth D everywhere: a cell the
    view's frustum reaches is kept exactly when its nearest corner lies at or
    in front of D."""
    cams = gi.ring_cameras(1, 80, 60, radius=4.0)
    origin, size, dims = np.array([-2, -2, -2], dtype=np.float32), 0.5, np.array([8, 8, 8])
    inf = O.cell_visible(cams, [np.full((60, 80), np.inf, np.float32)], origin, size, dims)
    for D in (3.0, 4.0, 5.5):
        vis = O.cell_visible(cams, [np.full((60, 80), D, np.float32)], origin, size, dims)
        # nearest corner depth per cell (camera 0 looks along -z from (0, 0, 4))
        zs = np.arange(8, dtype=np.float64) * 0.5 - 2.0
        zmin_axis = 4.0 - (zs + 0.5)            # the cell's corner with the largest world z
        zmin = np.broadcast_to(zmin_axis[:, None, None], (8, 8, 8))
        expect = inf.astype(bool) & (zmin <= D + 1e-6)
        # cells straddling the near plane use depth near; none here (near 0.2)
        np.testing.assert_array_equal(vis.astype(bool), expect)


def test_cell_visibility_is_conservative():
    """Every cell that an exact test (max of the depth buffer over the cell's
    full pixel rectangle, in float64) sees is kept; random depth buffers with
    occluders."""
    rng = np.random.default_rng(8)
    cams = _grid_cams()
    origin, size, dims = np.array([-3, -1.5, -3], dtype=np.float32), 0.6, np.array([10, 5, 10])
    depths = []
    for v in range(3):
        d = np.full((64, 96), np.inf, np.float32)
        for _ in range(6):
            y0, x0 = rng.integers(0, 64), rng.integers(0, 96)
            d[y0:y0 + rng.integers(5, 40), x0:x0 + rng.integers(5, 60)] = rng.uniform(2.0, 6.0)
        depths.append(d)
    vis = O.cell_visible(cams, depths, origin, size, dims).astype(bool)
    exact = np.zeros_like(vis)
    for v in range(3):
        R, t = np.asarray(cams["R"][v]), np.asarray(cams["t"][v])
        fx, fy, cx, cy = (float(cams[k][v]) for k in ("fx", "fy", "cx", "cy"))
        for cz in range(dims[2]):
            for cy_ in range(dims[1]):
                for cx_ in range(dims[0]):
                    corners = np.array([[cx_ + (k & 1), cy_ + ((k >> 1) & 1), cz + ((k >> 2) & 1)]
                                        for k in range(8)]) * size + origin
                    cc = corners @ R.T + t
                    if np.any(cc[:, 2] <= 0.2):
                        continue  # near-plane cells are kept conservatively; not tested here
                    u = fx * cc[:, 0] / cc[:, 2] + cx
                    w = fy * cc[:, 1] / cc[:, 2] + cy
                    x0, x1 = int(np.floor(u.min())), int(np.floor(u.max()))
                    y0, y1 = int(np.floor(w.min())), int(np.floor(w.max()))
                    if x1 < 0 or y1 < 0 or x0 > 95 or y0 > 63:
                        continue
                    x0, y0, x1, y1 = max(x0, 0), max(y0, 0), min(x1, 95), min(y1, 63)
                    m = depths[v][y0:y1 + 1, x0:x1 + 1].max()
                    if cc[:, 2].min() * (1 + 1e-5) <= m:
                        exact[cz, cy_, cx_] = True
    assert exact.any() and not exact.all()
    assert np.all(vis[exact])
    assert vis.sum() < vis.size   # something is culled


def test_cell_visibility_keeps_every_cell_a_sampled_point_shows():
    """No occluders: a cell is kept when any of its 5^3 sample points projects
    into an image in front of the near plane (the test may keep more)."""
    cams = _grid_cams()
    origin, size, dims = np.array([-6, -3, -6], dtype=np.float32), 1.0, np.array([12, 6, 12])
    depths = [np.full((64, 96), np.inf, np.float32)] * 3
    vis = O.cell_visible(cams, depths, origin, size, dims).astype(bool)
    f = np.linspace(0.02, 0.98, 5)
    off = np.stack(np.meshgrid(f, f, f, indexing="ij"), -1).reshape(-1, 3)
    for cz in range(dims[2]):
        for cy_ in range(dims[1]):
            for cx_ in range(dims[0]):
                pts = (np.array([cx_, cy_, cz]) + off) * size + origin
                seen = False
                for v in range(3):
                    cc = pts @ np.asarray(cams["R"][v]).T + np.asarray(cams["t"][v])
                    ok = cc[:, 2] > 0.2
                    u = cams["fx"][v] * cc[ok, 0] / cc[ok, 2] + cams["cx"][v]
                    w = cams["fy"][v] * cc[ok, 1] / cc[ok, 2] + cams["cy"][v]
                    if np.any((u >= 0) & (u < 96) & (w >= 0) & (w < 64)):
                        seen = True
                        break
                if seen:
                    assert vis[cz, cy_, cx_], (cz, cy_, cx_)
    assert not vis.all()


# ---------------------------------------------------------------- SH relighting (Sec. 3.4.1)
def _sh_light(env=None, direction=(0.0, 1.0, 0.0), radiance=(0.0, 0.0, 0.0)):
    L = np.zeros(56)
    if env is not None:
        L[:48] = np.asarray(env, dtype=float).reshape(48)
    d = np.asarray(direction, dtype=float)
    L[48:51] = d / np.linalg.norm(d)
    L[52:55] = radiance
    return L


def _visible(pr, v=0):
    return np.nonzero(pr[v, :, 14] > pr[v, :, 12])[0]


def test_relit_unit_lighting_is_orthonormality_of_the_basis():
    """Environment e_j (channel 0) against transfer e_k gives delta_jk: the
    exact sphere rule and the orthonormal basis together."""
    n = 256
    sc = gi.make_scene(n, 3, 40)
    sc[0, :, :3] *= 0.3
    sc[3:, :, :] = 0.0
    rows = gi.planes_to_rows(sc)
    for g in range(n):
        rows[g, 12 + 3 * (g % 16)] = 1.0  # transfer coefficient k = g % 16, channel 0
    cams = gi.ring_cameras(1, 64, 64)
    for j in (0, 2, 5, 9, 15):
        env = np.zeros((16, 3)); env[j, 0] = 1.0
        pr = O.project(gi.rows_to_planes(rows), 3, cams, dyn={"sh_light": _sh_light(env)})
        vis = _visible(pr)
        assert len(vis) > 200
        k = vis % 16
        np.testing.assert_allclose(pr[0, vis, 8], 0.5 + (k == j), atol=1e-13)
        np.testing.assert_allclose(pr[0, vis, 9:11], 0.5, atol=1e-13)


def test_relit_environment_term_matches_dense_integration_in_scipy():
    """int T(w) Lenv(R_g w) dw by numpy's 24-point Gauss-Legendre x 48
    azimuths with scipy's spherical harmonics and rotation."""
    rng = np.random.default_rng(41)
    n = 6
    sc = gi.make_scene(n, 3, 41, sh_std=0.5)
    sc[0, :, :3] *= 0.3
    env = rng.normal(size=(16, 3))
    q = rng.normal(size=4); q /= np.linalg.norm(q)
    d = {"sh_light": _sh_light(env), "group": np.zeros(n, dtype=np.int32),
         "poses": np.array([[*q, 0.0, 0.0, 0.0, 0.0]])}
    pr = O.project(sc, 3, gi.ring_cameras(1, 64, 64), dyn=d)
    Rg = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    z, wz = np.polynomial.legendre.leggauss(24)
    rows = gi.planes_to_rows(sc).astype(np.float64)
    acc = np.zeros((n, 3))
    for zi, wi in zip(z, wz):
        for j in range(48):
            ph = 2 * math.pi * j / 48
            w = np.array([math.sqrt(1 - zi * zi) * math.cos(ph), math.sqrt(1 - zi * zi) * math.sin(ph), zi])
            Yo = _real_sh_scipy(w)
            Yw = _real_sh_scipy(Rg @ w)
            Le = Yw @ env
            T = rows[:, 12:60].reshape(n, 16, 3).transpose(0, 2, 1) @ Yo
            acc += wi * (2 * math.pi / 48) * T * Le
    expect = np.maximum(acc + 0.5, 0.0)
    vis = _visible(pr)
    assert len(vis) == n
    np.testing.assert_allclose(pr[0, :, 8:11], expect, atol=1e-11)


def test_relit_light_along_the_view_reproduces_view_dependent_colour():
    """No environment, unit radiance from the view direction, fully visible:
    int T(w) delta(R_g w, dir) dw = T(R_g^T dir), the view-dependent colour."""
    n = 24
    sc = gi.make_scene(n, 3, 42, sh_std=0.4)
    cams = gi.ring_cameras(1, 64, 64)
    dd = _dyn(n, 3, 8, normals=False)
    base = O.project(sc, 3, cams, dyn=dd)
    rows = gi.planes_to_rows(sc).astype(np.float64)
    checked = 0
    for g in _visible(base):
        q = dd["poses"][dd["group"][g], :4]
        Rg = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        mu = Rg @ rows[g, :3] + dd["poses"][dd["group"][g], 4:7]
        centre = -cams["R"][0].T @ cams["t"][0]
        dirv = (mu - centre) / np.linalg.norm(mu - centre)
        d = {"sh_light": _sh_light(None, dirv, (1.0, 1.0, 1.0)), "group": dd["group"], "poses": dd["poses"]}
        pr = O.project(sc, 3, cams, dyn=d)
        np.testing.assert_allclose(pr[0, g, 8:12], base[0, g, 8:12], atol=1e-12)
        checked += 1
    assert checked > 15


def test_relit_visibility_attenuates_the_direct_light_only():
    n = 40
    sc = gi.make_scene(n, 2, 43)
    sc[3, :, :3] += 4.0  # a large DC transfer keeps every channel above the clamp
    cams = gi.ring_cameras(1, 64, 64)
    rng = np.random.default_rng(43)
    env = rng.normal(0, 0.3, (16, 3))
    env[0] = 1.0  # a positive ambient term
    L = _sh_light(env, (0.2, 0.9, -0.3), (0.9, 0.7, 0.5))
    out = {}
    for v in (0, 128, 255):
        out[v] = O.project(sc, 2, cams, dyn={"sh_light": L, "visibility": np.full(n, v, np.uint8)})[0, :, 8:11]
    assert np.all(out[0] > 0)
    np.testing.assert_allclose(out[128], out[0] + 128 / 255 * (out[255] - out[0]), atol=1e-12)
    none = O.project(sc, 2, cams, dyn={"sh_light": L})[0, :, 8:11]
    np.testing.assert_array_equal(none, out[255])
    # no light at all: only the offset is left
    dark = O.project(sc, 2, cams, dyn={"sh_light": _sh_light()})[0, _visible(O.project(sc, 2, cams)), 8:11]
    np.testing.assert_allclose(dark, 0.5, atol=1e-13)


def test_relit_gradient_matches_central_differences():
    n = 40
    sc = gi.make_scene(n, 2, 44, sh_std=0.3).astype(np.float64)
    sc[1, :, :3] += 1.2
    sc[0, :, :3] *= 0.6
    cams = gi.ring_cameras(2, 40, 32)
    rng = np.random.default_rng(44)
    dd = _dyn(n, 3, 9, normals=False)
    d = {"sh_light": _sh_light(rng.normal(0, 0.4, (16, 3)), (0.3, 0.8, 0.2), (0.8, 0.6, 0.9)),
         "visibility": rng.integers(0, 256, n).astype(np.uint8), "group": dd["group"], "poses": dd["poses"]}
    tgt = gi.make_scene(n, 2, 45).astype(np.float64)
    tgt[1, :, :3] += 1.2
    tgt[0, :, :3] *= 0.6
    target = O.forward(tgt, 2, cams, dyn=d)["image"]
    r = O.loss_and_grad(sc, 2, cams, target, dyn=d)
    g = r["dparams"]
    errs, checked, tries = [], 0, 0
    while checked < 40 and tries < 400:
        tries += 1
        p, i, c = int(rng.integers(0, 10)), int(rng.integers(0, n)), int(rng.integers(0, 4))
        if (p == 1 and c == 3) or np.all(r["proj"][:, i, 14] == 0):
            continue
        th = sc[p, i, c]
        h = 1e-6 * max(1.0, abs(th))
        sp_ = sc.copy(); sp_[p, i, c] = th + h
        sm_ = sc.copy(); sm_[p, i, c] = th - h
        fp, fm = O.forward(sp_, 2, cams, dyn=d), O.forward(sm_, 2, cams, dyn=d)
        if not (np.array_equal(fp["n_contrib"], r["n_contrib"]) and np.array_equal(fm["n_contrib"], r["n_contrib"])
                and np.array_equal(fp["proj"][..., 11:16], r["proj"][..., 11:16])
                and np.array_equal(fm["proj"][..., 11:16], r["proj"][..., 11:16])):
            continue
        Lp = O.loss(fp["image"], target, 2, 32, 40)[0]
        Lm = O.loss(fm["image"], target, 2, 32, 40)[0]
        fwd, bwd = (Lp - r["loss"]) / h, (r["loss"] - Lm) / h
        if abs(fwd - bwd) > 1e-3 * max(abs(fwd), abs(bwd), 1e-8):
            continue
        fd = (Lp - Lm) / (2 * h)
        noise = 100 * np.finfo(float).eps * abs(r["loss"]) / h
        errs.append(max(abs(fd - g[p, i, c]) - noise, 0.0) / max(abs(fd), abs(g[p, i, c]), 1e-12))
        checked += 1
    assert checked >= 30
    assert max(errs) <= 1e-5, sorted(errs)[-3:]


# ---------------------------------------------------------------- light visibility (Sec. 3.4.1)
def _light_cam(R, origin=(0.0, 0.0, 0.0), texel=0.05, W=48, H=40, alpha_min=0.5, bias=0.01):
    return {"R": np.asarray(R, dtype=float), "origin": np.asarray(origin, dtype=float), "texel": texel,
            "width": W, "height": H, "alpha_min": alpha_min, "bias": bias}


def _tilted_R():
    R, _ = gi.look_at((1.0, 2.0, 0.5))
    return R


def test_light_depth_bounding_box_equals_brute_force():
    sc = gi.make_scene(300, 0, 46)
    sc[1, :, :3] += 1.5
    lc = _light_cam(_tilted_R())
    for dyn in (None, _dyn(300, 4, 10, normals=False)):
        a = O.light_depth(sc, lc, dyn=dyn)
        b = O.light_depth(sc, lc, dyn=dyn, brute=True)
        np.testing.assert_array_equal(a, b)
        assert np.isfinite(a).mean() > 0.2


def _lone_gaussian(mean, scales, quat, logit):
    sc = np.zeros((15, 1, 4), dtype=np.float64)
    sc[0, 0] = [*mean, logit]
    sc[1, 0, :3] = np.log(scales)
    sc[2, 0] = quat
    return sc


def test_light_depth_footprint_closed_forms():
    """An isotropic Gaussian covers the disc |d|^2 <= tau ((s/h)^2 + 0.3); an
    axis-aligned anisotropic one covers the ellipse with the semi-axes its
    scales give along the light camera's x and y."""
    R = np.eye(3)
    h = 0.02
    lc = _light_cam(R, texel=h, W=64, H=48)
    o = 0.95
    logit = math.log(o / (1 - o))
    tau = 2 * math.log(o / 0.5)
    ii, jj = np.meshgrid(np.arange(64) + 0.5, np.arange(48) + 0.5)
    # isotropic; the quaternion is irrelevant
    mean = np.array([0.013, -0.021, 0.7])
    sc = _lone_gaussian(mean, [0.1, 0.1, 0.1], [0.3, 0.5, -0.2, 0.7], logit)
    u, v = mean[0] / h + 32, mean[1] / h + 24
    r2 = (ii - u) ** 2 + (jj - v) ** 2
    lim = tau * ((0.1 / h) ** 2 + 0.3)
    D = O.light_depth(sc, lc)
    sure = r2 < lim * (1 - 1e-9)
    out = r2 > lim * (1 + 1e-9)
    assert sure.sum() > 50
    assert np.all(D[sure] == mean[2]) and np.all(np.isinf(D[out]))
    # anisotropic: rotate 90 degrees about z, so the Gaussian's x axis lies along the map's y
    sx, sy = 0.15, 0.05
    qz = [math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)]
    sc = _lone_gaussian(mean, [sx, sy, 0.01], qz, logit)
    qf = (ii - u) ** 2 / ((sy / h) ** 2 + 0.3) + (jj - v) ** 2 / ((sx / h) ** 2 + 0.3)
    D = O.light_depth(sc, lc)
    sure = qf < tau * (1 - 1e-9)
    out = qf > tau * (1 + 1e-9)
    assert sure.sum() > 50
    assert np.all(D[sure] == mean[2]) and np.all(np.isinf(D[out]))
    # below alpha_min nothing is covered
    sc[0, 0, 3] = math.log(0.4 / 0.6)
    assert np.all(np.isinf(O.light_depth(sc, lc)))


def test_light_depth_is_invariant_under_a_rigid_motion_of_scene_and_light():
    """Moving every Gaussian by (R_g, t_g) and the light camera by the same
    motion (R_l' = R_l R_g^T, origin' = R_g origin + t_g) leaves the map as it was."""
    sc = gi.make_scene(200, 0, 47)
    sc[1, :, :3] += 1.5
    lc = _light_cam(_tilted_R(), origin=(0.1, -0.05, 0.2))
    q = np.array([0.8, -0.3, 0.4, 0.33]); q /= np.linalg.norm(q)
    t = np.array([0.2, -0.1, 0.15])
    Rg = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    d = {"group": np.zeros(200, dtype=np.int32), "poses": np.array([[*q, *t, 0.0]])}
    lc2 = dict(lc)
    lc2["R"] = lc["R"] @ Rg.T
    lc2["origin"] = Rg @ lc["origin"] + t
    moved = O.light_depth(sc, lc2, dyn=d)
    lo = O.light_depth(sc, lc, slack=1e-9)
    hi = O.light_depth(sc, lc, slack=-1e-9)
    fin = np.isfinite(moved)
    assert np.all((moved >= lo - 1e-12) | ~fin) and np.all((moved <= hi + 1e-12) | np.isinf(hi))
    assert fin.mean() > 0.2


def test_light_visibility_occluder_scene():
    """A large opaque Gaussian at depth 0.5 shadows a small one behind it at
    depth 1.5; itself, a small Gaussian beside it, one outside the map and one
    behind a faint (alpha < alpha_min) Gaussian are lit."""
    R = np.eye(3)
    lc = _light_cam(R, texel=0.02, W=64, H=64, bias=0.01)
    big = _lone_gaussian([0.0, 0.0, 0.5], [0.15, 0.15, 0.02], [1, 0, 0, 0], 4.0)
    parts = [big,
             _lone_gaussian([0.01, -0.01, 1.5], [0.01] * 3, [1, 0, 0, 0], 4.0),    # shadowed
             _lone_gaussian([0.5, 0.5, 1.5], [0.01] * 3, [1, 0, 0, 0], 4.0),       # beside: lit
             _lone_gaussian([2.0, 0.0, 1.5], [0.01] * 3, [1, 0, 0, 0], 4.0),       # outside the map: lit
             _lone_gaussian([-0.4, 0.4, 0.2], [0.1] * 3, [1, 0, 0, 0], -2.0),      # faint occluder
             _lone_gaussian([-0.4, 0.4, 1.0], [0.01] * 3, [1, 0, 0, 0], 4.0)]      # behind the faint one: lit
    sc = np.concatenate(parts, axis=1)
    D = O.light_depth(sc, lc)
    vis, uvz = O.light_visibility(sc, lc, D)
    np.testing.assert_array_equal(vis, [255, 0, 255, 255, 255, 255])
    np.testing.assert_allclose(uvz[1], [0.01 / 0.02 + 32, -0.01 / 0.02 + 32, 1.5], atol=1e-12)
    # every Gaussian alone in the scene is lit (bias >= 0)
    for g in range(sc.shape[1]):
        one = sc[:, g:g + 1]
        assert O.light_visibility(one, lc, O.light_depth(one, lc))[0][0] == 255
    # an empty map (+inf) lights everything
    v2, _ = O.light_visibility(sc, lc, np.full((64, 64), np.inf))
    assert np.all(v2 == 255)


# ---------------------------------------------------------------- splat rectangle
def _rect_case():
    sc = gi.make_scene(400, 1, 50)
    sc[1, :, :3] += 0.6
    sc[1, :, 0] += np.random.default_rng(50).normal(0, 0.7, 400)  # anisotropic splats
    sc[0, :30, 3] = -7.0  # opacity below 1/255
    cams = gi.ring_cameras(2, 96, 80)
    return sc, cams


def test_splat_rect_is_inside_the_square_and_covers_every_pixel_alpha_reaches():
    sc, cams = _rect_case()
    pr = O.project(sc, 1, cams)
    checked = 0
    for v in range(2):
        W, H = int(cams["width"][v]), int(cams["height"][v])
        ys, xs = np.mgrid[0:H, 0:W] + 0.5
        for g in range(pr.shape[1]):
            p = pr[v, g]
            if p[14] <= p[12]:
                continue
            u, vv, o, A, B, C, r = p[0], p[1], p[3], p[4], p[5], p[6], p[7]
            sq = O.rect(u, vv, r, W, H)
            assert sq[0] <= p[12] and sq[1] <= p[13] and p[14] <= sq[2] and p[15] <= sq[3]
            # pixels of the square where alpha >= 1/255 (brute force, FP64)
            dx, dy = xs - u, ys - vv
            alpha = o * np.exp(-0.5 * (A * dx * dx + 2 * B * dx * dy + C * dy * dy))
            tx, ty = (xs // 16).astype(int), (ys // 16).astype(int)
            in_sq = (tx >= sq[0]) & (tx < sq[2]) & (ty >= sq[1]) & (ty < sq[3])
            hit = in_sq & (alpha >= 1.0 / 255.0)
            in_rect = (tx >= p[12]) & (tx < p[14]) & (ty >= p[13]) & (ty < p[15])
            assert np.all(in_rect[hit])
            checked += 1
    assert checked > 300
    # faint splats get no tile
    assert np.all(pr[:, :30, 14] == 0)


def test_splat_rect_leaves_the_image_of_the_square_unchanged():
    """Binning by the 3-sigma squares and by the cut-down rectangles renders
    the same image, transmittance and contributor counts: the tiles dropped
    hold no pixel where the splat's alpha reaches 1/255."""
    sc, cams = _rect_case()
    f = O.forward(sc, 1, cams)
    pr = f["proj"]
    sq = np.zeros(pr.shape[:2] + (4,), dtype=np.int32)
    for v in range(2):
        W, H = int(cams["width"][v]), int(cams["height"][v])
        for g in range(pr.shape[1]):
            if pr[v, g, 7] > 0:
                sq[v, g] = O.rect(pr[v, g, 0], pr[v, g, 1], pr[v, g, 7], W, H)
    keys, vals, ranges = O.bin_sort(cams, sq, pr[..., 2].astype(np.float32))
    assert len(vals) > len(f["vals"])
    img, T, nc = O.render(cams, pr, vals, ranges)
    np.testing.assert_array_equal(img, f["image"])
    np.testing.assert_array_equal(T, f["T_final"])
    # contributor counts are list positions: compare the contributing sets instead
    assert np.array_equal(nc > 0, f["n_contrib"] > 0)
