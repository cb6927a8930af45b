"""FP64 CPU oracle of the online 3DGS optimisation step (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
the arithmetic lives in ``gs_oracle.c`` (plain C, double precision), and this
wrapper only converts array layouts and calls it.

Every stage takes its inputs explicitly so that a test can feed it either the
oracle's own upstream results (end to end) or the GPU's float32 upstream
results (stage-wise comparison).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from gs_inputs import planes_to_rows, rows_to_planes
from . import build as _build

_lib = None

_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_F = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_U32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_U64 = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_U8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")

TILE = 16
PROJ_FIELDS = ("u", "v", "depth", "opacity", "A", "B", "C", "radius", "r", "g", "b",
               "clamp", "x0", "y0", "x1", "y1")


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_sh_basis.argtypes = [_D, _D]
        L.or_sh_basis_grad.argtypes = [_D, _D]
        L.or_rect.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, _I32]
        L.or_splat_rect.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.c_int, C.c_int, C.c_int, _I32]
        L.or_project.argtypes = [C.c_int64, C.c_int, _D, C.c_int, _D, C.c_int, _D]
        L.or_project_dyn.argtypes = [C.c_int64, C.c_int, _D, C.c_int, _D, C.c_int, _I32, _D, C.c_void_p, _D,
                                     C.c_double, C.c_double, _D]
        L.or_project_bwd_dyn.argtypes = [C.c_int64, C.c_int, _D, C.c_int, _D, C.c_int, _D, _I32, _D, C.c_void_p,
                                         _D, C.c_double, C.c_double, _D]
        L.or_project_lit.argtypes = [C.c_int64, C.c_int, _D, C.c_int, _D, C.c_int, C.c_void_p, C.c_void_p, _D,
                                     C.c_void_p, _D]
        L.or_project_bwd_lit.argtypes = [C.c_int64, C.c_int, _D, C.c_int, _D, C.c_int, _D, C.c_void_p,
                                         C.c_void_p, _D, C.c_void_p, _D]
        L.or_light_depth.argtypes = [C.c_int64, _D, C.c_void_p, C.c_void_p, _D, C.c_double, C.c_int, _D]
        L.or_light_visibility.argtypes = [C.c_int64, _D, C.c_void_p, C.c_void_p, _D, _D, _U8, C.c_void_p]
        L.or_bin_count.argtypes = [C.c_int, C.c_int64, _I32]
        L.or_bin_count.restype = C.c_int64
        L.or_bin_sort.argtypes = [C.c_int, C.c_int64, _D, C.c_int, _I32, _F, _U64, _U32, _U32]
        L.or_bin_sort.restype = C.c_int64
        L.or_bin_ranges.argtypes = [C.c_int, C.c_int64, _D, C.c_int, _I32, _U32]
        L.or_bin_ranges.restype = C.c_int64
        L.or_bin_tiles.argtypes = [C.c_int, C.c_int64, _D, C.c_int, _I32, _F, C.c_int64, _I64, C.c_void_p, _I64]
        L.or_bin_tiles.restype = C.c_int64
        L.or_render.argtypes = [C.c_int, C.c_int64, _D, C.c_int, _D, _U32, _U32, _D, _D, _D, _I32]
        L.or_render_bwd.argtypes = [C.c_int, C.c_int64, _D, C.c_int, _D, _U32, _U32, _D, _D, _D]
        L.or_project_bwd.argtypes = [C.c_int64, C.c_int, _D, C.c_int, _D, C.c_int, _D, _D]
        L.or_ssim_map.argtypes = [C.c_int, C.c_int, _D, _D, _D, C.c_void_p]
        L.or_loss.argtypes = [C.c_int, C.c_int, C.c_int, _D, _D, C.c_double, C.c_double, _D]
        L.or_loss.restype = C.c_double
        L.or_adam.argtypes = [C.c_int64, _D, _D, _D, _D, _D, C.c_double, C.c_double, C.c_double, C.c_int]
        L.or_f32_to_f16.argtypes = [C.c_float]
        L.or_f16_to_f32.argtypes = [C.c_uint16]
        L.or_cell_of.argtypes = [_F, _F, C.c_float, _I32]
        L.or_cell_of.restype = C.c_int64
        L.or_depth_mips.argtypes = [_F, C.c_int, C.c_int, _F]
        L.or_cell_visible.argtypes = [C.c_int, _F, _F, _F, C.c_float, _I32, _U8]
        L.or_f16_to_f32.restype = C.c_float
        L.or_tensor_record_bytes.argtypes = [C.c_int]
        L.or_tensor_delta.argtypes = [C.c_int64, _F, _F, C.c_int, C.c_float, _U32, _U8]
        L.or_tensor_delta.restype = C.c_int64
        L.or_apply_tensor_delta.argtypes = [C.c_int64, _F, C.c_int, C.c_int64, _U32, _U8]
        L.or_apply_delta.argtypes = [C.c_int64, _F, C.c_int64, _U8]
        L.or_f32_to_f16.restype = C.c_uint16
        L.or_delta.argtypes = [C.c_int64, _F, _F, C.c_float, _U32, _U8]
        L.or_delta.restype = C.c_int64
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _rows(x):
    """Parameters as float64 rows [n][60]; accepts planes [15][n][4] or rows."""
    x = np.asarray(x)
    if x.ndim == 2 and x.shape[1] == 60:
        return _d(x)
    return _d(planes_to_rows(x))


# ------------------------------------------------------------------ layout
def cams_array(cams: dict) -> np.ndarray:
    """Camera dict (see gs_inputs) -> oracle records [V][20] float64."""
    V = len(cams["fx"])
    out = np.zeros((V, 20))
    out[:, 0:9] = np.asarray(cams["R"]).reshape(V, 9)
    out[:, 9:12] = cams["t"]
    out[:, 12] = cams["fx"]; out[:, 13] = cams["fy"]
    out[:, 14] = cams["cx"]; out[:, 15] = cams["cy"]
    out[:, 16] = cams["width"]; out[:, 17] = cams["height"]
    out[:, 18] = cams["near"]
    return out


def view_shapes(cams: dict):
    return [(int(h), int(w)) for w, h in zip(cams["width"], cams["height"])]


def n_tiles(cams: dict, tile: int = TILE) -> int:
    return int(sum(((int(w) + tile - 1) // tile) * ((int(h) + tile - 1) // tile)
                   for w, h in zip(cams["width"], cams["height"])))


def n_pixels(cams: dict) -> int:
    return int(sum(int(w) * int(h) for w, h in zip(cams["width"], cams["height"])))


# ------------------------------------------------------------------ stages
def sh_basis(d) -> np.ndarray:
    Y = np.zeros(16)
    lib().or_sh_basis(_d(d), Y)
    return Y


def sh_basis_grad(d) -> np.ndarray:
    dY = np.zeros(48)
    lib().or_sh_basis_grad(_d(d), dY)
    return dY.reshape(16, 3)


def rect(u, v, r, width, height, tile=TILE):
    """Tile rectangle of the square of half-side r around (u, v)."""
    out = np.zeros(4, dtype=np.int32)
    lib().or_rect(float(u), float(v), float(r), int(width), int(height), int(tile), out)
    return out


def splat_rect(u, v, r, a, c, opacity, width, height, tile=TILE):
    """Tile rectangle of a splat (the square cut to its alpha >= 1/255 box)."""
    out = np.zeros(4, dtype=np.int32)
    lib().or_splat_rect(float(u), float(v), float(r), float(a), float(c), float(opacity), int(width),
                        int(height), int(tile), out)
    return out


def _dyn_args(dyn):
    """dyn: dict with group (int [n]), poses ([G][8] quaternion wxyz,
    translation, 0), optional normals ([n][3]), light (3), ambient, diffuse."""
    group = np.ascontiguousarray(dyn["group"], dtype=np.int32)
    poses = _d(dyn["poses"])
    normals = dyn.get("normals")
    normals = None if normals is None else _d(normals)
    light = _d(dyn.get("light", (0.0, 1.0, 0.0)))
    keep = (group, poses, normals, light)
    nptr = None if normals is None else normals.ctypes.data_as(C.c_void_p)
    return keep, (group, poses, nptr, light, float(dyn.get("ambient", 0.3)), float(dyn.get("diffuse", 0.7)))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _lit_args(dyn, n):
    """SH relighting inputs of dyn: sh_light [56] (environment SH e[16][3],
    light direction xyz + 0, radiance rgb + 0), optional visibility (uint8
    [n]), optional group / poses (rigid objects)."""
    if dyn.get("normals") is not None:
        raise ValueError("SH relighting and the Lambertian DC factor are exclusive")
    L = _d(dyn["sh_light"])
    if L.shape != (56,):
        raise ValueError("sh_light must hold 56 values")
    vis = dyn.get("visibility")
    vis = None if vis is None else np.ascontiguousarray(vis, dtype=np.uint8)
    if vis is not None and vis.shape != (n,):
        raise ValueError("visibility must hold one value per Gaussian")
    group = dyn.get("group")
    group = None if group is None else np.ascontiguousarray(group, dtype=np.int32)
    poses = None if group is None else _d(dyn["poses"])
    keep = (L, vis, group, poses)
    return keep, (_ptr(group), _ptr(poses), L, _ptr(vis))


def light_cam_array(lcam: dict) -> np.ndarray:
    """Light camera dict (R [3][3] world -> light, origin [3], texel, width,
    height, alpha_min, bias) -> the oracle's [17] layout."""
    a = np.zeros(17)
    a[0:9] = np.asarray(lcam["R"], dtype=np.float64).reshape(9)
    a[9:12] = np.asarray(lcam["origin"], dtype=np.float64)
    a[12] = float(lcam["texel"])
    a[13] = int(lcam["width"])
    a[14] = int(lcam["height"])
    a[15] = float(lcam["alpha_min"])
    a[16] = float(lcam["bias"])
    return a


def _group_poses(dyn):
    if dyn is None or dyn.get("group") is None:
        return (None, None), (None, None)
    group = np.ascontiguousarray(dyn["group"], dtype=np.int32)
    poses = _d(dyn["poses"])
    return (group, poses), (_ptr(group), _ptr(poses))


def light_depth(planes, lcam: dict, dyn=None, slack: float = 0.0, brute: bool = False) -> np.ndarray:
    """Light-space depth map [H][W] float64 (+inf where no Gaussian covers)."""
    rows = _rows(planes)
    lc = light_cam_array(lcam)
    out = np.zeros((int(lcam["height"]), int(lcam["width"])))
    keep, gp = _group_poses(dyn)
    lib().or_light_depth(rows.shape[0], rows, gp[0], gp[1], lc, float(slack), int(bool(brute)), out)
    return out


def light_visibility(planes, lcam: dict, depth, dyn=None):
    """-> (visibility uint8 [n], uvz [n][3] light-map position and depth)."""
    rows = _rows(planes)
    n = rows.shape[0]
    lc = light_cam_array(lcam)
    vis = np.zeros(max(n, 1), dtype=np.uint8)
    uvz = np.zeros((max(n, 1), 3))
    keep, gp = _group_poses(dyn)
    lib().or_light_visibility(n, rows, gp[0], gp[1], lc, _d(depth), vis, _ptr(uvz))
    return vis[:n], uvz[:n]


def project(planes, sh_degree: int, cams: dict, tile: int = TILE, dyn=None) -> np.ndarray:
    """-> proj [V][n][16] float64 (fields PROJ_FIELDS; zero when culled).
    dyn: optional rigid-object poses and relighting (see _dyn_args, or
    _lit_args when it holds sh_light)."""
    rows = _rows(planes)
    n = rows.shape[0]
    V = len(cams["fx"])
    out = np.zeros((V, n, 16))
    if dyn is None:
        lib().or_project(n, sh_degree, rows, V, cams_array(cams), tile, out)
    elif dyn.get("sh_light") is not None:
        keep, a = _lit_args(dyn, n)
        lib().or_project_lit(n, sh_degree, rows, V, cams_array(cams), tile, *a, out)
    else:
        keep, a = _dyn_args(dyn)
        lib().or_project_dyn(n, sh_degree, rows, V, cams_array(cams), tile, *a, out)
    return out


def rects_of(proj) -> np.ndarray:
    return np.ascontiguousarray(proj[..., 12:16].astype(np.int32))


def bin_sort(cams: dict, rects, depth32, tile: int = TILE):
    """rects [V][n][4] int32, depth32 [V][n] float32 -> (keys u64, vals u32, ranges [T][2])."""
    rects = np.ascontiguousarray(rects, dtype=np.int32)
    depth32 = np.ascontiguousarray(depth32, dtype=np.float32)
    V, n = depth32.shape
    K = int(lib().or_bin_count(V, n, rects))
    keys = np.zeros(max(K, 1), dtype=np.uint64)
    vals = np.zeros(max(K, 1), dtype=np.uint32)
    ranges = np.zeros((n_tiles(cams, tile), 2), dtype=np.uint32)
    lib().or_bin_sort(V, n, cams_array(cams), tile, rects, depth32, keys, vals, ranges)
    return keys[:K], vals[:K], ranges


def bin_ranges(cams: dict, rects, tile: int = TILE):
    """rects [V][n][4] int32 -> (ranges [T][2] uint32 as bin_sort gives them, entry count),
    without forming the entries."""
    rects = np.ascontiguousarray(rects, dtype=np.int32)
    V, n = rects.shape[:2]
    ranges = np.zeros((n_tiles(cams, tile), 2), dtype=np.uint32)
    K = int(lib().or_bin_ranges(V, n, cams_array(cams), tile, rects, ranges))
    return ranges, K


def bin_tiles(cams: dict, rects, depth32, tiles, tile: int = TILE):
    """The sorted lists of the given global tiles only -> (vals u32, start int64 [len(tiles) + 1]):
    tile i's Gaussians, in bin_sort's order, are vals[start[i]:start[i + 1]]."""
    rects = np.ascontiguousarray(rects, dtype=np.int32)
    depth32 = np.ascontiguousarray(depth32, dtype=np.float32)
    req = np.ascontiguousarray(tiles, dtype=np.int64)
    V, n = depth32.shape
    start = np.zeros(len(req) + 1, dtype=np.int64)
    cams_a = cams_array(cams)
    total = int(lib().or_bin_tiles(V, n, cams_a, tile, rects, depth32, len(req), req, None, start))
    vals = np.zeros(max(total, 1), dtype=np.uint32)
    lib().or_bin_tiles(V, n, cams_a, tile, rects, depth32, len(req), req, vals.ctypes.data_as(C.c_void_p), start)
    return vals[:total], start


def render(cams: dict, proj, vals, ranges, bg=(0.0, 0.0, 0.0), tile: int = TILE):
    """-> (image [sum 3HW], T_final [sum HW], n_contrib [sum HW]) flat per view."""
    proj = _d(proj)
    V, n = proj.shape[:2]
    P = n_pixels(cams)
    img = np.zeros(3 * P); T = np.zeros(P); nc = np.zeros(P, dtype=np.int32)
    lib().or_render(V, n, cams_array(cams), tile, proj,
                    np.ascontiguousarray(vals, dtype=np.uint32),
                    np.ascontiguousarray(ranges, dtype=np.uint32), _d(bg), img, T, nc)
    return img, T, nc


def render_bwd(cams: dict, proj, vals, ranges, dimage, bg=(0.0, 0.0, 0.0), tile: int = TILE):
    """-> grad2d [V][n][9]."""
    proj = _d(proj)
    V, n = proj.shape[:2]
    g = np.zeros((V, n, 9))
    lib().or_render_bwd(V, n, cams_array(cams), tile, proj,
                        np.ascontiguousarray(vals, dtype=np.uint32),
                        np.ascontiguousarray(ranges, dtype=np.uint32), _d(bg), _d(dimage), g)
    return g


def project_bwd(planes, sh_degree: int, cams: dict, grad2d, tile: int = TILE, dyn=None) -> np.ndarray:
    """-> parameter gradient as planes [15][n][4] float64."""
    rows = _rows(planes)
    n = rows.shape[0]
    V = len(cams["fx"])
    d = np.zeros((n, 60))
    if dyn is None:
        lib().or_project_bwd(n, sh_degree, rows, V, cams_array(cams), tile, _d(grad2d), d)
    elif dyn.get("sh_light") is not None:
        keep, a = _lit_args(dyn, n)
        lib().or_project_bwd_lit(n, sh_degree, rows, V, cams_array(cams), tile, _d(grad2d), *a, d)
    else:
        keep, a = _dyn_args(dyn)
        lib().or_project_bwd_dyn(n, sh_degree, rows, V, cams_array(cams), tile, _d(grad2d), *a, d)
    return rows_to_planes(d)


def ssim_map(x, y, with_partials: bool = False):
    x = _d(x); y = _d(y)
    H, W = x.shape
    s = np.zeros((H, W))
    if with_partials:
        d = np.zeros((H, W, 3))
        lib().or_ssim_map(H, W, x, y, s, d.ctypes.data_as(C.c_void_p))
        return s, d
    lib().or_ssim_map(H, W, x, y, s, None)
    return s


def loss(image, target, V: int, H: int, W: int, w_l1: float = 0.8, w_ssim: float = 0.2):
    """-> (L, dL/dimage) for V equal-size views, planar [V][3][H][W]."""
    dimg = np.zeros(V * 3 * H * W)
    L = lib().or_loss(V, H, W, _d(image).ravel(), _d(target).ravel(), w_l1, w_ssim, dimg)
    return float(L), dimg


def adam(theta, grad, m, v, lr, step: int, b1=0.9, b2=0.999, eps=1e-8):
    """In place on float64 arrays; lr broadcast to theta's shape."""
    lr = np.ascontiguousarray(np.broadcast_to(lr, theta.shape), dtype=np.float64)
    lib().or_adam(theta.size, theta, _d(grad), m, v, lr, b1, b2, eps, step)


def f32_to_f16_bits(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float32).ravel()
    return np.array([lib().or_f32_to_f16(float(v)) for v in x], dtype=np.uint16)


def delta(theta_planes, base_planes, thr: float = 1e-3):
    """Float32 planes in; returns (idx u32[M], records u8[M][128], new baseline planes)."""
    th = np.ascontiguousarray(planes_to_rows(theta_planes), dtype=np.float32)
    base = np.ascontiguousarray(planes_to_rows(base_planes), dtype=np.float32)
    n = th.shape[0]
    idx = np.zeros(max(n, 1), dtype=np.uint32)
    rec = np.zeros((max(n, 1), 128), dtype=np.uint8)
    M = int(lib().or_delta(n, th, base, np.float32(thr), idx, rec))
    return idx[:M], rec[:M], rows_to_planes(base)


def cell_of(points, origin, size: float, dims):
    """Cell index of each point (float32 arithmetic, clamped)."""
    pts = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 3)
    o = np.ascontiguousarray(origin, dtype=np.float32)
    d = np.ascontiguousarray(dims, dtype=np.int32)
    return np.array([lib().or_cell_of(p, o, np.float32(size), d) for p in pts], dtype=np.int64)


def depth_mips(depth):
    """Max pyramid of one [H][W] buffer: list of levels (float32)."""
    dpt = np.ascontiguousarray(depth, dtype=np.float32)
    H, W = dpt.shape
    tot, w, h, shapes = 0, W, H, []
    while True:
        shapes.append((h, w)); tot += w * h
        if w == 1 and h == 1:
            break
        w, h = (w + 1) // 2, (h + 1) // 2
    out = np.zeros(tot, dtype=np.float32)
    lib().or_depth_mips(dpt, W, H, out)
    levels, off = [], 0
    for h, w in shapes:
        levels.append(out[off:off + h * w].reshape(h, w)); off += h * w
    return levels


def cell_visible(cams: dict, depths, origin, size: float, dims) -> np.ndarray:
    """Kept cells (uint8 [nz][ny][nx]) of the preculling test for the views'
    depth buffers (list of [H][W] float32)."""
    ca = np.ascontiguousarray(cams_array(cams), dtype=np.float32)
    dep = np.ascontiguousarray(np.concatenate([np.asarray(d, dtype=np.float32).ravel() for d in depths]))
    d = np.ascontiguousarray(dims, dtype=np.int32)
    vis = np.zeros(int(np.prod(dims)), dtype=np.uint8)
    lib().or_cell_visible(len(cams["fx"]), ca, dep, np.ascontiguousarray(origin, dtype=np.float32),
                          np.float32(size), d, vis)
    return vis.reshape(int(dims[2]), int(dims[1]), int(dims[0]))


ATTR_GROUPS = {"mean": 1, "opacity": 2, "scale": 4, "rotation": 8, "dc": 16, "sh_rest": 32}


def f16_bits_to_f32(bits) -> np.ndarray:
    b = np.asarray(bits, dtype=np.uint16).ravel()
    return np.array([lib().or_f16_to_f32(int(v)) for v in b], dtype=np.float32)


def tensor_record_bytes(attr: int) -> int:
    return int(lib().or_tensor_record_bytes(int(attr)))


def tensor_delta(theta_planes, base_planes, attr: int, thr: float = 1e-3):
    """-> (idx u32[M], vals u8[M][record bytes], new baseline planes)."""
    th = np.ascontiguousarray(planes_to_rows(theta_planes), dtype=np.float32)
    base = np.ascontiguousarray(planes_to_rows(base_planes), dtype=np.float32)
    n = th.shape[0]
    rb = tensor_record_bytes(attr)
    idx = np.zeros(max(n, 1), dtype=np.uint32)
    vals = np.zeros((max(n, 1), rb), dtype=np.uint8)
    M = int(lib().or_tensor_delta(n, th, base, int(attr), np.float32(thr), idx, vals))
    return idx[:M], vals[:M], rows_to_planes(base)


def apply_tensor_delta(params_planes, attr: int, idx, vals):
    rows = np.ascontiguousarray(planes_to_rows(params_planes), dtype=np.float32)
    idx = np.ascontiguousarray(idx, dtype=np.uint32)
    vals = np.ascontiguousarray(vals, dtype=np.uint8)
    lib().or_apply_tensor_delta(rows.shape[0], rows, int(attr), len(idx), idx, vals)
    return rows_to_planes(rows)


def apply_delta(params_planes, records):
    rows = np.ascontiguousarray(planes_to_rows(params_planes), dtype=np.float32)
    rec = np.ascontiguousarray(records, dtype=np.uint8)
    lib().or_apply_delta(rows.shape[0], rows, len(rec), rec)
    return rows_to_planes(rows)


# ------------------------------------------------------------------ composed
def forward(planes, sh_degree, cams, bg=(0.0, 0.0, 0.0), tile=TILE, dyn=None):
    proj = project(planes, sh_degree, cams, tile, dyn)
    keys, vals, ranges = bin_sort(cams, rects_of(proj), proj[..., 2].astype(np.float32), tile)
    img, T, nc = render(cams, proj, vals, ranges, bg, tile)
    return {"proj": proj, "keys": keys, "vals": vals, "ranges": ranges,
            "image": img, "T_final": T, "n_contrib": nc}


def loss_and_grad(planes, sh_degree, cams, target, w_l1=0.8, w_ssim=0.2,
                  bg=(0.0, 0.0, 0.0), tile=TILE, dyn=None):
    """Full FP64 chain: render, loss, image gradient, 2D and parameter gradients."""
    f = forward(planes, sh_degree, cams, bg, tile, dyn)
    V = len(cams["fx"])
    H, W = int(cams["height"][0]), int(cams["width"][0])
    L, dimg = loss(f["image"], target, V, H, W, w_l1, w_ssim)
    g2 = render_bwd(cams, f["proj"], f["vals"], f["ranges"], dimg, bg, tile)
    dp = project_bwd(planes, sh_degree, cams, g2, tile, dyn)
    f.update({"loss": L, "dimage": dimg, "grad2d": g2, "dparams": dp})
    return f


def render_loss(planes, sh_degree, cams, target, w_l1=0.8, w_ssim=0.2, bg=(0.0, 0.0, 0.0), tile=TILE,
                dyn=None):
    f = forward(planes, sh_degree, cams, bg, tile, dyn)
    V = len(cams["fx"])
    H, W = int(cams["height"][0]), int(cams["width"][0])
    return loss(f["image"], target, V, H, W, w_l1, w_ssim)[0]
