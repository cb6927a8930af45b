"""B300 (sm_103a) online 3D Gaussian Splatting step behind a C ABI.

Python names mirror the C entry points of include/gs.h; each function only
marshals torch tensors (device memory and streams) into the C call.  All
arithmetic runs in the CUDA kernels of libgs.so.  The library is required:
without it every call raises (there is no CPU path).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import GsError, check

CAMERA_DTYPE = np.dtype([("R", "<f4", (9,)), ("t", "<f4", (3,)), ("fx", "<f4"), ("fy", "<f4"),
                         ("cx", "<f4"), ("cy", "<f4"), ("width", "<i4"), ("height", "<i4"),
                         ("near_plane", "<f4"), ("_pad", "<f4")])
assert CAMERA_DTYPE.itemsize == 80
PROJ_STRIDE = 16
GRAD2D_STRIDE = 12
RECORD_BYTES = 128


def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ------------------------------------------------------------------ cameras
def pack_cameras(cams: dict) -> np.ndarray:
    """Camera dict (R [V,3,3], t [V,3], fx, fy, cx, cy, width, height, near)
    -> structured array in the gs_camera layout (80 bytes per view)."""
    V = len(cams["fx"])
    a = np.zeros(V, dtype=CAMERA_DTYPE)
    a["R"] = np.asarray(cams["R"], dtype=np.float64).reshape(V, 9)
    a["t"] = np.asarray(cams["t"], dtype=np.float64).reshape(V, 3)
    for k in ("fx", "fy", "cx", "cy"):
        a[k] = cams[k]
    a["width"] = cams["width"]
    a["height"] = cams["height"]
    a["near_plane"] = cams["near"]
    return a


def cameras_to_device(cams, device="cuda"):
    """-> uint8 tensor on the device holding gs_camera[V]."""
    torch = _torch()
    packed = cams if isinstance(cams, np.ndarray) else pack_cameras(cams)
    return torch.from_numpy(packed.view(np.uint8).copy()).to(device)


def _host_cams(cams):
    packed = cams if isinstance(cams, np.ndarray) else pack_cameras(cams)
    packed = np.ascontiguousarray(packed)
    return packed, packed.ctypes.data_as(C.POINTER(_lib.gs_camera))


def view_sizes(cams):
    packed = cams if isinstance(cams, np.ndarray) else pack_cameras(cams)
    return [(int(h), int(w)) for w, h in zip(packed["width"], packed["height"])]


def total_pixels(cams) -> int:
    return int(sum(h * w for h, w in view_sizes(cams)))


# ------------------------------------------------------------------ context
# gs_ctx_set_binning modes
BINNING = {"two_level": 0, "direct": 1}


class Context:
    """Owns a gs_ctx (device workspace, status word, graph)."""

    def __init__(self, device: int = 0, workspace_bytes: int = 0, tile: int = 16, sort_bits: int = 8,
                 sort_items: int = 16, binning: str = "two_level", raster_threads: int = 4,
                 raster_bwd_threads: "int | None" = None):
        L = _lib.lib()
        p = C.c_void_p()
        check("gs_ctx_create", L.gs_ctx_create(C.byref(p), device, workspace_bytes))
        self.ptr = p
        self.device = device
        self.tile = tile
        check("gs_ctx_set_tile", L.gs_ctx_set_tile(p, tile))
        check("gs_ctx_set_sort_bits", L.gs_ctx_set_sort_bits(p, sort_bits))
        check("gs_ctx_set_sort_items", L.gs_ctx_set_sort_items(p, sort_items))
        if binning not in BINNING:
            raise ValueError(f"binning must be one of {sorted(BINNING)}")
        self.binning = binning
        check("gs_ctx_set_binning", L.gs_ctx_set_binning(p, BINNING[binning]))
        self.raster_threads = raster_threads
        check("gs_ctx_set_raster_threads", L.gs_ctx_set_raster_threads(p, raster_threads))
        self.raster_bwd_threads = raster_threads if raster_bwd_threads is None else raster_bwd_threads
        check("gs_ctx_set_raster_bwd_threads", L.gs_ctx_set_raster_bwd_threads(p, self.raster_bwd_threads))

    def tuning(self) -> dict:
        """The context's current tunables (gs_ctx_get_tuning)."""
        v = [C.c_int32() for _ in range(5)]
        check("gs_ctx_get_tuning", _lib.lib().gs_ctx_get_tuning(self.ptr, *(C.byref(x) for x in v)))
        names = {val: k for k, val in BINNING.items()}
        return {"binning": names[v[0].value], "sort_bits": v[1].value, "sort_items": v[2].value,
                "raster_threads": v[3].value, "raster_bwd_threads": v[4].value}

    def set_wait_limit(self, cycles: int) -> None:
        """Bound of every inter-block wait in clock cycles (0: the default)."""
        check("gs_ctx_set_wait_limit", _lib.lib().gs_ctx_set_wait_limit(self.ptr, int(cycles)))

    def set_wait_test(self, tile: int) -> None:
        """Test hook of the bounded waits (gs_ctx_set_wait_test); -1 turns it off."""
        check("gs_ctx_set_wait_test", _lib.lib().gs_ctx_set_wait_test(self.ptr, int(tile)))

    def reserve(self, nbytes: int) -> None:
        check("gs_ctx_reserve", _lib.lib().gs_ctx_reserve(self.ptr, int(nbytes)))

    def status(self, stream=None):
        code, detail = C.c_int32(), C.c_int64()
        check("gs_get_status", _lib.lib().gs_get_status(self.ptr, _stream(stream), C.byref(code), C.byref(detail)))
        return code.value, detail.value

    def raise_status(self, stream=None) -> None:
        code, detail = self.status(stream)
        if code != _lib.GS_OK:
            err = GsError("device status", code)
            err.detail = detail
            raise err

    def total_tiles(self, cams) -> int:
        packed, p = _host_cams(cams)
        return int(_lib.lib().gs_total_tiles(self.ptr, p, len(packed)))

    def workspace_size(self, cams, n: int, keys_cap: int) -> int:
        packed, p = _host_cams(cams)
        return int(_lib.lib().gs_workspace_size(self.ptr, p, len(packed), int(n), int(keys_cap)))

    def close(self) -> None:
        if self.ptr:
            _lib.lib().gs_ctx_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Dynamics:
    """Rigid-object poses and a directional light for a scene (gs_dynamics).

    group: uint8 [n] object of each Gaussian; poses: float [G][8] (unit
    quaternion w,x,y,z; translation x,y,z; 0); normals: float [n][3] or [n][4]
    object-frame unit normals (None: no relighting); light: unit vector
    towards the light.  Device copies are kept here; set_frame() overwrites
    the poses and the light in place, so a captured graph sees new values."""

    def __init__(self, group, poses, normals=None, light=(0.0, 1.0, 0.0), ambient=0.3, diffuse=0.7,
                 device="cuda"):
        torch = _torch()
        self.group = torch.as_tensor(np.asarray(group, dtype=np.uint8)).to(device)
        self.poses = torch.as_tensor(np.asarray(poses, dtype=np.float32).reshape(-1, 8)).to(device)
        self.normals = None
        if normals is not None:
            nn = np.zeros((len(normals), 4), dtype=np.float32)
            nn[:, :3] = np.asarray(normals, dtype=np.float32)[:, :3]
            self.normals = torch.from_numpy(nn).to(device)
        self.light = torch.zeros(4, dtype=torch.float32, device=device)
        self.light[:3] = torch.as_tensor(np.asarray(light, dtype=np.float32))
        self.struct = _lib.gs_dynamics(
            n_groups=self.poses.shape[0], group=self.group.data_ptr(), poses=self.poses.data_ptr(),
            normals=self.normals.data_ptr() if self.normals is not None else None,
            light=self.light.data_ptr(), ambient=ambient, diffuse=diffuse)

    def set_frame(self, poses=None, light=None):
        torch = _torch()
        if poses is not None:
            self.poses.copy_(torch.as_tensor(np.asarray(poses, dtype=np.float32).reshape(-1, 8)))
        if light is not None:
            self.light[:3].copy_(torch.as_tensor(np.asarray(light, dtype=np.float32)))


class Precull:
    """Preculling grid (gs_precull): cell of a mean p is floor((p - origin) /
    cell_size) per axis, clamped; `visible` (uint8 [nz][ny][nx] on the
    device) marks the kept cells, filled by update() (gs_cell_visibility) or by
    the caller.  The struct holds the buffer's address, so a captured graph
    sees later updates."""

    def __init__(self, origin, cell_size: float, dims, device="cuda"):
        torch = _torch()
        self.dims = tuple(int(d) for d in dims)
        self.visible = torch.ones(self.dims[::-1], dtype=torch.uint8, device=device)
        self.struct = _lib.gs_precull(cell_visible=self.visible.data_ptr(), cell_size=float(cell_size))
        for a in range(3):
            self.struct.origin[a] = float(origin[a])
            self.struct.dims[a] = self.dims[a]

    def update(self, ctx, cams, depth, stream=None):
        """Keep the cells that some view sees (depth: the views' buffers of
        camera-space z, +inf where empty, back to back)."""
        packed, host = _host_cams(cams)
        d_cams = cameras_to_device(packed, depth.device)
        need = int(_lib.lib().gs_precull_workspace_size(host, len(packed)))
        ctx.reserve(need)
        check("gs_cell_visibility", _lib.lib().gs_cell_visibility(
            ctx.ptr, _ptr(d_cams), host, len(packed), _ptr(depth), C.byref(self.struct), _ptr(self.visible),
            _stream(stream)))
        return self.visible


class Lighting:
    """SH relighting inputs (gs_lighting, Sec. 3.4.1): the world-frame
    environment SH e[16][3], the unit vector towards the directional light and
    its radiance in one device buffer of 56 floats, and an optional uint8
    light visibility per Gaussian (255 = lit).  set() overwrites the buffer in
    place and update_visibility() recomputes the visibility from a light-space
    depth map, so a captured graph sees each frame's values."""

    def __init__(self, n: int, env=None, direction=(0.0, 1.0, 0.0), radiance=(1.0, 1.0, 1.0),
                 with_visibility: bool = True, device="cuda"):
        torch = _torch()
        self.light = torch.zeros(56, dtype=torch.float32, device=device)
        self.visibility = (torch.full((max(int(n), 1),), 255, dtype=torch.uint8, device=device)
                           if with_visibility else None)
        self.n = int(n)
        self._host = self.pack(env if env is not None else np.zeros((16, 3)), direction, radiance)
        self.light.copy_(torch.from_numpy(self._host))
        self.struct = _lib.gs_lighting(light=self.light.data_ptr(),
                                       visibility=self.visibility.data_ptr() if with_visibility else None)

    @staticmethod
    def pack(env, direction, radiance) -> np.ndarray:
        buf = np.zeros(56, dtype=np.float32)
        buf[:48] = np.asarray(env, dtype=np.float32).reshape(48)
        d = np.asarray(direction, dtype=np.float64)
        buf[48:51] = d / np.linalg.norm(d)
        buf[52:55] = np.asarray(radiance, dtype=np.float32)
        return buf

    def set(self, env=None, direction=None, radiance=None):
        """Overwrite the given parts of the lighting (the others stay)."""
        torch = _torch()
        cur = self._host
        e = cur[:48] if env is None else env
        d = cur[48:51] if direction is None else direction
        r = cur[52:55] if radiance is None else radiance
        self._host = self.pack(e, d, r)
        self.light.copy_(torch.from_numpy(self._host))

    def update_visibility(self, ctx, params, lcam, depth=None, dyn=None, stream=None, frozen=None):
        """Render the light-space depth map of params (and the frozen pool, if
        given) and test every centre against it; returns the depth map.  The
        frozen pool is taken as static (dyn applies to params only)."""
        if dyn is not None and frozen is not None and frozen.shape[1] > 0:
            raise ValueError("update_visibility: a frozen pool with rigid-object dynamics is not supported")
        depth = gs_light_depth_map(ctx, params, lcam, depth, dyn=dyn, stream=stream)
        if frozen is not None and frozen.shape[1] > 0:
            gs_light_depth_map(ctx, frozen, lcam, depth, accumulate=True, stream=stream)
        n = params.shape[1]
        gs_light_visibility(ctx, params, lcam, depth, dyn=dyn, out=self.visibility[:n], stream=stream)
        if frozen is not None and frozen.shape[1] > 0:
            gs_light_visibility(ctx, frozen, lcam, depth, out=self.visibility[n:n + frozen.shape[1]],
                                stream=stream)
        return depth


def light_camera(R=None, origin=(0.0, 0.0, 0.0), texel=0.01, width=1024, height=1024, alpha_min=0.5,
                 bias=0.01, direction=None, extent=None):
    """gs_light_camera.  Either R (world -> light rows: map x, map y, depth
    axis) or direction (unit vector towards the light: the depth axis points
    along the light's travel, -direction); extent (world units covered by the
    larger map side) sets texel when given."""
    if R is None:
        d = -np.asarray(direction, dtype=np.float64)
        d /= np.linalg.norm(d)
        up = np.array([0.0, 1.0, 0.0]) if abs(d[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
        x = np.cross(up, d); x /= np.linalg.norm(x)
        y = np.cross(d, x)
        R = np.stack([x, y, d])
    if extent is not None:
        texel = float(extent) / max(int(width), int(height))
    c = _lib.gs_light_camera()
    Rf = np.asarray(R, dtype=np.float64).reshape(9)
    for i in range(9):
        c.R[i] = float(Rf[i])
    for i in range(3):
        c.origin[i] = float(origin[i])
    c.texel, c.width, c.height = float(texel), int(width), int(height)
    c.alpha_min, c.bias = float(alpha_min), float(bias)
    return c


def light_camera_dict(c) -> dict:
    """The fields of a gs_light_camera as a dict of floats / ints."""
    return {"R": np.array(c.R[:], dtype=np.float64).reshape(3, 3), "origin": np.array(c.origin[:], dtype=np.float64),
            "texel": float(c.texel), "width": int(c.width), "height": int(c.height),
            "alpha_min": float(c.alpha_min), "bias": float(c.bias)}


def _scene(params, sh_degree, dyn: "Dynamics | None" = None, precull: "Precull | None" = None,
           lighting: "Lighting | None" = None):
    n = params.shape[1] if params is not None else 0
    sc = _lib.gs_scene(n=n, sh_degree=sh_degree, params=params.data_ptr() if n else None)
    if dyn is not None:
        sc.dyn = C.pointer(dyn.struct)
    if precull is not None:
        sc.precull = C.pointer(precull.struct)
    if lighting is not None:
        sc.lighting = C.pointer(lighting.struct)
    return sc


def gs_light_depth_map(ctx, params, lcam, depth=None, accumulate=False, dyn=None, stream=None):
    """Light-space depth map [height][width] float32 (+inf where empty)."""
    torch = _torch()
    if depth is None:
        depth = torch.empty((lcam.height, lcam.width), dtype=torch.float32, device=params.device)
        accumulate = False
    sc = _scene(params, 0, dyn)
    check("gs_light_depth_map", _lib.lib().gs_light_depth_map(ctx.ptr, C.byref(sc), C.byref(lcam), _ptr(depth),
                                                              int(bool(accumulate)), _stream(stream)))
    return depth


def gs_light_visibility(ctx, params, lcam, depth, dyn=None, out=None, stream=None):
    """uint8 [n]: 255 where the centre is lit, 0 where the map occludes it."""
    torch = _torch()
    if out is None:
        out = torch.empty(max(params.shape[1], 1), dtype=torch.uint8, device=params.device)
    sc = _scene(params, 0, dyn)
    check("gs_light_visibility", _lib.lib().gs_light_visibility(ctx.ptr, C.byref(sc), C.byref(lcam), _ptr(depth),
                                                                _ptr(out), _stream(stream)))
    return out[:params.shape[1]]


# ------------------------------------------------------------------ entry points
def gs_project(ctx, params, sh_degree, d_cams, n_views, proj=None, stream=None, dyn=None, precull=None,
               lighting=None):
    torch = _torch()
    n = params.shape[1]
    if proj is None:
        proj = torch.empty((n_views, n, PROJ_STRIDE), dtype=torch.float32, device=params.device)
    sc = _scene(params, sh_degree, dyn, precull, lighting)
    check("gs_project", _lib.lib().gs_project(ctx.ptr, C.byref(sc), _ptr(d_cams), n_views, _ptr(proj),
                                              _stream(stream)))
    return proj


def gs_bin_sort(ctx, proj, d_cams, n_views, n, total_tiles, keys_cap, sorted_keys=None, sorted_vals=None,
                ranges=None, d_num_keys=None, want_keys=True, stream=None):
    torch = _torch()
    dev = proj.device
    if sorted_vals is None:
        sorted_vals = torch.empty(max(keys_cap, 1), dtype=torch.int32, device=dev)
    if want_keys and sorted_keys is None:
        sorted_keys = torch.empty(max(keys_cap, 1), dtype=torch.int32, device=dev)
    if ranges is None:
        ranges = torch.empty((total_tiles, 2), dtype=torch.int32, device=dev)
    if d_num_keys is None:
        d_num_keys = torch.zeros(1, dtype=torch.int32, device=dev)
    check("gs_bin_sort", _lib.lib().gs_bin_sort(ctx.ptr, _ptr(proj), _ptr(d_cams), n_views, n, total_tiles,
                                                keys_cap, _ptr(sorted_keys), _ptr(sorted_vals), _ptr(ranges),
                                                _ptr(d_num_keys), _stream(stream)))
    return sorted_keys, sorted_vals, ranges, d_num_keys


def _bg(bg):
    a = (C.c_float * 3)(*(bg if bg is not None else (0.0, 0.0, 0.0)))
    return a


def gs_render_fwd(ctx, proj, d_cams, n_views, n, total_tiles, sorted_vals, ranges, npix, bg=None,
                  image=None, T_final=None, n_contrib=None, want_state=True, stream=None):
    torch = _torch()
    dev = proj.device
    if image is None:
        image = torch.empty(3 * npix, dtype=torch.float32, device=dev)
    if want_state and T_final is None:
        T_final = torch.empty(npix, dtype=torch.float32, device=dev)
    if want_state and n_contrib is None:
        n_contrib = torch.empty(npix, dtype=torch.int32, device=dev)
    check("gs_render_fwd", _lib.lib().gs_render_fwd(ctx.ptr, _ptr(proj), _ptr(d_cams), n_views, n, total_tiles,
                                                    _ptr(sorted_vals), _ptr(ranges), _bg(bg), _ptr(image),
                                                    _ptr(T_final), _ptr(n_contrib), _stream(stream)))
    return image, T_final, n_contrib


def gs_loss(ctx, image, target, n_views, height, width, w_l1=0.8, w_ssim=0.2, d_loss=None, dimage=None,
            stream=None):
    torch = _torch()
    if d_loss is None:
        d_loss = torch.zeros(1, dtype=torch.float32, device=image.device)
    if dimage is None:
        dimage = torch.empty_like(image)
    check("gs_loss", _lib.lib().gs_loss(ctx.ptr, _ptr(image), _ptr(target), n_views, height, width, w_l1, w_ssim,
                                        _ptr(d_loss), _ptr(dimage), _stream(stream)))
    return d_loss, dimage


def gs_raster_bwd(ctx, proj, d_cams, n_views, n, total_tiles, sorted_vals, ranges, T_final, n_contrib, dimage,
                  bg=None, grad2d=None, stream=None):
    torch = _torch()
    if grad2d is None:
        grad2d = torch.empty((n_views, n, GRAD2D_STRIDE), dtype=torch.float32, device=proj.device)
    check("gs_raster_bwd", _lib.lib().gs_raster_bwd(ctx.ptr, _ptr(proj), _ptr(d_cams), n_views, n, total_tiles,
                                                    _ptr(sorted_vals), _ptr(ranges), _bg(bg), _ptr(T_final),
                                                    _ptr(n_contrib), _ptr(dimage), _ptr(grad2d), _stream(stream)))
    return grad2d


def gs_project_bwd(ctx, params, sh_degree, d_cams, n_views, proj, grad2d, dparams=None, accumulate=False,
                   stream=None, dyn=None, lighting=None):
    torch = _torch()
    if dparams is None:
        dparams = torch.empty_like(params)
        accumulate = False
    sc = _scene(params, sh_degree, dyn, None, lighting)
    check("gs_project_bwd", _lib.lib().gs_project_bwd(ctx.ptr, C.byref(sc), _ptr(d_cams), n_views, _ptr(proj),
                                                      _ptr(grad2d), _ptr(dparams), int(bool(accumulate)),
                                                      _stream(stream)))
    return dparams


def gs_render_bwd(ctx, params, sh_degree, d_cams, n_views, total_tiles, proj, sorted_vals, ranges, T_final,
                  n_contrib, dimage, bg=None, grad2d=None, dparams=None, stream=None, dyn=None, lighting=None):
    torch = _torch()
    n = params.shape[1]
    if grad2d is None:
        grad2d = torch.empty((n_views, n, GRAD2D_STRIDE), dtype=torch.float32, device=params.device)
    if dparams is None:
        dparams = torch.empty_like(params)
    sc = _scene(params, sh_degree, dyn, None, lighting)
    check("gs_render_bwd", _lib.lib().gs_render_bwd(ctx.ptr, C.byref(sc), _ptr(d_cams), n_views, total_tiles,
                                                    _ptr(proj), _ptr(sorted_vals), _ptr(ranges), _bg(bg),
                                                    _ptr(T_final), _ptr(n_contrib), _ptr(dimage), _ptr(grad2d),
                                                    _ptr(dparams), _stream(stream)))
    return grad2d, dparams


def adam_cfg(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, step=1, d_step=None, increment=False):
    cfg = _lib.gs_adam_cfg()
    lrs = np.broadcast_to(np.asarray(lr, dtype=np.float32), (60,))
    for i in range(60):
        cfg.lr[i] = float(lrs[i])
    cfg.beta1, cfg.beta2, cfg.eps, cfg.step = beta1, beta2, eps, step
    cfg.d_step = d_step.data_ptr() if d_step is not None else None
    cfg.increment = int(bool(increment))
    return cfg


def gs_adam_step(ctx, theta, grad, m, v, cfg, stream=None):
    check("gs_adam_step", _lib.lib().gs_adam_step(ctx.ptr, _ptr(theta), _ptr(grad), _ptr(m), _ptr(v),
                                                  theta.shape[1], C.byref(cfg), _stream(stream)))


def gs_extract_delta(ctx, theta, baseline, thr=1e-3, d_idx=None, d_records=None, d_count=None, stream=None):
    torch = _torch()
    n = theta.shape[1]
    dev = theta.device
    if d_idx is None:
        d_idx = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    if d_records is None:
        d_records = torch.empty((max(n, 1), RECORD_BYTES), dtype=torch.uint8, device=dev)
    if d_count is None:
        d_count = torch.zeros(1, dtype=torch.int32, device=dev)
    check("gs_extract_delta", _lib.lib().gs_extract_delta(ctx.ptr, _ptr(theta), _ptr(baseline), n, float(thr),
                                                          _ptr(d_idx), _ptr(d_records), _ptr(d_count),
                                                          _stream(stream)))
    return d_idx, d_records, d_count


# attribute groups of tensor deltas (GS_ATTR_* in include/gs.h)
ATTR = {"mean": 1, "opacity": 2, "scale": 4, "rotation": 8, "dc": 16, "sh_rest": 32}


def tensor_record_bytes(attr) -> int:
    a = ATTR[attr] if isinstance(attr, str) else int(attr)
    return int(_lib.lib().gs_tensor_record_bytes(a))


def gs_extract_tensor_delta(ctx, theta, baseline, attr, thr=1e-3, d_idx=None, d_vals=None, d_count=None,
                            stream=None):
    """-> (d_idx, d_vals, d_count): the group's changed Gaussians (GS_ATTR_*)."""
    torch = _torch()
    a = ATTR[attr] if isinstance(attr, str) else int(attr)
    n = theta.shape[1]
    rb = tensor_record_bytes(a)
    if rb < 0:
        check("gs_extract_tensor_delta", _lib.GS_ERR_ARG)  # not one GS_ATTR_* group
    dev = theta.device
    if d_idx is None:
        d_idx = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    if d_vals is None:
        d_vals = torch.empty((max(n, 1), rb), dtype=torch.uint8, device=dev)
    if d_count is None:
        d_count = torch.zeros(1, dtype=torch.int32, device=dev)
    check("gs_extract_tensor_delta", _lib.lib().gs_extract_tensor_delta(
        ctx.ptr, _ptr(theta), _ptr(baseline), n, a, float(thr), _ptr(d_idx), _ptr(d_vals), _ptr(d_count),
        _stream(stream)))
    return d_idx, d_vals, d_count


def gs_apply_tensor_delta(ctx, params, attr, d_idx, d_vals, d_count, stream=None):
    a = ATTR[attr] if isinstance(attr, str) else int(attr)
    check("gs_apply_tensor_delta", _lib.lib().gs_apply_tensor_delta(
        ctx.ptr, _ptr(params), params.shape[1], a, _ptr(d_idx), _ptr(d_vals), _ptr(d_count), _stream(stream)))
    return params


def gs_apply_delta(ctx, params, d_records, d_count, stream=None):
    check("gs_apply_delta", _lib.lib().gs_apply_delta(ctx.ptr, _ptr(params), params.shape[1], _ptr(d_records),
                                                      _ptr(d_count), _stream(stream)))
    return params


def gs_render_batch(ctx, params, sh_degree, d_cams, n_requests, total_tiles, keys_cap, npix, bg=None,
                    image=None, stream=None, dyn=None, precull=None, lighting=None, host_cams=None):
    """host_cams (the cameras of d_cams, packed or as a dict): render through
    gs_render_batch_sized, which plans the tiles and super-tiles from them
    (total_tiles is then not used)."""
    torch = _torch()
    if image is None:
        image = torch.empty(3 * npix, dtype=torch.float32, device=params.device)
    sc = _scene(params, sh_degree, dyn, precull, lighting)
    if host_cams is not None:
        packed, host = _host_cams(host_cams)
        if len(packed) != n_requests:
            raise ValueError("host_cams must hold the n_requests cameras of d_cams")
        check("gs_render_batch_sized", _lib.lib().gs_render_batch_sized(ctx.ptr, C.byref(sc), _ptr(d_cams), host,
                                                                        n_requests, keys_cap, _bg(bg), _ptr(image),
                                                                        _stream(stream)))
        return image
    check("gs_render_batch", _lib.lib().gs_render_batch(ctx.ptr, C.byref(sc), _ptr(d_cams), n_requests,
                                                        total_tiles, keys_cap, _bg(bg), _ptr(image),
                                                        _stream(stream)))
    return image


def gs_autotune(ctx, params, sh_degree, cams, keys_cap, reps=3, stream=None, dyn=None, lighting=None):
    """Time the render/adjoint path over the tunables (gs_autotune) and leave
    `ctx` set to the fastest: binning and sort settings by their time outside
    compositing, the compositing and adjoint layouts each on its own.  Returns
    (chosen, entries): chosen is ctx.tuning(); entries are dicts with binning,
    sort_bits, sort_items, raster_threads, ms, ms_render_fwd, ms_render_bwd."""
    packed, host = _host_cams(cams)
    V = len(packed)
    d_cams = cameras_to_device(packed, params.device)
    out = (_lib.gs_tune_entry * 64)()
    cnt = C.c_int32(0)
    sc = _scene(params, sh_degree, dyn, None, lighting)
    check("gs_autotune", _lib.lib().gs_autotune(ctx.ptr, C.byref(sc), _ptr(d_cams), host, V, int(keys_cap),
                                                int(reps), out, 64, C.byref(cnt), _stream(stream)))
    names = {v: k for k, v in BINNING.items()}
    entries = [{"binning": names[e.binning], "sort_bits": e.sort_bits, "sort_items": e.sort_items,
                "raster_threads": e.raster_threads, "ms": float(e.ms), "ms_render_fwd": float(e.ms_render_fwd),
                "ms_render_bwd": float(e.ms_render_bwd)} for e in out[:cnt.value]]
    chosen = ctx.tuning()
    ctx.binning, ctx.raster_threads = chosen["binning"], chosen["raster_threads"]
    ctx.raster_bwd_threads = chosen["raster_bwd_threads"]
    return chosen, entries


def train_io(params, grads, m, v, baseline, targets, image, d_loss, d_idx, d_records, d_count, d_step, frozen=None):
    io = _lib.gs_train_io(*(t.data_ptr() for t in (params, grads, m, v, baseline, targets, image, d_loss,
                                                   d_idx, d_records, d_count, d_step)))
    if frozen is not None and frozen.shape[1] > 0:
        io.frozen = frozen.data_ptr()
    return io


def train_cfg(n, sh_degree, n_views, width, height, keys_cap, w_l1=0.8, w_ssim=0.2, bg=(0.0, 0.0, 0.0),
              delta_thr=1e-3, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, dyn: "Dynamics | None" = None,
              n_frozen: int = 0, precull: "Precull | None" = None, lighting: "Lighting | None" = None,
              phases: int = 0):
    """gs_train_cfg; phases: _lib.TRAIN_GRADIENT, TRAIN_UPDATE or TRAIN_ALL (0 = all)."""
    cfg = _lib.gs_train_cfg()
    cfg.n_frozen = int(n_frozen)
    cfg.phases = int(phases)
    if lighting is not None:
        cfg.lighting = C.pointer(lighting.struct)
    if precull is not None:
        cfg.precull = C.pointer(precull.struct)
    if dyn is not None:
        cfg.dyn = C.pointer(dyn.struct)
    cfg.n, cfg.sh_degree, cfg.n_views, cfg.width, cfg.height = n, sh_degree, n_views, width, height
    cfg.keys_cap, cfg.w_l1, cfg.w_ssim, cfg.delta_thr = keys_cap, w_l1, w_ssim, delta_thr
    for i in range(3):
        cfg.bg[i] = bg[i]
    cfg.adam = adam_cfg(lr, beta1, beta2, eps)
    return cfg


def gs_train_step(ctx, d_cams, io, cfg, stream=None):
    check("gs_train_step", _lib.lib().gs_train_step(ctx.ptr, _ptr(d_cams), C.byref(io), C.byref(cfg),
                                                    _stream(stream)))


def gs_train_graph_capture(ctx, d_cams, io, cfg, stream=None):
    check("gs_train_graph_capture", _lib.lib().gs_train_graph_capture(ctx.ptr, _ptr(d_cams), C.byref(io),
                                                                      C.byref(cfg), _stream(stream)))


def gs_graph_launch(ctx, stream=None):
    check("gs_graph_launch", _lib.lib().gs_graph_launch(ctx.ptr, _stream(stream)))
