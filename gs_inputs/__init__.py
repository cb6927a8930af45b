"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module draws random numbers and lays them out; it holds none of the
method's arithmetic (no projection, shading, compositing, loss or update).

The paper's scenes are live renders of a private Unity scene (Sec. 4.1), which
is not available; these seeded scenes stand in for them at the Gaussian counts
and camera rigs of the paper's experiments (Table 1: 208K-453K Gaussians,
4-8 reference cameras on a circle around the content, Sec. 4.2.1).

Parameter layout (one float32 array ``[15, n, 4]``, "planes"):

* plane 0: mean x, y, z, opacity logit
* plane 1: log-scale x, y, z, 0 (pad)
* plane 2: rotation quaternion (w, x, y, z), not normalised
* planes 3..14: 48 spherical-harmonics coefficients, coefficient ``k``
  (0..15, order l = 0..3, m = -l..l) of colour channel ``c`` at flat index
  ``3 * k + c``; flat index ``j`` lives in plane ``3 + j // 4``, lane ``j % 4``.

Cameras are returned as a dict of float64/int arrays (world-to-camera rotation
``R`` [V,3,3] and translation ``t`` [V,3], pinhole ``fx, fy, cx, cy``,
``width, height`` and ``near``), with x right, y down and +z forward.
"""
from __future__ import annotations

import math

import numpy as np

N_PLANES = 15
N_SH = 16
# 1 / (2 sqrt(pi)): the value of the degree-0 real spherical harmonic.  Used
# only to state the input distribution "degree-0 colour ~ N(0.5, 0.2)" as a
# distribution of the stored DC coefficient.
_Y00 = 0.5 / math.sqrt(math.pi)

SEED_MODEL = 0
SEED_TARGET = 1
SEED_CAMERAS = 2
SEED_SERVING = 3


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def make_scene(n: int, sh_degree: int, seed: int = SEED_MODEL,
               sh_std: float = 0.2) -> np.ndarray:
    """A seeded Gaussian set as float32 planes ``[15, n, 4]``.

    means ~ U[-1, 1]^3, log-scales ~ N(-4, 0.5), quaternions ~ N(0, 1)^4
    (normalised here so they are unit on input; the method normalises again),
    opacity logits ~ N(0, 1), degree-0 colour ~ N(0.5, 0.2) per channel stored
    as its DC coefficient, higher coefficients ~ N(0, sh_std) up to
    ``sh_degree`` and zero beyond it.
    """
    if not 0 <= sh_degree <= 3:
        raise ValueError("sh_degree must be in 0..3")
    rng = _rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(n, 3))
    log_s = rng.normal(-4.0, 0.5, size=(n, 3))
    quat = rng.normal(0.0, 1.0, size=(n, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    logit = rng.normal(0.0, 1.0, size=(n,))
    rgb = rng.normal(0.5, 0.2, size=(n, 3))
    sh = np.zeros((n, N_SH, 3))
    sh[:, 0, :] = (rgb - 0.5) / _Y00
    n_used = (sh_degree + 1) ** 2
    if n_used > 1:
        sh[:, 1:n_used, :] = rng.normal(0.0, sh_std, size=(n, n_used - 1, 3))
    flat = np.zeros((n, 60))
    flat[:, 0:3] = means
    flat[:, 3] = logit
    flat[:, 4:7] = log_s
    flat[:, 8:12] = quat
    flat[:, 12:60] = sh.reshape(n, 48)
    return np.ascontiguousarray(
        flat.reshape(n, N_PLANES, 4).transpose(1, 0, 2)).astype(np.float32)


def planes_to_rows(planes: np.ndarray) -> np.ndarray:
    """``[15, n, 4]`` planes -> ``[n, 60]`` rows (a transpose, nothing else)."""
    p = np.asarray(planes)
    return np.ascontiguousarray(p.transpose(1, 0, 2).reshape(p.shape[1], 60))


def rows_to_planes(rows: np.ndarray) -> np.ndarray:
    r = np.asarray(rows)
    return np.ascontiguousarray(r.reshape(r.shape[0], N_PLANES, 4).transpose(1, 0, 2))


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)):
    """World-to-camera (R, t) for a camera at ``eye`` looking at ``target``.

    Camera axes: x right, y down, z forward (towards the target)."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ eye
    return R, t


def _pinhole(width: int, height: int, fov_x_deg: float):
    fx = width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    return fx, fx, width / 2.0, height / 2.0


def cameras_from_eyes(eyes, widths, heights, fov_x_deg: float = 60.0,
                      near: float = 0.2, targets=None) -> dict:
    V = len(eyes)
    R = np.zeros((V, 3, 3))
    t = np.zeros((V, 3))
    fx = np.zeros(V); fy = np.zeros(V); cx = np.zeros(V); cy = np.zeros(V)
    for i, e in enumerate(eyes):
        tgt = (0.0, 0.0, 0.0) if targets is None else targets[i]
        R[i], t[i] = look_at(e, tgt)
        fx[i], fy[i], cx[i], cy[i] = _pinhole(int(widths[i]), int(heights[i]), fov_x_deg)
    return {"R": R, "t": t, "fx": fx, "fy": fy, "cx": cx, "cy": cy,
            "width": np.asarray(widths, dtype=np.int64),
            "height": np.asarray(heights, dtype=np.int64),
            "near": np.full(V, near)}


def ring_cameras(n_views: int, width: int, height: int, radius: float = 3.0,
                 fov_x_deg: float = 60.0, near: float = 0.2) -> dict:
    """``n_views`` cameras on a ring of ``radius`` in the y = 0 plane at angles
    2*pi*k/V, all looking at the origin; view 0 sits at (0, 0, radius)."""
    eyes = [(radius * math.sin(2 * math.pi * k / n_views), 0.0,
             radius * math.cos(2 * math.pi * k / n_views)) for k in range(n_views)]
    return cameras_from_eyes(eyes, [width] * n_views, [height] * n_views,
                             fov_x_deg, near)


def subset_cameras(cams: dict, idx) -> dict:
    idx = np.atleast_1d(np.asarray(idx))
    return {k: np.asarray(v)[idx] for k, v in cams.items()}


def drift_signs(n: int, seed: int = SEED_TARGET + 100) -> np.ndarray:
    """Fixed per-element signs (+1/-1) for the drifting target set, as planes
    ``[15, n, 4]``; the pad lane of plane 1 is 0."""
    s = _rng(seed).integers(0, 2, size=(N_PLANES, n, 4)).astype(np.float32) * 2 - 1
    s[1, :, 3] = 0.0
    return s


# ---------------------------------------------------------------- serving
SERVING_RESOLUTIONS = ((1280, 720), (1920, 1080), (1440, 1600))
STEREO_HALF_IPD = 0.032


def serving_requests(n_requests: int, rate_hz: float, n_clients: int = 64,
                     seed: int = SEED_SERVING, ring_radius: float = 3.0,
                     jitter: float = 0.3):
    """Poisson arrivals of forward-only render requests.

    Each of ``n_clients`` clients issues a Poisson process; the merged stream
    has rate ``rate_hz``.  Resolution is uniform over the three classes; the
    1440x1600 class is one eye of a stereo pair (eye offset +-0.032 along the
    camera's x axis).  The eye is a ring point plus a uniform offset in a ball
    of radius ``jitter``.  Returns a list of dicts with ``t_arrival`` (s),
    ``client``, ``width``, ``height`` and ``eye``.
    """
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    t = np.cumsum(gaps)
    out = []
    for i in range(n_requests):
        w, h = SERVING_RESOLUTIONS[int(rng.integers(0, 3))]
        ang = rng.uniform(0.0, 2 * math.pi)
        base = np.array([ring_radius * math.sin(ang), 0.0, ring_radius * math.cos(ang)])
        while True:
            o = rng.uniform(-1.0, 1.0, size=3)
            if o @ o <= 1.0:
                break
        eye = base + jitter * o
        if h == 1600:
            R, _ = look_at(eye)
            eye = eye + (1 if rng.integers(0, 2) else -1) * STEREO_HALF_IPD * R[0]
        out.append({"t_arrival": float(t[i]), "client": int(rng.integers(0, n_clients)),
                    "width": w, "height": h, "eye": eye})
    return out


# ---------------------------------------------------------------- dynamics
def rigid_groups(n: int, n_groups: int = 16) -> np.ndarray:
    """Group id of Gaussian i is i mod n_groups (uint8)."""
    return (np.arange(n) % n_groups).astype(np.uint8)


def unit_normals(n: int, seed: int = SEED_MODEL + 10) -> np.ndarray:
    v = _rng(seed).normal(size=(n, 3))
    return (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)


def frame_poses(n_frames: int, n_groups: int = 16, max_deg_per_frame: float = 2.0,
                amplitude: float = 0.1, period: int = 120, seed: int = SEED_MODEL + 20) -> np.ndarray:
    """Absolute object poses for frames 0..n_frames-1, float64 [F, G, 8]
    (unit quaternion w, x, y, z; translation x, y, z; 0).

    Group g spins about a fixed uniform axis at a rate U[0.25, 1] x
    max_deg_per_frame degrees per frame, and its translation follows
    amplitude * sin(2 pi f / period + phase_g) along a fixed uniform direction,
    so frame 0 is near identity and the objects stay within the camera ring."""
    rng = _rng(seed)
    axis = rng.normal(size=(n_groups, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    rate = np.radians(rng.uniform(0.25, 1.0, size=n_groups) * max_deg_per_frame)
    direc = rng.normal(size=(n_groups, 3))
    direc /= np.linalg.norm(direc, axis=1, keepdims=True)
    phase = rng.uniform(0.0, 2 * math.pi, size=n_groups)
    f = np.arange(n_frames)[:, None]
    ang = rate[None, :] * f
    out = np.zeros((n_frames, n_groups, 8))
    out[..., 0] = np.cos(ang / 2)
    out[..., 1:4] = np.sin(ang / 2)[..., None] * axis[None]
    out[..., 4:7] = (amplitude * (np.sin(2 * math.pi * f / period + phase[None]) - np.sin(phase[None])))[..., None] \
        * direc[None]
    return out


def light_directions(n_frames: int, zenith_deg: float = 45.0, step_deg: float = 1.0):
    """Directional light at a fixed zenith angle whose azimuth turns by
    ``step_deg`` per frame (unit vectors pointing towards the light, +y up)."""
    z = math.radians(zenith_deg)
    out = np.zeros((n_frames, 3))
    for f in range(n_frames):
        a = math.radians(step_deg * f)
        out[f] = (math.sin(z) * math.cos(a), math.cos(z), math.sin(z) * math.sin(a))
    return out
