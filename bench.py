"""Benchmark of the online 3DGS optimisation step (and the oracle reference arm).

Workload (default): 1M Gaussians, SH degree 3, a batch of 8 reference views
of 1280x720 on a ring of radius 3, L1 + 0.2 D-SSIM, Adam (lr 1e-3), delta
extraction (threshold 1e-3) every step, targets drifting by 1e-3 per
parameter per step.  One step = one graph launch of the whole batched step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 GPUs the views of each step are
split over the ranks (rank r renders views r, r + N, ...) and their
gradients are summed by an NCCL all-reduce before every rank runs the same
update (paper_2604_02851_b300.parallel); the throughput is steps of the whole
job over the slowest rank's time.  --parallelism replicas instead runs one
independent model per GPU.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gs_inputs as gi  # noqa: E402

METRIC = "train steps/s (1M Gaussians, 8×720p views, fwd+bwd+Adam); client render p99 ms"
WORKLOADS = {
    # name: (n, sh, views, width, height)
    "c3_1M_8x720p": (1_000_000, 3, 8, 1280, 720),
    "c2_100k_4x512": (100_000, 3, 4, 512, 512),
    "c1_10k_128": (10_000, 0, 1, 128, 128),
    "prof_200k_8x720p": (200_000, 3, 8, 1280, 720),
    "c5_3M_8x1080p_dynamic": (3_000_000, 3, 8, 1920, 1080),
    # the 1M-Gaussian 8 x 720p scene plus 3M Gaussians above it, outside every view (a large
    # world of which the cameras see a part; Sec. 3.3 preculling)
    "c3_far3M_8x720p": (4_000_000, 3, 8, 1280, 720),
}
FAR_WORKLOADS = {"c3_far3M_8x720p": 3_000_000}
DYNAMIC_WORKLOADS = {"c5_3M_8x1080p_dynamic"}
DEFAULT_WORKLOAD = "c3_1M_8x720p"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# FP32 operations per unit of work, counted from the kernels' source (FMA = 2;
# an ex2 / rcp, a min and a compare count 1 each).  Unit: one (pixel,
# fragment) evaluation up to the pixel's last contributor, counted as a full
# evaluation (pairs below the alpha cut-off stop after the exponent, so this
# is an upper bound on the work done).
#   compositing: offset 1, exponent 2 FMA + penalty 1, test 1, ex2 + scale 2,
#     min 1, 1 - alpha and T update 3, weight 1, three colour FMAs 6 = 20
#   adjoint: offset 1, exponent 2 FMA, test 1, ex2 + scale 2, min 1,
#     1 - alpha 2, rcp + T 2, weight 1, three colour-gradient FMAs 6,
#     dL/dC . (c - R) 7, dL/dalpha 1, X update 2, clamp select + dL/dP 2,
#     dL/dP dx 1 and the sums of dL/dP, dL/dP dx, dL/dP dx^2 4 = 37
RASTER_FWD_FLOP_PER_FRAGMENT = 20
RASTER_BWD_FLOP_PER_FRAGMENT = 37
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(sm_count: int, sm_mhz: float) -> float:
    """FP32 peak of the device at a clock: SMs x 128 FP32 lanes x 2 (FMA) x clock."""
    return sm_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def phase_model(n, V, K, total_tiles, npix, sum_nc, n_changed, binning, passes, Kc, chunks, n_train=None,
                depth_passes=4):
    """Algorithmic bytes (HBM) or FLOPs per launch of each phase.

    K fine (tile, Gaussian) entries; two-level binning moves Kc coarse
    (super-tile, Gaussian) entries through `passes` radix passes and writes
    the chunk bitmaps (2 KB per chunk); direct binning moves the K entries
    through `passes` passes; the depth sort runs `depth_passes` passes."""
    vn = V * n
    nt = n if n_train is None else n_train  # Gaussians that are trained (the active pool)
    if binning == "two_level":
        # the training step stops at the chunk bitmaps (2 KB per chunk)
        emit = vn * (8 + 4) + Kc * 8
        sort = Kc * 16 * passes + Kc * 8 + chunks * 2048
    else:
        emit = vn * (8 + 4) + K * 8
        sort = K * (16 * (passes - 1) + 12) + total_tiles * 16
    return {
        # parameters read; per (view, Gaussian) the 48-byte record of the
        # fused step, the 8-byte depth-sort item and the 4-byte tile rectangle
        # written
        "project": ("hbm", n * 240 + vn * (48 + 8 + 4)),
        # the key histogram reads 4 bytes, each pass reads and writes an
        # 8-byte item
        "depth_sort": ("hbm", vn * (depth_passes * 16 + 4)),
        "emit": ("hbm", emit),
        "tile_sort": ("hbm", sort),
        "render_fwd": ("alu", sum_nc * RASTER_FWD_FLOP_PER_FRAGMENT),
        "loss": ("hbm", 3 * npix * 44),
        "raster_bwd": ("alu", sum_nc * RASTER_BWD_FLOP_PER_FRAGMENT),
        "project_bwd": ("hbm", nt * 480 + V * nt * (48 + 32)),
        # Adam fused with the delta's changed test: theta, grad, m, v, baseline
        # read, theta, m, v written, one flag byte out
        "adam": ("hbm", 60 * nt * 4 * 8 + nt),
        # the records: block sums scanned, flags read, per changed Gaussian
        # theta re-read, index, record and baseline written
        "delta": ("hbm", nt + n_changed * (240 + 4 + 128 + 240)),
    }


def delta_bytes(n, n_changed):
    """Algorithmic bytes of one gs_extract_delta: theta and baseline read
    (2 x 240 B per Gaussian), per changed Gaussian the index, the 128-byte
    record and the rewritten baseline (240 B)."""
    return n * 480 + n_changed * (4 + 128 + 240)


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum of the
# kernel in one ncu capture), valid while the kernel's source file is
# unchanged (first 12 hex digits of its SHA-1).
MEASURED_TRAFFIC = {
    ("c3_1M_8x720p", "k_raster_bwd"): (277.7e6, "csrc/raster.cu", "4fb8691de8db"),
}

# Warp instructions per (pixel, fragment) evaluation of a raster kernel
# (smsp__inst_executed.sum of one launch over its sum of n_contrib, one ncu
# capture of the 200k-Gaussian, 8 x 720p case), valid while the kernel's
# source file is unchanged: with this run's sum of n_contrib it gives the
# kernel's instructions per launch for the issue-slot roofline.
MEASURED_INSTRUCTIONS = {
    "k_raster_bwd": (937934239 / 890192530, "csrc/raster.cu", "4fb8691de8db"),
}


def _source_unchanged(src, sha):
    import hashlib
    path = os.path.join(ROOT, "paper_2604_02851_b300", src)
    try:
        with open(path, "rb") as f:
            return hashlib.sha1(f.read()).hexdigest()[:12] == sha
    except OSError:
        return False


def measured_traffic(workload, kernel):
    ent = MEASURED_TRAFFIC.get((workload, kernel))
    if ent is None:
        return None
    nbytes, src, sha = ent
    return nbytes if _source_unchanged(src, sha) else None


def issue_roofline(kernel, sum_nc, ms, sm_count, sm_mhz):
    """Issue-slot roofline of a raster kernel: its warp instructions per
    launch (the measured per-fragment budget x this run's fragments) over its
    time, against SMs x 4 schedulers x 1 instruction a cycle."""
    ent = MEASURED_INSTRUCTIONS.get(kernel)
    if ent is None or not _source_unchanged(ent[1], ent[2]):
        return None
    inst = ent[0] * sum_nc
    ach = inst / (ms / 1e3) / 1e9
    peak = sm_count * 4 * sm_mhz / 1e3
    return {"achieved": ach, "peak": peak, "unit": "G warp instructions/s", "frac": ach / peak,
            "warp_instructions": inst,
            "source": "warp instructions per (pixel, fragment) from one ncu capture (smsp__inst_executed.sum / "
                      "sum of n_contrib, 200k Gaussians, 8 x 720p) x this run's sum of n_contrib"}


# phases that are one kernel (plus negligible set-up launches), by kernel name
SINGLE_KERNEL_PHASES = {"project": "k_project", "emit": "k_emit", "render_fwd": "k_render_fwd",
                        "raster_bwd": "k_raster_bwd", "project_bwd": "k_project_bwd", "adam": "k_adam_flags"}


def gpu_launches_per_step(binning, passes):
    """Kernels of one train step, counted from the launch sequence: view
    table, projection, depth sort (count, histogram, look-back clear, scan,
    4 passes), emission and sort (two-level: emission, fine total, ranges
    init, look-back clear, scan, passes, ranges fix, chunk table, chunk
    owners, bitmaps;
    direct: emission, ranges init, look-back clear, scan, passes, ranges
    fix), compositing, loss (2), adjoints (2), Adam with the delta's changed
    test and the step counter (2), delta scan and records (2)."""
    depth = 8
    sort = (9 + passes) if binning == "two_level" else (5 + passes)
    return 1 + 1 + depth + sort + 1 + 2 + 1 + 1 + 2 + 2


def replica_seeds(rank: int):
    """Seeds of rank r's replica: each rank trains its own model (independent
    problems, no data-path collective)."""
    return gi.SEED_MODEL + 1000 * rank, gi.SEED_TARGET + 1000 * rank


def replica_throughput(my_ms: float, steps: int, world: int, device):
    """Whole-job throughput of `world` replicas: the slowest rank's time for
    its `steps` steps (MAX over ranks), and world * steps over that time."""
    import torch
    t = torch.tensor([my_ms], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    total_ms = float(t.item())
    return total_ms, world * steps / (total_ms / 1e3)


def depth_passes(torch, proj, V, n):
    """Radix passes the depth sort runs on a projection: three when the
    visible Gaussians' keys (the float bits of their depths) span fewer than
    2^24 - 1 values, since it then orders key - smallest key, else four."""
    b = proj.view(torch.int32).view(V * n, 16)
    vis = b[:, 14] > 0
    if not bool(vis.any().item()):
        return 4
    k = b[:, 2][vis].to(torch.int64) & 0xFFFFFFFF
    return 3 if int((k.max() - k.min()).item()) < 0xFFFFFF else 4


def coarse_work(torch, proj, V, n):
    """Super-tile entries of a projection (a work count for the roofline)."""
    b = proj.view(torch.int32).view(V * n, 16)
    lo = b[:, 12].to(torch.int64) & 0xFFFFFFFF
    hi = b[:, 13].to(torch.int64) & 0xFFFFFFFF
    vis = b[:, 14] > 0
    x0, y0, x1, y1 = lo & 0xFFFF, lo >> 16, hi & 0xFFFF, hi >> 16
    per = ((((x1 - 1) >> 3) - (x0 >> 3) + 1) * (((y1 - 1) >> 3) - (y0 >> 3) + 1)) * vis
    return int(per.sum().item())


_CUDART = None


def event_ms(a, b) -> float:
    """cudaEventElapsedTime on two torch events' handles (graph-recorded
    events are not known to torch's own bookkeeping)."""
    import ctypes
    global _CUDART
    if _CUDART is None:
        for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
            try:
                _CUDART = ctypes.CDLL(name)
                break
            except OSError:
                continue
        _CUDART.cudaEventElapsedTime.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_void_p, ctypes.c_void_p]
    ms = ctypes.c_float()
    rc = _CUDART.cudaEventElapsedTime(ctypes.byref(ms), ctypes.c_void_p(a.cuda_event), ctypes.c_void_p(b.cuda_event))
    if rc != 0:
        raise RuntimeError(f"cudaEventElapsedTime failed ({rc})")
    return float(ms.value)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.strip().split(",") for r in open(self.f.name) if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1])); mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for nm, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle leg
class OracleSampler:
    """Times the FP64 oracle on bounded samples of one optimisation step.

    A sample takes one view and one 16-row band of it: projection of every
    Gaussian for that band's camera, binning, compositing, loss, both
    adjoints.  The mean band time is scaled by the bands per view and the
    views per step; Adam is timed on a slice of the parameters and scaled to
    all of them."""

    def __init__(self, n, sh, V, W, H, seed_offset=0, dynamic=False, relight=False):
        import oracle as O
        self.O = O
        self.dyn = None
        if dynamic:
            # the scene at frame 1 of the dynamic workload (poses, light, normals)
            self.dyn = {"group": gi.rigid_groups(n, 16), "poses": gi.frame_poses(2, 16)[1],
                        "normals": gi.unit_normals(n), "light": gi.light_directions(2)[1],
                        "ambient": 0.3, "diffuse": 0.7}
        if relight:
            # SH-lighting product with every Gaussian lit (the map is not sampled)
            L = np.zeros(56)
            L[:48] = relight_env().reshape(48)
            L[48:51] = gi.light_directions(2)[1]
            L[52:55] = RELIGHT_RADIANCE
            self.dyn = {"sh_light": L}
            if dynamic:
                self.dyn.update(group=gi.rigid_groups(n, 16), poses=gi.frame_poses(2, 16)[1])
        self.n, self.sh, self.V, self.W, self.H = n, sh, V, W, H
        self.planes = gi.planes_to_rows(gi.make_scene(n, sh, gi.SEED_MODEL + seed_offset)).astype(np.float64)
        self.target_planes = gi.planes_to_rows(gi.make_scene(n, sh, gi.SEED_TARGET + seed_offset)).astype(np.float64)
        self.cams = gi.ring_cameras(V, W, H)
        self.bands = math.ceil(H / 16)
        self.k = 0
        self.t_adam = None

    def _band_cam(self, k):
        v, b = k % self.V, (k * 7) % self.bands
        cam = gi.subset_cameras(self.cams, [v])
        cam["height"] = np.array([min(16, self.H - 16 * b)])
        cam["cy"] = cam["cy"] - 16 * b
        return cam

    def sample(self) -> float:
        cam = self._band_cam(self.k)
        self.k += 1
        tgt = self.O.forward(self.target_planes, self.sh, cam, dyn=self.dyn)["image"]  # reference view, not timed
        t0 = time.perf_counter()
        self.O.loss_and_grad(self.planes, self.sh, cam, tgt, dyn=self.dyn)
        return time.perf_counter() - t0

    def adam_seconds(self) -> float:
        if self.t_adam is None:
            m = min(self.n * 60, 2_000_000)
            th = np.zeros(m); g = np.random.default_rng(0).normal(size=m)
            mm = np.zeros(m); vv = np.zeros(m)
            t0 = time.perf_counter()
            self.O.adam(th, g, mm, vv, 1e-3, 1)
            self.t_adam = (time.perf_counter() - t0) * (self.n * 60 / m)
            self.adam_floats = m
        return self.t_adam

    def step_seconds(self, band_times) -> float:
        return float(np.mean(band_times)) * self.bands * self.V + self.adam_seconds()

    def describe(self, samples) -> str:
        self.adam_seconds()
        return (f"estimated from band samples: {samples} samples of one 16-row band of one view (all {self.n} "
                f"Gaussians projected, binned, composited, loss + both adjoints, FP64), scaled x{self.bands} bands "
                f"x{self.V} views; Adam on {self.adam_floats} floats scaled to {self.n * 60}")


RELIGHT_RADIANCE = (1.0, 0.95, 0.9)
RELIGHT_MAP = 2048          # light-space depth map, texels per side
RELIGHT_EXTENT = 4.0        # world units the map covers (the scene and its motion)


def relight_env():
    """Seeded world-frame environment SH [16][3]: a positive ambient term and
    small higher bands."""
    env = np.random.default_rng(gi.SEED_MODEL + 30).normal(0.0, 0.1, (16, 3))
    env[0] = 1.0
    return env


def omp_cores():
    try:
        return int(os.environ.get("OMP_NUM_THREADS", "")) or os.cpu_count()
    except ValueError:
        return os.cpu_count()


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, same metric and workload.
    Each step is a bounded sample sized so that warmup + steps end within a
    few minutes; under torchrun only rank 0 runs."""
    if rank != 0:
        return
    n, sh, V, W, H = WORKLOADS[args.workload]
    smp = OracleSampler(n, sh, V, W, H, dynamic=args.workload in DYNAMIC_WORKLOADS, relight=args.relight)
    one = smp.sample()
    budget_s = 150.0
    # one band sample is the smallest unit; when the requested steps do not
    # all fit in the budget, the steps share the samples that do
    total = max(1, min(args.steps + args.warmup, int(budget_s / max(one, 1e-3))))
    warm = min(args.warmup, max(0, total - 1)) if total > args.steps else min(args.warmup, total // 4)
    for _ in range(warm):
        smp.sample()
    times = []
    t0 = time.perf_counter()
    for _ in range(max(1, total - warm)):
        times.append(smp.sample())
    wall = time.perf_counter() - t0
    step_s = smp.step_seconds(times)
    value = 1.0 / step_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "gaussians": n, "sh_degree": sh, "views": V,
                       "resolution": [W, H]},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": omp_cores(), "kind": "oracle",
                             "sample": smp.describe(len(times)), "estimated": True, "wall_s": wall},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU leg
def run_sharded(args, rank, world, local_rank):
    """The training step with its views split over the ranks: per step, each
    rank's gradient part (one graph launch over its views), the all-reduce of
    the gradient, the update (the same on every rank).  Strong scaling: every
    step covers all views of the workload whatever the number of ranks."""
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300 import parallel
    from paper_2604_02851_b300.train import estimate_keys

    if args.frozen_frac > 0 or args.precull or args.relight or args.workload in FAR_WORKLOADS:
        raise SystemExit("view sharding runs the plain or dynamic workloads (no freezing, preculling or relighting)")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n, sh, V, W, H = WORKLOADS[args.workload]
    views = parallel.shard_views(V, world, rank)
    cams = gi.ring_cameras(V, W, H)
    sub = parallel.subset_cameras(cams, views)
    # one model, replicated on every rank
    params = torch.from_numpy(gi.make_scene(n, sh, gi.SEED_MODEL)).to(dev)
    tparams = torch.from_numpy(gi.make_scene(n, sh, gi.SEED_TARGET)).to(dev)
    dynamic = args.workload in DYNAMIC_WORKLOADS
    drift = None if dynamic else torch.from_numpy(gi.drift_signs(n)).to(dev) * 1e-3
    frames = max(args.steps, 1) + args.warmup + args.e2e_steps + 16
    dyn = None
    if dynamic:
        poses = gi.frame_poses(frames, 16)
        lights = gi.light_directions(frames)
        dyn = gs.Dynamics(gi.rigid_groups(n, 16), poses[0], gi.unit_normals(n), lights[0], 0.3, 0.7, device=dev)
    frame = [0]

    def make_ctx():
        return gs.Context(local_rank, 0, tile=args.tile, sort_bits=args.sort_bits, sort_items=args.sort_items,
                          binning=args.binning, raster_threads=args.raster_threads,
                          raster_bwd_threads=args.raster_bwd_threads)
    ctx = make_ctx()
    keys_cap = estimate_keys(ctx, params, sh, sub, slack=1.3, dyn=dyn)
    if args.autotune:
        ctx.reserve(ctx.workspace_size(sub, n, keys_cap))
        best, _ = gs.gs_autotune(ctx, params, sh, sub, keys_cap, reps=2, dyn=dyn)
        args.binning, args.sort_bits = best["binning"], best["sort_bits"]
        args.sort_items, args.raster_threads = best["sort_items"], best["raster_threads"]
        args.raster_bwd_threads = best["raster_bwd_threads"]
    st = parallel.ViewShardedTrainer(params, sh, cams, keys_cap, rank, world, ctx=ctx, dyn=dyn)
    tr = st.trainer
    tctx = make_ctx()
    tctx.reserve(tctx.workspace_size(sub, n, keys_cap))

    def next_targets():
        if dynamic:
            frame[0] = (frame[0] + 1) % frames
            dyn.set_frame(poses[frame[0]], lights[frame[0]])
        else:
            tparams.add_(drift)
        gs.gs_render_batch(tctx, tparams, sh, tr.d_cams, len(views), tr.total_tiles, keys_cap, tr.npix,
                           image=st.targets, dyn=dyn)

    phase_ev = [torch.cuda.Event(enable_timing=True) for _ in range(gs._lib.TRAIN_PHASE_EVENTS)]
    next_targets()
    tr.capture(phase_events=phase_ev)
    for _ in range(args.warmup):
        next_targets()
        st.step()
    torch.cuda.synchronize()
    st.raise_status()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    phase_ms = np.zeros(len(phase_ev) - 1)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    for k in range(args.steps):
        next_targets()
        ev0[k].record()
        st.step()
        ev1[k].record()
        ev1[k].synchronize()
        for i in range(8):  # the gradient part's phases (the update runs outside the graph)
            phase_ms[i] += event_ms(phase_ev[i], phase_ev[i + 1])
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])
    st.raise_status()
    t = torch.tensor([float(step_ms.sum())], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    total_ms = float(t.item())
    value = args.steps / (total_ms / 1e3)
    loss = st.loss()
    phase_avg = {name: float(ms / args.steps) for name, ms in zip(gs._lib.TRAIN_PHASES[:8], phase_ms[:8])}
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2032.0
    fp32_peak = fp32_peak_tflops(sm_count, sm_mhz)
    # work counts of this rank's views, for the dominant kernel's roofline
    proj = gs.gs_project(ctx, params, sh, tr.d_cams, len(views), dyn=dyn)
    _, vals, ranges, nk = gs.gs_bin_sort(ctx, proj, tr.d_cams, len(views), n, tr.total_tiles, keys_cap,
                                         want_keys=False)
    _, T, nc = gs.gs_render_fwd(ctx, proj, tr.d_cams, len(views), n, tr.total_tiles, vals, ranges, tr.npix)
    torch.cuda.synchronize()
    sum_nc = int(nc.to(torch.int64).sum().item())
    del proj, vals, ranges, T, nc
    ach = sum_nc * RASTER_BWD_FLOP_PER_FRAGMENT / (phase_avg["raster_bwd"] / 1e3) / 1e12
    roofline = {"kernel": "k_raster_bwd", "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": None,
                "peak_source": f"derived: {sm_count} SMs (queried) x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                               f"{sm_mhz:.0f} MHz (median sampled)"}
    # end to end: this rank's targets up from pinned host memory, the step,
    # rank 0 reads the loss, the delta count and the records back
    e2e = None
    if args.e2e_steps > 0:
        host = torch.empty(st.targets.numel(), dtype=torch.float32).pin_memory()
        next_targets()
        host.copy_(st.targets)
        h_loss = torch.empty(1, dtype=torch.float32).pin_memory()
        h_cnt = torch.empty(1, dtype=torch.int32).pin_memory()
        h_rec = torch.empty((n, gs.RECORD_BYTES), dtype=torch.uint8).pin_memory()
        h2d = d2h = 0
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.e2e_steps):
            st.targets.copy_(host, non_blocking=True)
            h2d += host.numel() * 4
            st.step()
            lt = tr.d_loss.clone()
            parallel.reduce_gradients(lt)  # the loss of all views: the sum of the ranks' shares
            if rank == 0:
                h_loss.copy_(lt, non_blocking=True)
                h_cnt.copy_(tr.d_count, non_blocking=True)
                torch.cuda.current_stream().synchronize()
                m = int(h_cnt.item())
                if m:
                    h_rec[:m].copy_(tr.d_records[:m], non_blocking=True)
                d2h += 8 + m * gs.RECORD_BYTES
        e1.record()
        torch.cuda.synchronize()
        t = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device=dev)
        if world > 1:
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e = {"value": args.e2e_steps / (float(t.item()) / 1e3), "unit": "steps/s",
               "h2d_bytes_per_step": h2d // args.e2e_steps, "d2h_bytes_per_step": d2h // args.e2e_steps,
               "steps": args.e2e_steps,
               "pipeline": "per step: each rank uploads its views' targets, the sharded step, rank 0 reads back "
                           "the loss and the delta records"}
    tctx.close()
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
               "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": args.workload, "gaussians": n, "sh_degree": sh, "views": V,
                          "views_per_rank": len(views), "resolution": [W, H], "keys_cap": keys_cap,
                          "binning": args.binning, "sort_digit_bits": args.sort_bits, "sort_items": args.sort_items,
                          "raster_threads_per_row": args.raster_threads,
                          "raster_bwd_threads_per_row": args.raster_bwd_threads,
                          "l2": "inputs larger than L2 (params 240 MB, keys > 1 GB per step)",
                          "parallelism": f"views over {world} ranks, NCCL all-reduce of the gradient"},
               "roofline": roofline, "cpu_baseline": None, "clocks": clk, "e2e": e2e,
               "gpu_launches": gpu_launches_per_step(
                   args.binning, math.ceil(math.ceil(math.log2(max(tr.total_tiles, 2))) / args.sort_bits)) * args.steps,
               "phases_ms_rank0_gradient_part": phase_avg, "loss_last": loss}
        print(json.dumps(out), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.train import OnlineTrainer, estimate_keys

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n, sh, V, W, H = WORKLOADS[args.workload]
    # replicas: rank r trains its own seeded model (independent problems)
    seed_model, seed_target = replica_seeds(rank)
    planes = gi.make_scene(n, sh, seed_model)
    target_planes = gi.make_scene(n, sh, seed_target)
    n_far = FAR_WORKLOADS.get(args.workload, 0)
    if n_far:
        # the last n_far Gaussians move to y in [3, 9], above the scene: every
        # view's frustum misses them
        for pl in (planes, target_planes):
            pl[0, n - n_far:, 1] = pl[0, n - n_far:, 1] * 3.0 + 6.0
    signs = gi.drift_signs(n)
    cams = gi.ring_cameras(V, W, H)
    params = torch.from_numpy(planes).to(dev)
    tparams = torch.from_numpy(target_planes).to(dev)
    dynamic = args.workload in DYNAMIC_WORKLOADS
    # static scene: the target set drifts by 1e-3 per parameter per step;
    # dynamic scene: 16 rigid objects move every frame and the light turns
    drift = None if dynamic else torch.from_numpy(signs).to(dev) * 1e-3
    dyn = None
    frames = max(args.steps, 1) + args.warmup + args.e2e_steps + 16
    lights = gi.light_directions(frames)
    frame = [0]
    if dynamic:
        G = 16
        poses = gi.frame_poses(frames, G)
        # relighting by the SH-lighting product replaces the Lambertian DC factor
        normals = None if args.relight else gi.unit_normals(n)
        dyn = gs.Dynamics(gi.rigid_groups(n, G), poses[0], normals, lights[0], 0.3, 0.7, device=dev)
    lighting = tlight = None
    if args.relight:
        # Sec. 3.4.1: SH lighting (environment + directional light turning
        # 1 deg per frame) and a per-Gaussian light visibility from a
        # light-space depth map, recomputed every frame inside the timed step
        lighting = gs.Lighting(n, relight_env(), lights[0], RELIGHT_RADIANCE, device=dev)
        tlight = gs.Lighting(n, relight_env(), lights[0], RELIGHT_RADIANCE, with_visibility=False, device=dev)
        ldepth = torch.empty((RELIGHT_MAP, RELIGHT_MAP), dtype=torch.float32, device=dev)

    ctx = gs.Context(local_rank, 0, tile=args.tile, sort_bits=args.sort_bits, sort_items=args.sort_items,
                     binning=args.binning, raster_threads=args.raster_threads,
                     raster_bwd_threads=args.raster_bwd_threads)
    keys_cap = estimate_keys(ctx, params, sh, cams, slack=1.3, dyn=dyn)
    tuned = None
    if args.autotune:
        # pick binning, digit width, items per thread and raster layout for this
        # workload (gs_autotune); the step graph is captured afterwards
        ctx.reserve(ctx.workspace_size(cams, n, keys_cap))
        best, entries = gs.gs_autotune(ctx, params, sh, cams, keys_cap, reps=2, dyn=dyn, lighting=lighting)
        args.binning, args.sort_bits = best["binning"], best["sort_bits"]
        args.sort_items, args.raster_threads = best["sort_items"], best["raster_threads"]
        args.raster_bwd_threads = best["raster_bwd_threads"]
        worst = max(e["ms"] for e in entries)
        tuned = {"configs_tried": len(entries), "best_ms": min(e["ms"] for e in entries), "worst_ms": worst,
                 "timed": "projection + bin/sort + compositing + its adjoint"}
    frozen = None
    if args.frozen_frac > 0:
        # Gaussian freezing: the last part of the model is an inference-only pool
        na = int(round(n * (1.0 - args.frozen_frac)))
        frozen = params[:, na:].contiguous()
        params = params[:, :na].contiguous()
    precull = None
    if args.precull:
        # grid over the whole world; kept cells from the views' depth buffers
        # (empty here: the frustum decides), computed once for the fixed rig
        precull = gs.Precull((-3.0, -3.0, -3.0), 0.5, (12, 26, 12), device=dev)
        far = torch.full((V * H * W,), float("inf"), dtype=torch.float32, device=dev)
        pctx = gs.Context(local_rank, 0)
        precull.update(pctx, cams, far)
        torch.cuda.synchronize()
        pctx.close()
        del far
    tr = OnlineTrainer(params, sh, cams, keys_cap, ctx=ctx, dyn=dyn, frozen=frozen, precull=precull,
                       lighting=lighting)
    packed = tr.packed
    tctx = gs.Context(local_rank, 0, tile=args.tile, sort_bits=args.sort_bits, sort_items=args.sort_items,
                     binning=args.binning, raster_threads=args.raster_threads,
                     raster_bwd_threads=args.raster_bwd_threads)
    tkeys = estimate_keys(tctx, tparams, sh, cams, slack=1.3, dyn=dyn)
    tctx.reserve(tctx.workspace_size(packed, n, tkeys))

    def next_targets():
        # the engine side: move the scene and render its reference views
        if dynamic or args.relight:
            frame[0] = (frame[0] + 1) % len(lights)
        if dynamic:
            dyn.set_frame(poses[frame[0]], lights[frame[0]])
        else:
            tparams.add_(drift)
        if args.relight:
            lighting.set(direction=lights[frame[0]])
            tlight.set(direction=lights[frame[0]])
        gs.gs_render_batch(tctx, tparams, sh, tr.d_cams, V, tr.total_tiles, tkeys, tr.npix, image=tr.targets,
                           dyn=dyn, lighting=tlight)

    def light_camera():
        return gs.light_camera(direction=lights[frame[0]], width=RELIGHT_MAP, height=RELIGHT_MAP,
                               extent=RELIGHT_EXTENT, alpha_min=0.5, bias=2.0 * RELIGHT_EXTENT / RELIGHT_MAP)

    def update_visibility():
        lighting.update_visibility(tr.ctx, params, light_camera(), ldepth, dyn=dyn, frozen=frozen)

    phase_ev = [torch.cuda.Event(enable_timing=True) for _ in range(gs._lib.TRAIN_PHASE_EVENTS)]
    next_targets()
    tr.capture(phase_events=phase_ev)
    for _ in range(args.warmup):
        next_targets()
        if args.relight:
            update_visibility()
        tr.step()
    torch.cuda.synchronize()
    tr.raise_status()
    tctx.raise_status()

    snapshot = params.clone()  # the model before the timed steps (tensor-delta measurement)
    # the end-to-end run starts from the same model and optimiser state as the
    # timed steps (the cost of a step depends on how far the synthetic model
    # has trained, and fresh Adam moments move every parameter at once)
    e2e_state = None
    if args.e2e_steps > 0:
        e2e_state = {"params": params.clone(), "m": tr.m.clone(), "v": tr.v.clone(),
                     "baseline": tr.baseline.clone(), "step": tr.d_step.clone()}
    # ---- timed region: K steps, device time of each step by CUDA events
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    phase_ms = np.zeros(len(phase_ev) - 1)
    lv_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    vis_ms = 0.0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        next_targets()
        ev0[k].record()
        if args.relight:
            lv_ev[0].record()
            update_visibility()
            lv_ev[1].record()
        tr.step()
        ev1[k].record()
        ev1[k].synchronize()
        for i in range(len(phase_ev) - 1):
            phase_ms[i] += event_ms(phase_ev[i], phase_ev[i + 1])
        if args.relight:
            vis_ms += event_ms(lv_ev[0], lv_ev[1])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])
    code, detail = tr.ctx.status()
    if code != 0:
        raise RuntimeError(f"device status {code} ({detail}) during the timed region")
    total_ms, value = replica_throughput(float(step_ms.sum()), args.steps, world, dev)
    ms_per_step = total_ms / args.steps
    loss_last = tr.loss()
    changed = tr.delta_count()
    phase_avg = {name: float(ms / args.steps) for name, ms in zip(gs._lib.TRAIN_PHASES, phase_ms)}
    relight = None
    if args.relight:
        vis_host = lighting.visibility[:n].cpu().numpy()
        dmap = ldepth.cpu().numpy()
        relight = {"visibility_ms": vis_ms / args.steps, "light_map": [RELIGHT_MAP, RELIGHT_MAP],
                   "extent": RELIGHT_EXTENT, "alpha_min": 0.5, "covered_texels": float(np.isfinite(dmap).mean()),
                   "shadowed_fraction": float((vis_host == 0).mean()),
                   "what": "per frame, inside each timed step: light-space depth map of every Gaussian "
                           "(clear + warp-per-Gaussian splat) and the centre test; the step's projection "
                           "evaluates the SH-lighting product (environment rotated per object + directional "
                           "light x visibility)"}

    # ---- work counts of the current model, for the roofline (outside the timed region)
    wc_params = params if frozen is None else torch.cat([params, frozen], 1)  # every rendered Gaussian
    proj = gs.gs_project(ctx, wc_params, sh, tr.d_cams, V, dyn=dyn, lighting=lighting)
    _, vals, ranges, nk = gs.gs_bin_sort(ctx, proj, tr.d_cams, V, n, tr.total_tiles, keys_cap, want_keys=False)
    _, T, nc = gs.gs_render_fwd(ctx, proj, tr.d_cams, V, n, tr.total_tiles, vals, ranges, tr.npix)
    torch.cuda.synchronize()
    K = int(nk.item())
    sum_nc = int(nc.to(torch.int64).sum().item())
    Kc = coarse_work(torch, proj, V, n)
    dpasses = depth_passes(torch, proj, V, n)
    st_px = args.tile * 8
    n_super = sum(((int(w) + st_px - 1) // st_px) * ((int(h) + st_px - 1) // st_px)
                  for w, h in zip(packed["width"], packed["height"]))
    chunks = Kc // 256 + n_super
    del proj, vals, ranges, T, nc
    tile_passes = math.ceil(math.ceil(math.log2(max(tr.total_tiles, 2))) / args.sort_bits)
    if args.binning == "two_level":
        # the fused step sorts the super-tile key; a key of sort_bits + 1 to
        # 9 bits takes one wide pass
        sbits = math.ceil(math.log2(max(n_super, 2)))
        tile_passes = 1 if args.sort_bits < sbits <= 9 else math.ceil(sbits / args.sort_bits)
    del wc_params
    model = phase_model(n, V, K, tr.total_tiles, tr.npix, sum_nc, changed, args.binning, tile_passes, Kc, chunks,
                        n_train=params.shape[1], depth_passes=dpasses)
    hbm_peak, peak_src = _peaks()
    # FP32 peak from the queried SM count at the median SM clock sampled in the timed region
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2032.0
    fp32_peak = fp32_peak_tflops(sm_count, sm_mhz)
    fp32_src = f"derived: {sm_count} SMs (queried) x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_mhz:.0f} MHz (median sampled)"
    kernels = {}
    for name, ms in phase_avg.items():
        if name not in model:
            # the delta extraction runs inside the Adam kernel: its phase is empty
            kernels[name] = {"ms": ms, "fused_into": "adam"}
            continue
        bound, work = model[name]
        if bound == "hbm":
            ach = work / (ms / 1e3) / 1e9
            kernels[name] = {"ms": ms, "bound": "hbm", "achieved": ach, "unit": "GB/s", "peak": hbm_peak,
                             "frac": ach / hbm_peak, "algorithmic_bytes": work}
        else:
            ach = work / (ms / 1e3) / 1e12
            kernels[name] = {"ms": ms, "bound": "alu", "achieved": ach, "unit": "TFLOP/s",
                             "peak": fp32_peak, "frac": ach / fp32_peak, "algorithmic_flop": work}
    dom = max(SINGLE_KERNEL_PHASES, key=lambda p: phase_avg[p])
    dk = kernels[dom]
    roofline = {"kernel": SINGLE_KERNEL_PHASES[dom], "bound": dk["bound"], "achieved": dk["achieved"],
                "peak": dk["peak"],
                "unit": dk["unit"], "frac": dk["frac"],
                "traffic": measured_traffic(args.workload, SINGLE_KERNEL_PHASES[dom]),
                "peak_source": peak_src if dk["bound"] == "hbm" else fp32_src,
                "issue": issue_roofline(SINGLE_KERNEL_PHASES[dom], sum_nc, phase_avg[dom], sm_count, sm_mhz)
                if dk["bound"] == "alu" else None}

    # ---- tensor deltas per attribute group since the start of the timed steps
    tensor_deltas = measure_tensor_deltas(gs, torch, params, snapshot, _peaks()[0]) if args.tensor_deltas else None
    del snapshot
    # ---- the standalone gs_extract_delta on the changed set of one step
    delta_standalone = measure_delta_standalone(gs, torch, tr, next_targets, hbm_peak) if args.delta_reps else None

    # ---- end to end through the public API: host targets in, loss + delta out
    host_targets = None
    if args.e2e_steps > 0:
        host_targets = []
        for _ in range(2):
            next_targets()
            h = torch.empty(tr.targets.numel(), dtype=torch.float32).pin_memory()
            h.copy_(tr.targets)
            host_targets.append(h)

    # ---- the unbatched reference point: one view per launch sequence
    plain = None
    if args.plain_steps > 0:
        for _ in range(3):
            next_targets()
            tr.step_plain()
        torch.cuda.synchronize()
        pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        plain_ms = 0.0
        for _ in range(args.plain_steps):
            next_targets()
            pe0.record()
            tr.step_plain()
            pe1.record()
            pe1.synchronize()
            plain_ms += pe0.elapsed_time(pe1)
        plain_ms /= args.plain_steps
        plain = {"ms_per_step": plain_ms, "steps": args.plain_steps,
                 "batched_graph_speedup": plain_ms / ms_per_step,
                 "what": "per view: projection, bin/sort with a host read of the key count, compositing, "
                         "loss, both adjoints as separate launches; then Adam and delta"}
    tr.ctx.close()
    tctx.close()
    del tr
    torch.cuda.empty_cache()
    e2e = None
    if args.e2e_steps > 0:
        def make_ctx():
            return gs.Context(local_rank, 0, tile=args.tile, sort_bits=args.sort_bits, sort_items=args.sort_items,
                              binning=args.binning, raster_threads=args.raster_threads,
                     raster_bwd_threads=args.raster_bwd_threads)
        e2e = run_e2e(args, host_targets, e2e_state, sh, cams, keys_cap, make_ctx, dyn, world, lighting)
        del host_targets, e2e_state
    serving = None
    if args.serve_requests > 0:
        torch.cuda.empty_cache()
        serving = run_serving(args, local_rank, rank)

    out = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            smp = OracleSampler(n, sh, V, W, H, dynamic=dynamic, relight=args.relight)
            times = [smp.sample() for _ in range(args.cpu_samples)]
            cpu = {"value": 1.0 / smp.step_seconds(times), "unit": "steps/s", "cores": omp_cores(),
                   "kind": "oracle", "sample": smp.describe(args.cpu_samples)}
        out = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": args.workload, "gaussians": n, "sh_degree": sh, "views": V,
                          "resolution": [W, H], "keys_per_step": K, "coarse_keys_per_step": Kc,
                          "keys_cap": keys_cap, "tile": args.tile, "depth_sort_passes": dpasses,
                          "dynamics": "16 rigid objects, new SE(3) pose per frame (spin <= 2 deg/frame, "
                                      "sinusoidal translation 0.1), light at 45 deg zenith turning 1 deg/frame; "
                                      + ("SH-lighting product with per-Gaussian light visibility"
                                         if args.relight else
                                         "Lambertian relight of the DC term (ambient 0.3, diffuse 0.7)")
                          if dynamic else None,
                          "relight": relight,
                          "sort_digit_bits": args.sort_bits, "sort_items": args.sort_items, "binning": args.binning,
                          "raster_threads_per_row": args.raster_threads,
                          "raster_bwd_threads_per_row": args.raster_bwd_threads, "autotune": tuned,
                          "frozen_fraction": args.frozen_frac, "precull": bool(args.precull),
                          "far_gaussians": n_far,
                          "graph": True,
                          "l2": "inputs larger than L2 (params 240 MB, keys > 1 GB per step)",
                          "targets": "re-rendered each step by gs_render_batch outside the step's events",
                          "parallelism": "replicas" if world > 1 else "single"},
               "roofline": roofline, "cpu_baseline": cpu, "clocks": clk, "e2e": e2e,
               "serving_p99_ms": serving_p99(serving),
               "serving_delivery_p99_ms": serving_p99(serving, "p99_ms"),
               "plain_step": plain, "serving": serving,
               "gpu_launches": (gpu_launches_per_step(args.binning, tile_passes)
                                + (1 + 3 + (2 if frozen is not None else 0) if args.relight else 0)
                                + (1 if frozen is not None else 0)) * args.steps,
               "tensor_deltas": tensor_deltas, "delta_standalone": delta_standalone,
               "phases_ms": phase_avg, "kernels": kernels, "loss_last": loss_last, "delta_changed_last": changed,
               "wall_s_timed_loop": wall}
        print(json.dumps(out), flush=True)
    return out


def serving_p99(serving, key="render_p99_ms"):
    """The p99 render latency (ms: arrival to the image complete in device
    memory) of the 2M-Gaussian serving run at 50 % of saturation (the metric's second
    half), or of the load nearest to it; key="p99_ms": arrival to the image
    in host memory."""
    if not serving or not serving.get("loads"):
        return None
    return min(serving["loads"], key=lambda r: abs(r["load"] - 0.5))[key]


def run_serving(args, local_rank, rank):
    """Serving: forward-only renders of a static 2M-Gaussian SH-3 model for
    64 clients with Poisson arrivals, resolutions mixed 1280x720 / 1920x1080 /
    1440x1600 per eye, eyes within 0.3 of the ring of radius 3; continuous
    batching on 3 slots.  Saturation is measured first with every request
    queued at once; open-loop runs of args.serve_requests requests then offer
    each load in args.serve_loads (fractions of saturation)."""
    import torch
    import paper_2604_02851_b300 as gs
    from paper_2604_02851_b300.serve import RenderServer, Request, measure_keys_per_pixel, percentiles
    dev = torch.device("cuda", local_rank)
    n, sh = 2_000_000, 3
    params = torch.from_numpy(gi.make_scene(n, sh, gi.SEED_SERVING + 1000 * rank)).to(dev)
    probe = gi.cameras_from_eyes([(3.0 * math.sin(a), 0.0, 3.0 * math.cos(a)) for a in (0.3, 2.0)],
                                 [1280, 1920], [720, 1080])
    kpp = measure_keys_per_pixel(params, sh, probe)
    srv = RenderServer(params, sh, kpp, slots=3, max_batch=6, max_pixels_per_batch=6_000_000,
                       memory_budget=64 << 30, slack=1.3)

    def requests(k, rate, seed):
        out = []
        for i, sp in enumerate(gi.serving_requests(k, rate_hz=rate, seed=seed)):
            cams = gi.cameras_from_eyes([sp["eye"]], [sp["width"]], [sp["height"]])
            out.append(Request(rid=i, width=sp["width"], height=sp["height"], cam=gs.pack_cameras(cams),
                               t_arrival=sp["t_arrival"]))
        return out

    srv.run(requests(12, 1e6, gi.SEED_SERVING + 50), realtime=False)  # warm-up
    done, el = srv.run(requests(max(args.serve_requests // 3, 64), 1e6, gi.SEED_SERVING + 51), realtime=False)
    saturation = len(done) / el
    loads = []
    for i, load in enumerate(args.serve_loads):
        rate = load * saturation
        srv.batches = 0
        srv.batch_sizes = []
        srv.launch_while_busy = 0
        srv.max_busy = 0
        retries0 = srv.retries
        done, el = srv.run(requests(args.serve_requests, rate, gi.SEED_SERVING + 52 + i), realtime=True)
        srv.check()
        p50, p99, lat = percentiles(done)
        r50, r99, _ = percentiles(done, rendered=True)
        loads.append({"load": load, "requests": len(done), "offered_rate_hz": rate, "renders_per_s": len(done) / el,
                      "render_p50_ms": r50, "render_p99_ms": r99, "p50_ms": p50, "p99_ms": p99,
                      "batches": srv.batches,
                      "mean_batch": float(np.mean(srv.batch_sizes)) if srv.batch_sizes else 0.0,
                      "max_slots_busy": srv.max_busy, "batches_started_while_busy": srv.launch_while_busy,
                      "capacity_retries": srv.retries - retries0})
    res = {"model": "2M Gaussians, SH3", "clients": 64, "saturation_renders_per_s": saturation, "slots": 3,
           "loads": loads, "latency": "render_*: arrival to the image complete in device memory; p50/p99: "
                                     "arrival to the image (float32, planar) in pinned host memory"}
    del srv, params
    torch.cuda.empty_cache()
    return res


def measure_delta_standalone(gs, torch, tr, next_targets, hbm_peak, reps=10):
    """gs_extract_delta on the inputs of one training step's delta: the
    parameters after one more step and the transmitted baseline before it
    (so the same changed set as the step's fused extraction).  Timed with
    CUDA events per call; the baseline is restored between calls outside
    the events."""
    b0 = tr.baseline.clone()
    next_targets()
    tr.step()
    torch.cuda.synchronize()
    fused_m = tr.delta_count()
    n = tr.params.shape[1]
    ctx = gs.Context(tr.params.device.index or 0, 1 << 26)
    base = b0.clone()
    idx = torch.empty(max(n, 1), dtype=torch.int32, device=tr.params.device)
    rec = torch.empty((max(n, 1), 128), dtype=torch.uint8, device=tr.params.device)
    cnt = torch.zeros(1, dtype=torch.int32, device=tr.params.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for r in range(reps + 2):
        base.copy_(b0)
        e0.record()
        gs.gs_extract_delta(ctx, tr.params, base, tr.delta_thr, d_idx=idx, d_records=rec, d_count=cnt)
        e1.record()
        e1.synchronize()
        if r >= 2:
            times.append(e0.elapsed_time(e1))
    ctx.raise_status()
    m = int(cnt.item())
    ctx.close()
    ms = float(np.median(times))
    work = delta_bytes(n, m)
    ach = work / (ms / 1e3) / 1e9
    return {"ms": ms, "changed": m, "changed_by_fused_step": fused_m, "bound": "hbm", "achieved": ach,
            "unit": "GB/s", "peak": hbm_peak, "frac": ach / hbm_peak, "algorithmic_bytes": work,
            "kernels": "k_delta_flags + k_scan_sums + k_delta_emit", "reps": reps}


TENSOR_GROUPS = (("mean", 0, 3, 4), ("opacity", 3, 4, 2), ("scale", 4, 7, 2), ("rotation", 8, 12, 2),
                 ("dc", 12, 15, 2), ("sh_rest", 15, 60, 2))


def measure_tensor_deltas(gs, torch, params, snapshot, hbm_peak, reps=5):
    """Per attribute group: extraction of the changes since `snapshot` and
    their client-side replay, timed with CUDA events (outside the timed
    steps).  Algorithmic bytes: the group's planes of theta and baseline read
    (16 B per plane per Gaussian each), index + record written and the
    baseline planes rewritten per sent Gaussian; replay reads index + record
    and rewrites the group's planes per sent Gaussian."""
    n = params.shape[1]
    ctx = gs.Context(params.device.index or 0, 1 << 26)
    out = {}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for name, lo, hi, width in TENSOR_GROUPS:
        planes = (hi - 1) // 4 - lo // 4 + 1
        rb = (hi - lo) * width
        base = snapshot.clone()
        idx, vals, cnt = gs.gs_extract_tensor_delta(ctx, params, base, name)
        torch.cuda.synchronize()
        m = int(cnt.item())
        ms_x = ms_a = 0.0
        client = snapshot.clone()
        for _ in range(reps):
            base.copy_(snapshot)
            ev[0].record()
            gs.gs_extract_tensor_delta(ctx, params, base, name, d_idx=idx, d_vals=vals, d_count=cnt)
            ev[1].record()
            gs.gs_apply_tensor_delta(ctx, client, name, idx, vals, cnt)
            ev[2].record()
            ev[2].synchronize()
            ms_x += ev[0].elapsed_time(ev[1]) / reps
            ms_a += ev[1].elapsed_time(ev[2]) / reps
        bx = n * planes * 32 + m * (4 + rb + planes * 16)
        ba = m * (4 + rb + planes * 32)
        out[name] = {"sent": m, "record_bytes": rb, "extract_ms": ms_x, "apply_ms": ms_a,
                     "extract_frac_hbm": bx / (ms_x / 1e3) / 1e9 / hbm_peak,
                     "apply_frac_hbm": ba / (ms_a / 1e3) / 1e9 / hbm_peak if ms_a > 0 else None}
    ctx.raise_status()
    ctx.close()
    return out


def run_e2e(args, host_targets, state, sh, cams, keys_cap, make_ctx, dyn, world, lighting=None):
    """The same metric through the public API with host buffers: every step
    uploads its targets from pinned host memory and returns its loss, delta
    count and delta records to pinned host memory.  The copies overlap the
    compute of the neighbouring steps (StreamingTrainer); the timed region
    runs from the first upload to the last record read-back."""
    import torch
    from paper_2604_02851_b300.train import StreamingTrainer
    st = StreamingTrainer(state["params"], sh, cams, keys_cap, make_ctx, dyn=dyn, lighting=lighting)
    # continue from the device-timed run's starting point: moments, baseline
    # and step counter (the slots share them)
    s0 = st.slots[0]
    s0.m.copy_(state["m"])
    s0.v.copy_(state["v"])
    s0.baseline.copy_(state["baseline"])
    s0.d_step.copy_(state["step"])
    st.capture()
    st.run(lambda k: host_targets[k % 2], 3)  # warm-up
    torch.cuda.synchronize()
    st.h2d_bytes = st.d2h_bytes = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st.h2d)
    st.compute.wait_event(e0)
    st.d2h.wait_event(e0)
    st.run(lambda k: host_targets[k % 2], args.e2e_steps)
    e1.record(st.d2h)
    torch.cuda.synchronize()
    st.raise_status()
    ms = e0.elapsed_time(e1)
    out = {"value": world * args.e2e_steps / (ms / 1e3), "unit": "steps/s",
           "h2d_bytes_per_step": st.h2d_bytes // args.e2e_steps, "d2h_bytes_per_step": st.d2h_bytes // args.e2e_steps,
           "steps": args.e2e_steps, "pipeline": "two graph slots; uploads and read-backs overlap compute",
           "model": "the model and optimiser state before the device-timed steps"}
    for t in st.slots:
        t.ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--sort-bits", type=int, default=8)
    ap.add_argument("--sort-items", type=int, default=16)
    ap.add_argument("--binning", choices=("two_level", "direct"), default="two_level")
    ap.add_argument("--raster-threads", type=int, choices=(2, 4), default=4)
    ap.add_argument("--raster-bwd-threads", type=int, choices=(2, 4), default=None,
                    help="threads per pixel row of the compositing adjoint (default: --raster-threads)")
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="choose binning / sort / raster settings with gs_autotune before timing")
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="steps of the end-to-end measurement (-1: as many as --steps)")
    ap.add_argument("--cpu-samples", type=int, default=12)
    ap.add_argument("--plain-steps", type=int, default=10)
    ap.add_argument("--serve-requests", type=int, default=10_000, help="requests per offered load (0: no serving)")
    ap.add_argument("--serve-loads", type=lambda x: [float(v) for v in x.split(",")], default=[0.25, 0.5, 0.9],
                    help="offered loads as fractions of the measured saturation, comma separated")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precull", action="store_true",
                    help="preculling grid (Sec. 3.3): Gaussians outside the views' cells are not processed")
    ap.add_argument("--frozen-frac", type=float, default=0.0,
                    help="fraction of the model held in the inference-only (frozen) pool")
    ap.add_argument("--relight", action="store_true",
                    help="SH-lighting product and per-frame light visibility (Sec. 3.4.1) in every step")
    ap.add_argument("--parallelism", choices=("auto", "views", "replicas"), default="auto",
                    help="N > 1 GPUs: split each step's views over the ranks (auto, views) or run one model per "
                         "GPU (replicas); views also forces the split path on one GPU")
    ap.add_argument("--delta-reps", type=int, default=10,
                    help="time the standalone gs_extract_delta on one step's changed set (0: skip)")
    ap.add_argument("--tensor-deltas", action=argparse.BooleanOptionalAction, default=True,
                    help="time per-attribute tensor-delta extraction and replay after the timed steps")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.e2e_steps < 0:
        args.e2e_steps = args.steps
    if args.raster_bwd_threads is None:
        args.raster_bwd_threads = args.raster_threads

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1 or args.parallelism == "views":
        import torch
        torch.distributed.init_process_group("nccl")
    if args.parallelism == "views" or (world > 1 and args.parallelism == "auto"):
        run_sharded(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
