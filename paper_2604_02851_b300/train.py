"""Online optimiser: the server-side refit loop of Sec. 3.1 / 3.2.3.

The paper's optimiser thread "iterates over ready reference cameras,
optionally grouping them as mini batches, renders the present Gaussian model
from those viewpoints, compares the result to the captured ground-truth
images, and updates the trainable Gaussian parameters" (Sec. 3.1), and the
changed Gaussians stream out as tensor deltas (Sec. 3.5).

``OnlineTrainer.step()`` runs one whole step over all reference views as one
CUDA-graph launch of ``gs_train_step`` (all views batched in every kernel).
``OnlineTrainer.step_plain()`` is the unbatched reference point: per view,
separate launches of projection, binning (with a host read of the key count),
compositing, loss and both adjoints, then Adam and delta extraction.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import (Context, RECORD_BYTES, GRAD2D_STRIDE, PROJ_STRIDE, _lib, _ptr, _stream, adam_cfg,
               cameras_to_device, check, gs_adam_step, gs_bin_sort, gs_extract_delta, gs_loss,
               gs_project, gs_project_bwd, gs_raster_bwd, gs_render_fwd, pack_cameras, train_cfg, train_io)


class OnlineTrainer:
    def __init__(self, params, sh_degree: int, cams: dict, keys_cap: int, lr=1e-3, w_l1=0.8, w_ssim=0.2,
                 delta_thr=1e-3, bg=(0.0, 0.0, 0.0), tile=16, sort_bits=8, ctx: Context | None = None,
                 dyn=None, share: "OnlineTrainer | None" = None, frozen=None, precull=None, lighting=None,
                 phases: int = 0):
        """share: another trainer of the same model whose gradient, Adam
        moments, delta baseline and step counter this one uses (a second
        graph slot with its own targets, image and delta outputs).
        frozen: planes [15][m][4] of an inference-only pool (Sec. 3.3,
        Gaussian freezing): rendered with `params`, never updated; gradients,
        Adam state and deltas cover `params` only.
        precull: a Precull grid (Sec. 3.3): Gaussians of culled cells are not
        rendered and keep their parameters and Adam state this step.
        lighting: a Lighting (Sec. 3.4.1): colours are the SH-lighting
        product, attenuated by its per-Gaussian light visibility.
        phases: the parts of the step that step() runs (_lib.TRAIN_GRADIENT,
        TRAIN_UPDATE, TRAIN_ALL; 0 = all); step_update() runs the update alone."""
        import torch
        self.torch = torch
        self.params = params
        self.n = n = params.shape[1]
        self.sh = sh_degree
        self.cams = cams
        self.packed = pack_cameras(cams)
        self.V = V = len(self.packed)
        self.W, self.H = int(self.packed["width"][0]), int(self.packed["height"][0])
        if not (np.all(self.packed["width"] == self.W) and np.all(self.packed["height"] == self.H)):
            raise ValueError("all reference views of a step share one resolution")
        self.keys_cap = int(keys_cap)
        self.lr, self.w_l1, self.w_ssim, self.delta_thr, self.bg = lr, w_l1, w_ssim, delta_thr, tuple(bg)
        dev = params.device
        self.ctx = ctx or Context(dev.index or 0, 0, tile=tile, sort_bits=sort_bits)
        self.frozen = frozen
        self.n_frozen = 0 if frozen is None else int(frozen.shape[1])
        self.ctx.reserve(self.ctx.workspace_size(self.packed, n + self.n_frozen, self.keys_cap))
        self.d_cams = cameras_to_device(self.packed, dev)
        self.total_tiles = self.ctx.total_tiles(self.packed)
        self.npix = V * self.W * self.H
        f32 = dict(dtype=torch.float32, device=dev)
        if share is not None:
            self.grads, self.m, self.v, self.baseline = share.grads, share.m, share.v, share.baseline
        else:
            self.grads = torch.zeros_like(params)
            self.m = torch.zeros_like(params)
            self.v = torch.zeros_like(params)
            self.baseline = params.clone()
        self.targets = torch.zeros(3 * self.npix, **f32)
        self.image = torch.zeros(3 * self.npix, **f32)
        self.d_loss = torch.zeros(1, **f32)
        self.d_idx = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
        self.d_records = torch.zeros((max(n, 1), RECORD_BYTES), dtype=torch.uint8, device=dev)
        self.d_count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.d_step = share.d_step if share is not None else torch.ones(1, dtype=torch.int32, device=dev)
        self.io = train_io(params, self.grads, self.m, self.v, self.baseline, self.targets, self.image,
                           self.d_loss, self.d_idx, self.d_records, self.d_count, self.d_step, frozen=frozen)
        self.dyn = dyn  # kept alive: the step reads its device buffers
        self.precull = precull
        self.lighting = lighting
        self.cfg = train_cfg(n, sh_degree, V, self.W, self.H, self.keys_cap, w_l1, w_ssim, self.bg, delta_thr, lr,
                             dyn=dyn, n_frozen=self.n_frozen, precull=precull, lighting=lighting, phases=phases)
        self.cfg_update = train_cfg(n, sh_degree, V, self.W, self.H, self.keys_cap, w_l1, w_ssim, self.bg, delta_thr,
                                    lr, dyn=dyn, n_frozen=self.n_frozen, precull=precull, lighting=lighting,
                                    phases=_lib.TRAIN_UPDATE)
        self._captured = False
        self._events = None
        self._plain = None

    # ------------------------------------------------------------ batched step
    def capture(self, stream=None, phase_events=None):
        """Capture the whole step into a CUDA graph (optionally with phase
        events recorded by every replay)."""
        if phase_events is not None:
            for e in phase_events:  # torch creates the CUDA event on its first record
                e.record()
            self.torch.cuda.synchronize()
            if any(not e.cuda_event for e in phase_events):
                raise RuntimeError("phase events must be timing-enabled CUDA events")
            arr = (C.c_void_p * len(phase_events))(*[e.cuda_event for e in phase_events])
            self._events = (phase_events, arr)
            check("gs_train_graph_capture_events",
                  _lib.lib().gs_train_graph_capture_events(self.ctx.ptr, _ptr(self.d_cams), C.byref(self.io),
                                                           C.byref(self.cfg), arr, _stream(stream)))
        else:
            check("gs_train_graph_capture",
                  _lib.lib().gs_train_graph_capture(self.ctx.ptr, _ptr(self.d_cams), C.byref(self.io),
                                                    C.byref(self.cfg), _stream(stream)))
        self._captured = True

    def step(self, stream=None):
        if not self._captured:
            self.capture(stream)
        check("gs_graph_launch", _lib.lib().gs_graph_launch(self.ctx.ptr, _stream(stream)))

    def step_eager(self, stream=None):
        """The same batched step without the graph (one launch sequence)."""
        check("gs_train_step", _lib.lib().gs_train_step(self.ctx.ptr, _ptr(self.d_cams), C.byref(self.io),
                                                        C.byref(self.cfg), _stream(stream)))

    def step_update(self, stream=None):
        """The update part alone (Adam on self.grads, delta extraction, step
        counter), without a graph: a few launches."""
        check("gs_train_step", _lib.lib().gs_train_step(self.ctx.ptr, _ptr(self.d_cams), C.byref(self.io),
                                                        C.byref(self.cfg_update), _stream(stream)))

    # ------------------------------------------------------------ plain step
    def _plain_buffers(self):
        if self._plain is None:
            torch = self.torch
            dev = self.params.device
            pv = {}
            for v in range(self.V):
                one = self.packed[v:v + 1]
                pv[v] = {"cams": cameras_to_device(one, dev), "tt": self.ctx.total_tiles(one)}
            self._plain = {
                "views": pv,
                "proj": torch.empty((1, self.n, PROJ_STRIDE), dtype=torch.float32, device=dev),
                "grad2d": torch.empty((1, self.n, GRAD2D_STRIDE), dtype=torch.float32, device=dev),
                "vals": torch.empty(self.keys_cap, dtype=torch.int32, device=dev),
                "ranges": torch.empty((max(x["tt"] for x in pv.values()), 2), dtype=torch.int32, device=dev),
                "nk": torch.zeros(1, dtype=torch.int32, device=dev),
                "T": torch.empty(self.W * self.H, dtype=torch.float32, device=dev),
                "nc": torch.empty(self.W * self.H, dtype=torch.int32, device=dev),
                "dimg": torch.empty(3 * self.W * self.H, dtype=torch.float32, device=dev),
                "loss": torch.zeros(self.V, dtype=torch.float32, device=dev),
                "step": 0,
            }
        return self._plain

    def step_plain(self, stream=None) -> float:
        """One view per launch sequence, host read of each view's key count."""
        if self.n_frozen:
            raise ValueError("the plain step has no frozen pool")
        b = self._plain_buffers()
        HW = self.W * self.H
        for v in range(self.V):
            pv = b["views"][v]
            gs_project(self.ctx, self.params, self.sh, pv["cams"], 1, proj=b["proj"], stream=stream, dyn=self.dyn)
            gs_bin_sort(self.ctx, b["proj"], pv["cams"], 1, self.n, pv["tt"], self.keys_cap, sorted_vals=b["vals"],
                        ranges=b["ranges"], d_num_keys=b["nk"], want_keys=False, stream=stream)
            k = int(b["nk"].item())  # host read of the key count
            if k > self.keys_cap:
                raise RuntimeError(f"key capacity {self.keys_cap} below {k}")
            img_v = self.image[3 * HW * v:3 * HW * (v + 1)]
            gs_render_fwd(self.ctx, b["proj"], pv["cams"], 1, self.n, pv["tt"], b["vals"], b["ranges"], HW,
                          bg=self.bg, image=img_v, T_final=b["T"], n_contrib=b["nc"], stream=stream)
            gs_loss(self.ctx, img_v, self.targets[3 * HW * v:3 * HW * (v + 1)], 1, self.H, self.W,
                    self.w_l1 / self.V, self.w_ssim / self.V, d_loss=b["loss"][v:v + 1], dimage=b["dimg"],
                    stream=stream)
            gs_raster_bwd(self.ctx, b["proj"], pv["cams"], 1, self.n, pv["tt"], b["vals"], b["ranges"], b["T"],
                          b["nc"], b["dimg"], bg=self.bg, grad2d=b["grad2d"], stream=stream)
            gs_project_bwd(self.ctx, self.params, self.sh, pv["cams"], 1, b["proj"], b["grad2d"], dparams=self.grads,
                           accumulate=v > 0, stream=stream, dyn=self.dyn)
        b["step"] += 1
        gs_adam_step(self.ctx, self.params, self.grads, self.m, self.v,
                     adam_cfg(self.lr, step=b["step"]), stream=stream)
        gs_extract_delta(self.ctx, self.params, self.baseline, self.delta_thr, d_idx=self.d_idx,
                         d_records=self.d_records, d_count=self.d_count, stream=stream)
        return float(b["loss"].sum().item())

    # ------------------------------------------------------------ results
    def loss(self) -> float:
        return float(self.d_loss.item())

    def delta_count(self) -> int:
        return int(self.d_count.item())

    def raise_status(self):
        self.ctx.raise_status()


class StreamingTrainer:
    """The server loop with host I/O overlapped (Sec. 3.1, 3.5): reference
    images arrive in host memory, changed-Gaussian records leave to host
    memory.  Two graph slots share one model (parameters, Adam state, delta
    baseline, step counter) and alternate: while slot k % 2 computes step k,
    the copy stream uploads the targets of step k + 1 into the other slot and
    the records of step k - 1 come back.  Steps run in order on one compute
    stream, so the result equals the one-slot loop.

    `make_ctx()` returns a fresh Context configured like the first slot's."""

    def __init__(self, params, sh_degree: int, cams: dict, keys_cap: int, make_ctx, dyn=None, **kw):
        import torch
        self.torch = torch
        self.slots = [OnlineTrainer(params, sh_degree, cams, keys_cap, ctx=make_ctx(), dyn=dyn, **kw)]
        self.slots.append(OnlineTrainer(params, sh_degree, cams, keys_cap, ctx=make_ctx(), dyn=dyn,
                                        share=self.slots[0], **kw))
        dev = params.device
        self.compute = torch.cuda.Stream(device=dev)
        self.h2d = torch.cuda.Stream(device=dev)
        self.d2h = torch.cuda.Stream(device=dev)
        n = self.slots[0].n
        self.host_loss = [torch.empty(1, dtype=torch.float32).pin_memory() for _ in range(2)]
        self.host_cnt = [torch.empty(1, dtype=torch.int32).pin_memory() for _ in range(2)]
        self.host_rec = [torch.empty((max(n, 1), RECORD_BYTES), dtype=torch.uint8).pin_memory() for _ in range(2)]
        self.h2d_bytes = 0
        self.d2h_bytes = 0

    def capture(self):
        for t in self.slots:
            t.capture(self.compute)
        self.torch.cuda.synchronize()

    def run(self, host_targets, steps: int, on_delta=None):
        """Run `steps` steps; host_targets(k) gives step k's targets as a
        pinned host tensor (planar [V][3][H][W] floats).  on_delta(k, loss,
        count, records) receives each step's outputs in host memory (the
        records view is valid during the call).  Returns the loss of the last
        step.

        Step k + 1's upload is queued right after step k is launched and
        starts when step k - 1 (the last user of that slot's targets) ends,
        so it overlaps all of step k; the read-backs of step k - 1 are
        queued on the (in-order) read-back stream before those of step k."""
        torch = self.torch
        Ev = torch.cuda.Event
        slot_free = [Ev(), Ev()]       # the slot's records have been copied out
        uploaded = [Ev(), Ev()]
        done = [Ev(), Ev()]            # the slot's step (and its reads of the targets) ended
        counted = [Ev(), Ev()]
        for e in slot_free + done:
            e.record(self.compute)
        last_loss = None

        def upload(k):
            s = k % 2
            t = self.slots[s]
            src = host_targets(k)
            with torch.cuda.stream(self.h2d):
                self.h2d.wait_event(done[s])
                t.targets.copy_(src, non_blocking=True)
                uploaded[s].record(self.h2d)
            self.h2d_bytes += t.targets.numel() * 4

        def drain(k):
            nonlocal last_loss
            s = k % 2
            counted[s].synchronize()
            m = int(self.host_cnt[s].item())
            with torch.cuda.stream(self.d2h):
                if m:
                    self.host_rec[s][:m].copy_(self.slots[s].d_records[:m], non_blocking=True)
                slot_free[s].record(self.d2h)
            slot_free[s].synchronize()
            self.d2h_bytes += 8 + m * RECORD_BYTES
            last_loss = float(self.host_loss[s].item())
            if on_delta is not None:
                on_delta(k, last_loss, m, self.host_rec[s][:m])

        if steps:
            upload(0)
        for k in range(steps):
            s = k % 2
            t = self.slots[s]
            self.compute.wait_event(uploaded[s])
            self.compute.wait_event(slot_free[s])
            t.step(self.compute)
            done[s].record(self.compute)
            if k + 1 < steps:
                upload(k + 1)
            # step k - 1's records go out before step k's read-backs are queued
            # on the (in-order) read-back stream, so they do not wait for step k
            if k >= 1:
                drain(k - 1)
            with torch.cuda.stream(self.d2h):
                self.d2h.wait_event(done[s])
                self.host_loss[s].copy_(t.d_loss, non_blocking=True)
                self.host_cnt[s].copy_(t.d_count, non_blocking=True)
                counted[s].record(self.d2h)
        if steps:
            drain(steps - 1)
        return last_loss

    def raise_status(self):
        for t in self.slots:
            t.raise_status()


def estimate_keys(ctx: Context, params, sh_degree: int, cams, slack: float = 1.25, dyn=None) -> int:
    """Key count of one bin/sort of the current model (through the C ABI,
    with the scene's current object poses when `dyn` is given), scaled by
    `slack` to leave room for the model to move."""
    import torch
    packed = cams if isinstance(cams, np.ndarray) else pack_cameras(cams)
    V = len(packed)
    n = params.shape[1]
    d_cams = cameras_to_device(packed, params.device)
    tt = ctx.total_tiles(packed)
    cap = 1 << 20
    while True:
        ctx.reserve(ctx.workspace_size(packed, n, cap))
        proj = gs_project(ctx, params, sh_degree, d_cams, V, dyn=dyn)
        _, vals, ranges, nk = gs_bin_sort(ctx, proj, d_cams, V, n, tt, cap, want_keys=False)
        torch.cuda.synchronize()
        code, detail = ctx.status()
        if code == 0:
            k = int(nk.item())
            break
        if code != _lib.GS_ERR_CAPACITY:
            raise RuntimeError(f"bin/sort failed with status {code}")
        cap = int(detail * 1.05) + 1024
    del proj, vals, ranges
    return int(k * slack) + 4096
