"""Continuous-batching render server for client viewpoints.

Sec. 3.1 / 3.5: clients render the streamed Gaussian model locally from the
viewpoint of the camera that tracks the user.  Serving many such viewpoints
from one device-resident model is done here with continuous batching:

* requests queue on arrival;
* each of S slots (own CUDA stream, context, workspace and output buffer)
  runs one batch at a time: all its requests, whatever their resolutions, in
  one gs_render_batch launch sequence (projection, binning/sort and
  compositing of every view), followed by the copy of each image to pinned
  host memory;
* whenever a slot is free, requests waiting at that moment are admitted into
  its next batch while the batch's memory estimate fits the slot's workspace
  and the server's budget, so work that arrives while other batches are on
  the device starts as soon as a slot and memory free up, and batches on
  different slots overlap on the GPU.

Two latencies are measured from a request's arrival: to the moment its image
is complete in device memory (the render, what a client displaying it waits
for) and to the moment it is in pinned host memory (delivery over the host
link).  Results do not depend on batch composition: each view's key
order, tile lists and pixels are computed independently of the other views.
"""
from __future__ import annotations

import gc
import time
from dataclasses import dataclass, field

import numpy as np

from . import Context, cameras_to_device, gs_render_batch, pack_cameras


@dataclass
class Request:
    rid: int
    width: int
    height: int
    cam: np.ndarray            # packed gs_camera record (1 element)
    t_arrival: float
    t_done: float = -1.0       # image in pinned host memory
    t_rendered: float = -1.0   # image complete in device memory
    image: object = None       # pinned host tensor [3, H, W] when done
    keys_est: int = 0
    bytes_est: int = 0


@dataclass
class _Slot:
    ctx: Context
    stream: object
    image: object              # device output buffer
    host: object               # pinned host buffer of the same size
    ws_bytes: int
    event: object = None
    rendered: object = None    # event after the render, before the host copy
    t_rendered: float = -1.0
    batch: list = field(default_factory=list)
    offsets: list = field(default_factory=list)


class RenderServer:
    """Forward-only renders of a static model for many client viewpoints."""

    def __init__(self, params, sh_degree: int, keys_per_pixel: float, slots: int = 3, max_batch: int = 6,
                 max_pixels_per_batch: int = 6_000_000, memory_budget: int = 48 << 30, slack: float = 1.3,
                 bg=(0.0, 0.0, 0.0), keep_images: bool = False):
        import torch
        self.torch = torch
        self.params = params
        self.n = params.shape[1]
        self.sh = sh_degree
        self.kpp = float(keys_per_pixel)
        self.slack = slack
        self.max_batch = max_batch
        self.max_pixels = max_pixels_per_batch
        self.budget = memory_budget
        self.bg = bg
        self.keep_images = keep_images
        dev = params.device
        self.slots = []
        # workspace per slot: sized for the largest admissible batch
        k_cap = int(self.kpp * self.max_pixels * slack) + 65536
        probe = pack_cameras({"R": np.eye(3)[None], "t": np.zeros((1, 3)), "fx": [1.0], "fy": [1.0], "cx": [0.0],
                              "cy": [0.0], "width": [1920], "height": [1600], "near": [0.2]})
        self.keys_cap_slot = k_cap
        for _ in range(slots):
            ctx = Context(dev.index or 0, 0)
            many = np.repeat(probe, max_batch)
            ws = ctx.workspace_size(many, self.n, k_cap)
            ctx.reserve(ws)
            self.slots.append(_Slot(ctx=ctx, stream=torch.cuda.Stream(device=dev),
                                    image=torch.empty(3 * self.max_pixels, dtype=torch.float32, device=dev),
                                    host=torch.empty(3 * self.max_pixels, dtype=torch.float32).pin_memory(),
                                    ws_bytes=ws))
        self.in_flight_bytes = 0
        self.batches = 0
        self.batch_sizes = []
        self.max_busy = 0          # most slots seen running at once
        self.retries = 0           # batches rendered again after a key-capacity overflow
        self._start = None
        self.launch_while_busy = 0  # batches started while another slot was running

    def estimate(self, req: Request) -> None:
        px = req.width * req.height
        req.keys_est = int(self.kpp * px * self.slack) + 4096
        req.bytes_est = self.n * 80 + req.keys_est * 24 + px * 16

    # ------------------------------------------------------------ scheduling
    def _launch(self, slot: _Slot, reqs, keys: int | None = None) -> None:
        torch = self.torch
        cams = np.concatenate([r.cam for r in reqs])
        tt = slot.ctx.total_tiles(cams)
        npix = sum(r.width * r.height for r in reqs)
        if keys is None:
            keys = min(self.keys_cap_slot, sum(r.keys_est for r in reqs))
        with torch.cuda.stream(slot.stream):
            d_cams = cameras_to_device(cams, self.params.device)
            gs_render_batch(slot.ctx, self.params, self.sh, d_cams, len(reqs), tt, keys, npix, bg=self.bg,
                            image=slot.image, stream=slot.stream, host_cams=cams)
            rendered = torch.cuda.Event()
            rendered.record(slot.stream)
            slot.host[:3 * npix].copy_(slot.image[:3 * npix], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
        offs, off = [], 0
        for r in reqs:
            offs.append(off)
            off += 3 * r.width * r.height
        busy = sum(1 for x in self.slots if x.event is not None)
        if busy:
            self.launch_while_busy += 1
        self.max_busy = max(self.max_busy, busy + 1)
        slot.event = ev
        slot.rendered = rendered
        slot.t_rendered = -1.0
        slot.batch = list(reqs)
        slot.offsets = offs
        slot.d_cams = d_cams
        self.in_flight_bytes += sum(r.bytes_est for r in reqs)
        self.batches += 1
        self.batch_sizes.append(len(reqs))

    def _complete(self, slot: _Slot, now: float) -> list:
        # a key count above the batch's estimate leaves truncated lists: render
        # the batch again with the count the device reported, and raise the
        # estimate for later requests
        code, detail = slot.ctx.status(slot.stream)
        if code == 2 and detail <= self.keys_cap_slot:
            est = sum(r.keys_est for r in slot.batch)
            self.slack *= max(1.0, 1.1 * detail / max(est, 1))
            self.retries += 1
            reqs = slot.batch
            self.in_flight_bytes -= sum(r.bytes_est for r in reqs)
            self.batches -= 1
            self.batch_sizes.pop()
            self._launch(slot, reqs, keys=min(self.keys_cap_slot, int(detail * 1.05) + 4096))
            slot.event.synchronize()
            now = max(now, time.perf_counter() - self._start) if self._start is not None else now
            code, detail = slot.ctx.status(slot.stream)
        if code != 0:
            raise RuntimeError(f"render batch failed on the device: status {code} ({detail})")
        done = []
        t_rendered = slot.t_rendered if slot.t_rendered >= 0 else now
        for r, off in zip(slot.batch, slot.offsets):
            r.t_done = now
            r.t_rendered = t_rendered
            if self.keep_images:
                m = 3 * r.width * r.height
                r.image = slot.host[off:off + m].numpy().reshape(3, r.height, r.width).copy()
            done.append(r)
        self.in_flight_bytes -= sum(r.bytes_est for r in slot.batch)
        slot.batch, slot.offsets, slot.event, slot.rendered = [], [], None, None
        return done

    def _admit(self, queue) -> list:
        """Requests from the head of the queue that fit one batch."""
        batch, px, mem = [], 0, 0
        while queue and len(batch) < self.max_batch:
            r = queue[0]
            p = r.width * r.height
            if batch and (px + p > self.max_pixels or self.in_flight_bytes + mem + r.bytes_est > self.budget):
                break
            if not batch and self.in_flight_bytes + r.bytes_est > self.budget and self.in_flight_bytes > 0:
                break
            batch.append(queue.pop(0))
            px += p
            mem += r.bytes_est
        return batch

    def run(self, requests, realtime: bool = True, t0: float | None = None):
        """Serve `requests` (sorted by t_arrival, seconds relative to start).
        With realtime=True arrivals follow the wall clock; otherwise every
        request is queued at time 0 (a closed, saturating load).  Returns the
        completed requests and the elapsed seconds."""
        for r in requests:
            self.estimate(r)
        # the loop allocates events and small tensors per batch; a cyclic
        # garbage collection pass in the middle of a burst would stall every
        # queued request, so collection waits until the run ends (reference
        # counting still frees everything the loop drops)
        gc_was_on = gc.isenabled()
        gc.disable()
        try:
            return self._serve(requests, realtime, t0)
        finally:
            if gc_was_on:
                gc.enable()

    def _serve(self, requests, realtime: bool, t0: float | None):
        pending = list(requests)
        nxt = 0  # pending[nxt:] have not arrived yet
        queue, done = [], []
        start = time.perf_counter() if t0 is None else t0
        self._start = start
        while len(done) < len(requests):
            now = time.perf_counter() - start
            while nxt < len(pending) and (not realtime or pending[nxt].t_arrival <= now):
                r = pending[nxt]
                nxt += 1
                if not realtime:
                    r.t_arrival = 0.0
                queue.append(r)
            progressed = False
            for slot in self.slots:
                if slot.rendered is not None and slot.t_rendered < 0 and slot.rendered.query():
                    slot.t_rendered = time.perf_counter() - start
                if slot.event is not None and slot.event.query():
                    done.extend(self._complete(slot, time.perf_counter() - start))
                    progressed = True
                if slot.event is None and queue:
                    batch = self._admit(queue)
                    if batch:
                        self._launch(slot, batch)
                        progressed = True
            if not progressed:
                # a timed sleep overshoots by the kernel's timer slack (about
                # 50 us), which would delay noticing a finished batch or an
                # arrival: sleep only while the next arrival is more than 2 ms
                # away and nothing runs, otherwise yield and poll again
                if nxt < len(pending) and not queue and all(s.event is None for s in self.slots):
                    wait = pending[nxt].t_arrival - (time.perf_counter() - start)
                    if wait > 2e-3:
                        time.sleep(min(wait - 1.5e-3, 1e-3))
                    else:
                        time.sleep(0)
                else:
                    time.sleep(0)
        return done, time.perf_counter() - start

    def render_now(self, reqs) -> list:
        """Render `reqs` as one batch on slot 0 and wait (tests, warm-up)."""
        for r in reqs:
            self.estimate(r)
        slot = self.slots[0]
        self._launch(slot, reqs)
        slot.event.synchronize()
        self._start = None
        return self._complete(slot, 0.0)

    def check(self) -> None:
        for s in self.slots:
            s.ctx.raise_status()


def measure_keys_per_pixel(params, sh_degree: int, cams) -> float:
    """Keys per pixel of the current model for a set of representative
    views (one bin/sort through the C ABI), for the server's memory estimate."""
    from .train import estimate_keys
    packed = cams if isinstance(cams, np.ndarray) else pack_cameras(cams)
    ctx = Context(params.device.index or 0, 0)
    k = estimate_keys(ctx, params, sh_degree, packed, slack=1.0)
    ctx.close()
    px = int(sum(int(w) * int(h) for w, h in zip(packed["width"], packed["height"])))
    return k / px


def percentiles(reqs, rendered: bool = False):
    """p50 and p99 (ms) of arrival-to-host latency, or with rendered=True of
    arrival-to-device-image latency, and the latencies."""
    lat = np.array([((r.t_rendered if rendered else r.t_done) - r.t_arrival) * 1e3 for r in reqs])
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99)), lat
