"""The views of one optimisation step spread over GPUs (one process per GPU).

The optimiser renders the current model from every ready reference camera
(Sec. 3.1).  Projection, binning, compositing, the loss and both adjoints
of a view need that view alone, so the step shards over views: rank r of N
takes views r, r + N, r + 2N, ...  Its loss weights are scaled by its share
of the views, so that its loss is its part of the mean loss over all views
and the sum of the ranks' gradients is the gradient of that mean.  One
collective follows, an all-reduce (sum) of the 60 n gradient floats; then
every rank runs the same Adam update and delta extraction on the same
gradient, so the model stays replicated and any rank can send the delta.

The gradient part of a rank runs as one CUDA-graph launch of gs_train_step
with GS_TRAIN_GRADIENT; the update part is gs_train_step with
GS_TRAIN_UPDATE (a few launches).  The reduction goes through
torch.distributed (NCCL between GPUs, gloo in the CPU tests); on one rank it
is skipped.
"""
from __future__ import annotations

import numpy as np

from . import _lib
from .train import OnlineTrainer


def shard_views(n_views: int, world: int, rank: int) -> list:
    """Views of rank `rank` among `world` ranks: rank, rank + world, ..."""
    if not (0 <= rank < world):
        raise ValueError("rank must lie in [0, world)")
    if world > n_views:
        raise ValueError(f"{world} ranks for {n_views} views: every rank needs a view")
    return list(range(rank, n_views, world))


def view_share(n_views: int, world: int, rank: int) -> float:
    """Fraction of the step's views that rank `rank` renders (its loss weight)."""
    return len(shard_views(n_views, world, rank)) / n_views


def subset_cameras(cams: dict, views) -> dict:
    idx = np.asarray(list(views))
    return {k: np.asarray(v)[idx] for k, v in cams.items()}


def reduce_gradients(grads, group=None):
    """Sum every rank's gradient into `grads`, in place (all-reduce); a
    no-op when torch.distributed is not initialised or has one rank."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grads, op=dist.ReduceOp.SUM, group=group)
    return grads


class ViewShardedTrainer:
    """One rank's share of the batched step over `cams` (all ranks pass the
    same cameras, parameters and settings).  step(targets): this rank's
    gradient (graph launch), the all-reduce, the update.  `targets` holds
    this rank's views only (planar [3][H][W] each, in shard order)."""

    def __init__(self, params, sh_degree: int, cams: dict, keys_cap: int, rank: int, world: int, group=None,
                 w_l1=0.8, w_ssim=0.2, **kw):
        V = len(cams["fx"])
        self.views = shard_views(V, world, rank)
        self.share = view_share(V, world, rank)
        self.rank, self.world, self.group = rank, world, group
        self.trainer = OnlineTrainer(params, sh_degree, subset_cameras(cams, self.views), keys_cap,
                                     w_l1=w_l1 * self.share, w_ssim=w_ssim * self.share,
                                     phases=_lib.TRAIN_GRADIENT, **kw)
        self.targets = self.trainer.targets

    def capture(self, stream=None):
        self.trainer.capture(stream)

    def step(self, stream=None):
        import torch
        t = self.trainer
        t.step(stream)
        s = stream if stream is not None else torch.cuda.current_stream(t.params.device)
        with torch.cuda.stream(s):
            reduce_gradients(t.grads, self.group)
        t.step_update(stream)

    def loss(self) -> float:
        """The mean loss over all views of the step (sum of the ranks' shares)."""
        t = self.trainer.d_loss.clone()
        reduce_gradients(t, self.group)
        return float(t.item())

    def delta_count(self) -> int:
        return self.trainer.delta_count()

    @property
    def ctx(self):
        return self.trainer.ctx

    def raise_status(self):
        self.trainer.raise_status()
