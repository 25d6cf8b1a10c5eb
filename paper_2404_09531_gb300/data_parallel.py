"""Data-parallel training over ranks of torch.distributed (one process per GPU).

Rays are independent (Eq. 1 composites each ray on its own), so a training
batch shards by rays: rank r takes a contiguous slice of n_r of the N rays,
runs the fused training step (omerf_train_step) on it with the per-ray
weights lambda_1 and lambda_8 scaled by n_r / N, and lambda_7 (the
interval-span term of Eq. 5, a sum over occupancy cells, not over rays) kept
on rank 0 only; the sum over ranks of the loss and of every gradient is then
the full-batch value (the batch means of Eqs. 10 and 12 are sums over the
shards).  One all-reduce (sum) over a single flat FP32 buffer that holds the
six gradient tensors and the loss carries the only exchange of the step
(NCCL on GPUs, gloo for the CPU tests).  The paper trains on one GPU
(Sec. 4.3); this is the sharded form of the same step.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

GRAD_KEYS = ("grid", "p_xy", "p_xz", "p_yz", "occ", "mlp")


def shard(n: int, rank: int, world: int) -> slice:
    """Contiguous slice of rank `rank` of n rays: sizes differ by at most one,
    the first n % world ranks taking the larger share."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n >= 0")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return slice(lo, lo + base + (1 if rank < extra else 0))


def shard_lambda(lam, n_local: int, n_total: int, rank: int):
    """The weights of rank `rank`'s shard: the per-ray means of Eqs. 10 and 12
    scaled by n_local / n_total, the per-cell Eq. 5 term on rank 0 only."""
    f = n_local / n_total if n_total else 0.0
    return (float(lam[0]) * f, float(lam[1]) * f, float(lam[2]) if rank == 0 else 0.0)


def _pad16(n: int) -> int:
    return (n + 3) // 4 * 4  # float32 elements: every view starts 16-byte aligned


class FlatGrads:
    """The six FP32 gradient buffers and the loss [4] as views of one flat
    buffer, each view 16-byte aligned, so that one collective reduces all."""

    def __init__(self, shapes: dict, device):
        sizes = [_pad16(int(torch.Size(shapes[k]).numel())) for k in GRAD_KEYS]
        self.flat = torch.zeros(sum(sizes) + 4, dtype=torch.float32, device=device)
        self.grads, off = {}, 0
        for k, sz in zip(GRAD_KEYS, sizes):
            n = int(torch.Size(shapes[k]).numel())
            self.grads[k] = self.flat[off:off + n].view(shapes[k])
            off += sz
        self.loss = self.flat[off:off + 4]

    def zero_(self):
        self.flat.zero_()


def default_step(scene, rays, target, dirs, lam, grads, loss, saved=None):
    """The fused CUDA training step of one shard (gradients accumulate)."""
    from . import binding
    binding.train_step(scene, rays, target, dirs, lam=lam, grads=grads, saved=saved, loss=loss)


class DataParallelStep:
    """Ray-sharded training step: each rank computes its shard's loss and
    gradients with the CUDA step, then one all-reduce sums them over ranks.

    ``shapes`` gives each parameter's shape (keys of GRAD_KEYS); ``step_fn``
    computes one shard into the given grads / loss views (the CUDA step by
    default).  After __call__, ``grads`` and ``loss`` hold the full-batch
    values on every rank."""

    def __init__(self, shapes: dict, device, group=None, step_fn=default_step):
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.buf = FlatGrads(shapes, device)
        self.step_fn = step_fn

    @property
    def grads(self):
        return self.buf.grads

    @property
    def loss(self):
        return self.buf.loss

    def __call__(self, scene, rays, target, dirs, lam, saved=None):
        n = int(rays.shape[0])
        sl = shard(n, self.rank, self.world)
        n_local = sl.stop - sl.start
        self.buf.zero_()
        if n_local > 0 or self.rank == 0:  # rank 0 adds the interval-span term even without rays
            d = None if dirs is None else dirs[sl]
            self.step_fn(scene, rays[sl], target[sl], d, shard_lambda(lam, n_local, n, self.rank), self.grads,
                         self.loss, saved)
        if self.world > 1:
            dist.all_reduce(self.buf.flat, op=dist.ReduceOp.SUM, group=self.group)
        return self.loss
