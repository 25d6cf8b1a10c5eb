"""Host logic of the ray-sharded data-parallel training step (CPU, gloo,
world size 2): shards, the per-shard loss weights and the single all-reduce
give the full-batch loss and gradients.  The per-shard computation here is
the FP64 oracle's (injected as the step function: no GPU), so a mistake in
the sharding or the weights, not in the kernels, is what these tests catch;
tests/test_gpu_data_parallel.py runs the same step with the CUDA kernels."""
import os
import tempfile

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
from paper_2404_09531_gb300 import data_parallel as dp  # noqa: E402

LAM = (1.0, 1e-2, 1e-3)


@pytest.mark.parametrize("n,world", [(10, 3), (2, 4), (0, 2), (1 << 18, 8), (7, 1)])
def test_shards_partition_the_batch(n, world):
    parts = [dp.shard(n, r, world) for r in range(world)]
    assert parts[0].start == 0 and parts[-1].stop == n
    for a, b in zip(parts, parts[1:]):
        assert a.stop == b.start
    sizes = [p.stop - p.start for p in parts]
    assert max(sizes) - min(sizes) <= 1 and sum(sizes) == n


def test_shard_weights_sum_to_the_batch():
    n, world = 1001, 3
    lams = [dp.shard_lambda(LAM, dp.shard(n, r, world).stop - dp.shard(n, r, world).start, n, r)
            for r in range(world)]
    np.testing.assert_allclose(sum(l[0] for l in lams), LAM[0])
    np.testing.assert_allclose(sum(l[1] for l in lams), LAM[1])
    assert [l[2] for l in lams] == [LAM[2], 0.0, 0.0]


def test_flat_views_are_aligned_and_disjoint():
    shapes = {"grid": (3, 5, 7, 8), "p_xy": (5, 3, 8), "p_xz": (5, 2, 8), "p_yz": (3, 2, 8), "occ": (3, 3, 2),
              "mlp": (883,)}
    fg = dp.FlatGrads(shapes, "cpu")
    base = fg.flat.data_ptr()
    spans = []
    for k in dp.GRAD_KEYS:
        v = fg.grads[k]
        assert tuple(v.shape) == shapes[k] and v.is_contiguous()
        assert (v.data_ptr() - base) % 16 == 0
        spans.append((v.data_ptr(), v.data_ptr() + 4 * v.numel()))
    spans.append((fg.loss.data_ptr(), fg.loss.data_ptr() + 16))
    spans.sort()
    for a, b in zip(spans, spans[1:]):
        assert a[1] <= b[0]


def _oracle_step(sc):
    """A step function that fills the views from the oracle (FP64 -> FP32)."""
    def step(scene, rays, target, dirs, lam, grads, loss, saved=None):
        r = oracle.train(oracle.OracleScene(sc), rays.numpy(), target.numpy(), dirs.numpy(), lam=lam)
        for k in dp.GRAD_KEYS:
            grads[k] += torch.as_tensor(r["grads"][k].reshape(grads[k].shape), dtype=torch.float32)
        loss[0] += float(r["loss"])
    return step


def _worker(rank, world, init, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=init, rank=rank, world_size=world)
    sc = synth.tiny_scene(seed=2, n_rays=37)
    shapes = {"grid": sc["grid"].shape, "p_xy": sc["p_xy"].shape, "p_xz": sc["p_xz"].shape,
              "p_yz": sc["p_yz"].shape, "occ": sc["occ"].shape, "mlp": sc["mlp"].shape}
    step = dp.DataParallelStep(shapes, "cpu", step_fn=_oracle_step(sc))
    step(None, torch.as_tensor(sc["rays"]), torch.as_tensor(sc["target"]), torch.as_tensor(sc["smooth_dirs"]), LAM)
    if rank == 0:
        np.savez(out, loss=step.loss.numpy(), **{k: v.numpy() for k, v in step.grads.items()})
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sum_to_the_full_batch():
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as tmp:
        init = "file://" + os.path.join(tmp, "store")
        out = os.path.join(tmp, "rank0.npz")
        mp.start_processes(_worker, args=(2, init, out), nprocs=2, join=True, start_method="spawn")
        got = np.load(out)
    sc = synth.tiny_scene(seed=2, n_rays=37)
    ref = oracle.train(oracle.OracleScene(sc), sc["rays"], sc["target"], sc["smooth_dirs"], lam=LAM)
    np.testing.assert_allclose(got["loss"][0], ref["loss"], rtol=1e-6)
    for k in dp.GRAD_KEYS:
        g, r = got[k].astype(np.float64).reshape(-1), ref["grads"][k].reshape(-1)
        assert np.linalg.norm(g - r) <= 1e-6 * np.linalg.norm(r) + 1e-12, k
