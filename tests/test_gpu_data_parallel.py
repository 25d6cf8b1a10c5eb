"""The ray-sharded data-parallel training step with the CUDA kernels: two
processes on cuda:0 (gloo carrying the CUDA gradient buffer; each process
runs its own kernels, none waits on the other's), each computing its shard
of a config-3 batch; after the all-reduce the loss and gradients equal the
single-process full-batch step within 1e-5 relative and the FP64 oracle
within the 1e-3 gradient bar."""
import os
import tempfile

import numpy as np
import pytest

import oracle
import synth
from _util import GRAD_RTOL, grad_errors

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
import paper_2404_09531_gb300 as om  # noqa: E402
from paper_2404_09531_gb300 import data_parallel as dp  # noqa: E402

LAM = (1.0, 1e-2, 1e-4)
N = 6000


def _batch():
    sc = synth.make_scene(3)
    b = synth.make_train_batch(3, N, seed=4)
    b["target"] = oracle.render(oracle.OracleScene(synth.perturb_scene(sc)), b["rays"])["rgb"].astype(np.float32)
    return sc, b


def _worker(rank, world, init, out, batch_path):
    import torch.distributed as dist
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=init, rank=rank, world_size=world)
    z = np.load(batch_path)
    sc = synth.make_scene(3)
    scene = om.scene_from_synth(sc, device="cuda")
    shapes = {k: tuple(getattr(scene, k).shape) for k in dp.GRAD_KEYS}
    step = dp.DataParallelStep(shapes, torch.device("cuda"))
    rays, tgt, dirs = (torch.as_tensor(z[k]).cuda() for k in ("rays", "target", "smooth_dirs"))
    step(scene, rays, tgt, dirs, LAM)
    torch.cuda.synchronize()
    if rank == 0:
        np.savez(out, loss=step.loss.cpu().numpy(), **{k: v.cpu().numpy() for k, v in step.grads.items()})
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_match_the_full_batch_and_the_oracle():
    import torch.multiprocessing as mp
    sc, b = _batch()
    with tempfile.TemporaryDirectory() as tmp:
        bp = os.path.join(tmp, "batch.npz")
        np.savez(bp, **b)
        out = os.path.join(tmp, "rank0.npz")
        mp.start_processes(_worker, args=(2, "file://" + os.path.join(tmp, "store"), out, bp), nprocs=2, join=True,
                           start_method="spawn")
        got = np.load(out)
    scene = om.scene_from_synth(sc, device="cuda")
    full = om.train_step(scene, b["rays"], b["target"], b["smooth_dirs"], lam=LAM)
    torch.cuda.synchronize()
    np.testing.assert_allclose(got["loss"], full["loss"].cpu().numpy(), rtol=1e-5, atol=1e-9)
    ref = oracle.train(oracle.OracleScene(sc), b["rays"], b["target"], b["smooth_dirs"], lam=LAM)
    np.testing.assert_allclose(float(got["loss"][0]), ref["loss"], rtol=1e-5)
    for k in dp.GRAD_KEYS:
        g = got[k].astype(np.float64).reshape(-1)
        f = full["grads"][k].cpu().numpy().astype(np.float64).reshape(-1)
        assert np.linalg.norm(g - f) <= 1e-5 * np.linalg.norm(f) + 1e-12, k
        nrel, mrel = grad_errors(got[k], ref["grads"][k])
        assert nrel <= GRAD_RTOL and mrel <= GRAD_RTOL, (k, nrel, mrel)


def _worker_small(rank, world, init, out, n):
    import torch.distributed as dist
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=init, rank=rank, world_size=world)
    sc = synth.make_scene(3)
    b = synth.make_train_batch(3, max(n, 1), seed=9)
    scene = om.scene_from_synth(sc, device="cuda")
    shapes = {k: tuple(getattr(scene, k).shape) for k in dp.GRAD_KEYS}
    step = dp.DataParallelStep(shapes, torch.device("cuda"))
    rays, tgt, dirs = (torch.as_tensor(b[k][:n]).cuda() for k in ("rays", "target", "smooth_dirs"))
    step(scene, rays, tgt, dirs, LAM)
    torch.cuda.synchronize()
    if rank == 0:
        np.savez(out, loss=step.loss.cpu().numpy(), **{k: v.cpu().numpy() for k, v in step.grads.items()})
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("n", [0, 1])
def test_batches_smaller_than_the_world(n):
    """One ray (rank 1's shard is empty) and no ray at all (rank 0 still adds
    the interval-span term): equal to the single-process step."""
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as tmp:
        out = os.path.join(tmp, "rank0.npz")
        mp.start_processes(_worker_small, args=(2, "file://" + os.path.join(tmp, "store"), out, n), nprocs=2,
                           join=True, start_method="spawn")
        got = np.load(out)
    sc = synth.make_scene(3)
    b = synth.make_train_batch(3, max(n, 1), seed=9)
    scene = om.scene_from_synth(sc, device="cuda")
    full = om.train_step(scene, b["rays"][:n], b["target"][:n], b["smooth_dirs"][:n], lam=LAM)
    torch.cuda.synchronize()
    np.testing.assert_allclose(got["loss"], full["loss"].cpu().numpy(), rtol=1e-6, atol=1e-12)
    for k in dp.GRAD_KEYS:
        np.testing.assert_allclose(got[k], full["grads"][k].cpu().numpy(), rtol=1e-6, atol=1e-12, err_msg=k)
