"""Failure paths on the GPU without a GPU fault: host fault injection
(OMERF_FAULT) and a bounded device wait that runs out.

- OMERF_FAULT=extract_wait makes every CTA of the tensor-memory-accelerator
  brick extraction give up its first mbarrier wait at once: the kernel
  records the timeout in the device error word, waits (bounded) for the load
  still in flight and stops.  omerf_sync, or the next extraction call,
  reports OMERF_ETIMEOUT; a later extraction without the fault is complete.
- OMERF_FAULT=alloc / launch make scene creation / a launch fail on the host.
"""
import numpy as np
import pytest

import synth
from _util import gpu_scene

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
import paper_2404_09531_gb300 as om  # noqa: E402

ETIMEOUT, ENOMEM, ECUDA = -5, -6, -4


def _dense_and_table():
    sc = synth.make_scene(1)
    spec = sc["spec"]
    grid = torch.as_tensor(sc["grid"]).cuda().contiguous()
    occ = torch.as_tensor(sc["occ"]).cuda()
    table, n_alloc = om.build_brick_table(spec.aabb, spec.L, 8, occ)
    return spec, grid, table, int(n_alloc.item())


def test_extract_wait_that_runs_out_is_reported(monkeypatch):
    if not om.lib().omerf_tma_available():
        pytest.skip("no tensor-map encoder: the extraction has no device wait")
    spec, grid, table, nb = _dense_and_table()
    ref = om.extract_bricks(spec.L, 8, table, grid, n_bricks=nb)
    om.sync(timeout_ms=10000)
    monkeypatch.setenv("OMERF_FAULT", "extract_wait")
    om.extract_bricks(spec.L, 8, table, grid, n_bricks=nb)
    with pytest.raises(om.OmerfError, match="status -5"):
        om.sync(timeout_ms=10000)
    om.sync(timeout_ms=10000)  # reported once
    # without omerf_sync, the next extraction call reports it
    om.extract_bricks(spec.L, 8, table, grid, n_bricks=nb)
    torch.cuda.synchronize()
    with pytest.raises(om.OmerfError, match="status -5"):
        om.extract_bricks(spec.L, 8, table, grid, n_bricks=nb)
    monkeypatch.delenv("OMERF_FAULT")
    pool = om.extract_bricks(spec.L, 8, table, grid, n_bricks=nb)
    om.sync(timeout_ms=10000)
    assert torch.equal(pool, ref)
    # the context is still usable: a render after the reported timeouts
    scene = gpu_scene(synth.make_scene(1))
    rgb, cnt = om.render(scene, camera=synth.make_cameras(1)[0])
    torch.cuda.synchronize()
    assert int(cnt.sum().item()) > 0


def test_injected_allocation_failure(monkeypatch):
    sc = synth.make_scene(1)
    monkeypatch.setenv("OMERF_FAULT", "alloc")
    with pytest.raises(om.OmerfError, match="status -6"):
        gpu_scene(sc)
    monkeypatch.delenv("OMERF_FAULT")
    gpu_scene(sc)


def test_injected_launch_failure(monkeypatch):
    sc = synth.make_scene(1)
    scene = gpu_scene(sc)
    cam = synth.make_cameras(1)[0]
    ref = om.render(scene, camera=cam)[0]
    batch = synth.make_train_batch(3, 256)
    monkeypatch.setenv("OMERF_FAULT", "launch")
    with pytest.raises(om.OmerfError, match="status -4"):
        om.render(scene, camera=cam)
    with pytest.raises(om.OmerfError, match="status -4"):
        om.train_step(scene, batch["rays"], batch["target"], batch["smooth_dirs"])
    with pytest.raises(om.OmerfError, match="status -4"):
        om.render_cameras(scene, [cam])
    monkeypatch.delenv("OMERF_FAULT")
    rgb = om.render(scene, camera=cam)[0]
    torch.cuda.synchronize()
    np.testing.assert_array_equal(rgb.cpu().numpy(), ref.cpu().numpy())
