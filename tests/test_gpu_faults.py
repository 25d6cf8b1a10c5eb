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


def test_host_arrays_rejected_before_any_launch():
    """A pageable host array handed to an entry point as device data is
    refused on the host (OMERF_EDEVICE, naming the argument) before anything
    is launched, and the scene keeps working."""
    import ctypes
    scene = gpu_scene(synth.make_scene(1))
    L = om.lib()
    n = 64
    rays_h = np.zeros((n, 6), np.float32)
    rays_h[:, 2], rays_h[:, 5] = 1.0, -1.0
    rays_d = torch.as_tensor(rays_h).cuda()
    target = torch.zeros((n, 3), device="cuda")
    saved = torch.empty(n * om.saved_bytes_per_ray() // 4, device="cuda")
    loss = torch.zeros(4, device="cuda")
    grads = om.zero_grads(scene)
    g_host = np.zeros(scene.grid.numel(), np.float32)
    lam = (ctypes.c_float * 3)(1.0, 0.0, 0.0)
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    H = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    gp = [P(grads[k]) for k in ("grid", "p_xy", "p_xz", "p_yz", "occ", "mlp")]

    rc = L.omerf_train_step(scene.handle, H(rays_h), P(target), None, n, 0, lam, P(saved), P(loss), *gp, None)
    assert rc == -3 and "rays" in L.omerf_last_error().decode()
    rc = L.omerf_train_step(scene.handle, P(rays_d), P(target), None, n, 0, lam, P(saved), P(loss), H(g_host),
                            *gp[1:], None)
    assert rc == -3 and "gradient" in L.omerf_last_error().decode()
    rgb = torch.empty((n, 3), device="cuda")
    rc = L.omerf_render(scene.handle, None, H(rays_h), n, P(rgb), None, None)
    assert rc == -3 and "rays" in L.omerf_last_error().decode()
    rc = L.omerf_sparsity_loss(scene.handle, H(rays_h[:, :3].copy()), n, ctypes.c_float(1.0), None, P(loss),
                               *gp[:4], None)
    assert rc == -3
    assert not np.any(g_host)
    # nothing was launched on the bad calls; the device arrays still work
    rgb2, cnt = om.render(scene, rays=rays_d)
    torch.cuda.synchronize()
    assert torch.isfinite(rgb2).all() and cnt.shape == (n,)
    om.sync()  # no error is pending from the refused calls
