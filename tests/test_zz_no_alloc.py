"""The allocation-free render entry point, omerf_render_noalloc, against omerf_render.

It serves callers that cannot allocate device memory: a host framework that
owns all device memory and hands the renderer fixed buffers, or a frame loop
that must not call cudaMalloc because it can synchronise the device.  Its
scratch (work counters, occupancy hulls) lives in one static device array
shared by every call, so the checks below render several scenes back to back
and compare each call with the regular entry point.

This file is collected last (test_zz_*) so that a failure here does not hide
the results of the other GPU tests; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from _util import RGB_ATOL, gpu_scene

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
import paper_2404_09531_gb300 as om  # noqa: E402
from paper_2404_09531_gb300 import binding  # noqa: E402


def _check_same(ref, got, what):
    rgb_ref, cnt_ref = ref
    rgb, cnt = got
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cnt.cpu().numpy(), cnt_ref.cpu().numpy(), err_msg=what)
    err = (rgb - rgb_ref).abs().max().item() if rgb.numel() else 0.0
    assert err <= RGB_ATOL, f"{what}: max-abs {err:.3e}"


def test_two_calls_in_a_row_match_the_regular_render():
    sc1 = synth.make_scene(1)
    s1 = gpu_scene(sc1)
    cam1 = synth.make_cameras(1)[0]
    sc2 = synth.make_scene(2)
    s2 = gpu_scene(sc2)
    cam2 = synth.make_cameras(2)[0]
    rays1 = oracle.camera_rays(cam1)[::3]
    ref1 = om.render(s1, camera=cam1)
    ref2 = om.render(s2, camera=cam2)
    ref3 = om.render(s1, rays=rays1)
    # the caller's own preallocated outputs
    n1, n2, n3 = 64 * 64, 1920 * 1080, rays1.shape[0]
    out1 = (torch.empty((n1, 3), device="cuda"), torch.empty(n1, dtype=torch.int32, device="cuda"))
    out2 = (torch.empty((n2, 3), device="cuda"), torch.empty(n2, dtype=torch.int32, device="cuda"))
    out3 = (torch.empty((n3, 3), device="cuda"), torch.empty(n3, dtype=torch.int32, device="cuda"))
    rays1_d = torch.as_tensor(rays1).cuda()
    for call in range(2):
        _check_same(ref1, om.render_noalloc(s1, camera=cam1, rgb=out1[0], count=out1[1]), f"scene 1, call {call}")
        _check_same(ref2, om.render_noalloc(s2, camera=cam2, rgb=out2[0], count=out2[1]), f"scene 2, call {call}")
        _check_same(ref3, om.render_noalloc(s1, rays=rays1_d, rgb=out3[0], count=out3[1]), f"ray list, call {call}")


def test_rejects_an_occupancy_plane_beyond_the_scratch():
    sc = synth.make_scene(1)
    scene = gpu_scene(sc)
    d = binding._SceneDesc.from_buffer_copy(scene._desc)
    # a 16384^2 occupancy plane at a fine step needs a 16384^2 coarse grid:
    # rejected on the host before anything reads the (small) occ array
    d.occ_res = 16384
    d.step = 2.0 ** -20
    rgb = torch.empty((4, 3), device="cuda")
    rays = torch.as_tensor(oracle.camera_rays(synth.make_cameras(1)[0])[:4]).cuda()
    lib = om.lib()
    rc = lib.omerf_render_noalloc(ctypes.byref(d), None, ctypes.c_void_p(rays.data_ptr()), 4,
                                  ctypes.c_void_p(rgb.data_ptr()), None, None)
    assert rc == -2
    assert b"no-allocation render reserves" in lib.omerf_last_error()


def test_bf16_brick_scene_matches_the_regular_render():
    sc = synth.make_scene(4)
    scene = gpu_scene(sc)
    cam = synth.make_cameras(4)[2]
    ref = om.render(scene, camera=cam)
    for call in range(2):
        _check_same(ref, om.render_noalloc(scene, camera=cam, count=torch.empty_like(ref[1])), f"bf16 call {call}")


def test_output_pointers_are_checked_like_the_regular_render():
    """A pageable host buffer is rejected with OMERF_EDEVICE before any launch
    (as omerf_render rejects it); page-locked host buffers are written
    through their device alias and match the regular render."""
    sc = synth.make_scene(1)
    scene = gpu_scene(sc)
    cam = synth.make_cameras(1)[0]
    n = cam["width"] * cam["height"]
    ref = om.render(scene, camera=cam)
    lib = om.lib()
    cs = binding.camera_struct(cam)
    pageable = np.zeros((n, 3), np.float32)
    rc = lib.omerf_render_noalloc(ctypes.byref(scene._desc), ctypes.byref(cs), None, n,
                                  ctypes.c_void_p(pageable.ctypes.data), None, None)
    assert rc == -3
    assert b"rgb" in lib.omerf_last_error()
    assert not pageable.any()
    pinned = torch.zeros((n, 3), dtype=torch.float32, pin_memory=True)
    pinned_cnt = torch.zeros(n, dtype=torch.int32, pin_memory=True)
    for call in range(2):
        rc = lib.omerf_render_noalloc(ctypes.byref(scene._desc), ctypes.byref(cs), None, n,
                                      ctypes.c_void_p(pinned.data_ptr()), ctypes.c_void_p(pinned_cnt.data_ptr()),
                                      None)
        assert rc == 0
        torch.cuda.synchronize()
        _check_same(ref, (pinned.cuda(), pinned_cnt.cuda()), f"page-locked output, call {call}")


def test_host_ray_list_is_refused():
    """A ray list in pageable host memory is refused with OMERF_EDEVICE."""
    sc = synth.make_scene(1)
    scene = gpu_scene(sc)
    n = 64
    rays = np.zeros((n, 6), np.float32)
    rays[:, 5] = -1.0
    rgb = torch.zeros((n, 3), device="cuda")
    lib = om.lib()
    rc = lib.omerf_render_noalloc(ctypes.byref(scene._desc), None, ctypes.c_void_p(rays.ctypes.data), n,
                                  ctypes.c_void_p(rgb.data_ptr()), None, None)
    assert rc == -3
    assert b"rays" in lib.omerf_last_error()


def test_repeated_calls_leave_no_device_allocation_behind():
    """After a first call (which loads the module and its static scratch),
    50 more calls on preallocated outputs leave the device's free memory
    unchanged: no call keeps an allocation.  (A cudaMalloc / cudaFree pair
    within one call would not show here.)"""
    sc = synth.make_scene(2)
    scene = gpu_scene(sc)
    cam = synth.make_cameras(2)[1]
    n = cam["width"] * cam["height"]
    rgb = torch.empty((n, 3), device="cuda")
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    om.render_noalloc(scene, camera=cam, rgb=rgb, count=cnt)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(50):
        om.render_noalloc(scene, camera=cam, rgb=rgb, count=cnt)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
