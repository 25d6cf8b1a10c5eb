"""Host fault injection (OMERF_FAULT) on the CPU: every entry point that can
reach its launch site without a GPU returns OMERF_ECUDA with the injected
message, before anything is launched.  The pointers passed are never
dereferenced (the fault stands in for the launch)."""
import ctypes
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2404_09531_gb300", "libomerf.so")
EDEVICE, ECUDA = -3, -4
FAKE = ctypes.c_void_p(1 << 20)  # 1 MiB: aligned for every argument, never read


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    import paper_2404_09531_gb300 as om
    return om.lib()


@pytest.fixture
def fault(monkeypatch):
    def set_(v):
        monkeypatch.setenv("OMERF_FAULT", v)
    return set_


def _f32(*v):
    return (ctypes.c_float * len(v))(*v)


def _i32(*v):
    return (ctypes.c_int32 * len(v))(*v)


def _calls(lib):
    aabb = _f32(-1, 1, -1, 1, -0.1, 0.1)
    return {
        "omerf_build_brick_table": lambda: lib.omerf_build_brick_table(aabb, _i32(16, 16, 8), 4, FAKE, 4, FAKE, FAKE,
                                                                       None),
        "omerf_occupancy_grid": lambda: lib.omerf_occupancy_grid(aabb, FAKE, 4, _i32(8, 8, 40), FAKE, None, None),
        "omerf_extract_bricks": lambda: lib.omerf_extract_bricks(_i32(16, 16, 8), 4, FAKE, 3, FAKE, FAKE, 3, 0, FAKE,
                                                                 None),
        "omerf_plane_crop_rows": lambda: lib.omerf_plane_crop_rows(_f32(-0.1, 0.1), 32, FAKE, 4, FAKE, FAKE, None),
        "omerf_crop_planes": lambda: lib.omerf_crop_planes(FAKE, 16, 32, 3, 9, 0, FAKE, None),
    }


@pytest.mark.parametrize("entry", ["omerf_build_brick_table", "omerf_occupancy_grid", "omerf_extract_bricks",
                                   "omerf_plane_crop_rows", "omerf_crop_planes"])
def test_injected_launch_failure(lib, fault, entry):
    fault("launch")
    assert _calls(lib)[entry]() == ECUDA
    msg = lib.omerf_last_error().decode()
    assert entry in msg and "fault injected" in msg


def test_injected_launch_failure_adam(lib, fault):
    import paper_2404_09531_gb300.binding as b
    g = b._AdamGroup(FAKE.value, FAKE.value, FAKE.value, FAKE.value, None, 1024, 1e-3)
    arr = (b._AdamGroup * 1)(g)
    fault("other,launch")  # a comma-separated list of sites
    assert lib.omerf_adam_step(arr, 1, 0.9, 0.99, 1e-15, 1, None) == ECUDA
    assert "omerf_adam_step" in lib.omerf_last_error().decode()


def test_validation_comes_before_the_fault(lib, fault):
    """A bad argument is still reported as such (the fault site is the launch)."""
    fault("launch")
    assert lib.omerf_build_brick_table(_f32(-1, 1, -1, 1, -0.1, 0.1), _i32(16, 16, 8), 3, FAKE, 4, FAKE, FAKE,
                                       None) == -1


def test_binding_raises_the_status(lib, fault):
    import paper_2404_09531_gb300.binding as b
    fault("launch")
    rc = lib.omerf_crop_planes(FAKE, 16, 32, 3, 9, 0, FAKE, None)
    with pytest.raises(b.OmerfError, match="status -4"):
        b._check(rc, "omerf_crop_planes")


def _no_cuda_device():
    try:
        import torch
        return not torch.cuda.is_available()
    except Exception:
        return True


@pytest.mark.skipif(not _no_cuda_device(), reason="would launch a kernel on fake pointers")
def test_unnamed_sites_do_not_fire(lib, fault):
    """Only the named sites fire: with near-miss names the call goes on past
    the launch hook to the device-memory check of its arrays, which fails for
    want of a device (this runs only where there is no CUDA device), with
    that check's message instead of the injected one."""
    fault("launchx,xlaunch,alloc")
    rc = lib.omerf_build_brick_table(_f32(-1, 1, -1, 1, -0.1, 0.1), _i32(16, 16, 8), 4, FAKE, 4, FAKE, FAKE, None)
    assert rc == EDEVICE
    msg = lib.omerf_last_error().decode()
    assert "fault injected" not in msg and "occ" in msg
