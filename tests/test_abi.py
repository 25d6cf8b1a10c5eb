"""The C ABI library loads, exports every entry point declared in
include/omerf.h, and rejects bad arguments on the host.  CPU only: no call here
launches a kernel."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "omerf.h")
LIB = os.path.join(ROOT, "paper_2404_09531_gb300", "libomerf.so")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(omerf_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    import paper_2404_09531_gb300 as om
    return om.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("omerf_scene_create", "omerf_render", "omerf_train_fwd", "omerf_train_bwd",
                     "omerf_train_step", "omerf_ray_interval", "omerf_build_brick_table"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(LIB)
    for name in _declared():
        assert hasattr(raw, name), name


def test_binding_covers_every_declared_symbol():
    import paper_2404_09531_gb300.binding as b
    assert sorted(b.SIGNATURES) == _declared()


def test_host_validation_without_gpu(lib):
    import paper_2404_09531_gb300.binding as b
    d = b._SceneDesc()
    d.aabb[:] = [-1, 1, -1, 1, -0.1, 0.1]
    d.grid_res[:] = [4, 4, 4]
    d.plane_res[:] = [4, 4, 4]
    d.occ_res = 2
    d.step = 0.3  # not a power of two
    d.eps_occ = 0.01
    d.n_max = 16
    d.grid = d.plane_xy = d.plane_xz = d.plane_yz = d.occ = d.mlp = 4096
    out = ctypes.c_void_p()
    assert lib.omerf_scene_create(ctypes.byref(d), None, ctypes.byref(out)) == -1
    assert b"power of two" in lib.omerf_last_error()
    d.step = 1 / 64
    d.grid_res[:] = [1, 4, 4]
    assert lib.omerf_scene_create(ctypes.byref(d), None, ctypes.byref(out)) == -2
    d.grid_res[:] = [4, 4, 4]
    d.feat_dtype = 7
    assert lib.omerf_scene_create(ctypes.byref(d), None, ctypes.byref(out)) == -1
    d.feat_dtype = 0
    d.grid = 4100  # misaligned
    assert lib.omerf_scene_create(ctypes.byref(d), None, ctypes.byref(out)) == -1
    assert b"aligned" in lib.omerf_last_error()
    assert lib.omerf_scene_create(None, None, ctypes.byref(out)) == -1
    # size query: host-only, the same validation; a brick grid adds one
    # 32-byte neighbour record per brick of the grid
    lib.omerf_scene_device_bytes.restype = ctypes.c_int64
    d.grid = 4096
    dense = lib.omerf_scene_device_bytes(ctypes.byref(d))
    assert dense > 0
    d.grid_res[:] = [16, 24, 8]
    d.brick, d.brick_table, d.n_bricks = 4, 4096, 10
    assert lib.omerf_scene_device_bytes(ctypes.byref(d)) - dense == 32 * (4 * 6 * 2)
    d.brick, d.brick_table, d.n_bricks = 0, None, 0
    d.grid_res[:] = [4, 4, 4]
    d.step = 0.3
    assert lib.omerf_scene_device_bytes(ctypes.byref(d)) == -1
    d.step = 1 / 64
    # texels are addressed with 32-bit element offsets: arrays of 2^31 or more
    # elements are refused (dense grid, brick pool, each plane)
    d.grid = 4096
    d.grid_res[:] = [2048, 2048, 64]  # 2^31 elements
    assert lib.omerf_scene_create(ctypes.byref(d), None, ctypes.byref(out)) == -2
    assert b"2^31" in lib.omerf_last_error()
    d.grid_res[:] = [2048, 2048, 63]
    d.plane_res[:] = [16384, 16384, 4]  # XY plane 2^31 elements
    assert lib.omerf_scene_create(ctypes.byref(d), None, ctypes.byref(out)) == -2
    d.plane_res[:] = [4, 4, 4]
    d.brick, d.brick_table, d.n_bricks = 8, 4096, 1 << 19  # pool of 2^19 bricks of 8^3 x 8 = 2^31 elements
    assert lib.omerf_scene_create(ctypes.byref(d), None, ctypes.byref(out)) == -2
    d.brick, d.brick_table, d.n_bricks = 0, None, 0
    d.grid_res[:] = [4, 4, 4]
    aabb = (ctypes.c_float * 6)(-1, 1, -1, 1, -1, 1)
    res = (ctypes.c_int32 * 3)(8, 8, 8)
    assert lib.omerf_build_brick_table(aabb, res, 3, ctypes.c_void_p(4096), 4, ctypes.c_void_p(4096),
                                       ctypes.c_void_p(4096), None) == -1
    assert lib.omerf_render(None, None, None, 10, None, None, None) == -1
    assert lib.omerf_saved_bytes_per_ray() == 80
    # the regularisers reject a missing scene before touching the device
    assert lib.omerf_sparsity_loss(None, None, 0, 0.05, None, None, None, None, None, None, None) == -1
    assert lib.omerf_entropy_loss(None, None, 0, 1e-3, None, None, None, None, None, None, None, None) == -1
    assert b"NULL scene" in lib.omerf_last_error()
    # extraction entry points validate sizes before launching
    aabb = (ctypes.c_float * 6)(-1, 1, -1, 1, -1, 1)
    n = (ctypes.c_int32 * 3)(4, 4, 0)
    assert lib.omerf_occupancy_grid(aabb, ctypes.c_void_p(4096), 2, n, ctypes.c_void_p(4096), None, None) == -2
    g = (ctypes.c_int32 * 3)(8, 8, 8)
    assert lib.omerf_extract_bricks(g, 3, ctypes.c_void_p(4096), 1, ctypes.c_void_p(4096), None, 0, 0,
                                    ctypes.c_void_p(4096), None) == -1
    pz = (ctypes.c_float * 2)(0.5, 0.5)
    assert lib.omerf_plane_crop_rows(pz, 8, ctypes.c_void_p(4096), 2, ctypes.c_void_p(4096),
                                     ctypes.c_void_p(4096), None) == -1
    assert lib.omerf_crop_planes(ctypes.c_void_p(4096), 4, 8, 5, 5, 0, ctypes.c_void_p(8192), None) == -2


def test_host_schedules_match_reference(lib):
    from oracle import adam
    for step in (0, 1000, 40000, 80000):
        assert lib.omerf_lr_exponential(5e-5, 1e-5, step, 80000) == pytest.approx(adam.lr_exponential(5e-5, 1e-5, step, 80000), rel=1e-6)
    for step in (0, 9999, 10000, 14000, 10 ** 8):
        assert lib.omerf_lambda_occ(step) == pytest.approx(adam.lambda_occ(step), rel=1e-6)


def test_camera_validation_without_gpu(lib):
    """Host cameras with a non-finite pose or intrinsics, or a singular
    rotation (rays without direction), are rejected with OMERF_EINVAL before
    any pointer is inspected or anything launched."""
    import paper_2404_09531_gb300.binding as b
    d = b._SceneDesc()
    d.aabb[:] = [-1, 1, -1, 1, -0.1, 0.1]
    d.grid_res[:] = [4, 4, 4]
    d.plane_res[:] = [4, 4, 4]
    d.occ_res = 2
    d.step = 2.0 ** -8
    d.eps_occ = 0.01
    d.n_max = 16
    d.grid = d.plane_xy = d.plane_xz = d.plane_yz = d.occ = d.mlp = 1 << 20
    good = {"c2w": [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 2]], "fx": 8.0, "fy": 8.0, "cx": 4.0, "cy": 4.0,
            "width": 8, "height": 8}
    bad = [dict(good, fx=float("inf")), dict(good, cy=float("nan")),
           dict(good, c2w=[[1, 0, 0, 0], [0, float("nan"), 0, 0], [0, 0, 1, 2]]),
           dict(good, c2w=[[1, 0, 0, 0], [1, 0, 0, 0], [0, 0, 1, 2]]),   # singular: rows 0 and 1 equal
           dict(good, c2w=[[0, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 2]])]
    for cam in bad:
        cs = b.camera_struct(cam)
        rc = lib.omerf_render_noalloc(ctypes.byref(d), ctypes.byref(cs), None, 64, ctypes.c_void_p(1 << 20), None,
                                      None)
        assert rc == -1, cam
    assert b"camera" in lib.omerf_last_error()


def test_new_entry_points_validate_on_the_host(lib):
    """Arguments the new entry points reject before touching the GPU."""
    FAKE = ctypes.c_void_p(1 << 20)
    f6 = (ctypes.c_float * 6)(-1, 1, -1, 1, -0.1, 0.1)
    g3 = (ctypes.c_int32 * 3)(16, 16, 8)
    # grow: NULL old table / missing counter, table aliasing old_table, bad brick edge
    assert lib.omerf_grow_brick_table(f6, g3, 4, FAKE, 4, None, FAKE, FAKE, FAKE, None) == -1
    assert lib.omerf_grow_brick_table(f6, g3, 4, FAKE, 4, FAKE, FAKE, FAKE, None, None) == -1
    assert lib.omerf_grow_brick_table(f6, g3, 4, FAKE, 4, FAKE, FAKE, FAKE, FAKE, None) == -1  # table == old_table
    assert lib.omerf_grow_brick_table(f6, g3, 3, FAKE, 4, ctypes.c_void_p(2 << 20), FAKE, FAKE, FAKE, None) == -1
    # load probe: slice sizes must be whole 256-thread x 32-byte sweeps, buffers aligned
    assert lib.omerf_probe_load_bandwidth(FAKE, 4096, 4, 1, FAKE, None) == -2
    assert lib.omerf_probe_load_bandwidth(FAKE, 8192 + 16, 4, 1, FAKE, None) == -2
    assert lib.omerf_probe_load_bandwidth(FAKE, 8192, 0, 1, FAKE, None) == -2
    assert lib.omerf_probe_load_bandwidth(ctypes.c_void_p((1 << 20) + 16), 8192, 4, 1, FAKE, None) == -1
    assert lib.omerf_probe_load_bandwidth(None, 8192, 4, 1, FAKE, None) == -1
    # reduction probe: regions of whole 4 KB steps, a 16-byte aligned buffer
    assert lib.omerf_probe_red_bandwidth(FAKE, 2048, 4, 1, None) == -2
    assert lib.omerf_probe_red_bandwidth(FAKE, 4096 + 16, 4, 1, None) == -2
    assert lib.omerf_probe_red_bandwidth(FAKE, (1 << 24) + 4096, 4, 1, None) == -2
    assert lib.omerf_probe_red_bandwidth(FAKE, 4096, 4, 0, None) == -2
    assert lib.omerf_probe_red_bandwidth(ctypes.c_void_p((1 << 20) + 8), 4096, 4, 1, None) == -1
    assert lib.omerf_probe_red_bandwidth(None, 4096, 4, 1, None) == -1
    # checking-build counters: a NULL scene or output
    counts = (ctypes.c_uint64 * 2)()
    assert lib.omerf_check_counts(None, counts, 0, None) == -1
    assert lib.omerf_check_build() in (0, 1)
