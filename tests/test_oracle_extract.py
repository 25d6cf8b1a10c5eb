"""Pins for the oracle's extraction after training (Sec. 4.4 and Sec. 5.3):
the 3D occupancy grid derived from the occupancy plane, the brick pool of an
occupancy-driven brick table, and the XZ/YZ plane rows cropped to the
occupancy bounds.  CPU only.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth


def _rule_evaluates(aabb, occ, M, p):
    """The sample rule restated for points p [n][3] in float32: inside the
    closed box, nearest cell by floor((x - x0) (M / (x1 - x0))), z strictly
    inside the cell's interval."""
    p = np.asarray(p, np.float32)
    x0, x1, y0, y1, z0, z1 = [np.float32(v) for v in aabb]
    inside = (p[:, 0] >= x0) & (p[:, 0] <= x1) & (p[:, 1] >= y0) & (p[:, 1] <= y1) & (p[:, 2] >= z0) & (p[:, 2] <= z1)
    cx = np.clip(np.floor((p[:, 0] - x0) * (np.float32(M) / (x1 - x0))), 0, M - 1).astype(int)
    cy = np.clip(np.floor((p[:, 1] - y0) * (np.float32(M) / (y1 - y0))), 0, M - 1).astype(int)
    zb = occ[cx, cy]
    return inside & (zb[:, 0] < p[:, 2]) & (p[:, 2] < zb[:, 1])


# ---------------------------------------------------------------- Sec. 5.3 occupancy grid
def test_occupancy_grid_uniform_interval_closed_form():
    aabb = (-1.0, 1.0, -1.0, 1.0, -0.5, 0.5)
    occ = np.tile(np.array([-0.15, 0.25], np.float32), (4, 4, 1))
    N = (6, 5, 10)  # z voxels of height 0.1 with edges at -0.5, -0.4, ..., 0.5
    grid, cnt = oracle.occupancy_grid(aabb, occ, N)
    # voxel k spans [-0.5 + 0.1 k, -0.4 + 0.1 k): it meets (-0.15, 0.25) for k = 3..7
    want_k = np.zeros(10, bool)
    want_k[3:8] = True
    assert cnt == 6 * 5 * 5
    assert np.all(grid == want_k[None, None, :])
    # empty cells (z_min >= z_max) occupy nothing
    empty = np.tile(np.array([0.3, 0.3], np.float32), (4, 4, 1))
    assert oracle.occupancy_grid(aabb, empty, N)[1] == 0


def test_occupancy_grid_matches_dense_point_sampling():
    """A voxel is occupied iff some point in it is evaluated: dense random
    points in each voxel find a witness exactly in the occupied voxels."""
    rng = np.random.default_rng(0)
    M = 5
    aabb = (-1.0, 1.0, -0.5, 1.5, 0.0, 1.0)
    occ = np.empty((M, M, 2), np.float32)
    h = rng.uniform(0.2, 0.8, (M, M))
    occ[..., 0] = h - rng.uniform(0.05, 0.3, (M, M))
    occ[..., 1] = h + rng.uniform(0.05, 0.3, (M, M))
    occ[1, 3] = (0.6, 0.4)  # an empty cell
    N = (7, 6, 9)
    grid, cnt = oracle.occupancy_grid(aabb, occ, N)
    assert 0 < cnt < np.prod(N)
    x0, x1, y0, y1, z0, z1 = aabb
    witness = np.zeros(N, bool)
    per = 4000
    for i in range(N[0]):
        for j in range(N[1]):
            for k in range(N[2]):
                u = rng.uniform(0, 1, (per, 3))
                p = np.stack([x0 + (i + u[:, 0]) * (x1 - x0) / N[0], y0 + (j + u[:, 1]) * (y1 - y0) / N[1],
                              z0 + (k + u[:, 2]) * (z1 - z0) / N[2]], 1)
                witness[i, j, k] = _rule_evaluates(aabb, occ, M, p).any()
    # every witnessed voxel is marked; marked voxels without a witness have
    # only a sliver of overlap (checked: none on this seed)
    assert np.all(grid[witness] == 1)
    assert np.array_equal(grid.astype(bool), witness)


def test_occupancy_grid_refines_consistently():
    """Halving the voxels: a coarse voxel is occupied iff one of its 8
    children is (the footprints and z-ranges nest exactly for these sizes)."""
    sc = synth.make_scene(1)
    aabb, occ = sc["spec"].aabb, sc["occ"]
    fine, _ = oracle.occupancy_grid(aabb, occ, (64, 64, 32))
    coarse, _ = oracle.occupancy_grid(aabb, occ, (32, 32, 16))
    pooled = fine.reshape(32, 2, 32, 2, 16, 2).max(axis=(1, 3, 5))
    np.testing.assert_array_equal(coarse, pooled)


# ---------------------------------------------------------------- Sec. 4.4 bricks
def test_extracted_pool_renders_like_the_dense_grid():
    spec = dataclasses.replace(synth.scene_spec(1), brick=8, L=(40, 36, 16))
    sc = synth.make_scene(1)
    rng = np.random.default_rng(4)
    dense = rng.normal(0, 0.5, (*spec.L, 8)).astype(np.float32)
    dense[..., 0] += 1.0
    table = oracle.brick_table(spec, sc["occ"])
    pool = oracle.extract_bricks(spec.L, 8, table, dense)
    # the definition: each pool brick is the grid's block, zero beyond the grid
    for (bi, bj, bk), b in np.ndenumerate(table):
        if b < 0:
            continue
        blk = dense[bi * 8:bi * 8 + 8, bj * 8:bj * 8 + 8, bk * 8:bk * 8 + 8]
        np.testing.assert_array_equal(pool[b, :blk.shape[0], :blk.shape[1], :blk.shape[2]], blk)
        assert np.all(pool[b, blk.shape[0]:] == 0) and np.all(pool[b, :, blk.shape[1]:] == 0)
    sc_d = dict(sc, grid=dense, spec=dataclasses.replace(spec, brick=0))
    sc_s = dict(sc, grid=pool, table=table, spec=spec)
    rays = oracle.camera_rays(synth.make_cameras(1)[0])
    a = oracle.render(oracle.OracleScene(sc_s), rays)
    b = oracle.render(oracle.OracleScene(sc_d), rays)
    assert a["unalloc"] == 0 and (a["count"] > 0).mean() > 0.3
    np.testing.assert_array_equal(a["rgb"], b["rgb"])


def test_reextraction_from_an_older_pool():
    """A new table from a changed occupancy plane: bricks the old pool held
    keep their values, new ones are zero."""
    spec = dataclasses.replace(synth.scene_spec(1), brick=4, L=(64, 64, 32))
    sc = synth.make_scene(1)
    dense = np.random.default_rng(5).normal(0, 1, (*spec.L, 8)).astype(np.float32)
    t1 = oracle.brick_table(spec, sc["occ"])
    occ2 = sc["occ"].copy()
    occ2[:, :, 1] += 0.05  # occupied space grows upwards
    occ2[:8, :8] = (0.5, -0.5)  # and a corner empties
    t2 = oracle.brick_table(spec, occ2)
    assert ((t2 >= 0) & (t1 < 0)).any() and ((t1 >= 0) & (t2 < 0)).any()
    p1 = oracle.extract_bricks(spec.L, 4, t1, dense)
    p2 = oracle.extract_bricks(spec.L, 4, t2, p1, src_table=t1)
    full = oracle.extract_bricks(spec.L, 4, t2, dense)
    for idx, b in np.ndenumerate(t2):
        if b < 0:
            continue
        if t1[idx] >= 0:
            np.testing.assert_array_equal(p2[b], full[b])
        else:
            assert np.all(p2[b] == 0)


# ---------------------------------------------------------------- Sec. 4.4 plane z-range
def test_plane_crop_rows_hand_case():
    aabb = (-1.0, 1.0, -1.0, 1.0, -1.0, 1.0)
    occ = np.array([[[-0.3, 0.1], [0.5, 0.4]], [[-0.2, 0.2], [0.0, 0.1]]], np.float32)
    # Rz = 9: u = (z + 1) * 4; u(-0.3) = 2.8 -> row 2 - 1 = 1; u(0.2) = 4.8 -> row 4 + 2 = 6
    rows, zr = oracle.plane_crop_rows(aabb, 9, occ)
    assert rows == (1, 6)
    assert zr == (-0.75, 0.5)
    assert oracle.plane_crop_rows(aabb, 9, np.array([[[0.5, 0.4]]], np.float32)) is None
    # clamped at the plane's ends
    full = np.array([[[-0.99, 0.99]]], np.float32)
    assert oracle.plane_crop_rows(aabb, 9, full)[0] == (0, 8)


@pytest.mark.parametrize("cfg", [1, "city"])
def test_cropped_planes_render_like_full_planes(cfg):
    if cfg == "city":
        spec = dataclasses.replace(synth.scene_spec(2), L=(64, 64, 8), brick=0, R=(256, 256, 64), M=64,
                                   step=1 / 512, width=48, height=32, n_cams=2)
        sc = synth.make_scene(spec)
        sc["grid"] = np.random.default_rng(1).normal(0, 0.3, (*spec.L, 8)).astype(np.float32)
        cams = synth.make_cameras(spec)
    else:
        sc = synth.make_scene(1)
        spec = sc["spec"]
        cams = synth.make_cameras(1)
    (k0, k1), zr = oracle.plane_crop_rows(spec.aabb, spec.R[2], sc["occ"])
    assert 0 < k1 - k0 + 1 < spec.R[2]
    spec_c = dataclasses.replace(spec, R=(spec.R[0], spec.R[1], k1 - k0 + 1))
    sc_c = dict(sc, spec=spec_c, p_xz=sc["p_xz"][:, k0:k1 + 1].copy(), p_yz=sc["p_yz"][:, k0:k1 + 1].copy(),
                plane_z=zr)
    rays = np.concatenate([oracle.camera_rays(c) for c in cams])
    a = oracle.render(oracle.OracleScene(sc), rays)
    b = oracle.render(oracle.OracleScene(sc_c), rays)
    assert (a["count"] > 0).mean() > 0.2
    np.testing.assert_array_equal(a["count"], b["count"])
    # the same texels, weights from the cropped z-range, whose bounds are FP32
    # values (2^-24 relative): equal up to that rounding of the texel coordinate
    np.testing.assert_allclose(b["rgb"], a["rgb"], rtol=0, atol=1e-6)
    assert math.isclose(zr[1] - zr[0], (k1 - k0) * (spec.aabb[5] - spec.aabb[4]) / (spec.R[2] - 1), rel_tol=1e-6)
