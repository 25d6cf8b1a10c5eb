"""Pins for the oracle's working-set count (the parameters a render reads at
least once, used for the compulsory-bytes figure of the render roofline).
CPU only."""
import dataclasses

import numpy as np

import oracle
import synth


def _vertical_scene():
    sc = synth.tiny_scene(seed=0, L=(5, 5, 5), R=(9, 9, 9), M=4)
    sc["occ"][:] = (-1.0, 1.0)  # every cell holds the whole box: all in-box samples evaluated
    return sc


def test_vertical_ray_hand_case():
    """A ray straight down at (x, y) = (0.1, -0.3) through a box of z-extent
    [-0.5, 0.5], step 1/16, no termination.  Vertex-aligned coordinates:
    grid x u = 2.2 -> vertices 2, 3; y u = 1.4 -> 1, 2; z spans 0..4.
    Planes (9 texels per axis): x u = 4.4 -> 4, 5; y u = 2.8 -> 2, 3; z 0..8.
    Occupancy (4 cells): cell (2, 1).  Samples: z = 1.5 - k/16 in [-0.5, 0.5]
    for k = 16..32, i.e. 17."""
    sc = _vertical_scene()
    ray = np.array([[0.1, -0.3, 1.5, 0.0, 0.0, -1.0]], np.float32)
    ws = oracle.working_set(oracle.OracleScene(sc, t_thr=0.0), ray)
    assert ws["samples"] == 17
    want = np.zeros((5, 5, 5), bool)
    want[2:4, 1:3, :] = True
    np.testing.assert_array_equal(ws["grid"], want)
    xy = np.zeros((9, 9), bool)
    xy[4:6, 2:4] = True
    xz = np.zeros((9, 9), bool)
    xz[4:6, :] = True
    yz = np.zeros((9, 9), bool)
    yz[2:4, :] = True
    np.testing.assert_array_equal(ws["p_xy"], xy)
    np.testing.assert_array_equal(ws["p_xz"], xz)
    np.testing.assert_array_equal(ws["p_yz"], yz)
    occ = np.zeros((4, 4), bool)
    occ[2, 1] = True
    np.testing.assert_array_equal(ws["occ"], occ)


def test_features_read_are_the_gradient_support():
    """Every feature a render reads receives a gradient, and nothing else
    does: with random features and oblique rays (interpolation weights are
    never exactly zero), the nonzero pattern of the oracle's loss gradient
    equals the working set, on a dense grid and on a brick pool, with and
    without early termination."""
    for brick, t_thr in ((0, 0.0), (0, 1e-2), (4, 1e-2)):
        sc = synth.tiny_scene(seed=3, n_rays=64, L=(10, 9, 8), R=(12, 11, 9), M=3)
        if brick:
            spec = dataclasses.replace(sc["spec"], brick=brick)
            table = oracle.brick_table(spec, sc["occ"])
            sc = dict(sc, spec=spec, table=table, grid=oracle.extract_bricks(spec.L, brick, table, sc["grid"]))
        osc = oracle.OracleScene(sc, t_thr=t_thr)
        ws = oracle.working_set(osc, sc["rays"])
        ref = oracle.train(osc, sc["rays"], sc["target"], sc["smooth_dirs"], lam=(1.0, 0.0, 0.0))
        assert ws["samples"] == int(oracle.render(osc, sc["rays"])["count"].sum()) > 100
        for k in ("grid", "p_xy", "p_xz", "p_yz"):
            support = np.any(ref["grads"][k] != 0, axis=-1)
            np.testing.assert_array_equal(ws[k], support, err_msg=f"{k} brick={brick} t_thr={t_thr}")


def test_occupancy_cells_brute_force():
    """Occupancy cells: restated in numpy -- every lattice sample k inside the
    closed box (FP32 positions) up to the ray's last evaluated sample when it
    stopped early, else to its exit, marks its nearest cell."""
    sc = synth.make_scene(1)
    spec = sc["spec"]
    n_max, t_thr = 12, 0.05  # so that some rays stop on each rule
    osc = oracle.OracleScene(sc, n_max=n_max, t_thr=t_thr)
    rays = oracle.camera_rays(synth.make_cameras(1)[0])[::7]
    ws = oracle.working_set(osc, rays)
    r = oracle.render(osc, rays)
    x0, x1, y0, y1, z0, z1 = [np.float32(v) for v in spec.aabb]
    step = np.float32(spec.step)
    M = spec.M
    want = np.zeros((M, M), bool)
    capped, ended = r["count"] >= n_max, (r["count"] > 0) & (r["TN"] < t_thr)
    stopped = capped | ended
    for i, ray in enumerate(rays):
        k = np.arange(0, 4096, dtype=np.int64)
        t = k.astype(np.float32) * step
        p = ray[None, :3] + t[:, None] * ray[None, 3:]
        inside = ((p[:, 0] >= x0) & (p[:, 0] <= x1) & (p[:, 1] >= y0) & (p[:, 1] <= y1) & (p[:, 2] >= z0)
                  & (p[:, 2] <= z1))
        if stopped[i]:
            inside &= k <= r["k_last"][i]
        p = p[inside]
        cx = np.clip(np.floor((p[:, 0] - x0) * (np.float32(M) / (x1 - x0))), 0, M - 1).astype(int)
        cy = np.clip(np.floor((p[:, 1] - y0) * (np.float32(M) / (y1 - y0))), 0, M - 1).astype(int)
        want[cx, cy] = True
    assert capped.any() and ended.any() and (~stopped & (r["count"] > 0)).any() and want.sum() > 10
    np.testing.assert_array_equal(ws["occ"], want)
