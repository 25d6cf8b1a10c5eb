"""Pins for the FP64 oracle: closed forms, invariants, hand-derived schedules,
library restatements and finite differences.  CPU only.

Each test names the part of Oblique-MERF (arXiv 2404.09531) it pins and is
chosen so that a plausible slip (dropped term, wrong sign or index, swapped
axis) makes it fail.
"""
import dataclasses
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "schedule_cases.json")


def _const_scene(occ, n_max=128, t_thr=0.0, dens=1.5, other=0.0, eps=0.001, step=1 / 64,
                 L=(4, 4, 4), R=(4, 4, 4)):
    sc = synth.tiny_scene(L=L, R=R, M=np.asarray(occ).shape[0], step=step, eps=eps)
    sc["grid"][:] = other
    sc["grid"][..., 0] = dens
    for k in ("p_xy", "p_xz", "p_yz"):
        sc[k][:] = 0.0
    sc["occ"] = np.asarray(occ, np.float32)
    return oracle.OracleScene(sc, n_max=n_max, t_thr=t_thr)


# ---------------------------------------------------------------- Eq. 6
def test_occupancy_function_points():
    eps = 0.01
    zmin, zmax = -0.1, 0.1
    assert oracle.occupancy_value(zmin + eps / 2, zmin, zmax, eps) == pytest.approx(0.25, abs=1e-15)
    assert oracle.occupancy_value(zmax - eps / 4, zmin, zmax, eps) == pytest.approx(1 / 16, abs=1e-15)
    assert oracle.occupancy_value(0.0, zmin, zmax, eps) == 1.0
    assert oracle.occupancy_value(zmin + eps, zmin, zmax, eps) == pytest.approx(1.0, abs=1e-14)
    for z in (-0.2, zmin, zmax, 0.3):
        assert oracle.occupancy_value(z, zmin, zmax, eps) == 0.0
    # monotone rise on the lower ramp, fall on the upper ramp
    lo = [oracle.occupancy_value(zmin + f * eps, zmin, zmax, eps) for f in np.linspace(0.05, 0.95, 10)]
    hi = [oracle.occupancy_value(zmax - f * eps, zmin, zmax, eps) for f in np.linspace(0.05, 0.95, 10)]
    assert np.all(np.diff(lo) > 0) and np.all(np.diff(hi) > 0)
    # overlapping ramps (interval narrower than 2 eps): min of the two ramps
    assert oracle.occupancy_value(0.0, -eps / 2, eps / 2, eps) == pytest.approx(0.25, abs=1e-15)
    assert oracle.occupancy_value(eps / 4, -eps / 2, eps / 2, eps) == pytest.approx(1 / 16, abs=1e-15)


# ---------------------------------------------------------------- appendix A
def test_view_encoding_closed_form():
    d = np.array([0.6, -0.8, 0.0])
    enc = oracle.view_encoding(d)
    assert enc.shape == (27,)
    np.testing.assert_array_equal(enc[:3], d)
    for k in range(4):
        f = 2.0 ** k
        assert enc[3 + 6 * k + 0] == pytest.approx(math.sin(f * 0.6), abs=1e-15)
        assert enc[3 + 6 * k + 1] == pytest.approx(math.sin(-f * 0.8), abs=1e-15)
        assert enc[3 + 6 * k + 2] == 0.0
        assert enc[3 + 6 * k + 3] == pytest.approx(math.cos(f * 0.6), abs=1e-15)
        assert enc[3 + 6 * k + 5] == 1.0
    # sin^2 + cos^2 = 1 for every frequency and axis
    for k in range(4):
        s = enc[3 + 6 * k:6 + 6 * k]
        c = enc[6 + 6 * k:9 + 6 * k]
        np.testing.assert_allclose(s * s + c * c, 1.0, atol=1e-15)


# ---------------------------------------------------------------- Eq. 4, deferred MLP
def test_mlp_matches_numpy_matmul():
    rng = np.random.default_rng(3)
    P = rng.normal(0, 0.3, 883)
    F = rng.uniform(0, 1, (50, 7))
    d = rng.normal(0, 1, (50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    got = oracle.mlp(P, F, d)
    W1 = P[:544].reshape(16, 34)
    b1 = P[544:560]
    W2 = P[560:816].reshape(16, 16)
    b2 = P[816:832]
    W3 = P[832:880].reshape(3, 16)
    b3 = P[880:883]
    freqs = 2.0 ** np.arange(4)
    enc = [d]
    for f in freqs:
        enc += [np.sin(f * d), np.cos(f * d)]
    x = np.concatenate([F] + enc, 1)
    h1 = np.maximum(x @ W1.T + b1, 0)
    h2 = np.maximum(h1 @ W2.T + b2, 0)
    y = 1 / (1 + np.exp(-(h2 @ W3.T + b3)))
    np.testing.assert_allclose(got, y, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- Eq. 2, feature field
def _affine_scene(brick=0):
    sc = synth.tiny_scene(L=(5, 7, 6), R=(9, 11, 8))
    spec = sc["spec"]
    x0, x1, y0, y1, z0, z1 = spec.aabb
    rng = np.random.default_rng(11)
    A = rng.normal(0, 1, (4, 3, 8))  # per source, per axis, per channel slopes
    c0 = rng.normal(0, 1, (4, 8))

    def axis(n, lo, hi):
        return lo + np.arange(n) * (hi - lo) / (n - 1)

    gx, gy, gz = axis(5, x0, x1), axis(7, y0, y1), axis(6, z0, z1)
    sc["grid"] = (c0[0] + gx[:, None, None, None] * A[0, 0] + gy[None, :, None, None] * A[0, 1]
                  + gz[None, None, :, None] * A[0, 2])
    px, py, pz = axis(9, x0, x1), axis(11, y0, y1), axis(8, z0, z1)
    sc["p_xy"] = c0[1] + px[:, None, None] * A[1, 0] + py[None, :, None] * A[1, 1]
    sc["p_xz"] = c0[2] + px[:, None, None] * A[2, 0] + pz[None, :, None] * A[2, 2]
    sc["p_yz"] = c0[3] + py[:, None, None] * A[3, 1] + pz[None, :, None] * A[3, 2]

    def truth(p):
        t = c0.sum(0) + p[:, 0:1] * (A[0, 0] + A[1, 0] + A[2, 0]) + p[:, 1:2] * (A[0, 1] + A[1, 1] + A[3, 1])
        return t + p[:, 2:3] * (A[0, 2] + A[2, 2] + A[3, 2])

    return sc, truth


def test_features_reproduce_affine_fields():
    sc, truth = _affine_scene()
    os_ = oracle.OracleScene(sc)
    rng = np.random.default_rng(5)
    p = np.stack([rng.uniform(-1, 1, 400), rng.uniform(-1, 1, 400), rng.uniform(-0.5, 0.5, 400)], 1)
    p[:4] = [[-1, -1, -0.5], [1, 1, 0.5], [1, -1, 0.5], [0, 0, 0]]  # corners and faces
    got, ua = oracle.features(os_, p)
    assert ua == 0
    np.testing.assert_allclose(got, truth(p), atol=1e-12)


def test_features_single_vertex_is_a_tent():
    sc = synth.tiny_scene(L=(5, 5, 5), R=(4, 4, 4))
    sc["grid"][:] = 0.0
    for k in ("p_xy", "p_xz", "p_yz"):
        sc[k][:] = 0.0
    sc["grid"][2, 3, 1, 4] = 1.0  # one vertex, channel 4
    os_ = oracle.OracleScene(sc)
    rng = np.random.default_rng(6)
    p = np.stack([rng.uniform(-1, 1, 500), rng.uniform(-1, 1, 500), rng.uniform(-0.5, 0.5, 500)], 1)
    got, _ = oracle.features(os_, p)
    u = (p[:, 0] + 1) / 2 * 4
    v = (p[:, 1] + 1) / 2 * 4
    w = (p[:, 2] + 0.5) * 4
    tent = np.maximum(0, 1 - abs(u - 2)) * np.maximum(0, 1 - abs(v - 3)) * np.maximum(0, 1 - abs(w - 1))
    np.testing.assert_allclose(got[:, 4], tent, atol=1e-14)
    assert np.abs(np.delete(got, 4, axis=1)).max() == 0.0
    # plane texel tents: XZ texel (ix=1, iz=2), channel 0
    sc["grid"][:] = 0.0
    sc["p_xz"][1, 2, 0] = 1.0
    got, _ = oracle.features(oracle.OracleScene(sc), p)
    u = (p[:, 0] + 1) / 2 * 3
    w = (p[:, 2] + 0.5) * 3
    tent = np.maximum(0, 1 - abs(u - 1)) * np.maximum(0, 1 - abs(w - 2))
    np.testing.assert_allclose(got[:, 0], tent, atol=1e-14)


# ---------------------------------------------------------------- schedule (hand-derived)
@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"])
def test_hand_derived_schedules(case):
    os_ = _const_scene(case["occ"], n_max=case["n_max"])
    ray = np.asarray(case["ray"], np.float32)[None]
    out = oracle.render(os_, ray)
    assert out["count"][0] == case["count"]
    assert out["k_first"][0] == case["k_first"]
    assert out["k_last"][0] == case["k_last"]
    if case["name"].startswith("vertical"):
        assert out["TN"][0] == pytest.approx(case["T_N"], rel=1e-13)
    if case["count"] == 0:
        np.testing.assert_array_equal(out["rgb"][0], os_.bg)
        assert out["TN"][0] == 1.0


# ---------------------------------------------------------------- Eq. 1, constant slab
def test_constant_slab_closed_form_and_colour():
    occ = [[[-0.3, 0.3]] * 2] * 2
    os_ = _const_scene(occ, other=0.75)
    ray = np.array([[0.3, 0.2, 1.0, 0.0, 0.0, -1.0]], np.float32)
    out = oracle.render(os_, ray)
    tn = math.exp(-39 * math.exp(1.5) / 64)
    assert out["TN"][0] == pytest.approx(tn, rel=1e-13)
    xc = 1 / (1 + math.exp(-0.75))
    np.testing.assert_allclose(out["F"][0], (1 - tn) * xc, rtol=1e-13)
    g = oracle.mlp(os_.mlp, out["F"][0], ray[0, 3:].astype(np.float64))[0]
    np.testing.assert_allclose(out["rgb"][0], (1 - tn) * xc + g, rtol=1e-13)


@pytest.mark.parametrize("dz", [-1.0, -0.6])
def test_slab_transmittance_converges_with_step(dz):
    """T_N -> exp(-tau * (b - a) / |d_z|) with O(step) error as the lattice refines."""
    a, b = -0.2013, 0.2511  # not aligned with any lattice
    dens = float(np.float32(math.log(3.0)))  # the grid stores FP32
    tau = math.exp(dens)
    d = np.array([math.sqrt(1 - dz * dz), 0.0, dz])
    o = np.array([-0.9, 0.1, 0.9])
    exact = math.exp(-tau * (b - a) / abs(dz))
    errs = []
    steps = [1 / 64, 1 / 256, 1 / 1024, 1 / 4096]
    for st in steps:
        os_ = _const_scene([[[a, b]] * 2] * 2, n_max=100000, dens=dens, step=st, eps=1e-9)
        out = oracle.render(os_, np.concatenate([o, d])[None].astype(np.float32))
        n = out["count"][0]
        assert out["TN"][0] == pytest.approx(math.exp(-tau * n * st), rel=1e-12)
        errs.append(abs(out["TN"][0] - exact))
        # the evaluated run length differs from (b - a)/|d_z| by at most one step
        assert errs[-1] <= 1.01 * tau * st / abs(dz) * exact * math.exp(tau * st / abs(dz))
    assert max(errs[2:]) < errs[0] or errs[0] < 1e-3


# ---------------------------------------------------------------- Eq. 8 invariant
def test_weights_plus_transmittance_is_one():
    sc = synth.make_scene(1)
    os_ = oracle.OracleScene(sc, t_thr=0.0)
    rays = oracle.camera_rays(synth.make_cameras(1)[0])
    rng = np.random.default_rng(0)
    for r in rng.choice(len(rays), 60, replace=False):
        w, tn = oracle.ray_weights(os_, rays[r])
        assert np.all(w >= 0)
        assert w.sum() + tn == pytest.approx(1.0, abs=1e-12)
    os_t = oracle.OracleScene(sc)
    out = oracle.render(os_t, rays)
    hit = out["count"] > 0
    F = out["F"][hit]
    assert np.all(F >= 0) and np.all(F[:, :3] <= 1 + 1e-12)
    # termination: a ray that stopped early has T_N below the threshold
    stopped = out["TN"] < sc["spec"].t_thr
    assert np.all(out["count"][stopped] < sc["spec"].n_max + 1)


def test_termination_and_cap_are_first_crossing():
    sc = synth.make_scene(1)
    sc["grid"] = sc["grid"].copy()
    sc["grid"][..., 0] += 1.5  # denser than the config so that rays terminate
    rays = oracle.camera_rays(synth.make_cameras(1)[0])
    base = oracle.render(oracle.OracleScene(sc, t_thr=0.0), rays)
    thr = oracle.render(oracle.OracleScene(sc), rays)
    assert np.all(thr["count"] <= base["count"])
    # stopping only shortens rays whose T fell below 1e-4
    shorter = thr["count"] < base["count"]
    assert shorter.any()
    assert np.all(thr["TN"][shorter] < 1e-4)
    capped = oracle.render(oracle.OracleScene(sc, t_thr=0.0, n_max=5), rays)
    np.testing.assert_array_equal(capped["count"], np.minimum(base["count"], 5))


# ---------------------------------------------------------------- pinhole rays
def test_camera_rays_geometry():
    cam = {"c2w": np.array([[1, 0, 0, 0.5], [0, 1, 0, -0.25], [0, 0, 1, 2.0]], np.float32),
           "fx": np.float32(10.0), "fy": np.float32(10.0), "cx": np.float32(2.0), "cy": np.float32(1.5),
           "width": 4, "height": 3}
    rays = oracle.camera_rays(cam)
    assert rays.shape == (12, 6)
    np.testing.assert_array_equal(rays[:, :3], np.tile([0.5, -0.25, 2.0], (12, 1)))
    # pixel (1, 1): centre (1.5, 1.5) -> u = -0.05, v = 0
    d = rays[1 * 4 + 1, 3:]
    want = np.array([-0.05, 0.0, -1.0]) / math.sqrt(0.05 ** 2 + 1)
    np.testing.assert_allclose(d, want, atol=2e-7)
    cams = synth.make_cameras(2, n=2)
    cams[0]["width"], cams[0]["height"] = 64, 36
    cams[0]["cx"], cams[0]["cy"] = np.float32(32), np.float32(18)
    r = oracle.camera_rays(cams[0])
    np.testing.assert_allclose(np.linalg.norm(r[:, 3:].astype(np.float64), axis=1), 1.0, atol=3e-7)
    # image rows go down (-y camera), columns go right (+x camera)
    c2w = cams[0]["c2w"].astype(np.float64)
    right, up = c2w[:, 0], c2w[:, 1]
    assert (r[1, 3:] - r[0, 3:]) @ right > 0
    assert (r[64, 3:] - r[0, 3:]) @ up < 0


# ---------------------------------------------------------------- losses
def test_losses_closed_forms():
    sc = synth.tiny_scene(n_rays=6)
    os_ = oracle.OracleScene(sc, bg=(0.2, 0.3, 0.4))
    # all cells empty: every ray returns bg; only the Charbonnier and L_occ terms remain
    sc_e = dict(sc)
    sc_e["occ"] = np.array([[[0.4, -0.4]] * 2] * 2, np.float32)
    os_e = oracle.OracleScene(sc_e, bg=(0.2, 0.3, 0.4))
    res = oracle.train(os_e, sc["rays"], sc["target"], sc["smooth_dirs"], lam=(1.0, 0.1, 0.01))
    bg = np.array([0.2, 0.3, 0.4], np.float32).astype(np.float64)  # bg is an FP32 setting
    charb = np.sqrt(((bg - sc["target"].astype(np.float64)) ** 2).sum(1) + 1e-6).mean()
    occ = 4 * 0.8 ** 2
    assert res["loss_terms"][0] == pytest.approx(charb, rel=1e-12)
    assert res["loss_terms"][1] == 0.0
    assert res["loss_terms"][2] == pytest.approx(0.01 * occ, rel=1e-6)
    for k in ("grid", "p_xy", "p_xz", "p_yz", "mlp"):
        assert np.abs(res["grads"][k]).max() == 0.0
    # dL_occ/dz_max = 2 lam (z_max - z_min) = 2 * 0.01 * (-0.8)
    np.testing.assert_allclose(res["grads"]["occ"][..., 1], -0.016, rtol=1e-6)
    np.testing.assert_allclose(res["grads"]["occ"][..., 0], 0.016, rtol=1e-6)
    # smoothness: s = d gives no penalty; s = -d gives cosine -1 times |G(-d) - G(d)|^2
    same = np.repeat(sc["rays"][:, None, 3:], 1, axis=1)
    r0 = oracle.train(os_, sc["rays"], sc["target"], same, lam=(0.0, 1.0, 0.0), want_grad=False)
    assert abs(r0["loss_terms"][1]) < 1e-14  # s/|s| differs from d by rounding only
    out = oracle.render(os_, sc["rays"])
    hit = out["count"] > 0
    d64 = sc["rays"][:, 3:].astype(np.float64)
    gd = oracle.mlp(os_.mlp, out["F"], d64)
    gm = oracle.mlp(os_.mlp, out["F"], -d64 / np.linalg.norm(d64, axis=1, keepdims=True))
    want = -(((gm - gd) ** 2).sum(1) * hit).mean()
    r1 = oracle.train(os_, sc["rays"], sc["target"], -same, lam=(0.0, 1.0, 0.0), want_grad=False)
    assert r1["loss_terms"][1] == pytest.approx(want, rel=1e-12)
    # Charbonnier on rendered colours
    r2 = oracle.train(os_, sc["rays"], sc["target"], same, lam=(1.0, 0.0, 0.0), want_grad=False)
    want2 = np.sqrt(((out["rgb"] - sc["target"]) ** 2).sum(1) + 1e-6).mean()
    assert r2["loss_terms"][0] == pytest.approx(want2, rel=1e-12)


# ---------------------------------------------------------------- analytic gradient vs FD
def _fd_check(sc, lam, bg, h=1e-6, rng_sel=None):
    os_ = oracle.OracleScene(sc, bg=bg)
    args = (sc["rays"], sc["target"], sc["smooth_dirs"])
    an = oracle.train(os_, *args, lam=lam)
    assert an["loss"] > 0
    keys = {"grid": "grid", "p_xy": "pxy", "p_xz": "pxz", "p_yz": "pyz", "occ": "occ", "mlp": "mlp"}
    checked = skipped = 0
    worst = 0.0
    for gk, attr in keys.items():
        arr = getattr(os_, attr)
        flat = arr.reshape(-1)
        idx = range(flat.size) if rng_sel is None else rng_sel(flat.size)
        g = an["grads"][gk].reshape(-1)
        for i in idx:
            v = flat[i]
            flat[i] = v + h
            rp = oracle.train(os_, *args, lam=lam, want_grad=False)
            flat[i] = v - h
            rm = oracle.train(os_, *args, lam=lam, want_grad=False)
            flat[i] = v
            if rp["signature"] != rm["signature"] or rp["signature"] != an["signature"]:
                skipped += 1
                continue
            fd = (rp["loss"] - rm["loss"]) / (2 * h)
            err = abs(fd - g[i])
            worst = max(worst, err / (1e-6 + abs(g[i])))
            assert err <= 1e-7 + 1e-6 * abs(g[i]), (gk, i, fd, g[i])
            checked += 1
    return checked, skipped, an


def test_gradient_matches_central_differences_everywhere():
    """Every parameter of a 4^3 grid, 4x4 planes, 2x2 occupancy, 4 rays, full MLP."""
    sc = synth.tiny_scene(n_rays=4)
    checked, skipped, an = _fd_check(sc, lam=(1.0, 0.1, 0.01), bg=(0.2, 0.3, 0.4))
    assert checked > 1500 and skipped < 40
    # every parameter group receives gradient
    for k, g in an["grads"].items():
        assert np.abs(g).max() > 0, k
    # the ramp branches were exercised (z-bound gradients beyond L_occ's)
    os_ = oracle.OracleScene(sc, bg=(0.2, 0.3, 0.4))
    no_occ = oracle.train(os_, sc["rays"], sc["target"], sc["smooth_dirs"], lam=(1.0, 0.1, 0.0))
    assert np.abs(no_occ["grads"]["occ"]).max() > 1e-4


def test_gradient_central_differences_brick_grid():
    sc = synth.tiny_scene(n_rays=4, L=(6, 6, 6), seed=2)
    spec = dataclasses.replace(sc["spec"], brick=4)
    sc["spec"] = spec
    dense = sc["grid"]
    table = oracle.brick_table(spec, sc["occ"])
    nb = int(table.max()) + 1
    pool = np.zeros((nb, 4, 4, 4, 8), np.float32)
    for (bi, bj, bk), b in np.ndenumerate(table):
        if b < 0:
            continue
        blk = dense[bi * 4:bi * 4 + 4, bj * 4:bj * 4 + 4, bk * 4:bk * 4 + 4]
        pool[b, :blk.shape[0], :blk.shape[1], :blk.shape[2]] = blk
    sc["grid"], sc["table"] = pool, table
    rng = np.random.default_rng(1)
    checked, skipped, _ = _fd_check(sc, lam=(1.0, 0.1, 0.01), bg=(0.1, 0.0, 0.2),
                                    rng_sel=lambda n: rng.choice(n, min(n, 150), replace=False))
    assert checked > 600


def test_gradient_grad_scale_and_linearity():
    sc = synth.tiny_scene(n_rays=4)
    os_ = oracle.OracleScene(sc, bg=(0.2, 0.3, 0.4))
    args = (sc["rays"], sc["target"], sc["smooth_dirs"])
    a = oracle.train(os_, *args, lam=(1.0, 0.1, 0.01), grad_scale=1.0)
    b = oracle.train(os_, *args, lam=(1.0, 0.1, 0.01), grad_scale=-2.5)
    for k in a["grads"]:
        np.testing.assert_allclose(b["grads"][k], -2.5 * a["grads"][k], rtol=1e-13, atol=1e-300)


# ---------------------------------------------------------------- Sec. 4.4 bricks
def _brute_table(spec, occ):
    """Continuous-geometry restatement in float64: brick footprint dilated by a voxel."""
    B = spec.brick
    x0, x1, y0, y1, z0, z1 = spec.aabb
    nb = [(l + B - 1) // B for l in spec.L]
    vx = [(x1 - x0) / (spec.L[0] - 1), (y1 - y0) / (spec.L[1] - 1), (z1 - z0) / (spec.L[2] - 1)]
    cxs = (x1 - x0) / spec.M
    cys = (y1 - y0) / spec.M
    alloc = np.zeros(nb, bool)
    for bi in range(nb[0]):
        xa, xb = x0 + (bi * B - 1) * vx[0], x0 + (bi * B + B) * vx[0]
        for bj in range(nb[1]):
            ya, yb = y0 + (bj * B - 1) * vx[1], y0 + (bj * B + B) * vx[1]
            ci = [i for i in range(spec.M) if x0 + i * cxs <= xb and x0 + (i + 1) * cxs >= xa]
            cj = [j for j in range(spec.M) if y0 + j * cys <= yb and y0 + (j + 1) * cys >= ya]
            for bk in range(nb[2]):
                za, zb = z0 + (bk * B - 1) * vx[2], z0 + (bk * B + B) * vx[2]
                for i in ci:
                    for j in cj:
                        lo, hi = occ[i, j]
                        if lo <= hi and hi >= za and lo <= zb:
                            alloc[bi, bj, bk] = True
    return alloc


def test_brick_table_matches_geometric_definition():
    spec = dataclasses.replace(synth.scene_spec(2), L=(50, 45, 20), brick=8, M=23)
    rng = np.random.default_rng(4)
    h = rng.uniform(-0.04, 0.03, (23, 23))
    occ = np.stack([h - 0.006, h + 0.006], -1).astype(np.float32)
    occ[rng.uniform(size=(23, 23)) < 0.3] = [1.0, -1.0]
    table = oracle.brick_table(spec, occ)
    alloc = _brute_table(spec, occ.astype(np.float64))
    np.testing.assert_array_equal(table >= 0, alloc)
    # pool indices are dense and in x-major brick order
    ids = table[table >= 0]
    np.testing.assert_array_equal(ids, np.arange(ids.size))
    assert 0 < ids.size < table.size


def test_brick_grid_renders_like_dense_grid():
    """No evaluated sample reads an unallocated brick, so sparse == dense exactly."""
    spec = dataclasses.replace(synth.scene_spec(2), L=(128, 128, 16), R=(256, 256, 32), M=64,
                               step=1 / 512, width=48, height=32, n_cams=2)
    sc = synth.make_scene(spec)
    table = oracle.brick_table(spec, sc["occ"])
    pool = synth.fill_brick_pool(sc, table)
    sc_sparse = dict(sc, grid=pool, table=table)
    # the dense grid equal to the pool where allocated and garbage elsewhere
    B = spec.brick
    dense = np.full((*spec.L, 8), 1e3, np.float32)
    for (bi, bj, bk), b in np.ndenumerate(table):
        if b >= 0:
            dense[bi * B:(bi + 1) * B, bj * B:(bj + 1) * B, bk * B:(bk + 1) * B] = pool[b]
    sc_dense = dict(sc, grid=dense, table=None, spec=dataclasses.replace(spec, brick=0))
    rays = np.concatenate([oracle.camera_rays(c) for c in synth.make_cameras(spec)])
    a = oracle.render(oracle.OracleScene(sc_sparse), rays)
    b = oracle.render(oracle.OracleScene(sc_dense), rays)
    assert a["unalloc"] == 0
    assert (a["count"] > 0).mean() > 0.2
    np.testing.assert_array_equal(a["count"], b["count"])
    np.testing.assert_array_equal(a["rgb"], b["rgb"])
