"""Pins for the oracle's regularisers of Sec. 4.3: the sparsity loss (Eq. 13)
and the entropy loss (Eq. 14).  CPU only.

Readings: the sparsity loss averages the opacity alpha = 1 - exp(-tau delta)
(delta the lattice step) over caller-given points in the occupied space; the
entropy loss uses a_i = M_i alpha_i over each ray's evaluated samples (no
early termination) with p_i = a_i / sum_j a_j, and its gradient reaches both
the density features and the occupancy plane through M.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _const_scene(occ, dens=1.5, eps=1e-9, step=1 / 64, n_max=4096, L=(4, 4, 4), R=(4, 4, 4)):
    sc = synth.tiny_scene(L=L, R=R, M=np.asarray(occ).shape[0], step=step, eps=eps)
    sc["grid"][:] = 0.25
    sc["grid"][..., 0] = dens
    for k in ("p_xy", "p_xz", "p_yz"):
        sc[k][:] = 0.0
    sc["occ"] = np.asarray(occ, np.float32)
    return sc, oracle.OracleScene(sc, n_max=n_max, t_thr=0.0)


# ---------------------------------------------------------------- Eq. 13
def test_sparsity_constant_density_closed_form():
    sc, os_ = _const_scene([[[-0.3, 0.3]] * 2] * 2)
    pts = synth.sparsity_points(sc, 37, seed=3)
    lam = 0.05
    res = oracle.sparsity(os_, pts, lam=lam)
    sigma = math.exp(1.5) / 64
    alpha = -math.expm1(-sigma)
    assert res["loss"] == pytest.approx(lam * alpha, rel=1e-14)
    g = res["grads"]
    # each point spreads dL/dt0 = lam/n (1 - alpha) sigma over weights summing to one
    want = lam * (1 - alpha) * sigma
    assert g["grid"][..., 0].sum() == pytest.approx(want, rel=1e-12)
    for k in ("p_xy", "p_xz", "p_yz"):
        assert g[k][..., 0].sum() == pytest.approx(want, rel=1e-12)
        assert np.abs(g[k][..., 1:]).max() == 0.0
    assert np.abs(g["grid"][..., 1:]).max() == 0.0
    assert np.all(g["grid"][..., 0] >= 0)


def test_sparsity_point_on_a_vertex_touches_one_vertex():
    sc, os_ = _const_scene([[[-0.3, 0.3]] * 2] * 2, L=(5, 5, 5))
    # vertex (1, 3, 2) of a 5^3 grid over [-1,1]^2 x [-0.5,0.5]: x = -0.5, y = 0.5, z = 0
    pt = np.array([[-0.5, 0.5, 0.0]], np.float32)
    res = oracle.sparsity(os_, pt, lam=1.0)
    sigma = math.exp(1.5) / 64
    g = res["grads"]
    nz = np.argwhere(g["grid"][..., 0] != 0)
    assert nz.tolist() == [[1, 3, 2]]
    assert g["grid"][1, 3, 2, 0] == pytest.approx(math.exp(-sigma) * sigma, rel=1e-13)


def test_sparsity_empty_and_linear():
    sc = synth.tiny_scene()
    os_ = oracle.OracleScene(sc)
    assert oracle.sparsity(os_, np.zeros((0, 3), np.float32))["loss"] == 0.0
    pts = synth.sparsity_points(sc, 11, seed=1)
    a = oracle.sparsity(os_, pts, lam=0.05)
    b = oracle.sparsity(os_, pts, lam=0.05, grad_scale=-3.0)
    for k in a["grads"]:
        np.testing.assert_allclose(b["grads"][k], -3.0 * a["grads"][k], rtol=1e-14, atol=1e-300)
    # the mean over a duplicated point set is unchanged
    c = oracle.sparsity(os_, np.concatenate([pts, pts]), lam=0.05)
    assert c["loss"] == pytest.approx(a["loss"], rel=1e-14)


def _fd(fn, os_, groups, h=1e-6, skip=None, rtol=1e-6, atol=1e-8):
    an = fn(os_)
    checked = skipped = 0
    attrs = {"grid": "grid", "p_xy": "pxy", "p_xz": "pxz", "p_yz": "pyz", "occ": "occ"}
    for gk in groups:
        flat = getattr(os_, attrs[gk]).reshape(-1)
        g = an["grads"][gk].reshape(-1)
        for i in range(flat.size):
            v = flat[i]
            flat[i] = v + h
            lp = fn(os_, want_grad=False)["loss"]
            sp = skip(os_) if skip else None
            flat[i] = v - h
            lm = fn(os_, want_grad=False)["loss"]
            sm = skip(os_) if skip else None
            flat[i] = v
            if skip and (sp != sm or sp != skip(os_)):
                skipped += 1
                continue
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[i]) <= atol + rtol * abs(g[i]), (gk, i, fd, g[i])
            checked += 1
    return an, checked, skipped


def test_sparsity_gradient_matches_central_differences():
    sc = synth.tiny_scene(seed=4)
    os_ = oracle.OracleScene(sc)
    pts = synth.sparsity_points(sc, 9, seed=2)
    an, checked, _ = _fd(lambda o, want_grad=True: oracle.sparsity(o, pts, lam=0.05, want_grad=want_grad),
                         os_, ("grid", "p_xy", "p_xz", "p_yz"), atol=1e-10)
    assert checked == sum(an["grads"][k].size for k in ("grid", "p_xy", "p_xz", "p_yz"))
    # only the density channel receives gradient
    for k in ("grid", "p_xy", "p_xz", "p_yz"):
        assert np.abs(an["grads"][k][..., 0]).max() > 0
        assert np.abs(an["grads"][k][..., 1:]).max() == 0.0


# ---------------------------------------------------------------- Eq. 14
def test_entropy_uniform_slab_is_log_n_and_stationary():
    """Equal a_i on every sample: p = 1/N, loss = log N, zero gradient (the maximum)."""
    sc, os_ = _const_scene([[[-0.3, 0.3]] * 2] * 2)
    rays = np.array([[0.3, 0.2, 1.0, 0.0, 0.0, -1.0], [-0.4, 0.1, 1.2, 0.0, 0.0, -1.0]], np.float32)
    n = oracle.render(os_, rays)["count"]
    assert n[0] > 30 and n[1] > 30
    lam = 1e-3
    res = oracle.entropy(os_, rays, lam=lam)
    assert res["loss"] == pytest.approx(lam * (math.log(n[0]) + math.log(n[1])) / 2, rel=1e-13)
    for k, g in res["grads"].items():
        assert np.abs(g).max() < 1e-15, k


def test_entropy_matches_normalised_weights_of_the_render():
    """a_i recovered from the compositing weights w_i = T_i a_i of the render
    (Eq. 8, no termination), then -sum p log p written out in numpy."""
    sc = synth.make_scene(1)
    os_ = oracle.OracleScene(sc, t_thr=0.0)
    rays = synth.entropy_rays(sc, 40, seed=5)
    lam = 1e-3
    total = 0.0
    for r in rays:
        w, _ = oracle.ray_weights(os_, r)
        if w.size == 0:
            continue
        T = 1.0 - np.concatenate([[0.0], np.cumsum(w)[:-1]])
        a = w / T
        if a.sum() <= 0:
            continue
        p = a / a.sum()
        p = p[p > 0]
        total += -(p * np.log(p)).sum()
    res = oracle.entropy(os_, rays, lam=lam, want_grad=False)
    assert res["loss"] > 0
    assert res["loss"] == pytest.approx(lam * total / len(rays), rel=1e-9)


def test_entropy_two_samples_binary_entropy():
    """Two evaluated samples with a_1 = alpha on a ramp-free cell and a_2 in a
    second cell: loss = H(a_1 / (a_1 + a_2)) with H the binary entropy."""
    # cells of a 2x2 plane at x < 0 and x > 0; a horizontal ray at z = 0 with
    # step 1/4 from x = -0.375 evaluates x = -0.375 (+ k/4) -> samples in both cells
    occ = [[[-0.1, 0.1]] * 2, [[-0.1, 0.1]] * 2]
    sc, _ = _const_scene(occ, step=0.25, dens=0.0)
    sc["grid"][..., 0] = 0.0
    sc["grid"][2:, ..., 0] = 2.0  # denser at x >= 1/3 of the vertex range
    os_ = oracle.OracleScene(sc, t_thr=0.0, n_max=4096)
    ray = np.array([[-0.375, 0.25, 0.0, 1.0, 0.0, 0.0]], np.float32)
    w, _ = oracle.ray_weights(os_, ray[0])
    T = 1.0 - np.concatenate([[0.0], np.cumsum(w)[:-1]])
    a = w / T
    H = -sum(x / a.sum() * math.log(x / a.sum()) for x in a)
    assert oracle.entropy(os_, ray, lam=1.0)["loss"] == pytest.approx(H, rel=1e-12)
    assert a.size >= 2 and len(set(np.round(a, 12))) >= 2


def test_entropy_gradient_matches_central_differences():
    sc = synth.tiny_scene(seed=6, n_rays=3)
    os_ = oracle.OracleScene(sc)
    rays = synth.entropy_rays(sc, 3, seed=9, tilt=0.3)
    assert np.all(oracle.render(os_, rays)["count"] > 3)

    def counts(o):
        return tuple(oracle.render(o, rays)["count"].tolist())

    an, checked, skipped = _fd(lambda o, want_grad=True: oracle.entropy(o, rays, lam=1.0, want_grad=want_grad),
                               os_, ("grid", "p_xy", "p_xz", "p_yz", "occ"), skip=counts, rtol=2e-6,
                               atol=1e-9)
    assert checked > 600 and skipped < 10
    assert np.abs(an["grads"]["occ"]).max() > 1e-3  # the ramps carry gradient to z_min / z_max
    for k in ("grid", "p_xy", "p_xz", "p_yz"):
        assert np.abs(an["grads"][k][..., 1:]).max() == 0.0


def test_entropy_empty_cases():
    sc = synth.tiny_scene()
    os_ = oracle.OracleScene(sc)
    assert oracle.entropy(os_, np.zeros((0, 6), np.float32))["loss"] == 0.0
    miss = np.array([[5.0, 5.0, 1.0, 0.0, 0.0, -1.0]], np.float32)  # outside the box
    res = oracle.entropy(os_, miss)
    assert res["loss"] == 0.0
    assert all(np.abs(g).max() == 0.0 for g in res["grads"].values())
    # a single evaluated sample has p = 1 and no entropy
    sc1, os1 = _const_scene([[[-0.3, 0.3]] * 2] * 2, step=1.0)
    one = np.array([[0.3, 0.2, 0.0, 0.0, 0.0, -1.0]], np.float32)
    assert oracle.render(os1, one)["count"][0] == 1
    assert oracle.entropy(os1, one)["loss"] == 0.0
