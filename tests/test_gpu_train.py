"""GPU parity of the training forward + backward (through the C ABI) against the
FP64 oracle, whose analytic gradient is pinned by central differences.

Bar: loss within 1e-5 relative; per parameter tensor, gradient error
||g_gpu - g_ref|| / ||g_ref|| <= 1e-3 and max |g_gpu - g_ref| <= 1e-3 max |g_ref|.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from _util import GRAD_RTOL, brick_inputs, gpu_scene, grad_errors

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
import paper_2404_09531_gb300 as om  # noqa: E402

LAM = (1.0, 1e-2, 1e-4)
KEYS = ("grid", "p_xy", "p_xz", "p_yz", "occ", "mlp")


def _check_grads(res, ref, rtol=GRAD_RTOL, what=""):
    for k in KEYS:
        g = res["grads"][k].cpu().numpy()
        nrel, mrel = grad_errors(g, ref["grads"][k])
        assert nrel <= rtol and mrel <= rtol, f"{what} {k}: norm-rel {nrel:.2e}, max-rel {mrel:.2e}"


def _run(sc, batch, lam=LAM, **over):
    scene = gpu_scene(sc, **over)
    res = om.train_step(scene, batch["rays"], batch["target"], batch["smooth_dirs"], lam=lam)
    torch.cuda.synchronize()
    ref = oracle.train(oracle.OracleScene(sc, **over), batch["rays"], batch["target"], batch["smooth_dirs"],
                       lam=lam)
    return scene, res, ref


def test_config3_subset_loss_and_gradients():
    sc = synth.make_scene(3)
    batch = synth.make_train_batch(3, 8192)
    batch["target"] = oracle.render(oracle.OracleScene(synth.perturb_scene(sc)), batch["rays"])["rgb"].astype(
        np.float32)
    scene, res, ref = _run(sc, batch)
    loss = res["loss"].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(loss[0], ref["loss"], rtol=1e-5)
    np.testing.assert_allclose(loss[1:], ref["loss_terms"], rtol=1e-4, atol=1e-9)
    _check_grads(res, ref, what="config 3")


@pytest.mark.parametrize("K", [0, 1, 3])
def test_smoothness_directions(K):
    sc = synth.make_scene(3)
    batch = synth.make_train_batch(3, 1500, K=max(K, 1), seed=11)
    if K == 0:
        batch["smooth_dirs"] = np.zeros((1500, 0, 3), np.float32)
    else:
        batch["smooth_dirs"] = batch["smooth_dirs"][:, :K]
    scene, res, ref = _run(sc, batch, lam=(1.0, 0.1, 0.0))
    _check_grads(res, ref, what=f"K={K}")


@pytest.mark.parametrize("seed", range(4))
def test_tiny_scenes_all_parameters(seed):
    """Tiny scenes whose oracle gradient is checked against central differences."""
    sc = synth.tiny_scene(seed=seed, n_rays=64)
    batch = {k: sc[k] for k in ("rays", "target", "smooth_dirs")}
    _, res, ref = _run(sc, batch, lam=(1.0, 0.1, 0.01), bg=(0.2, 0.3, 0.4))
    _check_grads(res, ref, what=f"tiny {seed}")


def test_brick_grid_gradients():
    sc = synth.tiny_scene(seed=5, n_rays=256, L=(10, 9, 8))
    B = 4
    spec = dataclasses.replace(sc["spec"], brick=B)
    table = oracle.brick_table(spec, sc["occ"])
    nb = int(table.max()) + 1
    pool = np.zeros((nb, B, B, B, 8), np.float32)
    for (bi, bj, bk), b in np.ndenumerate(table):
        if b >= 0:
            blk = sc["grid"][bi * B:(bi + 1) * B, bj * B:(bj + 1) * B, bk * B:(bk + 1) * B]
            pool[b, :blk.shape[0], :blk.shape[1], :blk.shape[2]] = blk
    sb = dict(sc, spec=spec, grid=pool, table=table)
    batch = {k: sc[k] for k in ("rays", "target", "smooth_dirs")}
    _, res, ref = _run(sb, batch, lam=(1.0, 0.1, 0.01))
    _check_grads(res, ref, what="brick")


def test_64_rays_against_central_differences():
    """64 config-3 rays: GPU gradient vs oracle central differences on sampled parameters."""
    sc = synth.make_scene(3)
    batch = synth.make_train_batch(3, 64, seed=21)
    lam = (1.0, 1e-2, 1e-4)
    scene = gpu_scene(sc, t_thr=0.0)
    res = om.train_step(scene, batch["rays"], batch["target"], batch["smooth_dirs"], lam=lam)
    torch.cuda.synchronize()
    osc = oracle.OracleScene(sc, t_thr=0.0)
    base = oracle.train(osc, batch["rays"], batch["target"], batch["smooth_dirs"], lam=lam)
    rng = np.random.default_rng(0)
    h = 1e-5
    attrs = {"grid": "grid", "p_xy": "pxy", "p_xz": "pxz", "p_yz": "pyz", "occ": "occ", "mlp": "mlp"}
    checked = 0
    for k, attr in attrs.items():
        ref_g = base["grads"][k].reshape(-1)
        nz = np.nonzero(ref_g)[0]
        flat = getattr(osc, attr).reshape(-1)
        gpu_g = res["grads"][k].cpu().numpy().reshape(-1)
        scale = np.abs(ref_g).max()
        for i in rng.choice(nz, min(12, nz.size), replace=False):
            v = flat[i]
            flat[i] = v + h
            rp = oracle.train(osc, batch["rays"], batch["target"], batch["smooth_dirs"], lam=lam, want_grad=False)
            flat[i] = v - h
            rm = oracle.train(osc, batch["rays"], batch["target"], batch["smooth_dirs"], lam=lam, want_grad=False)
            flat[i] = v
            if rp["signature"] != rm["signature"]:
                continue
            fd = (rp["loss"] - rm["loss"]) / (2 * h)
            assert abs(gpu_g[i] - fd) <= 1e-3 * scale + 1e-6 * abs(fd), (k, i, gpu_g[i], fd)
            checked += 1
    assert checked >= 50


def test_autograd_function_and_grad_scale():
    sc = synth.make_scene(3)
    batch = synth.make_train_batch(3, 2048, seed=3)
    scene = gpu_scene(sc)
    params = [scene.grid, scene.p_xy, scene.p_xz, scene.p_yz, scene.occ, scene.mlp]
    for p in params:
        p.requires_grad_(True)
    loss = om.TrainStep.apply(scene, batch["rays"], batch["target"], batch["smooth_dirs"], LAM, *params)
    (2.5 * loss).backward()
    torch.cuda.synchronize()
    ref = oracle.train(oracle.OracleScene(sc), batch["rays"], batch["target"], batch["smooth_dirs"], lam=LAM,
                       grad_scale=2.5)
    np.testing.assert_allclose(loss.item(), ref["loss"], rtol=1e-5)
    for k, p in zip(KEYS, params):
        nrel, mrel = grad_errors(p.grad.cpu().numpy(), ref["grads"][k])
        assert nrel <= GRAD_RTOL and mrel <= GRAD_RTOL, (k, nrel, mrel)


def test_bf16_features_train_against_rounded_oracle():
    """BF16 features (FP32 master copy and FP32 gradients) vs the oracle on the
    BF16-rounded values: only the arithmetic differs."""
    sc = synth.make_scene(5)
    rb = lambda a: torch.as_tensor(a).to(torch.bfloat16).float().numpy()  # noqa: E731
    sc_b = dict(sc, grid=rb(sc["grid"]), p_xy=rb(sc["p_xy"]), p_xz=rb(sc["p_xz"]), p_yz=rb(sc["p_yz"]))
    batch = synth.make_train_batch(5, 4096)
    scene = gpu_scene(sc)
    assert scene.feat_dtype == torch.bfloat16
    res = om.train_step(scene, batch["rays"], batch["target"], batch["smooth_dirs"], lam=LAM)
    torch.cuda.synchronize()
    ref = oracle.train(oracle.OracleScene(sc_b), batch["rays"], batch["target"], batch["smooth_dirs"], lam=LAM)
    _check_grads(res, ref, what="bf16")


def _view_encoding(d):
    parts = [d]
    for k in range(4):
        parts += [np.sin((2.0 ** k) * d), np.cos((2.0 ** k) * d)]
    return np.concatenate(parts, 1)


def _unambiguous(sc, batch, margin=1e-4):
    """Drop the few rays where FP32 and FP64 may take different branches:
    (a) the transmittance passes within 1e-4 (relative) of the termination
    threshold at a sample (they may stop one sample apart, as in the render
    parity), and (b) a hidden unit of an MLP evaluation of the ray (at d or
    at a smoothness direction) has a pre-activation within `margin` of the
    ReLU kink, where the two sides take different derivatives.  Both are a
    fraction of a percent of the rays of a large batch."""
    out = oracle.render(oracle.OracleScene(sc), batch["rays"])
    amb = out["ambiguous"] != 0
    P = np.asarray(sc["mlp"], np.float64)
    W1, b1 = P[0:544].reshape(16, 34), P[544:560]
    W2, b2 = P[560:816].reshape(16, 16), P[816:832]
    d = batch["rays"][:, 3:].astype(np.float64)
    dirs = [d] + [batch["smooth_dirs"][:, k].astype(np.float64) for k in range(batch["smooth_dirs"].shape[1])]
    kink = np.zeros(len(d), bool)
    for v in dirs:
        v = v / np.linalg.norm(v, axis=1, keepdims=True)
        a1 = np.concatenate([out["F"], _view_encoding(v)], 1) @ W1.T + b1
        a2 = np.maximum(a1, 0.0) @ W2.T + b2
        kink |= (np.abs(a1).min(1) < margin) | (np.abs(a2).min(1) < margin)
    drop = amb | (kink & (out["count"] > 0))
    assert drop.mean() < 1e-2
    return {k: v[~drop] for k, v in batch.items()}


def test_config3_full_batch_as_benchmarked():
    """The benchmarked training workload at full size: 2^18 config-3 rays
    (less the ambiguous ones),
    K = 1, lambda = (1, 1e-2, 1e-4), one fused step through the C ABI; every
    parameter tensor's gradient and the loss against the FP64 oracle."""
    sc = synth.make_scene(3)
    batch = _unambiguous(sc, synth.make_train_batch(3, 1 << 18))
    batch["target"] = oracle.render(oracle.OracleScene(synth.perturb_scene(sc)), batch["rays"])["rgb"].astype(
        np.float32)
    scene, res, ref = _run(sc, batch)
    loss = res["loss"].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(loss[0], ref["loss"], rtol=1e-5)
    np.testing.assert_allclose(loss[1:], ref["loss_terms"], rtol=1e-4, atol=1e-9)
    _check_grads(res, ref, what="config 3 full")


def test_config5_full_batch_bf16_as_benchmarked():
    """2^20 rays of 64 cameras with BF16 features (the large precision
    workload): gradients against the oracle on the BF16-rounded features."""
    sc = synth.make_scene(5)
    rb = lambda a: torch.as_tensor(a).to(torch.bfloat16).float().numpy()  # noqa: E731
    sc_b = dict(sc, grid=rb(sc["grid"]), p_xy=rb(sc["p_xy"]), p_xz=rb(sc["p_xz"]), p_yz=rb(sc["p_yz"]))
    batch = _unambiguous(sc_b, synth.make_train_batch(5, 1 << 20))
    scene = gpu_scene(sc)
    assert scene.feat_dtype == torch.bfloat16
    res = om.train_step(scene, batch["rays"], batch["target"], batch["smooth_dirs"], lam=LAM)
    torch.cuda.synchronize()
    ref = oracle.train(oracle.OracleScene(sc_b), batch["rays"], batch["target"], batch["smooth_dirs"], lam=LAM)
    np.testing.assert_allclose(float(res["loss"][0]), ref["loss"], rtol=1e-5)
    _check_grads(res, ref, what="config 5 full bf16")


def test_bf16_brick_grid_gradients():
    """BF16 features in a brick pool (the sparse BF16 forward and re-march
    variants) against the oracle on the BF16-rounded pool and planes."""
    sc = synth.tiny_scene(seed=7, n_rays=256, L=(10, 9, 8))
    B = 4
    spec = dataclasses.replace(sc["spec"], brick=B)
    table = oracle.brick_table(spec, sc["occ"])
    rb = lambda a: torch.as_tensor(a).to(torch.bfloat16).float().numpy()  # noqa: E731
    pool = rb(oracle.extract_bricks(spec.L, B, table, sc["grid"]))
    sb = dict(sc, spec=spec, grid=pool, table=table, p_xy=rb(sc["p_xy"]), p_xz=rb(sc["p_xz"]), p_yz=rb(sc["p_yz"]))
    batch = {k: sc[k] for k in ("rays", "target", "smooth_dirs")}
    scene = gpu_scene(sb, feat_dtype=torch.bfloat16)
    assert scene.feat_dtype == torch.bfloat16 and scene.brick == B
    res = om.train_step(scene, batch["rays"], batch["target"], batch["smooth_dirs"], lam=(1.0, 0.1, 0.01))
    torch.cuda.synchronize()
    ref = oracle.train(oracle.OracleScene(sb), batch["rays"], batch["target"], batch["smooth_dirs"],
                       lam=(1.0, 0.1, 0.01))
    np.testing.assert_allclose(float(res["loss"][0]), ref["loss"], rtol=1e-5)
    _check_grads(res, ref, what="bf16 brick")


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_city_scene_training(dtype):
    """Training at the city scene's sizes (the large-scene reading of the big
    training workload): 512x512x32 grid in 8^3 bricks, 2048^2 / 2048x128
    planes, 256^2 occupancy, step 1/2048, rays from 64 oblique 1920x1080
    cameras.  Every gradient tensor against the oracle (on the BF16-rounded
    pool and planes for BF16)."""
    spec = dataclasses.replace(synth.scene_spec(2), n_cams=64)
    sc = synth.make_scene(spec)
    table, pool = brick_inputs(sc)
    sb = dict(sc, grid=pool, table=table)
    if dtype == torch.bfloat16:
        rb = lambda a: torch.as_tensor(a).to(torch.bfloat16).float().numpy()  # noqa: E731
        sb.update(grid=rb(pool), p_xy=rb(sc["p_xy"]), p_xz=rb(sc["p_xz"]), p_yz=rb(sc["p_yz"]))
    batch = _unambiguous(sb, synth.make_train_batch(spec, 8192))
    scene = gpu_scene(sb, feat_dtype=dtype)
    assert scene.brick == 8
    res = om.train_step(scene, batch["rays"], batch["target"], batch["smooth_dirs"], lam=LAM)
    torch.cuda.synchronize()
    ref = oracle.train(oracle.OracleScene(sb), batch["rays"], batch["target"], batch["smooth_dirs"], lam=LAM)
    assert np.count_nonzero(ref["grads"]["grid"]) > 10000
    np.testing.assert_allclose(float(res["loss"][0]), ref["loss"], rtol=1e-5)
    _check_grads(res, ref, what=f"city {dtype}")


@pytest.mark.parametrize("n", [1, 31, 33])
def test_ragged_small_batches(n):
    """Batches that fill part of one or two 32-ray bundles."""
    sc = synth.make_scene(3)
    batch = synth.make_train_batch(3, n, seed=5 + n)
    scene, res, ref = _run(sc, batch)
    np.testing.assert_allclose(float(res["loss"][0]), ref["loss"], rtol=1e-5)
    _check_grads(res, ref, what=f"n={n}")


def test_zero_rays_leave_only_the_interval_span_term():
    """An empty batch: the loss and gradients are those of the span term
    lambda_7 sum (z_max - z_min)^2 alone (Eq. 5), the oracle's with the ray
    terms switched off."""
    sc = synth.make_scene(3)
    scene = gpu_scene(sc)
    empty = {k: v[:0] for k, v in synth.make_train_batch(3, 1, seed=2).items()}
    res = om.train_step(scene, empty["rays"], empty["target"], empty["smooth_dirs"], lam=LAM)
    torch.cuda.synchronize()
    one = synth.make_train_batch(3, 1, seed=2)
    ref = oracle.train(oracle.OracleScene(sc), one["rays"], one["target"], one["smooth_dirs"], lam=(0.0, 0.0, LAM[2]))
    np.testing.assert_allclose(float(res["loss"][0]), ref["loss"], rtol=1e-5)
    for k in KEYS:
        g = res["grads"][k].cpu().numpy()
        if k == "occ":
            nrel, mrel = grad_errors(g, ref["grads"][k])
            assert nrel <= GRAD_RTOL and mrel <= GRAD_RTOL, f"occ: {nrel:.2e} {mrel:.2e}"
        else:
            assert not np.any(g), k
