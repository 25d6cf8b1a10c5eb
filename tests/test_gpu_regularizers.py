"""GPU parity of the regularisers of Sec. 4.3 (through the C ABI) against the
FP64 oracle: the sparsity loss (Eq. 13) and the entropy loss (Eq. 14).

Bar: loss within 1e-5 relative (sparsity) and 1e-4 relative (entropy, whose
per-ray value log S - sum a log a / S is formed in FP32); per parameter
tensor, gradient error ||g_gpu - g_ref|| / ||g_ref|| <= 1e-3 and
max |g_gpu - g_ref| <= 1e-3 max |g_ref|.  Sample decisions are the exact FP32
rule, so the set of samples on every ray is the oracle's.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from _util import GRAD_RTOL, brick_inputs, edge_rays, gpu_scene, grad_errors, oracle_scene_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
import paper_2404_09531_gb300 as om  # noqa: E402

FEAT = ("grid", "p_xy", "p_xz", "p_yz")


def _check(grads, ref, keys, what):
    for k in keys:
        nrel, mrel = grad_errors(grads[k].cpu().numpy(), ref["grads"][k])
        assert nrel <= GRAD_RTOL and mrel <= GRAD_RTOL, f"{what} {k}: norm-rel {nrel:.2e}, max-rel {mrel:.2e}"


def _sparsity(scene, osc, pts, lam=0.05):
    grads = om.zero_grads(scene)
    loss = om.sparsity_loss(scene, pts, lam=lam, grads=grads)
    torch.cuda.synchronize()
    ref = oracle.sparsity(osc, pts, lam=lam)
    return float(loss.item()), grads, ref


def _entropy(scene, osc, rays, lam=1e-3):
    grads = om.zero_grads(scene)
    loss = om.entropy_loss(scene, rays, lam=lam, grads=grads)
    torch.cuda.synchronize()
    ref = oracle.entropy(osc, rays, lam=lam)
    return float(loss.item()), grads, ref


# ---------------------------------------------------------------- Eq. 13
def test_sparsity_dense_grid_paper_batch():
    """2^14 points in the occupied space of the 64x64x16 scene (the paper's batch)."""
    sc = synth.make_scene(3)
    scene = gpu_scene(sc)
    pts = synth.sparsity_points(sc, 1 << 14)
    loss, grads, ref = _sparsity(scene, oracle.OracleScene(sc), pts)
    assert loss == pytest.approx(ref["loss"], rel=1e-5)
    _check(grads, ref, FEAT, "sparsity dense")
    for k in FEAT:
        assert grads[k][..., 1:].abs().max().item() == 0.0


def test_sparsity_brick_grid_and_clamped_points():
    """The 512x512x32 brick grid, plus points outside the box (clamped to its
    faces) and in unallocated bricks (zero grid part, no grid gradient)."""
    sc = synth.make_scene(2)
    table, pool = brick_inputs(sc)
    scene = gpu_scene(sc, table=table)
    rng = np.random.default_rng(3)
    outside = np.stack([rng.uniform(-1.5, 1.5, 256), rng.uniform(-1.5, 1.5, 256), rng.uniform(-0.2, 0.2, 256)], 1)
    pts = np.concatenate([synth.sparsity_points(sc, 1 << 14), outside]).astype(np.float32)
    loss, grads, ref = _sparsity(scene, oracle_scene_for(sc, table, pool), pts)
    assert loss == pytest.approx(ref["loss"], rel=1e-5)
    _check(grads, ref, FEAT, "sparsity bricks")


def test_sparsity_bf16_features_against_rounded_oracle():
    sc = synth.make_scene(5)
    rb = lambda a: torch.as_tensor(a).to(torch.bfloat16).float().numpy()  # noqa: E731
    sc_b = dict(sc, grid=rb(sc["grid"]), p_xy=rb(sc["p_xy"]), p_xz=rb(sc["p_xz"]), p_yz=rb(sc["p_yz"]))
    scene = gpu_scene(sc)
    assert scene.feat_dtype == torch.bfloat16
    pts = synth.sparsity_points(sc, 4096)
    loss, grads, ref = _sparsity(scene, oracle.OracleScene(sc_b), pts)
    assert loss == pytest.approx(ref["loss"], rel=1e-5)
    _check(grads, ref, FEAT, "sparsity bf16")


def test_sparsity_empty_accumulate_and_grad_scale():
    sc = synth.make_scene(3)
    scene = gpu_scene(sc)
    pts = synth.sparsity_points(sc, 3000, seed=4)
    grads = om.zero_grads(scene)
    loss = torch.full((1,), 2.0, device="cuda")
    om.sparsity_loss(scene, np.zeros((0, 3), np.float32), grads=grads, loss=loss)
    torch.cuda.synchronize()
    assert loss.item() == 2.0 and all(g.abs().max().item() == 0.0 for g in grads.values())
    om.sparsity_loss(scene, pts, lam=0.05, grads=grads, loss=loss, grad_scale=-0.5)
    torch.cuda.synchronize()
    ref = oracle.sparsity(oracle.OracleScene(sc), pts, lam=0.05, grad_scale=-0.5)
    # the sum is rounded at magnitude 2 in FP32 (an ulp there is 2.4e-7)
    assert loss.item() - 2.0 == pytest.approx(ref["loss"], abs=4.8e-7)
    _check(grads, ref, FEAT, "grad_scale")


# ---------------------------------------------------------------- Eq. 14
def test_entropy_dense_grid_paper_batch():
    """2^10 top-down rays over the 64x64x16 scene (the paper's batch)."""
    sc = synth.make_scene(3)
    scene = gpu_scene(sc)
    rays = synth.entropy_rays(sc, 1 << 10)
    loss, grads, ref = _entropy(scene, oracle.OracleScene(sc), rays)
    assert ref["loss"] > 0
    assert loss == pytest.approx(ref["loss"], rel=1e-4)
    _check(grads, ref, FEAT + ("occ",), "entropy dense")


def test_entropy_brick_grid():
    sc = synth.make_scene(2)
    table, pool = brick_inputs(sc)
    scene = gpu_scene(sc, table=table)
    rays = synth.entropy_rays(sc, 1 << 10)
    loss, grads, ref = _entropy(scene, oracle_scene_for(sc, table, pool), rays)
    assert loss == pytest.approx(ref["loss"], rel=1e-4)
    _check(grads, ref, FEAT + ("occ",), "entropy bricks")


@pytest.mark.parametrize("seed", range(3))
def test_entropy_tiny_scenes_with_ramps(seed):
    """Tiny scenes with wide occupancy ramps (every sample's M < 1 somewhere),
    whose oracle gradient is pinned by central differences."""
    sc = synth.tiny_scene(seed=seed, step=1 / 64)
    rays = np.concatenate([synth.entropy_rays(sc, 200, seed=seed, tilt=0.3), edge_rays(sc["spec"], 100, seed)])
    loss, grads, ref = _entropy(gpu_scene(sc), oracle.OracleScene(sc), rays, lam=1.0)
    assert loss == pytest.approx(ref["loss"], rel=1e-4)
    assert np.abs(ref["grads"]["occ"]).max() > 0
    _check(grads, ref, FEAT + ("occ",), f"entropy tiny {seed}")


def test_entropy_sample_cap_and_edge_rays():
    """n_max caps each ray at its first n_max evaluated samples; rays that miss
    the box, start inside it or run along an axis behave as the oracle's."""
    sc = synth.make_scene(1)
    spec = dataclasses.replace(sc["spec"], n_max=7)
    sc = dict(sc, spec=spec)
    rays = np.concatenate([synth.entropy_rays(sc, 512, tilt=0.6), edge_rays(spec, 300)])
    osc = oracle.OracleScene(sc, t_thr=0.0)
    assert (oracle.render(osc, rays)["count"] == 7).sum() > 100
    loss, grads, ref = _entropy(gpu_scene(sc), oracle.OracleScene(sc), rays, lam=0.5)
    assert loss == pytest.approx(ref["loss"], rel=1e-4)
    _check(grads, ref, FEAT + ("occ",), "entropy cap")


def test_entropy_bf16_features_against_rounded_oracle():
    sc = synth.make_scene(5)
    rb = lambda a: torch.as_tensor(a).to(torch.bfloat16).float().numpy()  # noqa: E731
    sc_b = dict(sc, grid=rb(sc["grid"]), p_xy=rb(sc["p_xy"]), p_xz=rb(sc["p_xz"]), p_yz=rb(sc["p_yz"]))
    scene = gpu_scene(sc)
    rays = synth.entropy_rays(sc, 1 << 10)
    loss, grads, ref = _entropy(scene, oracle.OracleScene(sc_b), rays)
    assert loss == pytest.approx(ref["loss"], rel=1e-4)
    _check(grads, ref, FEAT + ("occ",), "entropy bf16")


def test_entropy_without_gradients_and_empty():
    sc = synth.make_scene(3)
    scene = gpu_scene(sc)
    rays = synth.entropy_rays(sc, 300, seed=8)
    loss = om.entropy_loss(scene, rays, lam=1e-3)
    torch.cuda.synchronize()
    assert loss.item() == pytest.approx(oracle.entropy(oracle.OracleScene(sc), rays, lam=1e-3,
                                                       want_grad=False)["loss"], rel=1e-4)
    empty = om.entropy_loss(scene, np.zeros((0, 6), np.float32))
    torch.cuda.synchronize()
    assert empty.item() == 0.0


def test_regularisers_bf16_brick_grid():
    """Both regularisers on a BF16 brick pool (the sparse BF16 kernel variants)
    against the oracle on the rounded pool and planes."""
    sc = synth.make_scene(1)
    spec = dataclasses.replace(sc["spec"], brick=8)
    table = oracle.brick_table(spec, sc["occ"])
    rb = lambda a: torch.as_tensor(a).to(torch.bfloat16).float().numpy()  # noqa: E731
    pool = rb(oracle.extract_bricks(spec.L, 8, table, sc["grid"]))
    sb = dict(sc, spec=spec, grid=pool, table=table, p_xy=rb(sc["p_xy"]), p_xz=rb(sc["p_xz"]), p_yz=rb(sc["p_yz"]))
    scene = gpu_scene(sb, feat_dtype=torch.bfloat16)
    osc = oracle.OracleScene(sb)
    loss, grads, ref = _sparsity(scene, osc, synth.sparsity_points(sc, 4096))
    assert loss == pytest.approx(ref["loss"], rel=1e-5)
    _check(grads, ref, FEAT, "sparsity bf16 bricks")
    loss, grads, ref = _entropy(scene, osc, synth.entropy_rays(sc, 512))
    assert loss == pytest.approx(ref["loss"], rel=1e-4)
    _check(grads, ref, FEAT + ("occ",), "entropy bf16 bricks")
