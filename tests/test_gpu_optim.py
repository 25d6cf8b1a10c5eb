"""GPU parity of the fused Adam step (appendix A optimiser) against the FP64
reference in oracle/adam.py, and a short end-to-end training loop."""
import numpy as np
import pytest

import oracle
import synth
from oracle import adam as ref_adam

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
import paper_2404_09531_gb300 as om  # noqa: E402


def test_adam_matches_reference_over_steps():
    rng = np.random.default_rng(7)
    sizes = [1000, 33, 4097]
    lrs = [1e-2, 5e-5, 3e-3]
    p_ref = [rng.normal(size=n) for n in sizes]
    m_ref = [np.zeros(n) for n in sizes]
    v_ref = [np.zeros(n) for n in sizes]
    p = [torch.tensor(x, dtype=torch.float32, device="cuda") for x in p_ref]
    p_ref = [x.astype(np.float32).astype(np.float64) for x in p_ref]
    m = [torch.zeros(n, device="cuda") for n in sizes]
    v = [torch.zeros(n, device="cuda") for n in sizes]
    shadow = torch.empty(sizes[2], dtype=torch.bfloat16, device="cuda")
    for step in range(1, 9):
        grads = [rng.normal(size=n).astype(np.float32) for n in sizes]
        gd = [torch.tensor(g, device="cuda") for g in grads]
        groups = [{"param": p[i], "grad": gd[i], "m": m[i], "v": v[i], "lr": lrs[i]} for i in range(3)]
        groups[2]["shadow"] = shadow
        om.adam_step(groups, step)
        for i in range(3):
            p_ref[i], m_ref[i], v_ref[i] = ref_adam.adam_step(p_ref[i], grads[i], m_ref[i], v_ref[i], lrs[i], step)
    torch.cuda.synchronize()
    for i in range(3):
        np.testing.assert_allclose(p[i].cpu().numpy(), p_ref[i], rtol=0, atol=1e-5 * lrs[i] / 1e-3 + 1e-6)
        np.testing.assert_allclose(m[i].cpu().numpy(), m_ref[i], rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(v[i].cpu().numpy(), v_ref[i], rtol=1e-5, atol=1e-9)
    np.testing.assert_array_equal(shadow.float().cpu().numpy(), p[2].to(torch.bfloat16).float().cpu().numpy())


def test_schedule_functions_match_reference():
    for step in (0, 5000, 40000, 80000, 90000):
        assert om.lr_exponential(1e-2, 1e-3, step, 80000) == pytest.approx(ref_adam.lr_exponential(1e-2, 1e-3, step, 80000), rel=1e-6)
    for step in (0, 9999, 10000, 12000, 30000, 10 ** 6):
        assert om.lambda_occ(step) == pytest.approx(ref_adam.lambda_occ(step), rel=1e-6)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_training_loop_reduces_the_loss(dtype):
    sc = synth.make_scene(3)
    target_scene = synth.perturb_scene(sc, sigma=0.3)
    batch = synth.make_train_batch(3, 1 << 14, seed=5)
    target = oracle.render(oracle.OracleScene(target_scene), batch["rays"])["rgb"].astype(np.float32)
    scene = om.scene_from_synth(sc, device="cuda", feat_dtype=torch.bfloat16 if dtype == "bf16" else torch.float32)
    tr = om.Trainer(scene, total_steps=200, lam_occ=1e-4)
    losses = [float(tr.step(batch["rays"], target, batch["smooth_dirs"])[0]) for _ in range(30)]
    assert losses[-1] < 0.7 * losses[0], losses
    assert np.all(np.isfinite(losses))


def test_trainer_adds_the_regularisers_to_loss_and_gradients():
    """One Trainer step with the sparsity points and entropy rays: the loss
    total and the gradients are those of train_step plus both terms."""
    sc = synth.make_scene(3)
    batch = synth.make_train_batch(3, 4096, seed=6)
    pts = synth.sparsity_points(sc, 1 << 14)
    erays = synth.entropy_rays(sc, 1 << 10)
    s1 = om.scene_from_synth(sc, device="cuda")
    tr = om.Trainer(s1, total_steps=100, lam_occ=0.0, lr=(1e-30, 1e-30), lr_occ=(1e-30, 1e-30))
    loss = tr.step(batch["rays"], batch["target"], batch["smooth_dirs"], sparsity_points=pts, entropy_rays=erays)
    torch.cuda.synchronize()
    s2 = om.scene_from_synth(sc, device="cuda")
    res = om.train_step(s2, batch["rays"], batch["target"], batch["smooth_dirs"], lam=(1.0, 0.1, 0.0))
    osc = oracle.OracleScene(sc)
    sp = oracle.sparsity(osc, pts, lam=0.05, want_grad=False)["loss"]
    en = oracle.entropy(osc, erays, lam=1e-3, want_grad=False)["loss"]
    torch.cuda.synchronize()
    want = float(res["loss"][0]) + sp + en
    assert float(loss[0]) == pytest.approx(want, rel=1e-5)
    om.sparsity_loss(s2, pts, lam=0.05, grads=res["grads"])
    om.entropy_loss(s2, erays, lam=1e-3, grads=res["grads"])
    torch.cuda.synchronize()
    for k in ("grid", "p_xy", "p_xz", "p_yz", "occ", "mlp"):
        a, b = tr.grads[k], res["grads"][k]
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-7 * float(b.abs().max()) + 1e-30), k


@pytest.mark.parametrize("form", ["f32-dense", "bf16-bricks"])
def test_checkpoint_resume(form, tmp_path):
    """Train 3 steps, save, train 2 more; a trainer loaded from the file
    repeats those 2 steps (losses and parameters equal up to the ordering of
    float atomics), with the scene layout (brick table, dtype, march
    settings) and the optimiser state (moments, step counter, schedules)
    restored."""
    if form == "f32-dense":
        sc = synth.make_scene(3)
        scene = om.scene_from_synth(sc, device="cuda")
    else:
        import dataclasses
        sc = synth.make_scene(3)
        spec = dataclasses.replace(sc["spec"], brick=8)
        table = oracle.brick_table(spec, sc["occ"])
        pool = oracle.extract_bricks(spec.L, 8, table, sc["grid"])
        scene = om.scene_from_synth(dict(sc, spec=spec, grid=pool, table=table), device="cuda",
                                    feat_dtype=torch.bfloat16)
    batch = synth.make_train_batch(3, 1 << 13, seed=9)
    pts = synth.sparsity_points(sc, 1 << 10)
    erays = synth.entropy_rays(sc, 256)
    tr = om.Trainer(scene, total_steps=100)
    for _ in range(3):
        tr.step(batch["rays"], batch["target"], batch["smooth_dirs"], sparsity_points=pts, entropy_rays=erays)
    path = tmp_path / "ckpt.npz"
    tr.save(path)
    la = [float(tr.step(batch["rays"], batch["target"], batch["smooth_dirs"], sparsity_points=pts,
                        entropy_rays=erays)[0]) for _ in range(2)]
    tr2 = om.Trainer.load(path)
    assert tr2.step_no == 3 and tr2.total == 100 and tr2.scene.brick == scene.brick
    assert tr2.scene.feat_dtype == scene.feat_dtype
    lb = [float(tr2.step(batch["rays"], batch["target"], batch["smooth_dirs"], sparsity_points=pts,
                         entropy_rays=erays)[0]) for _ in range(2)]
    np.testing.assert_allclose(lb, la, rtol=1e-5)
    torch.cuda.synchronize()
    for k in ("grid", "p_xy", "p_xz", "p_yz", "occ", "mlp"):
        a, b = tr.master[k], tr2.master[k]
        assert (a - b).abs().max().item() <= 1e-5 * max(a.abs().max().item(), 1.0), k
    if form == "bf16-bricks":
        assert torch.equal(tr2.scene.table, scene.table)
        assert torch.equal(tr2.scene.grid, tr2.master["grid"].to(torch.bfloat16))
