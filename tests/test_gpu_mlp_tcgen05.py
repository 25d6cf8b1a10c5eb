"""The tcgen05 form of the deferred-MLP backward (OMERF_MLP_BWD=tcgen05):
128-ray tiles, each MLP layer and its backward one M = 128 tensor-core
product from shared memory into tensor memory (TF32 split operands), the
weight gradient one BF16-split product per evaluation accumulated in tensor
memory.  The same gradient bar against the FP64 oracle as the default
mma.sync form, agreement with that form, and a bounded wait that runs out
(OMERF_FAULT=mlp_wait) reported as OMERF_ETIMEOUT without a fault."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from _util import GRAD_RTOL, gpu_scene, grad_errors

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
import paper_2404_09531_gb300 as om  # noqa: E402

KEYS = ("grid", "p_xy", "p_xz", "p_yz", "occ", "mlp")


def _check(res, ref, what):
    for k in KEYS:
        nrel, mrel = grad_errors(res["grads"][k].cpu().numpy(), ref["grads"][k])
        assert nrel <= GRAD_RTOL and mrel <= GRAD_RTOL, f"{what} {k}: norm-rel {nrel:.2e}, max-rel {mrel:.2e}"


@pytest.mark.parametrize("K", [0, 1, 3])
def test_tcgen05_mlp_backward_against_oracle(monkeypatch, K):
    sc = synth.make_scene(3)
    b = synth.make_train_batch(3, 3000, K=max(K, 1), seed=17)
    if K == 0:
        b["smooth_dirs"] = np.zeros((3000, 0, 3), np.float32)
    else:
        b["smooth_dirs"] = b["smooth_dirs"][:, :K]
    b["target"] = oracle.render(oracle.OracleScene(synth.perturb_scene(sc)), b["rays"])["rgb"].astype(np.float32)
    lam = (1.0, 0.1, 1e-4)
    scene = gpu_scene(sc)
    default = om.train_step(scene, b["rays"], b["target"], b["smooth_dirs"], lam=lam)
    monkeypatch.setenv("OMERF_MLP_BWD", "tcgen05")
    res = om.train_step(scene, b["rays"], b["target"], b["smooth_dirs"], lam=lam)
    torch.cuda.synchronize()
    ref = oracle.train(oracle.OracleScene(sc), b["rays"], b["target"], b["smooth_dirs"], lam=lam)
    np.testing.assert_allclose(float(res["loss"][0].item()), ref["loss"], rtol=1e-5)
    _check(res, ref, f"tcgen05 K={K}")
    for k in KEYS:  # both forms are about FP32 accurate
        g, d = res["grads"][k].double(), default["grads"][k].double()
        assert float((g - d).norm() / d.norm().clamp_min(1e-30)) <= 1e-4, k


def test_tcgen05_mlp_backward_brick_bf16_and_grad_scale(monkeypatch):
    sc = synth.tiny_scene(seed=5, n_rays=300, L=(10, 9, 8))
    B = 4
    spec = dataclasses.replace(sc["spec"], brick=B)
    table = oracle.brick_table(spec, sc["occ"])
    nb = int(table.max()) + 1
    pool = np.zeros((nb, B, B, B, 8), np.float32)
    for (bi, bj, bk), bb in np.ndenumerate(table):
        if bb >= 0:
            blk = sc["grid"][bi * B:(bi + 1) * B, bj * B:(bj + 1) * B, bk * B:(bk + 1) * B]
            pool[bb, :blk.shape[0], :blk.shape[1], :blk.shape[2]] = blk
    sb = dict(sc, spec=spec, grid=pool, table=table)
    monkeypatch.setenv("OMERF_MLP_BWD", "tcgen05")
    scene = gpu_scene(sb)
    lam = (1.0, 0.1, 0.01)
    loss, saved, inputs = om.train_fwd(scene, sc["rays"], sc["target"], sc["smooth_dirs"], lam=lam)
    grads = om.train_bwd(scene, saved, inputs, lam=lam, grad_scale=2.5)
    torch.cuda.synchronize()
    ref = oracle.train(oracle.OracleScene(sb), sc["rays"], sc["target"], sc["smooth_dirs"], lam=lam, grad_scale=2.5)
    _check({"grads": grads}, ref, "tcgen05 brick")


def test_tcgen05_wait_that_runs_out_is_reported(monkeypatch):
    sc = synth.make_scene(3)
    b = synth.make_train_batch(3, 1000, seed=2)
    scene = gpu_scene(sc)
    monkeypatch.setenv("OMERF_MLP_BWD", "tcgen05")
    monkeypatch.setenv("OMERF_FAULT", "mlp_wait")
    om.train_step(scene, b["rays"], b["target"], b["smooth_dirs"])
    with pytest.raises(om.OmerfError, match="status -5"):
        om.sync(timeout_ms=20000)
    monkeypatch.delenv("OMERF_FAULT")
    res = om.train_step(scene, b["rays"], b["target"], b["smooth_dirs"])
    om.sync(timeout_ms=20000)
    ref = oracle.train(oracle.OracleScene(sc), b["rays"], b["target"], b["smooth_dirs"], lam=(1.0, 1e-2, 0.0))
    _check(res, ref, "after the reported timeout")
