"""Brick grids on the GPU against the FP64 oracle on every table the ABI
accepts (Eq. 2 with Sec. 4.4's sparse storage), and brick tables that follow
the occupancy plane while training moves it.

- A table sparser than the allocation rule: each corner vertex is read
  through its own brick (zero where that brick is not stored), on both sides,
  including samples whose lowest-corner brick is missing while a neighbour
  brick holding some of their corners is stored.
- omerf_grow_brick_table: bit-exact against a numpy restatement over the
  oracle's rule table.
- Trainer on a brick scene whose occupancy bounds move by more than the
  allocation rule's one-voxel dilation: the table grows, the pool, the FP32
  master and both Adam moments are re-extracted into the new layout (kept
  bricks keep their values, new ones start at zero), and the trained scene
  renders and differentiates like the oracle on the same table and pool.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from _util import GRAD_RTOL, bf16_mlp_error_bound, compare_render, gpu_scene, grad_errors

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
import paper_2404_09531_gb300 as om  # noqa: E402

KEYS = ("grid", "p_xy", "p_xz", "p_yz", "occ", "mlp")
LAM = (1.0, 1e-2, 1e-4)
B = 4


def _pool_from_dense(grid, table, B):
    nb = int(table.max()) + 1 if (table >= 0).any() else 0
    pool = np.zeros((max(nb, 1), B, B, B, 8), np.float32)
    for (bi, bj, bk), b in np.ndenumerate(table):
        if b >= 0:
            blk = grid[bi * B:(bi + 1) * B, bj * B:(bj + 1) * B, bk * B:(bk + 1) * B]
            pool[b, :blk.shape[0], :blk.shape[1], :blk.shape[2]] = blk
    return pool


def _reindex(flags):
    """x-major pool indices of a boolean brick mask (-1 where not stored)."""
    t = np.full(flags.shape, -1, np.int32)
    t[flags] = np.arange(int(flags.sum()), dtype=np.int32)
    return t


def _brick_scene(cfg=1):
    sc = synth.make_scene(cfg)
    spec = dataclasses.replace(sc["spec"], brick=B)
    return sc, spec


def _check_grads(res, ref, what):
    for k in KEYS:
        nrel, mrel = grad_errors(res["grads"][k].cpu().numpy(), ref["grads"][k])
        assert nrel <= GRAD_RTOL and mrel <= GRAD_RTOL, f"{what} {k}: norm-rel {nrel:.2e}, max-rel {mrel:.2e}"


def test_sparser_table_renders_and_trains_like_the_oracle():
    sc, spec = _brick_scene()
    rule = oracle.brick_table(spec, sc["occ"])
    rng = np.random.default_rng(7)
    keep = (rule >= 0) & (rng.uniform(size=rule.shape) < 0.6)
    table = _reindex(keep)
    pool = _pool_from_dense(sc["grid"], table, B)
    sb = dict(sc, spec=spec, grid=pool, table=table)
    scene = gpu_scene(sb)
    cam = synth.make_cameras(1)[0]
    rgb, cnt = om.render(scene, camera=cam)
    torch.cuda.synchronize()
    ref = oracle.render(oracle.OracleScene(sb), oracle.camera_rays(cam))
    assert ref["unalloc"] > 0  # the case where the two readings of a table differ is exercised
    compare_render(rgb.cpu().numpy(), cnt.cpu().numpy(), ref, what="sparser table")
    batch = synth.make_train_batch(3, 4096, seed=5)
    res = om.train_step(scene, batch["rays"], batch["target"], batch["smooth_dirs"], lam=LAM)
    torch.cuda.synchronize()
    oref = oracle.train(oracle.OracleScene(sb), batch["rays"], batch["target"], batch["smooth_dirs"], lam=LAM)
    np.testing.assert_allclose(float(res["loss"][0].item()), oref["loss"], rtol=1e-5)
    _check_grads(res, oref, "sparser table")


def test_grow_brick_table_bit_exact():
    sc, spec = _brick_scene()
    rng = np.random.default_rng(3)
    rule0 = oracle.brick_table(spec, sc["occ"])
    old_flags = ((rule0 >= 0) & (rng.uniform(size=rule0.shape) < 0.7)) | (rng.uniform(size=rule0.shape) < 0.05)
    old = _reindex(old_flags)
    occ = sc["occ"].copy()
    sel = rng.uniform(size=occ.shape[:2]) < 0.3
    occ[sel, 1] += 0.06
    occ[sel, 0] -= 0.04
    rule = oracle.brick_table(spec, occ)
    want = _reindex(old_flags | (rule >= 0))
    table, n_alloc, missing = om.grow_brick_table(spec.aabb, spec.L, B, torch.as_tensor(occ).cuda(),
                                                  torch.as_tensor(old).cuda())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(table.cpu().numpy(), want)
    assert int(n_alloc.item()) == int((want >= 0).sum())
    assert int(missing.item()) == int(((rule >= 0) & ~old_flags).sum()) > 0
    # a table that already covers the rule: nothing to add, same bricks
    t2, n2, m2 = om.grow_brick_table(spec.aabb, spec.L, B, torch.as_tensor(occ).cuda(), table)
    torch.cuda.synchronize()
    assert int(m2.item()) == 0
    np.testing.assert_array_equal(t2.cpu().numpy(), want)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_trainer_grows_bricks_as_bounds_move(dtype):
    sc, spec = _brick_scene()
    table = oracle.brick_table(spec, sc["occ"])
    sb = dict(sc, spec=spec, grid=_pool_from_dense(sc["grid"], table, B), table=table)
    scene = gpu_scene(sb, feat_dtype=dtype)
    batch = synth.make_train_batch(3, 4096, seed=9)
    batch["target"] = oracle.render(oracle.OracleScene(synth.perturb_scene(sc)), batch["rays"])["rgb"].astype(
        np.float32)
    # bounds move ~lr_occ per Adam step: far beyond the one-voxel (0.0167) dilation
    tr = om.Trainer(scene, lr=(1e-2, 1e-2), lr_occ=(2e-2, 2e-2), lam_occ=0.0, lam_smooth=1e-2,
                    grow_bricks_every=0)
    grown = 0
    for _ in range(5):
        tr.step(batch["rays"], batch["target"], batch["smooth_dirs"])
        old_table = tr.scene.table.cpu().numpy()
        old = {k: t.cpu().numpy() for k, t in (("master", tr.master["grid"]), ("m", tr.moments["grid"][0]),
                                               ("v", tr.moments["grid"][1]), ("grid", tr.scene.grid.float()))}
        if not tr.grow_bricks():
            continue
        grown += 1
        new_table = tr.scene.table.cpu().numpy()
        assert np.all(new_table[old_table >= 0] >= 0)  # no brick is dropped
        new = {k: t.cpu().numpy() for k, t in (("master", tr.master["grid"]), ("m", tr.moments["grid"][0]),
                                               ("v", tr.moments["grid"][1]), ("grid", tr.scene.grid.float()))}
        kept = old_table >= 0
        added = (new_table >= 0) & ~kept
        for k in new:
            np.testing.assert_array_equal(new[k][new_table[kept]], old[k][old_table[kept]], err_msg=k)
            assert not new[k][new_table[added]].any(), k
        assert tr.grads["grid"].shape == tr.scene.grid.shape
        # the grown table covers the rule for the moved bounds
        rule = oracle.brick_table(spec, tr.scene.occ.cpu().numpy())
        assert np.all(new_table[rule >= 0] >= 0)
        assert not tr.grow_bricks()
    assert grown >= 1
    # the trained scene against the oracle on the same table, pool and bounds
    st = dict(sc, spec=spec, grid=tr.scene.grid.float().cpu().numpy(), table=tr.scene.table.cpu().numpy(),
              occ=tr.scene.occ.cpu().numpy(), mlp=tr.scene.mlp.cpu().numpy(),
              **{k: getattr(tr.scene, k).float().cpu().numpy() for k in ("p_xy", "p_xz", "p_yz")})
    cam = synth.make_cameras(1)[0]
    rgb, cnt = om.render(tr.scene, camera=cam)
    torch.cuda.synchronize()
    ref = oracle.render(oracle.OracleScene(st), oracle.camera_rays(cam))
    if dtype == torch.float32:
        compare_render(rgb.cpu().numpy(), cnt.cpu().numpy(), ref, what="trained FP32")
    else:
        # the oracle reads the same BF16 values; the BF16 MLP's operand
        # rounding bounds the colour error per ray
        ok = ref["ambiguous"] == 0
        cnt_np, rgb_np = cnt.cpu().numpy(), rgb.cpu().numpy().astype(np.float64)
        assert np.array_equal(cnt_np[ok], ref["count"][ok])
        bound = bf16_mlp_error_bound(ref["F"], oracle.camera_rays(cam)[:, 3:], st["mlp"])
        assert np.all(np.abs(rgb_np - ref["rgb"]).max(1)[ok] <= bound[ok])
    res = om.train_step(tr.scene, batch["rays"], batch["target"], batch["smooth_dirs"], lam=LAM)
    torch.cuda.synchronize()
    oref = oracle.train(oracle.OracleScene(st), batch["rays"], batch["target"], batch["smooth_dirs"], lam=LAM)
    _check_grads(res, oref, f"trained {dtype}")
