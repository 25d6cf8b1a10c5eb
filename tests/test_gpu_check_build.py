"""The checking build (libomerf_check.so, OMERF_CHECK=1), run in a child
process that loads it instead of the default library:
- the benchmarked render (all 8 config-2 cameras, tables of Sec. 4.4's rule),
  a training step and the two regularisers on the brick scene read no
  feature outside the arrays and no corner of an unstored brick;
- on a table sparser than the rule, with early termination off (so that
  both sides evaluate exactly the same samples), the count of corner reads
  of unstored bricks equals the FP64 oracle's count of the same reads."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
import torch, dataclasses
import oracle, synth
import paper_2404_09531_gb300 as om
from test_gpu_bricks import _pool_from_dense, _reindex
assert om.lib().omerf_check_build() == 1
out = {}
sc = synth.make_scene(2)
table = oracle.brick_table(sc["spec"], sc["occ"])
scene = om.scene_from_synth(sc, device="cuda", table=table)
om.render_cameras(scene, synth.make_cameras(2))
out["render"] = om.check_counts(scene)
b = synth.make_train_batch(2, 4096)
om.train_step(scene, b["rays"], b["target"], b["smooth_dirs"], lam=(1.0, 1e-2, 1e-4))
g = om.zero_grads(scene)
om.sparsity_loss(scene, synth.sparsity_points(sc, 4096), grads=g)
om.entropy_loss(scene, synth.entropy_rays(sc, 512), grads=g)
out["train"] = om.check_counts(scene)
s1 = synth.make_scene(1)
spec = dataclasses.replace(s1["spec"], brick=4)
rule = oracle.brick_table(spec, s1["occ"])
keep = (rule >= 0) & (np.random.default_rng(7).uniform(size=rule.shape) < 0.6)
t1 = _reindex(keep)
sb = dict(s1, spec=spec, grid=_pool_from_dense(s1["grid"], t1, 4), table=t1)
sparse = om.scene_from_synth(sb, device="cuda", t_thr=0.0)
rays = oracle.camera_rays(synth.make_cameras(1)[0])
om.render(sparse, rays=rays)
out["sparser"] = om.check_counts(sparse)
out["sparser_oracle"] = oracle.render(oracle.OracleScene(sb, t_thr=0.0), rays)["unalloc"]
print("RESULT " + json.dumps(out))
"""


def test_checking_build_counts():
    lib = os.path.join(ROOT, "paper_2404_09531_gb300", "libomerf_check.so")
    if not os.path.exists(lib):
        pytest.skip("the checking build is not built")
    env = dict(os.environ, OMERF_CHECK="1")
    res = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True,
                         text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    line = [l for l in res.stdout.splitlines() if l.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    assert out["render"] == [0, 0]
    assert out["train"] == [0, 0]
    assert out["sparser"][1] == 0
    assert out["sparser_oracle"] > 0
    assert out["sparser"][0] == out["sparser_oracle"]


def test_default_build_has_no_counters():
    import paper_2404_09531_gb300 as om
    import synth
    if os.environ.get("OMERF_CHECK") == "1":
        pytest.skip("this process loaded the checking build")
    assert om.lib().omerf_check_build() == 0
    scene = om.scene_from_synth(synth.make_scene(1), device="cuda")
    with pytest.raises(om.OmerfError, match="without OMERF_CHECK"):
        om.check_counts(scene)
