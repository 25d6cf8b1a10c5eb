"""The BF16 error model of the deferred MLP (tests/_util.py), checked on the
CPU against a direct simulation of the BF16 form's arithmetic: input row,
weights and hidden ReLU outputs rounded to bfloat16 (torch's round-to-nearest
conversion), biases and sums kept wide.  The worst-case bound must hold for
every ray, and the probabilistic model must predict the observed spread."""
import numpy as np
import pytest

import synth
from _util import _view_encoding64, bf16_mlp_error_bound, bf16_mlp_error_sigma

torch = pytest.importorskip("torch")


def _bf16(a):
    return torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16).double().numpy()


def _mlp(x, mlp, rnd):
    W1 = np.asarray(mlp[0:544], np.float64).reshape(16, 34)
    W2 = np.asarray(mlp[560:816], np.float64).reshape(16, 16)
    W3 = np.asarray(mlp[832:880], np.float64).reshape(3, 16)
    b1, b2, b3 = (np.asarray(mlp[a:b], np.float64) for a, b in ((544, 560), (816, 832), (880, 883)))
    h1 = np.maximum(rnd(x) @ rnd(W1).T + b1, 0.0)
    h2 = np.maximum(rnd(h1) @ rnd(W2).T + b2, 0.0)
    return 1.0 / (1.0 + np.exp(-(rnd(h2) @ rnd(W3).T + b3)))


@pytest.mark.parametrize("cfg", [1, 4])
def test_bf16_mlp_error_model(cfg):
    mlp = synth.make_scene(cfg)["mlp"]
    rng = np.random.default_rng(cfg)
    n = 20000
    F = rng.uniform(0.0, 1.0, (n, 7)) * rng.uniform(0.0, 1.0, (n, 1))  # sum of weights <= 1
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    x = np.concatenate([F, _view_encoding64(d)], 1)
    exact = _mlp(x, mlp, lambda a: np.asarray(a, np.float64))
    bf = _mlp(x, mlp, _bf16)
    err = np.abs(bf - exact)
    bound = bf16_mlp_error_bound(F, d, mlp, f32_atol=0.0)
    sig = bf16_mlp_error_sigma(F, d, mlp)
    assert np.all(err.max(1) <= bound)
    assert (err / sig).max() <= 6.0
    # the spread the model predicts, to within a small factor
    ratio = np.mean(err ** 2) / np.mean(sig ** 2)
    assert 0.2 <= ratio <= 2.0, ratio
    # and a plainly wrong model fails: rounding units one bit coarser/finer
    assert (err / (sig / 4)).max() > 6.0
