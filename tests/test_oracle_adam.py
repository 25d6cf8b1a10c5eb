"""Pins for the optimiser reference (appendix A schedules, Adam update)."""
import numpy as np
import pytest

from oracle import adam


def test_first_step_closed_form():
    rng = np.random.default_rng(0)
    p0 = rng.normal(size=100)
    g = rng.normal(size=100)
    p, m, v = adam.adam_step(p0, g, np.zeros(100), np.zeros(100), lr=0.01, step=1)
    np.testing.assert_allclose(p, p0 - 0.01 * g / (np.abs(g) + 1e-15), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-13)
    np.testing.assert_allclose(v, 0.01 * g * g, rtol=1e-13)


def test_matches_torch_adam_float64():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    p0 = rng.normal(size=64)
    grads = rng.normal(size=(7, 64))
    t = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=3e-3, betas=(0.9, 0.99), eps=1e-15)
    p, m, v = p0.copy(), np.zeros(64), np.zeros(64)
    for k, g in enumerate(grads, start=1):
        t.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = adam.adam_step(p, g, m, v, lr=3e-3, step=k)
    np.testing.assert_allclose(p, t.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_schedules():
    assert adam.lr_exponential(1e-2, 1e-3, 0, 80000) == pytest.approx(1e-2)
    assert adam.lr_exponential(1e-2, 1e-3, 80000, 80000) == pytest.approx(1e-3)
    assert adam.lr_exponential(1e-2, 1e-3, 40000, 80000) == pytest.approx(1e-2 * 0.1 ** 0.5)
    assert adam.lambda_occ(9999) == 0.0
    assert adam.lambda_occ(10000) == pytest.approx(1e-4)
    assert adam.lambda_occ(11999) == pytest.approx(1e-4)
    assert adam.lambda_occ(12000) == pytest.approx(1.5e-4)
    assert adam.lambda_occ(10 ** 7) == 0.2
