"""FP64 reference of the optimiser step and schedules -- TEST INFRASTRUCTURE ONLY.

Oblique-MERF trains with Adam (appendix A: beta1 = 0.9, beta2 = 0.99,
eps = 1e-15), learning rates decaying exponentially from 1e-2 to 1e-3
(occupancy plane: 5e-5 to 1e-5), and the occupancy-loss weight lambda_7 = 0
until iteration 10,000, then 1e-4, multiplied by 1.5 every 2,000 iterations up
to 0.2.  The update is Adam's (Kingma and Ba) with bias correction:

    m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2
    p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)

Pinned in tests/test_oracle_adam.py by a closed form (the first step moves
every parameter by lr * g / (|g| + eps)) and by torch.optim.Adam in float64.
"""
import numpy as np


def adam_step(p, g, m, v, lr, step, beta1=0.9, beta2=0.99, eps=1e-15):
    """One Adam step in float64 on copies; returns (p, m, v)."""
    p = np.asarray(p, np.float64).copy()
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    p -= lr * mh / (np.sqrt(vh) + eps)
    return p, m, v


def lr_exponential(lr0, lr1, step, total):
    """Exponential decay from lr0 (step 0) to lr1 (step total), clamped."""
    s = min(max(step, 0), total) / float(total)
    return lr0 * (lr1 / lr0) ** s


def lambda_occ(step):
    """Occupancy-loss weight of appendix A at iteration `step`."""
    if step < 10000:
        return 0.0
    k = (step - 10000) // 2000
    return 0.2 if k >= 20 else min(1e-4 * 1.5 ** k, 0.2)  # 1e-4 * 1.5^19 > 0.2 already
