"""Shared helpers for the GPU parity tests (CUDA path vs FP64 oracle)."""
import numpy as np

import oracle
import synth

# tolerances (FP32 path): pixel max-abs error and gradient relative error
RGB_ATOL = 1e-4
GRAD_RTOL = 1e-3
BF16_PSNR_DB = 45.0


def gpu_scene(sc, device="cuda", **kw):
    import paper_2404_09531_gb300 as om
    return om.scene_from_synth(sc, device=device, **kw)


def oracle_scene_for(sc, table=None, pool=None, **over):
    """Oracle view of a synth scene; brick grids use the given table/pool."""
    if sc["spec"].brick and sc.get("grid") is None:
        sc = dict(sc, grid=pool, table=table)
    return oracle.OracleScene(sc, **over)


def brick_inputs(sc):
    """Brick table from the oracle's allocation rule and the generator's pool."""
    table = oracle.brick_table(sc["spec"], sc["occ"])
    pool = synth.fill_brick_pool(sc, table)
    return table, pool


def compare_render(rgb, count, ref, atol=RGB_ATOL, what=""):
    """Counts bit-exact and rgb within atol on rays the oracle marks unambiguous."""
    rgb = np.asarray(rgb, np.float64)
    count = np.asarray(count)
    ok = ref["ambiguous"] == 0
    assert ok.mean() > 0.99, f"{what}: too many ambiguous rays ({(~ok).sum()})"
    bad = np.nonzero(count[ok] != ref["count"][ok])[0]
    assert bad.size == 0, (f"{what}: {bad.size} count mismatches, first rays "
                           f"{np.nonzero(ok)[0][bad[:5]]}: gpu {count[ok][bad[:5]]} oracle {ref['count'][ok][bad[:5]]}")
    err = np.abs(rgb - ref["rgb"])[ok]
    assert err.max() <= atol, f"{what}: rgb max-abs {err.max():.3e} > {atol}"
    return float(err.max()), int((~ok).sum())


def psnr(a, b, peak=1.0):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(peak * peak / mse)


def grad_errors(g_gpu, g_ref):
    """(norm-relative error, max-abs error / max |ref|) of one gradient tensor."""
    a = np.asarray(g_gpu, np.float64).reshape(-1)
    b = np.asarray(g_ref, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.linalg.norm(a)), float(np.abs(a).max(initial=0.0))
    return float(np.linalg.norm(a - b) / nb), float(np.abs(a - b).max() / np.abs(b).max())


def edge_rays(spec, n_random=600, seed=0):
    """Rays covering the cases the method has: oblique, axis-parallel, grazing,
    missing the box, starting inside it, pointing away from it."""
    rng = np.random.default_rng(seed)
    x0, x1, y0, y1, z0, z1 = spec.aabb
    rays = []
    # oblique rays from above
    o = np.stack([rng.uniform(x0, x1, n_random), rng.uniform(y0, y1, n_random),
                  np.full(n_random, z1 + 0.5)], 1)
    t = np.stack([rng.uniform(x0, x1, n_random), rng.uniform(y0, y1, n_random),
                  np.full(n_random, z0)], 1)
    d = t - o
    rays.append(np.concatenate([o, d / np.linalg.norm(d, axis=1, keepdims=True)], 1))
    # straight down / straight along x and y / grazing nearly horizontal
    m = 64
    xs, ys = rng.uniform(x0, x1, m), rng.uniform(y0, y1, m)
    zc = 0.5 * (z0 + z1) + rng.uniform(-0.3, 0.3, m) * (z1 - z0)
    rays.append(np.stack([xs, ys, np.full(m, z1 + 1.0), np.zeros(m), np.zeros(m), -np.ones(m)], 1))
    rays.append(np.stack([np.full(m, x0 - 0.5), ys, zc, np.ones(m), np.zeros(m), np.zeros(m)], 1))
    rays.append(np.stack([xs, np.full(m, y1 + 0.5), zc, np.zeros(m), -np.ones(m), np.zeros(m)], 1))
    g = np.stack([np.full(m, x0 - 0.3), ys, zc, np.ones(m), rng.uniform(-0.2, 0.2, m),
                  rng.uniform(-1e-4, 1e-4, m)], 1)
    g[:, 3:] /= np.linalg.norm(g[:, 3:], axis=1, keepdims=True)
    rays.append(g)
    # missing the box, starting inside, pointing away
    rays.append(np.stack([xs, ys, np.full(m, z1 + 1.0), np.zeros(m), np.zeros(m), np.ones(m)], 1))
    inside = np.stack([xs, ys, zc], 1)
    dd = rng.normal(0, 1, (m, 3))
    dd /= np.linalg.norm(dd, axis=1, keepdims=True)
    rays.append(np.concatenate([inside, dd], 1))
    return np.concatenate(rays).astype(np.float32)


BF16_U = 2.0 ** -8  # unit roundoff of bfloat16: 8 significant bits, round to nearest: |x~ - x| <= 2^-8 |x|


def _view_encoding64(d):
    d = np.asarray(d, np.float64)
    parts = [d]
    for k in range(4):
        parts += [np.sin((2.0 ** k) * d), np.cos((2.0 ** k) * d)]
    return np.concatenate(parts, 1)


def bf16_mlp_error_bound(F, d, mlp, f32_atol=RGB_ATOL):
    """Per-ray bound on |rgb_bf16 - rgb_ref| for the BF16 form of the render
    against a reference that uses the same (BF16-rounded) features.

    The BF16 form runs the deferred MLP (Eq. 4) with the input row
    [F, encoding(d)], the three weight matrices and the two hidden ReLU
    outputs rounded to bfloat16 (relative error <= u = 2^-8 each) and FP32
    accumulation and biases.  First-order propagation, layer by layer, with
    a and h the reference pre-activations and ReLU outputs (FP64), u = 2^-8:
      input    |dx_i| <= u |x_i| + f32_atol (F in FP32 vs FP64; the encoding ~1e-7)
      layer l  e_j <= sum_i (1 + u) |W_ji| dh_i + u |W_ji| |h_i|   (+ FP32 sums, n 2^-24 sum |W h|)
      ReLU     dh_j <= e_j + u (|h_j| + e_j)   (1-Lipschitz, then the rounding)
      output   |dy| <= e_3 / 4                  (sigmoid slope <= 1/4)
    plus f32_atol for the composited colour's own FP32 error (the FP32 bar).
    Rays without samples (F = 0, the background) get f32_atol.
    Returns an array [n] (the bound on every channel of the ray)."""
    u = BF16_U
    F = np.asarray(F, np.float64)
    W1 = np.asarray(mlp[0:544], np.float64).reshape(16, 34)
    b1 = np.asarray(mlp[544:560], np.float64)
    W2 = np.asarray(mlp[560:816], np.float64).reshape(16, 16)
    b2 = np.asarray(mlp[816:832], np.float64)
    W3 = np.asarray(mlp[832:880], np.float64).reshape(3, 16)
    x = np.concatenate([F, _view_encoding64(d)], 1)
    dx = u * np.abs(x)
    dx[:, :7] += f32_atol
    dx[:, 7:] += 1e-6

    def layer(W, b, h, dh, n):
        a = h @ W.T + b
        s = np.abs(h) @ np.abs(W).T
        e = (np.abs(dh) @ np.abs(W).T) * (1 + u) + u * s + n * 2.0 ** -24 * (s + np.abs(b))
        return a, e

    a1, e1 = layer(W1, b1, x, dx, 35)
    h1 = np.maximum(a1, 0.0)
    d1 = e1 + u * (h1 + e1)
    a2, e2 = layer(W2, b2, h1, d1, 17)
    h2 = np.maximum(a2, 0.0)
    d2 = e2 + u * (h2 + e2)
    _, e3 = layer(W3, np.asarray(mlp[880:883], np.float64), h2, d2, 17)
    bound = e3.max(1) / 4.0 + f32_atol
    live = np.abs(F).sum(1) > 0
    return np.where(live, bound, f32_atol)


def bf16_mlp_error_sigma(F, d, mlp):
    """Per-ray standard deviation of the BF16 form's colour error under the
    standard probabilistic model of rounding (independent relative errors,
    uniform on [-u, u], variance u^2 / 3), linearised at the reference
    activations: every rounded quantity q (input, weight, hidden output)
    contributes (dy/dq * q)^2 u^2 / 3.  Returns [n, 3]."""
    u = BF16_U
    F = np.asarray(F, np.float64)
    W1 = np.asarray(mlp[0:544], np.float64).reshape(16, 34)
    b1 = np.asarray(mlp[544:560], np.float64)
    W2 = np.asarray(mlp[560:816], np.float64).reshape(16, 16)
    b2 = np.asarray(mlp[816:832], np.float64)
    W3 = np.asarray(mlp[832:880], np.float64).reshape(3, 16)
    b3 = np.asarray(mlp[880:883], np.float64)
    x = np.concatenate([F, _view_encoding64(d)], 1)
    a1 = x @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    a3 = h2 @ W3.T + b3
    y = 1.0 / (1.0 + np.exp(-a3))
    s3 = y * (1.0 - y)                                   # [n, 3]
    J2 = s3[:, :, None] * W3[None] * (a2 > 0)[:, None, :]  # dy/da2 [n, 3, 16]
    G2 = J2 @ W2                                         # dy/dh1 [n, 3, 16]
    J1 = G2 * (a1 > 0)[:, None, :]                       # dy/da1 [n, 3, 16]
    G1 = J1 @ W1                                         # dy/dx  [n, 3, 34]
    var = (G1 * x[:, None, :]) ** 2                      # input rounding
    var = var.sum(2)
    var += ((J1[:, :, :, None] * W1[None, None] * x[:, None, None, :]) ** 2).sum((2, 3))   # W1
    var += ((G2 * h1[:, None, :]) ** 2).sum(2)                                           # h1
    var += ((J2[:, :, :, None] * W2[None, None] * h1[:, None, None, :]) ** 2).sum((2, 3))  # W2
    G3 = s3[:, :, None] * W3[None]                                                       # dy/dh2
    var += ((G3 * h2[:, None, :]) ** 2).sum(2)                                           # h2 rounding
    var += ((s3[:, :, None] * W3[None] * h2[:, None, :]) ** 2).sum(2)                    # W3
    sig = np.sqrt(var * u * u / 3.0)
    live = np.abs(F).sum(1) > 0
    return np.where(live[:, None], sig, 0.0)
