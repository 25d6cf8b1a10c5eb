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
