"""Seeded synthetic oblique-photography scenes, cameras and training batches.

The paper's datasets (Campus-Oblique, Matrix City) are not available, so these
scenes stand in for their shape: a flat axis-aligned box whose xy-plane is the
ground, a height field that the occupancy plane of Sec. 4.1 brackets from below
and above, and cameras looking down at 30-60 degrees of pitch.

Everything here is scene *content*: feature values, occupancy bounds, MLP
weights, camera poses and training rays.  None of the renderer's arithmetic
lives here.

Array layouts (all channel-last, x-major):
  grid   dense [Lx][Ly][Lz][8] float32, or a brick pool [nb][B][B][B][8]
         addressed through an int32 brick table [ceil(Lx/B)][ceil(Ly/B)][ceil(Lz/B)]
  p_xy   [Rx][Ry][8]   p_xz [Rx][Rz][8]   p_yz [Ry][Rz][8]
  occ    [M][M][2]     (z_min, z_max) per occupancy cell, cell-centred
  mlp    883 float32   W1[16][34] b1[16] W2[16][16] b2[16] W3[3][16] b3[3]
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NCH = 8
MLP_NPARAM = 16 * 34 + 16 + 16 * 16 + 16 + 3 * 16 + 3  # 883
SEED_BASE = 20240415


@dataclasses.dataclass(frozen=True)
class SceneSpec:
    """Sizes and constants of one synthetic workload."""

    name: str
    cfg: int
    aabb: tuple  # (x0, x1, y0, y1, z0, z1)
    L: tuple  # grid vertices (Lx, Ly, Lz)
    brick: int  # brick edge in vertices, 0 = dense grid
    R: tuple  # plane texels (Rx, Ry, Rz)
    M: int  # occupancy cells per axis
    step: float  # lattice spacing (a power of two)
    n_max: int
    eps: float  # occupancy ramp width (Eq. 6)
    margin: float  # occupancy interval half-width around the surface
    t_thr: float = 1e-4
    city: bool = False  # heightfield with buildings and a void outside the city
    city_radius: float = 0.0
    n_cams: int = 1
    width: int = 64
    height: int = 64
    fov_y_deg: float = 45.0
    cam_dist: float = 2.5
    feat_dtype: str = "f32"  # storage type of grid and planes on the GPU
    lookat_range: float = 0.5  # camera targets uniform in [-r, r]^2 at z = 0


CONFIGS = {
    # Forward render 64x64, FP32 (small case the oracle finishes in seconds).
    1: SceneSpec("render-64x64-heightfield-fp32", 1, (-1.0, 1.0, -1.0, 1.0, -0.125, 0.125),
                 (64, 64, 16), 0, (256, 256, 32), 32, 1.0 / 256, 128, 0.01, 0.03,
                 n_cams=1, width=64, height=64, fov_y_deg=45.0, cam_dist=2.5),
    # Forward render 1920x1080 x 8 oblique cameras, sparse 512x512x32 grid, FP32.
    2: SceneSpec("render-1920x1080x8-oblique-city-fp32", 2, (-1.0, 1.0, -1.0, 1.0, -0.0625, 0.0625),
                 (512, 512, 32), 8, (2048, 2048, 128), 256, 1.0 / 2048, 512, 0.002, 0.006,
                 city=True, city_radius=0.555, n_cams=8, width=1920, height=1080,
                 fov_y_deg=50.0, cam_dist=0.6, lookat_range=0.25),
    # Training fwd+bwd on the config-1 scene, 2^18 rays from 16 cameras.
    3: SceneSpec("train-2^18-rays-heightfield-fp32", 3, (-1.0, 1.0, -1.0, 1.0, -0.125, 0.125),
                 (64, 64, 16), 0, (256, 256, 32), 32, 1.0 / 256, 128, 0.01, 0.03,
                 n_cams=16, width=256, height=256, fov_y_deg=45.0, cam_dist=2.5),
    # BF16 render 3840x2160 x 4 cameras, sparse 1024x1024x64 grid.
    4: SceneSpec("render-3840x2160x4-oblique-city-bf16", 4, (-1.0, 1.0, -1.0, 1.0, -0.0625, 0.0625),
                 (1024, 1024, 64), 8, (4096, 4096, 256), 512, 1.0 / 2048, 512, 0.002, 0.006,
                 city=True, city_radius=0.63, n_cams=4, width=3840, height=2160,
                 fov_y_deg=50.0, cam_dist=0.6, lookat_range=0.3, feat_dtype="bf16"),
    # Large training: 2^20 rays from 64 cameras, BF16 features with FP32 master copy.
    5: SceneSpec("train-2^20-rays-heightfield-bf16", 5, (-1.0, 1.0, -1.0, 1.0, -0.125, 0.125),
                 (64, 64, 16), 0, (256, 256, 32), 32, 1.0 / 256, 128, 0.01, 0.03,
                 n_cams=64, width=256, height=256, fov_y_deg=45.0, cam_dist=2.5,
                 feat_dtype="bf16"),
}


def scene_spec(cfg: int, **overrides) -> SceneSpec:
    spec = CONFIGS[cfg]
    return dataclasses.replace(spec, **overrides) if overrides else spec


# --------------------------------------------------------------------------
# Height fields (scene content)
# --------------------------------------------------------------------------

class _Heightfield:
    """Sum of 4 seeded sines, optionally plus axis-aligned box buildings."""

    def __init__(self, rng: np.random.Generator, city: bool):
        self.city = city
        if not city:
            self.a = rng.uniform(0.01, 0.02, 4)
            self.base = 0.0
        else:
            self.a = rng.uniform(0.001, 0.0025, 4)  # total amplitude <= 0.01
            self.base = -0.03
        self.u = rng.uniform(-2.0, 2.0, 4)
        self.v = rng.uniform(-2.0, 2.0, 4)
        self.phi = rng.uniform(0.0, 2.0 * math.pi, 4)
        if city:
            nb = 64
            self.bc = rng.uniform(-0.55, 0.55, (nb, 2))
            self.bs = rng.uniform(0.02, 0.1, (nb, 2))
            self.bh = rng.uniform(0.005, 0.04, nb)

    def ground(self, x, y):
        h = np.full(np.broadcast(x, y).shape, self.base, dtype=np.float64)
        for k in range(4):
            h += self.a[k] * np.sin(2.0 * math.pi * (self.u[k] * x + self.v[k] * y) + self.phi[k])
        return h

    def surface(self, x, y):
        g = self.ground(x, y)
        if not self.city:
            return g
        extra = np.zeros_like(g)
        for c, s, hb in zip(self.bc, self.bs, self.bh):
            inside = (np.abs(x - c[0]) <= 0.5 * s[0]) & (np.abs(y - c[1]) <= 0.5 * s[1])
            extra = np.where(inside, np.maximum(extra, hb), extra)
        return g + extra


def _rng(cfg_seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + cfg_seed + stream))


def _features(rng, shape, dens_std=0.1, other_std=0.5):
    out = rng.normal(0.0, other_std, shape).astype(np.float32)
    out[..., 0] = rng.normal(0.0, dens_std, shape[:-1]).astype(np.float32)
    return out


def _vertex_xyz(spec: SceneSpec, i, j, k):
    x0, x1, y0, y1, z0, z1 = spec.aabb
    Lx, Ly, Lz = spec.L
    return (x0 + i * (x1 - x0) / (Lx - 1), y0 + j * (y1 - y0) / (Ly - 1),
            z0 + k * (z1 - z0) / (Lz - 1))


def make_scene(cfg: int | SceneSpec, seed: int | None = None) -> dict:
    """Draw the feature volume, occupancy plane and MLP of one workload.

    For a brick grid (spec.brick > 0) the returned dict has no ``grid``: the
    brick set depends on the allocation rule, so the caller builds a table and
    then calls :func:`fill_brick_pool`.
    """
    spec = CONFIGS[cfg] if isinstance(cfg, int) else cfg
    s = spec.cfg if seed is None else seed
    rng = _rng(s)
    hf = _Heightfield(rng, spec.city)
    x0, x1, y0, y1, z0, z1 = spec.aabb
    Lx, Ly, Lz = spec.L
    Rx, Ry, Rz = spec.R
    M = spec.M

    scene = {"spec": spec, "heightfield": hf, "seed": s}
    scene["p_xy"] = _features(rng, (Rx, Ry, NCH))
    scene["p_xz"] = _features(rng, (Rx, Rz, NCH))
    scene["p_yz"] = _features(rng, (Ry, Rz, NCH))
    scene["mlp"] = rng.normal(0.0, 0.3, MLP_NPARAM).astype(np.float32)

    # occupancy plane: interval [surface - margin, surface + margin] per cell
    cx = x0 + (np.arange(M) + 0.5) * (x1 - x0) / M
    cy = y0 + (np.arange(M) + 0.5) * (y1 - y0) / M
    X, Y = np.meshgrid(cx, cy, indexing="ij")
    occ = np.empty((M, M, 2), np.float32)
    if not spec.city:
        h = hf.surface(X, Y)
        occ[..., 0] = h - spec.margin
        occ[..., 1] = h + spec.margin
    else:
        # supersample each cell 3x3: the interval spans ground to roof
        hx = (x1 - x0) / M
        hy = (y1 - y0) / M
        lo = np.full((M, M), np.inf)
        hi = np.full((M, M), -np.inf)
        for a in (-0.45, 0.0, 0.45):
            for b in (-0.45, 0.0, 0.45):
                g = hf.ground(X + a * hx, Y + b * hy)
                t = hf.surface(X + a * hx, Y + b * hy)
                lo = np.minimum(lo, g)
                hi = np.maximum(hi, t)
        occ[..., 0] = lo - spec.margin
        occ[..., 1] = hi + spec.margin
        void = (X * X + Y * Y) > spec.city_radius ** 2
        occ[void, 0] = 1.0
        occ[void, 1] = -1.0  # z_max < z_min: an empty cell
    scene["occ"] = occ

    if spec.brick == 0:
        i, j, k = np.meshgrid(np.arange(Lx), np.arange(Ly), np.arange(Lz), indexing="ij")
        grid = _features(np.random.Generator(np.random.PCG64(SEED_BASE + s + 500)), (Lx, Ly, Lz, NCH))
        vx, vy, vz = _vertex_xyz(spec, i, j, k)
        below = vz < hf.surface(vx, vy)
        grid[..., 0] += np.where(below, 5.0, -5.0).astype(np.float32)
        scene["grid"] = grid
        scene["table"] = None
    return scene


def fill_brick_pool(scene: dict, table: np.ndarray) -> np.ndarray:
    """Feature values of the allocated bricks, in pool order given by ``table``.

    ``table[bi, bj, bk]`` holds the pool index of a brick or -1.  Vertices
    past the grid's end (when L is not a multiple of B) are zero.
    """
    spec: SceneSpec = scene["spec"]
    B = spec.brick
    Lx, Ly, Lz = spec.L
    hf = scene["heightfield"]
    nb = int(table.max()) + 1 if table.size and table.max() >= 0 else 0
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + scene["seed"] + 500))
    pool = _features(rng, (max(nb, 1), B, B, B, NCH))[:nb].copy()
    coords = np.argwhere(table >= 0)
    idx = table[table >= 0]
    order = np.argsort(idx)
    coords = coords[order]
    li = np.arange(B)
    LI, LJ, LK = np.meshgrid(li, li, li, indexing="ij")
    chunk = 4096
    for c0 in range(0, nb, chunk):
        cc = coords[c0:c0 + chunk]
        I = cc[:, 0, None, None, None] * B + LI[None]
        J = cc[:, 1, None, None, None] * B + LJ[None]
        K = cc[:, 2, None, None, None] * B + LK[None]
        vx, vy, vz = _vertex_xyz(spec, I, J, K)
        below = vz < hf.surface(vx, vy)
        pool[c0:c0 + chunk, ..., 0] += np.where(below, 5.0, -5.0).astype(np.float32)
        outside = (I >= Lx) | (J >= Ly) | (K >= Lz)
        pool[c0:c0 + chunk][outside] = 0.0
    return pool


def perturb_scene(scene: dict, sigma: float = 0.05) -> dict:
    """A copy with every feature perturbed by N(0, sigma) (training targets)."""
    rng = _rng(scene["seed"], 2000)
    out = dict(scene)
    for key in ("grid", "p_xy", "p_xz", "p_yz"):
        if out.get(key) is not None:
            out[key] = (out[key] + rng.normal(0.0, sigma, out[key].shape)).astype(np.float32)
    return out


# --------------------------------------------------------------------------
# Cameras and training rays
# --------------------------------------------------------------------------

def _look_at_pose(pitch_deg, yaw_deg, target, dist):
    p = math.radians(pitch_deg)
    y = math.radians(yaw_deg)
    fwd = np.array([math.cos(p) * math.cos(y), math.cos(p) * math.sin(y), -math.sin(p)])
    origin = np.asarray(target, np.float64) - dist * fwd
    right = np.cross(fwd, [0.0, 0.0, 1.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    c2w = np.zeros((3, 4))
    c2w[:, 0] = right
    c2w[:, 1] = up
    c2w[:, 2] = -fwd  # the camera looks down its -z axis
    c2w[:, 3] = origin
    return c2w


def make_cameras(cfg: int | SceneSpec, n: int | None = None, seed: int | None = None) -> list:
    """Pinhole cameras as dicts: c2w (3x4 float32), fx, fy, cx, cy, width, height."""
    spec = CONFIGS[cfg] if isinstance(cfg, int) else cfg
    n = spec.n_cams if n is None else n
    rng = _rng(spec.cfg if seed is None else seed, 1000)
    W, H = spec.width, spec.height
    f = 0.5 * H / math.tan(0.5 * math.radians(spec.fov_y_deg))
    cams = []
    for c in range(n):
        if spec.cfg == 1 and c == 0:
            pitch, yaw, target = 45.0, 0.0, (0.0, 0.0, 0.0)
        else:
            pitch = rng.uniform(30.0, 60.0)
            yaw = rng.uniform(0.0, 360.0)
            t = rng.uniform(-spec.lookat_range, spec.lookat_range, 2)
            target = (t[0], t[1], 0.0)
        c2w = _look_at_pose(pitch, yaw, target, spec.cam_dist)
        cams.append({"c2w": c2w.astype(np.float32), "fx": np.float32(f), "fy": np.float32(f),
                     "cx": np.float32(0.5 * W), "cy": np.float32(0.5 * H),
                     "width": W, "height": H})
    return cams


def make_train_batch(cfg: int | SceneSpec, n_rays: int, K: int = 1, seed: int | None = None,
                     smooth_var: float = 0.3) -> dict:
    """Random training rays through random image points of the config's cameras.

    Directions are unit float32 vectors; smoothness directions s = d + delta
    with delta ~ N(0, smooth_var * I) (Eq. 9), drawn per ray and per k.
    """
    spec = CONFIGS[cfg] if isinstance(cfg, int) else cfg
    s = spec.cfg if seed is None else seed
    cams = make_cameras(spec, seed=s)
    rng = _rng(s, 1500)
    ci = rng.integers(0, len(cams), n_rays)
    px = rng.uniform(0.0, spec.width, n_rays)
    py = rng.uniform(0.0, spec.height, n_rays)
    rays = np.empty((n_rays, 6), np.float32)
    for c, cam in enumerate(cams):
        sel = ci == c
        if not sel.any():
            continue
        c2w = cam["c2w"].astype(np.float64)
        u = (px[sel] - float(cam["cx"])) / float(cam["fx"])
        v = -(py[sel] - float(cam["cy"])) / float(cam["fy"])
        dcam = np.stack([u, v, -np.ones_like(u)], 1)
        d = dcam @ c2w[:, :3].T
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        rays[sel, :3] = c2w[:, 3].astype(np.float32)
        rays[sel, 3:] = d.astype(np.float32)
    rng2 = _rng(s, 2000)
    delta = rng2.normal(0.0, math.sqrt(smooth_var), (n_rays, K, 3))
    smooth = (rays[:, None, 3:].astype(np.float64) + delta).astype(np.float32)
    target = rng2.uniform(0.0, 1.0, (n_rays, 3)).astype(np.float32)
    return {"rays": rays, "smooth_dirs": smooth, "target": target}


def sparsity_points(scene: dict, n: int, seed: int | None = None) -> np.ndarray:
    """Random points in the occupied space (the point set of Eq. 13): a
    uniformly chosen non-empty occupancy cell, x and y uniform inside it, z
    uniform in the cell's open interval (z_min, z_max).  float32 [n][3]."""
    spec = scene["spec"]
    rng = _rng(spec.cfg if seed is None else seed, 2500)
    occ = np.asarray(scene["occ"], np.float64).reshape(-1, 2)
    live = np.flatnonzero(occ[:, 0] < occ[:, 1])
    pts = np.zeros((n, 3), np.float32)
    if n == 0 or live.size == 0:
        return pts
    x0, x1, y0, y1 = spec.aabb[:4]
    M = spec.M
    cell = live[rng.integers(0, live.size, n)]
    cx, cy = cell // M, cell % M
    x = x0 + (cx + rng.uniform(0.0, 1.0, n)) * (x1 - x0) / M
    y = y0 + (cy + rng.uniform(0.0, 1.0, n)) * (y1 - y0) / M
    lo, hi = occ[cell, 0], occ[cell, 1]
    z = lo + rng.uniform(0.02, 0.98, n) * (hi - lo)
    pts[:, 0], pts[:, 1], pts[:, 2] = x, y, z
    return pts


def entropy_rays(scene: dict, n: int, seed: int | None = None, tilt: float = 0.2) -> np.ndarray:
    """Rays from high altitude to the ground (the ray set of Eq. 14): origins
    uniform over the box footprint, half the box height above its top,
    directions -z tilted by up to `tilt` (tangent) in x and y.  float32 [n][6]."""
    spec = scene["spec"]
    rng = _rng(spec.cfg if seed is None else seed, 3000)
    x0, x1, y0, y1, z0, z1 = spec.aabb
    o = np.stack([rng.uniform(x0, x1, n), rng.uniform(y0, y1, n), np.full(n, z1 + 0.5 * (z1 - z0))], 1)
    d = np.stack([rng.uniform(-tilt, tilt, n), rng.uniform(-tilt, tilt, n), -np.ones(n)], 1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.concatenate([o, d], 1).astype(np.float32)


def tiny_scene(seed: int = 0, L=(4, 4, 4), R=(4, 4, 4), M=2, n_rays=4, brick=0,
               occ_margin=0.35, step=1.0 / 16, eps=0.1) -> dict:
    """A few-parameter scene for finite-difference and hand-checked tests."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 9000 + seed))
    spec = SceneSpec("tiny", 0, (-1.0, 1.0, -1.0, 1.0, -0.5, 0.5), tuple(L), brick, tuple(R), M,
                     step, 64, eps, occ_margin, t_thr=0.0)
    scene = {"spec": spec, "seed": 9000 + seed}
    scene["grid"] = rng.normal(0.0, 0.5, (*L, NCH)).astype(np.float32)
    scene["grid"][..., 0] += 1.0
    scene["table"] = None
    scene["p_xy"] = rng.normal(0.0, 0.5, (R[0], R[1], NCH)).astype(np.float32)
    scene["p_xz"] = rng.normal(0.0, 0.5, (R[0], R[2], NCH)).astype(np.float32)
    scene["p_yz"] = rng.normal(0.0, 0.5, (R[1], R[2], NCH)).astype(np.float32)
    h = rng.uniform(-0.1, 0.1, (M, M))
    occ = np.empty((M, M, 2), np.float32)
    occ[..., 0] = h - occ_margin
    occ[..., 1] = h + occ_margin
    scene["occ"] = occ
    scene["mlp"] = rng.normal(0.0, 0.3, MLP_NPARAM).astype(np.float32)
    # rays from above at oblique angles through the box
    o = np.stack([rng.uniform(-0.6, 0.6, n_rays), rng.uniform(-0.6, 0.6, n_rays),
                  np.full(n_rays, 1.5)], 1)
    tgt = np.stack([rng.uniform(-0.4, 0.4, n_rays), rng.uniform(-0.4, 0.4, n_rays),
                    np.full(n_rays, -0.5)], 1)
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([o, d], 1).astype(np.float32)
    scene["rays"] = rays
    delta = rng.normal(0.0, math.sqrt(0.3), (n_rays, 1, 3))
    scene["smooth_dirs"] = (rays[:, None, 3:] + delta).astype(np.float32)
    scene["target"] = rng.uniform(0.0, 1.0, (n_rays, 3)).astype(np.float32)
    return scene
