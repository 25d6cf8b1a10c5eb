"""FP64 CPU oracle for the Oblique-MERF hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package imports nothing from it.

Functions follow Oblique-MERF (arXiv 2404.09531):
  render / features / occupancy_value / mlp / view_encoding   Eqs. 1-4, 6-8, appendix A
  train (loss + analytic gradient)                             Eqs. 5, 9-10, 12
  camera_rays                                                  pinhole rays (FP32 rule)
  brick_table                                                  Sec. 4.4 brick allocation
  sparsity / entropy (loss + analytic gradient)                Eqs. 13, 14 (Sec. 4.3)
  occupancy_grid / extract_bricks / plane_crop_rows            Sec. 4.4, Sec. 5.3 extraction
  working_set                                                  parameters a render reads (Sec. 4.4 viewer)

Parity status: every function is pinned in tests/test_oracle*.py by closed
forms, invariants, library routines or brute force (see that file).  No
function is pinned to a value the paper prints: the paper prints no worked
example for any synthetic input.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "omerf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

NPARAM = 883


def build(force: bool = False) -> str:
    """Compile the oracle with the system C compiler (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["cc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Scene(ctypes.Structure):
    _fields_ = [
        ("aabb", ctypes.c_float * 6),
        ("L", ctypes.c_int32 * 3),
        ("brick", ctypes.c_int32),
        ("table", ctypes.c_void_p),
        ("grid", ctypes.c_void_p),
        ("R", ctypes.c_int32 * 3),
        ("pxy", ctypes.c_void_p),
        ("pxz", ctypes.c_void_p),
        ("pyz", ctypes.c_void_p),
        ("M", ctypes.c_int32),
        ("occ", ctypes.c_void_p),
        ("mlp", ctypes.c_void_p),
        ("step", ctypes.c_float),
        ("eps", ctypes.c_float),
        ("t_thr", ctypes.c_float),
        ("bg", ctypes.c_float * 3),
        ("n_max", ctypes.c_int32),
        ("pz", ctypes.c_float * 2),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.or_render.restype = ctypes.c_long
        lib.or_render.argtypes = [P, P, ctypes.c_long, P, P, P, P, P, P, P, ctypes.c_int]
        lib.or_train.restype = ctypes.c_int
        lib.or_train.argtypes = [P, P, P, P, ctypes.c_long, ctypes.c_int, P, ctypes.c_double, P,
                                 P, P, P, P, P, P, P]
        lib.or_features.restype = ctypes.c_long
        lib.or_features.argtypes = [P, P, ctypes.c_long, P]
        lib.or_occupancy_value.restype = ctypes.c_double
        lib.or_occupancy_value.argtypes = [ctypes.c_double] * 4
        lib.or_view_encoding.restype = None
        lib.or_view_encoding.argtypes = [P, P]
        lib.or_mlp.restype = None
        lib.or_mlp.argtypes = [P, P, P, ctypes.c_long, P]
        lib.or_camera_rays.restype = None
        lib.or_camera_rays.argtypes = [P, ctypes.c_int, ctypes.c_int, P]
        lib.or_brick_table.restype = ctypes.c_long
        lib.or_brick_table.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, P]
        lib.or_ray_weights.restype = ctypes.c_int
        lib.or_ray_weights.argtypes = [P, P, P, P]
        lib.or_sparsity.restype = ctypes.c_double
        lib.or_sparsity.argtypes = [P, P, ctypes.c_long, ctypes.c_double, ctypes.c_double, P, P, P, P]
        lib.or_occupancy_grid.restype = ctypes.c_long
        lib.or_occupancy_grid.argtypes = [P, P, ctypes.c_int, P, P]
        lib.or_extract_bricks.restype = None
        lib.or_extract_bricks.argtypes = [P, ctypes.c_int, P, P, P, P]
        lib.or_plane_crop_rows.restype = ctypes.c_int
        lib.or_plane_crop_rows.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P, P]
        lib.or_entropy.restype = ctypes.c_double
        lib.or_entropy.argtypes = [P, P, ctypes.c_long, ctypes.c_double, ctypes.c_double, P, P, P, P, P]
        lib.or_working_set.restype = ctypes.c_long
        lib.or_working_set.argtypes = [P, P, ctypes.c_long, P, P, P, P, P, ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class OracleScene:
    """FP64 copies of a scene's arrays plus the C descriptor that points at them.

    ``scene`` is a dict as produced by ``synth.make_scene`` (keys grid, table,
    p_xy, p_xz, p_yz, occ, mlp, spec); values are widened to float64 exactly.
    Keyword overrides replace scalar settings (step, eps, t_thr, n_max, bg).
    """

    def __init__(self, scene: dict, **over):
        spec = scene["spec"]
        self.spec = spec
        self.grid = _f64(scene["grid"])
        self.table = None if scene.get("table") is None else np.ascontiguousarray(scene["table"], np.int32)
        self.pxy = _f64(scene["p_xy"])
        self.pxz = _f64(scene["p_xz"])
        self.pyz = _f64(scene["p_yz"])
        self.occ = _f64(scene["occ"])
        self.mlp = _f64(scene["mlp"])
        self.step = np.float32(over.get("step", spec.step))
        self.eps = np.float32(over.get("eps", spec.eps))
        self.t_thr = np.float32(over.get("t_thr", spec.t_thr))
        self.n_max = int(over.get("n_max", spec.n_max))
        self.bg = np.asarray(over.get("bg", (0.0, 0.0, 0.0)), np.float32)
        self.brick = int(spec.brick if self.table is not None else 0)
        pz = scene.get("plane_z")
        self.pz = np.zeros(2, np.float32) if pz is None else np.asarray(pz, np.float32)

    def desc(self) -> _Scene:
        s = _Scene()
        spec = self.spec
        s.aabb[:] = [float(np.float32(v)) for v in spec.aabb]
        s.L[:] = list(spec.L)
        s.brick = self.brick
        s.table = _ptr(self.table)
        s.grid = _ptr(self.grid)
        s.R[:] = list(spec.R)
        s.pxy, s.pxz, s.pyz = _ptr(self.pxy), _ptr(self.pxz), _ptr(self.pyz)
        s.M = spec.M
        s.occ = _ptr(self.occ)
        s.mlp = _ptr(self.mlp)
        s.step = float(self.step)
        s.eps = float(self.eps)
        s.t_thr = float(self.t_thr)
        s.bg[:] = [float(v) for v in self.bg]
        s.n_max = self.n_max
        s.pz[:] = [float(v) for v in self.pz]
        return s


def render(oscene: OracleScene, rays: np.ndarray, nthreads: int = 0) -> dict:
    """Forward render (Eqs. 1-4, 6-8) of rays [n][6] float32."""
    lib = _load()
    rays = np.ascontiguousarray(rays, np.float32)
    n = rays.shape[0]
    out = {
        "rgb": np.zeros((n, 3)), "count": np.zeros(n, np.int32), "F": np.zeros((n, 7)),
        "TN": np.zeros(n), "ambiguous": np.zeros(n, np.int32),
        "k_first": np.zeros(n, np.int32), "k_last": np.zeros(n, np.int32),
    }
    d = oscene.desc()
    ua = lib.or_render(ctypes.byref(d), _ptr(rays), n, _ptr(out["rgb"]), _ptr(out["count"]),
                       _ptr(out["F"]), _ptr(out["TN"]), _ptr(out["ambiguous"]),
                       _ptr(out["k_first"]), _ptr(out["k_last"]), int(nthreads))
    out["unalloc"] = int(ua)
    return out


def working_set(oscene: OracleScene, rays: np.ndarray, nthreads: int = 0) -> dict:
    """Which parameters a render of the rays reads at least once: boolean masks
    over the grid vertices (dense [Lx, Ly, Lz] or pool [nb, B, B, B]), the
    texels of each plane and the occupancy cells, plus the evaluated-sample
    count.  A vertex or texel is read by every evaluated sample whose
    interpolation stencil holds it (all 8 grid corners, 4 texels per plane,
    whatever their weight); an occupancy cell by every in-box lattice sample
    the march tests before the ray stops."""
    lib = _load()
    rays = np.ascontiguousarray(rays, np.float32)
    m = {"grid": np.zeros(oscene.grid.shape[:-1], np.uint8), "p_xy": np.zeros(oscene.pxy.shape[:-1], np.uint8),
         "p_xz": np.zeros(oscene.pxz.shape[:-1], np.uint8), "p_yz": np.zeros(oscene.pyz.shape[:-1], np.uint8),
         "occ": np.zeros(oscene.occ.shape[:-1], np.uint8)}
    d = oscene.desc()
    samples = lib.or_working_set(ctypes.byref(d), _ptr(rays), rays.shape[0], _ptr(m["grid"]), _ptr(m["p_xy"]),
                                 _ptr(m["p_xz"]), _ptr(m["p_yz"]), _ptr(m["occ"]), int(nthreads))
    out = {k: v.astype(bool) for k, v in m.items()}
    out["samples"] = int(samples)
    return out


def ray_weights(oscene: OracleScene, ray: np.ndarray):
    lib = _load()
    ray = np.ascontiguousarray(ray, np.float32).reshape(6)
    w = np.zeros(max(oscene.n_max, 1))
    tn = np.zeros(1)
    d = oscene.desc()
    cnt = lib.or_ray_weights(ctypes.byref(d), _ptr(ray), _ptr(w), _ptr(tn))
    return w[:cnt], float(tn[0])


def train(oscene: OracleScene, rays, target, smooth_dirs, lam=(1.0, 1e-2, 0.0), grad_scale=1.0,
          want_grad=True) -> dict:
    """Loss (Eqs. 5, 10, 12) and its FP64 gradient w.r.t. every parameter."""
    lib = _load()
    rays = np.ascontiguousarray(rays, np.float32)
    target = np.ascontiguousarray(target, np.float32)
    smooth_dirs = np.ascontiguousarray(smooth_dirs, np.float32)
    n = rays.shape[0]
    K = smooth_dirs.shape[1] if smooth_dirs.ndim == 3 else 1
    if K > 16:
        raise ValueError("the oracle supports at most 16 smoothness directions per ray")
    lam = np.asarray(lam, np.float64)
    loss = np.zeros(4)
    sig = np.zeros(1, np.uint64)
    g = {}
    if want_grad:
        g = {"grid": np.zeros_like(oscene.grid), "p_xy": np.zeros_like(oscene.pxy),
             "p_xz": np.zeros_like(oscene.pxz), "p_yz": np.zeros_like(oscene.pyz),
             "occ": np.zeros_like(oscene.occ), "mlp": np.zeros_like(oscene.mlp)}
    d = oscene.desc()
    rc = lib.or_train(ctypes.byref(d), _ptr(rays), _ptr(target), _ptr(smooth_dirs), n, K, _ptr(lam),
                      float(grad_scale), _ptr(loss), _ptr(g.get("grid")), _ptr(g.get("p_xy")),
                      _ptr(g.get("p_xz")), _ptr(g.get("p_yz")), _ptr(g.get("occ")), _ptr(g.get("mlp")),
                      _ptr(sig))
    if rc != 0:
        raise MemoryError("oracle train failed")
    return {"loss": float(loss[0]), "loss_terms": loss[1:].copy(), "grads": g, "signature": int(sig[0])}


def features(oscene: OracleScene, pts: np.ndarray):
    lib = _load()
    pts = np.ascontiguousarray(pts, np.float64)
    out = np.zeros((pts.shape[0], 8))
    d = oscene.desc()
    ua = lib.or_features(ctypes.byref(d), _ptr(pts), pts.shape[0], _ptr(out))
    return out, int(ua)


def occupancy_value(z, zmin, zmax, eps) -> float:
    return float(_load().or_occupancy_value(float(z), float(zmin), float(zmax), float(eps)))


def view_encoding(direction) -> np.ndarray:
    d = np.ascontiguousarray(direction, np.float64).reshape(3)
    enc = np.zeros(27)
    _load().or_view_encoding(_ptr(d), _ptr(enc))
    return enc


def mlp(params, F, dirs) -> np.ndarray:
    params = _f64(params)
    F = _f64(np.atleast_2d(F))
    dirs = _f64(np.atleast_2d(dirs))
    out = np.zeros((F.shape[0], 3))
    _load().or_mlp(_ptr(params), _ptr(F), _ptr(dirs), F.shape[0], _ptr(out))
    return out


def camera_rays(cam: dict) -> np.ndarray:
    """Pixel-centre pinhole rays [H*W][6] float32 (row-major pixels)."""
    c = np.zeros(16, np.float32)
    c[:12] = np.asarray(cam["c2w"], np.float32).reshape(12)
    c[12:] = [cam["fx"], cam["fy"], cam["cx"], cam["cy"]]
    W, H = int(cam["width"]), int(cam["height"])
    rays = np.zeros((H * W, 6), np.float32)
    _load().or_camera_rays(_ptr(c), W, H, _ptr(rays))
    return rays


def brick_table(spec, occ: np.ndarray) -> np.ndarray:
    """Sec. 4.4 brick allocation -> int32 table [nbx][nby][nbz] (-1 = empty)."""
    B = spec.brick
    nb = [(l + B - 1) // B for l in spec.L]
    table = np.zeros(nb, np.int32)
    aabb = np.asarray(spec.aabb, np.float32)
    L = np.asarray(spec.L, np.int32)
    occ = np.ascontiguousarray(occ, np.float32)
    _load().or_brick_table(_ptr(aabb), _ptr(L), B, _ptr(occ), spec.M, _ptr(table))
    return table


def _reg_grads(oscene, want_grad, occ=False):
    if not want_grad:
        return {}
    g = {"grid": np.zeros_like(oscene.grid), "p_xy": np.zeros_like(oscene.pxy),
         "p_xz": np.zeros_like(oscene.pxz), "p_yz": np.zeros_like(oscene.pyz)}
    if occ:
        g["occ"] = np.zeros_like(oscene.occ)
    return g


def sparsity(oscene: OracleScene, points, lam=0.05, grad_scale=1.0, want_grad=True) -> dict:
    """Eq. 13: lam * mean opacity at the given points [n][3]; FP64 gradient."""
    pts = np.ascontiguousarray(points, np.float64)
    g = _reg_grads(oscene, want_grad)
    d = oscene.desc()
    loss = _load().or_sparsity(ctypes.byref(d), _ptr(pts), pts.shape[0], float(lam), float(grad_scale),
                               _ptr(g.get("grid")), _ptr(g.get("p_xy")), _ptr(g.get("p_xz")), _ptr(g.get("p_yz")))
    return {"loss": float(loss), "grads": g}


def entropy(oscene: OracleScene, rays, lam=1e-3, grad_scale=1.0, want_grad=True) -> dict:
    """Eq. 14: lam * mean over rays of -sum p log p, p = M alpha / sum M alpha."""
    rays = np.ascontiguousarray(rays, np.float32)
    g = _reg_grads(oscene, want_grad, occ=True)
    d = oscene.desc()
    loss = _load().or_entropy(ctypes.byref(d), _ptr(rays), rays.shape[0], float(lam), float(grad_scale),
                              _ptr(g.get("grid")), _ptr(g.get("p_xy")), _ptr(g.get("p_xz")), _ptr(g.get("p_yz")),
                              _ptr(g.get("occ")))
    return {"loss": float(loss), "grads": g}


def occupancy_grid(aabb, occ, N):
    """Sec. 5.3: voxel occupancy [Nx][Ny][Nz] (uint8) from the occupancy plane, and the count."""
    aabb = np.asarray(aabb, np.float32)
    occ = np.ascontiguousarray(occ, np.float32)
    N = np.asarray(N, np.int32)
    out = np.zeros(tuple(int(v) for v in N), np.uint8)
    cnt = _load().or_occupancy_grid(_ptr(aabb), _ptr(occ), occ.shape[0], _ptr(N), _ptr(out))
    return out, int(cnt)


def extract_bricks(L, B, table, src, src_table=None) -> np.ndarray:
    """Brick pool for ``table`` from a dense grid or (with src_table) an older pool."""
    L = np.asarray(L, np.int32)
    table = np.ascontiguousarray(table, np.int32)
    src = np.ascontiguousarray(src, np.float32)
    st = None if src_table is None else np.ascontiguousarray(src_table, np.int32)
    nb = int(table.max()) + 1 if table.size else 0
    pool = np.zeros((max(nb, 0), B, B, B, 8), np.float32)
    _load().or_extract_bricks(_ptr(L), int(B), _ptr(table), _ptr(src), _ptr(st), _ptr(pool))
    return pool


def plane_crop_rows(aabb, Rz, occ):
    """Rows (k0, k1) of the XZ/YZ planes any evaluated sample touches and their z-range; None if empty."""
    aabb = np.asarray(aabb, np.float32)
    occ = np.ascontiguousarray(occ, np.float32)
    rows = np.zeros(2, np.int32)
    zr = np.zeros(2, np.float32)
    rc = _load().or_plane_crop_rows(_ptr(aabb), int(Rz), _ptr(occ), occ.shape[0], _ptr(rows), _ptr(zr))
    return None if rc != 0 else ((int(rows[0]), int(rows[1])), (float(zr[0]), float(zr[1])))

