"""ctypes binding of the C ABI in include/omerf.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# OMERF_CHECK=1 in the environment selects the checking build (bounds and
# unstored-brick counters; see include/omerf.h)
_LIB_PATH = os.path.join(_HERE, "libomerf_check.so" if os.environ.get("OMERF_CHECK") == "1" else "libomerf.so")
_lib = None

OMERF_F32 = 0
OMERF_BF16 = 1
MLP_NPARAM = 883


class OmerfError(RuntimeError):
    """A negative status returned by the library, with its message."""


class _SceneDesc(ctypes.Structure):
    _fields_ = [
        ("aabb", ctypes.c_float * 6),
        ("grid_res", ctypes.c_int32 * 3),
        ("brick", ctypes.c_int32),
        ("n_bricks", ctypes.c_int32),
        ("plane_res", ctypes.c_int32 * 3),
        ("occ_res", ctypes.c_int32),
        ("feat_dtype", ctypes.c_int32),
        ("step", ctypes.c_float),
        ("eps_occ", ctypes.c_float),
        ("t_thr", ctypes.c_float),
        ("bg", ctypes.c_float * 3),
        ("n_max", ctypes.c_int32),
        ("grid", ctypes.c_void_p),
        ("brick_table", ctypes.c_void_p),
        ("plane_xy", ctypes.c_void_p),
        ("plane_xz", ctypes.c_void_p),
        ("plane_yz", ctypes.c_void_p),
        ("occ", ctypes.c_void_p),
        ("mlp", ctypes.c_void_p),
        ("plane_z", ctypes.c_float * 2),
    ]


class _Camera(ctypes.Structure):
    _fields_ = [
        ("c2w", ctypes.c_float * 12),
        ("fx", ctypes.c_float),
        ("fy", ctypes.c_float),
        ("cx", ctypes.c_float),
        ("cy", ctypes.c_float),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
    ]


# name -> (restype, argtypes) for every entry point of include/omerf.h
_P = ctypes.c_void_p
_I = ctypes.c_int32
_L = ctypes.c_int64
SIGNATURES = {
    "omerf_scene_create": (ctypes.c_int, [_P, _P, _P]),
    "omerf_scene_update": (ctypes.c_int, [_P, _P]),
    "omerf_scene_destroy": (None, [_P]),
    "omerf_build_brick_table": (ctypes.c_int, [_P, _P, _I, _P, _I, _P, _P, _P]),
    "omerf_grow_brick_table": (ctypes.c_int, [_P, _P, _I, _P, _I, _P, _P, _P, _P, _P]),
    "omerf_ray_interval": (ctypes.c_int, [_P, _P, _P, _L, _P, _P]),
    "omerf_render": (ctypes.c_int, [_P, _P, _P, _L, _P, _P, _P]),
    "omerf_render_noalloc": (ctypes.c_int, [_P, _P, _P, _L, _P, _P, _P]),
    "omerf_render_cameras": (ctypes.c_int, [_P, _P, _I, _P, _P, _P]),
    "omerf_saved_bytes_per_ray": (ctypes.c_int64, []),
    "omerf_train_fwd": (ctypes.c_int, [_P, _P, _P, _P, _L, _I, _P, _P, _P, _P]),
    "omerf_train_bwd": (ctypes.c_int, [_P, _P, _P, _P, _L, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "omerf_train_step": (ctypes.c_int, [_P, _P, _P, _P, _L, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "omerf_sparsity_loss": (ctypes.c_int, [_P, _P, _L, ctypes.c_float, _P, _P, _P, _P, _P, _P, _P]),
    "omerf_entropy_loss": (ctypes.c_int, [_P, _P, _L, ctypes.c_float, _P, _P, _P, _P, _P, _P, _P, _P]),
    "omerf_occupancy_grid": (ctypes.c_int, [_P, _P, _I, _P, _P, _P, _P]),
    "omerf_extract_bricks": (ctypes.c_int, [_P, _I, _P, _I, _P, _P, _I, _I, _P, _P]),
    "omerf_tma_available": (ctypes.c_int32, []),
    "omerf_plane_crop_rows": (ctypes.c_int, [_P, _I, _P, _I, _P, _P, _P]),
    "omerf_crop_planes": (ctypes.c_int, [_P, _L, _I, _I, _I, _I, _P, _P]),
    "omerf_adam_step": (ctypes.c_int, [_P, _I, ctypes.c_float, ctypes.c_float, ctypes.c_float, _L, _P]),
    "omerf_lr_exponential": (ctypes.c_float, [ctypes.c_float, ctypes.c_float, _L, _L]),
    "omerf_lambda_occ": (ctypes.c_float, [_L]),
    "omerf_probe_load_bandwidth": (ctypes.c_int, [_P, _L, _I, _I, _P, _P]),
    "omerf_probe_red_bandwidth": (ctypes.c_int, [_P, _L, _I, _I, _P]),
    "omerf_scene_device_bytes": (ctypes.c_int64, [_P]),
    "omerf_check_build": (ctypes.c_int32, []),
    "omerf_check_counts": (ctypes.c_int, [_P, _P, _I, _P]),
    "omerf_check_totals": (None, [_P]),
    "omerf_sync": (ctypes.c_int, [_P, _I]),
    "omerf_last_error": (ctypes.c_char_p, []),
}


def lib():
    """Load libomerf.so from the package directory (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise OmerfError(f"{_LIB_PATH} is missing: build it with __graft_entry__.build()")
        handle = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _check(status: int, what: str):
    if status != 0:
        msg = lib().omerf_last_error()
        raise OmerfError(f"{what} failed with status {status}: {msg.decode() if msg else ''}")


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev_f32(x, device, shape=None):
    if x is None:
        return None
    t = torch.as_tensor(x)
    t = t.to(device=device, dtype=torch.float32).contiguous()
    if shape is not None and tuple(t.shape) != tuple(shape):
        t = t.reshape(shape)
    return t


def _require_cuda(t, name):
    if not t.is_cuda:
        raise OmerfError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise OmerfError(f"{name} must be contiguous")


def camera_struct(cam) -> _Camera:
    """A C camera from a dict with c2w (3x4), fx, fy, cx, cy, width, height."""
    c = _Camera()
    c.c2w[:] = [float(v) for v in np.asarray(cam["c2w"], np.float32).reshape(12)]
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(cam[k])) for k in ("fx", "fy", "cx", "cy"))
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


class Scene:
    """A scene handle over caller-owned device tensors.

    Tensors (channel-last, x-major; see include/omerf.h):
      grid     dense [Lx, Ly, Lz, 8] or brick pool [nb, B, B, B, 8]
      table    int32 brick table [nbx, nby, nbz] (brick grids) or None
      p_xy, p_xz, p_yz   planes [Rx, Ry, 8], [Rx, Rz, 8], [Ry, Rz, 8]
      occ      float32 [M, M, 2]      mlp float32 [883]
      plane_z  (z0, z1) the z-range of the XZ/YZ planes' Rz rows when they are
               cropped to the occupancy bounds (crop_planes); None = the box's
    Features are float32 or bfloat16 (both grid and planes the same dtype).
    The tensors are referenced, not copied: in-place updates are seen by the
    next call (call update() after changing occ).
    """

    def __init__(self, *, aabb, grid, p_xy, p_xz, p_yz, occ, mlp, step, eps, t_thr=1e-4, n_max=128,
                 bg=(0.0, 0.0, 0.0), table=None, brick=0, grid_res=None, plane_z=None, stream=None):
        self.grid, self.table = grid, table
        self.p_xy, self.p_xz, self.p_yz = p_xy, p_xz, p_yz
        self.occ, self.mlp = occ, mlp
        for name in ("grid", "p_xy", "p_xz", "p_yz", "occ", "mlp"):
            _require_cuda(getattr(self, name), name)
        if table is not None:
            _require_cuda(table, "table")
        dt = grid.dtype
        if dt not in (torch.float32, torch.bfloat16) or any(t.dtype != dt for t in (p_xy, p_xz, p_yz)):
            raise OmerfError("grid and planes must share one dtype, float32 or bfloat16")
        if occ.dtype != torch.float32 or mlp.dtype != torch.float32 or mlp.numel() != MLP_NPARAM:
            raise OmerfError("occ and mlp must be float32; mlp has 883 values")
        self.device = grid.device
        self.brick = int(brick)
        if grid_res is None:
            if self.brick:
                raise OmerfError("grid_res is required for a brick grid")
            grid_res = tuple(grid.shape[:3])
        self.grid_res = tuple(int(v) for v in grid_res)
        self.plane_res = (int(p_xy.shape[0]), int(p_xy.shape[1]), int(p_xz.shape[1]))
        self.occ_res = int(occ.shape[0])
        self.aabb = tuple(float(np.float32(v)) for v in aabb)
        self.step, self.eps, self.t_thr, self.n_max = float(step), float(eps), float(t_thr), int(n_max)
        self.bg = tuple(float(v) for v in bg)
        self.plane_z = None if plane_z is None else tuple(float(np.float32(v)) for v in plane_z)
        d = _SceneDesc()
        d.aabb[:] = list(self.aabb)
        d.grid_res[:] = list(self.grid_res)
        d.brick = self.brick
        d.n_bricks = int(grid.shape[0]) if self.brick else 0
        d.plane_res[:] = list(self.plane_res)
        d.occ_res = self.occ_res
        d.feat_dtype = OMERF_BF16 if dt == torch.bfloat16 else OMERF_F32
        d.step, d.eps_occ, d.t_thr = self.step, self.eps, self.t_thr
        d.bg[:] = list(self.bg)
        d.n_max = self.n_max
        d.grid = grid.data_ptr()
        d.brick_table = table.data_ptr() if table is not None else None
        d.plane_xy, d.plane_xz, d.plane_yz = p_xy.data_ptr(), p_xz.data_ptr(), p_yz.data_ptr()
        d.occ, d.mlp = occ.data_ptr(), mlp.data_ptr()
        d.plane_z[:] = list(self.plane_z) if self.plane_z is not None else [0.0, 0.0]
        self._desc = d
        h = ctypes.c_void_p()
        _check(lib().omerf_scene_create(ctypes.byref(d), _stream(stream), ctypes.byref(h)), "omerf_scene_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def feat_dtype(self):
        return self.grid.dtype

    def update(self, stream=None):
        """Recompute the occupancy hull after occ changed in place."""
        _check(lib().omerf_scene_update(self._h, _stream(stream)), "omerf_scene_update")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().omerf_scene_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_brick_table(aabb, grid_res, brick, occ: torch.Tensor, stream=None):
    """Sec. 4.4 brick allocation on the GPU -> (int32 table [nbx, nby, nbz], n_alloc tensor)."""
    _require_cuda(occ, "occ")
    nb = [(int(l) + brick - 1) // brick for l in grid_res]
    table = torch.empty(nb, dtype=torch.int32, device=occ.device)
    n_alloc = torch.empty(1, dtype=torch.int32, device=occ.device)
    a = (ctypes.c_float * 6)(*[float(v) for v in aabb])
    g = (ctypes.c_int32 * 3)(*[int(v) for v in grid_res])
    _check(lib().omerf_build_brick_table(a, g, int(brick), _ptr(occ), int(occ.shape[0]), _ptr(table),
                                         _ptr(n_alloc), _stream(stream)), "omerf_build_brick_table")
    return table, n_alloc


def grow_brick_table(aabb, grid_res, brick, occ: torch.Tensor, old_table: torch.Tensor, stream=None):
    """The stored bricks of ``old_table`` plus those Sec. 4.4's rule allocates
    for ``occ`` -> (table, n_alloc tensor, missing tensor: bricks added)."""
    _require_cuda(occ, "occ")
    _require_cuda(old_table, "old_table")
    table = torch.empty_like(old_table)
    n_alloc = torch.empty(1, dtype=torch.int32, device=occ.device)
    missing = torch.empty(1, dtype=torch.int32, device=occ.device)
    a = (ctypes.c_float * 6)(*[float(v) for v in aabb])
    g = (ctypes.c_int32 * 3)(*[int(v) for v in grid_res])
    _check(lib().omerf_grow_brick_table(a, g, int(brick), _ptr(occ), int(occ.shape[0]), _ptr(old_table), _ptr(table),
                                        _ptr(n_alloc), _ptr(missing), _stream(stream)), "omerf_grow_brick_table")
    return table, n_alloc, missing


def scene_from_synth(sc: dict, device="cuda", feat_dtype=None, table=None, stream=None, **over) -> Scene:
    """Upload a scene dict (keys grid/table, p_xy, p_xz, p_yz, occ, mlp, spec).

    For a brick grid without a pool, the brick table is built on the GPU
    (unless ``table`` is given) and the dict's generator fills the pool.
    """
    spec = sc["spec"]
    device = torch.device(device)
    dt = feat_dtype or (torch.bfloat16 if getattr(spec, "feat_dtype", "f32") == "bf16" else torch.float32)
    occ = torch.as_tensor(sc["occ"], dtype=torch.float32).to(device).contiguous()
    brick = int(spec.brick) if (sc.get("grid") is None or sc.get("table") is not None) else 0
    if brick:
        if sc.get("grid") is not None and sc.get("table") is not None:
            tab = torch.as_tensor(np.asarray(sc["table"], np.int32)).to(device)
            pool = sc["grid"]
        else:
            if table is None:
                tab, _ = build_brick_table(spec.aabb, spec.L, brick, occ, stream)
                table = tab.cpu().numpy()
            tab = torch.as_tensor(np.asarray(table, np.int32)).to(device)
            import synth  # the generator draws the feature values of the allocated bricks
            pool = synth.fill_brick_pool(sc, np.asarray(table))
        grid = torch.as_tensor(pool).to(device=device, dtype=dt).contiguous()
    else:
        tab = None
        grid = torch.as_tensor(sc["grid"]).to(device=device, dtype=dt).contiguous()
    kw = dict(aabb=spec.aabb, grid=grid, table=tab, brick=brick, grid_res=spec.L,
              p_xy=torch.as_tensor(sc["p_xy"]).to(device=device, dtype=dt).contiguous(),
              p_xz=torch.as_tensor(sc["p_xz"]).to(device=device, dtype=dt).contiguous(),
              p_yz=torch.as_tensor(sc["p_yz"]).to(device=device, dtype=dt).contiguous(),
              occ=occ, mlp=torch.as_tensor(sc["mlp"], dtype=torch.float32).to(device).contiguous(),
              step=spec.step, eps=spec.eps, t_thr=spec.t_thr, n_max=spec.n_max, stream=stream,
              plane_z=sc.get("plane_z"))
    kw.update(over)
    return Scene(**kw)


def render(scene: Scene, camera=None, rays=None, out=None, count_out=None, stream=None, want_count=True):
    """Forward render (Eqs. 1-4, 6-8) of a camera (dict) or of rays [n, 6].

    Returns (rgb [n, 3] float32, count [n] int32 or None) on the scene's
    device.  With ``out`` (and ``count_out``) given as page-locked CPU
    tensors the kernel writes the pixels straight into them; other CPU
    tensors receive a copy enqueued on the stream.
    """
    dev = scene.device
    cam_p = None
    if camera is not None:
        cs = camera_struct(camera)
        n = cs.width * cs.height
        cam_p = ctypes.byref(cs)
        rays_t = None
    else:
        rays_t = _dev_f32(rays, dev)
        n = int(rays_t.shape[0])
    st = _stream(stream)
    direct = out is not None and not out.is_cuda and out.is_pinned() and out.is_contiguous() and \
        out.dtype == torch.float32 and out.numel() == 3 * n and \
        (count_out is None or (count_out.is_pinned() and count_out.is_contiguous() and
                               count_out.dtype == torch.int32 and count_out.numel() == n))
    if direct:
        _check(lib().omerf_render(scene.handle, cam_p, _ptr(rays_t), n, _ptr(out), _ptr(count_out), st),
               "omerf_render")
        return out, count_out
    rgb = torch.empty((n, 3), dtype=torch.float32, device=dev)
    count = torch.empty(n, dtype=torch.int32, device=dev) if (want_count or count_out is not None) else None
    _check(lib().omerf_render(scene.handle, cam_p, _ptr(rays_t), n, _ptr(rgb), _ptr(count), st), "omerf_render")
    if out is not None:
        out.copy_(rgb, non_blocking=True)
        if count_out is not None:
            count_out.copy_(count, non_blocking=True)
        return out, count_out
    return rgb, count


def render_cameras(scene: Scene, cameras, out=None, count_out=None, stream=None, want_count=True):
    """Render several cameras in one launch: (rgb [sum n, 3], count [sum n])
    in camera order.  ``out`` / ``count_out`` may be device tensors or
    page-locked CPU tensors, which the kernel writes directly."""
    cams = list(cameras)
    arr = (_Camera * max(len(cams), 1))(*[camera_struct(c) for c in cams])
    n = sum(int(c["width"]) * int(c["height"]) for c in cams)
    dev = scene.device
    rgb = out if out is not None else torch.empty((n, 3), dtype=torch.float32, device=dev)
    count = count_out if count_out is not None else (
        torch.empty(n, dtype=torch.int32, device=dev) if want_count else None)
    for t, name in ((rgb, "out"), (count, "count_out")):
        if t is not None and (not t.is_contiguous() or (not t.is_cuda and not t.is_pinned())):
            raise OmerfError(f"{name} must be a contiguous device tensor or page-locked CPU tensor")
    if rgb.numel() != 3 * n or (count is not None and count.numel() != n):
        raise OmerfError("output sizes do not match the cameras")
    _check(lib().omerf_render_cameras(scene.handle, arr, len(cams), _ptr(rgb), _ptr(count), _stream(stream)),
           "omerf_render_cameras")
    return rgb, count


def render_noalloc(scene: Scene, camera=None, rays=None, rgb=None, count=None, stream=None):
    """Render through omerf_render_noalloc, which allocates no device memory.

    For callers that must not allocate: pass preallocated ``rgb`` [n, 3]
    float32 and ``count`` [n] int32 device tensors (allocated here only when
    omitted).  The scene's description is used directly; its handle is not.
    Calls that overlap on the GPU share one static scratch array and race.
    """
    dev = scene.device
    cam_p = None
    if camera is not None:
        cs = camera_struct(camera)
        n = cs.width * cs.height
        cam_p = ctypes.byref(cs)
        rays_t = None
    else:
        rays_t = _dev_f32(rays, dev)
        n = int(rays_t.shape[0])
    if rgb is None:
        rgb = torch.empty((n, 3), dtype=torch.float32, device=dev)
    _check(lib().omerf_render_noalloc(ctypes.byref(scene._desc), cam_p, _ptr(rays_t), n, _ptr(rgb), _ptr(count),
                                      _stream(stream)), "omerf_render_noalloc")
    return rgb, count


def ray_interval(scene: Scene, camera=None, rays=None, stream=None):
    """Per-ray lattice range [k_lo, k_hi] scanned by the march (int32 [n, 2])."""
    dev = scene.device
    cam_p = None
    if camera is not None:
        cs = camera_struct(camera)
        n = cs.width * cs.height
        cam_p = ctypes.byref(cs)
        rays_t = None
    else:
        rays_t = _dev_f32(rays, dev)
        n = int(rays_t.shape[0])
    out = torch.empty((n, 2), dtype=torch.int32, device=dev)
    _check(lib().omerf_ray_interval(scene.handle, cam_p, _ptr(rays_t), n, _ptr(out), _stream(stream)),
           "omerf_ray_interval")
    return out


def saved_bytes_per_ray() -> int:
    return int(lib().omerf_saved_bytes_per_ray())


def _train_inputs(scene, rays, target, smooth_dirs):
    dev = scene.device
    rays_t = _dev_f32(rays, dev)
    n = int(rays_t.shape[0])
    target_t = _dev_f32(target, dev, (n, 3))
    if smooth_dirs is None:
        dirs_t, K = None, 0
    else:
        dirs_t = _dev_f32(smooth_dirs, dev)
        if n == 0:
            # an empty batch: K from a [0][K][3] array (nothing is read)
            K = int(dirs_t.shape[1]) if dirs_t.dim() == 3 else 0
            dirs_t = dirs_t.reshape(0, K, 3)
        else:
            dirs_t = dirs_t.reshape(n, -1, 3)
            K = int(dirs_t.shape[1])
    return rays_t, target_t, dirs_t, n, K


def _lam(lam):
    return (ctypes.c_float * 3)(*[float(v) for v in lam])


def train_fwd(scene, rays, target, smooth_dirs=None, lam=(1.0, 1e-2, 0.0), stream=None):
    """Training forward: loss [4] (total, rgb, smooth, occ) and the saved state."""
    rays_t, target_t, dirs_t, n, K = _train_inputs(scene, rays, target, smooth_dirs)
    saved = torch.empty(max(n, 1) * saved_bytes_per_ray() // 4, dtype=torch.float32, device=scene.device)
    loss = torch.empty(4, dtype=torch.float32, device=scene.device)
    _check(lib().omerf_train_fwd(scene.handle, _ptr(rays_t), _ptr(target_t), _ptr(dirs_t), n, K, _lam(lam),
                                 _ptr(saved), _ptr(loss), _stream(stream)), "omerf_train_fwd")
    return loss, saved, (rays_t, target_t, dirs_t, n, K)


def zero_grads(scene):
    """Zeroed float32 gradient buffers shaped like the scene's parameters
    (keys grid, p_xy, p_xz, p_yz, occ, mlp), as the training calls take them."""
    z = lambda t: torch.zeros(t.shape, dtype=torch.float32, device=t.device)  # noqa: E731
    return {"grid": z(scene.grid), "p_xy": z(scene.p_xy), "p_xz": z(scene.p_xz), "p_yz": z(scene.p_yz),
            "occ": z(scene.occ), "mlp": z(scene.mlp)}



def train_bwd(scene, saved, inputs, lam=(1.0, 1e-2, 0.0), grad_scale=None, grads=None, stream=None):
    """Training backward: accumulates grad_scale * dL/dparam into ``grads`` (float32)."""
    rays_t, target_t, dirs_t, n, K = inputs
    if grads is None:
        grads = zero_grads(scene)
    gs = _grad_scale(scene, grad_scale)
    _check(lib().omerf_train_bwd(scene.handle, _ptr(rays_t), _ptr(target_t), _ptr(dirs_t), n, K, _lam(lam),
                                 _ptr(saved), _ptr(gs), _ptr(grads["grid"]), _ptr(grads["p_xy"]),
                                 _ptr(grads["p_xz"]), _ptr(grads["p_yz"]), _ptr(grads["occ"]),
                                 _ptr(grads["mlp"]), _stream(stream)), "omerf_train_bwd")
    return grads


def train_step(scene, rays, target, smooth_dirs=None, lam=(1.0, 1e-2, 0.0), grads=None, saved=None,
               stream=None, loss=None):
    """One fused forward + backward: returns {"loss": [4] tensor, "grads": dict}.
    ``loss`` may be a caller's float32 [4] device tensor (overwritten)."""
    rays_t, target_t, dirs_t, n, K = _train_inputs(scene, rays, target, smooth_dirs)
    if saved is None:
        saved = torch.empty(max(n, 1) * saved_bytes_per_ray() // 4, dtype=torch.float32, device=scene.device)
    if loss is None:
        loss = torch.empty(4, dtype=torch.float32, device=scene.device)
    elif not loss.is_cuda or loss.dtype != torch.float32 or loss.numel() < 4 or not loss.is_contiguous():
        raise OmerfError("loss must be a contiguous float32 CUDA tensor of 4 values")
    if grads is None:
        grads = zero_grads(scene)
    _check(lib().omerf_train_step(scene.handle, _ptr(rays_t), _ptr(target_t), _ptr(dirs_t), n, K, _lam(lam),
                                  _ptr(saved), _ptr(loss), _ptr(grads["grid"]), _ptr(grads["p_xy"]),
                                  _ptr(grads["p_xz"]), _ptr(grads["p_yz"]), _ptr(grads["occ"]),
                                  _ptr(grads["mlp"]), _stream(stream)), "omerf_train_step")
    return {"loss": loss, "grads": grads, "saved": saved}


def _grad_scale(scene, grad_scale):
    if grad_scale is None:
        return None
    return torch.as_tensor(grad_scale, dtype=torch.float32, device=scene.device).reshape(1).contiguous()


def _reg_loss(loss, scene):
    if loss is None:
        return torch.zeros(1, dtype=torch.float32, device=scene.device)
    _require_cuda(loss, "loss")
    return loss


def sparsity_loss(scene, points, lam=0.05, grads=None, loss=None, grad_scale=None, stream=None):
    """Eq. 13: adds lam * mean alpha over ``points`` [n][3] to ``loss`` (a new
    [1] tensor when None) and grad_scale * dL/dparam to ``grads`` (a dict as
    from train_step; None skips the gradient).  Returns the loss tensor."""
    pts = _dev_f32(points, scene.device)
    n = int(pts.shape[0]) if pts.numel() else 0
    loss = _reg_loss(loss, scene)
    g = grads or {}
    _check(lib().omerf_sparsity_loss(scene.handle, _ptr(pts), n, float(lam), _ptr(_grad_scale(scene, grad_scale)),
                                     _ptr(loss), _ptr(g.get("grid")), _ptr(g.get("p_xy")), _ptr(g.get("p_xz")),
                                     _ptr(g.get("p_yz")), _stream(stream)), "omerf_sparsity_loss")
    return loss


def entropy_loss(scene, rays, lam=1e-3, grads=None, loss=None, grad_scale=None, stream=None):
    """Eq. 14: adds lam * mean over ``rays`` [n][6] of -sum p log p
    (p = M alpha / sum M alpha) to ``loss`` and its gradient (features and
    occupancy plane) to ``grads``.  Returns the loss tensor."""
    r = _dev_f32(rays, scene.device)
    n = int(r.shape[0]) if r.numel() else 0
    loss = _reg_loss(loss, scene)
    g = grads or {}
    _check(lib().omerf_entropy_loss(scene.handle, _ptr(r), n, float(lam), _ptr(_grad_scale(scene, grad_scale)),
                                    _ptr(loss), _ptr(g.get("grid")), _ptr(g.get("p_xy")), _ptr(g.get("p_xz")),
                                    _ptr(g.get("p_yz")), _ptr(g.get("occ")), _stream(stream)), "omerf_entropy_loss")
    return loss


def _feat_enum(t):
    if t.dtype == torch.float32:
        return OMERF_F32
    if t.dtype == torch.bfloat16:
        return OMERF_BF16
    raise OmerfError("features must be float32 or bfloat16")


def occupancy_grid(aabb, occ, N, stream=None):
    """Sec. 5.3 occupancy grid from the occupancy plane: (bits uint32 tensor
    [Nx, Ny, ceil(Nz/32)] viewed as int32, count tensor [1] int64)."""
    _require_cuda(occ, "occ")
    N = [int(v) for v in N]
    bits = torch.empty((N[0], N[1], (N[2] + 31) // 32), dtype=torch.int32, device=occ.device)
    count = torch.zeros(1, dtype=torch.int64, device=occ.device)
    a = (ctypes.c_float * 6)(*[float(v) for v in aabb])
    n = (ctypes.c_int32 * 3)(*N)
    _check(lib().omerf_occupancy_grid(a, _ptr(occ), int(occ.shape[0]), n, _ptr(bits), _ptr(count),
                                      _stream(stream)), "omerf_occupancy_grid")
    return bits, count


def unpack_occupancy_bits(bits, Nz):
    """[Nx, Ny, W] int32 words -> bool [Nx, Ny, Nz] (host numpy)."""
    w = np.asarray(bits.cpu().numpy() if hasattr(bits, "cpu") else bits).view(np.uint32)
    shifts = np.arange(32, dtype=np.uint32)
    out = ((w[..., None] >> shifts) & 1).astype(bool).reshape(w.shape[0], w.shape[1], -1)
    return out[..., :Nz]


def extract_bricks(grid_res, brick, table, src, src_table=None, n_bricks=None, src_n_bricks=None, stream=None):
    """Sec. 4.4 brick pool for ``table`` from a dense grid or an older pool
    (``src_table``); returns the new pool tensor [n_bricks, B, B, B, 8]."""
    _require_cuda(table, "table")
    _require_cuda(src, "src")
    if n_bricks is None:
        n_bricks = int(table.max().item()) + 1 if table.numel() else 0
    if src_table is not None:
        _require_cuda(src_table, "src_table")
        if src_n_bricks is None:
            src_n_bricks = int(src.shape[0])
    B = int(brick)
    pool = torch.empty((max(int(n_bricks), 0), B, B, B, 8), dtype=src.dtype, device=src.device)
    if n_bricks == 0:
        return pool
    g = (ctypes.c_int32 * 3)(*[int(v) for v in grid_res])
    _check(lib().omerf_extract_bricks(g, B, _ptr(table), int(n_bricks), _ptr(src), _ptr(src_table),
                                      int(src_n_bricks or 0), _feat_enum(src), _ptr(pool), _stream(stream)),
           "omerf_extract_bricks")
    return pool


def plane_crop_rows(scene, stream=None):
    """Rows (k0, k1) of the scene's XZ/YZ planes any evaluated sample reads and
    the cropped z-range, or None if no cell is occupied (one small readback)."""
    rows = torch.empty(2, dtype=torch.int32, device=scene.device)
    zr = torch.empty(2, dtype=torch.float32, device=scene.device)
    pz = scene.plane_z if scene.plane_z is not None else (scene.aabb[4], scene.aabb[5])
    _check(lib().omerf_plane_crop_rows((ctypes.c_float * 2)(*pz), int(scene.plane_res[2]), _ptr(scene.occ),
                                       int(scene.occ_res), _ptr(rows), _ptr(zr), _stream(stream)),
           "omerf_plane_crop_rows")
    r = rows.cpu().tolist()
    if r[0] < 0:
        return None
    return (r[0], r[1]), tuple(float(v) for v in zr.cpu().tolist())


def crop_planes(scene, stream=None):
    """A new Scene whose XZ and YZ planes keep only the rows any evaluated
    sample reads (Sec. 4.4); grid, XY plane, occupancy and MLP are shared."""
    cr = plane_crop_rows(scene, stream)
    if cr is None:
        raise OmerfError("the occupancy plane is empty")
    (k0, k1), zr = cr
    out = []
    for p in (scene.p_xz, scene.p_yz):
        dst = torch.empty((p.shape[0], k1 - k0 + 1, 8), dtype=p.dtype, device=p.device)
        _check(lib().omerf_crop_planes(_ptr(p), int(p.shape[0]), int(p.shape[1]), k0, k1, _feat_enum(p), _ptr(dst),
                                       _stream(stream)), "omerf_crop_planes")
        out.append(dst)
    return Scene(aabb=scene.aabb, grid=scene.grid, table=scene.table, brick=scene.brick, grid_res=scene.grid_res,
                 p_xy=scene.p_xy, p_xz=out[0], p_yz=out[1], occ=scene.occ, mlp=scene.mlp, step=scene.step,
                 eps=scene.eps, t_thr=scene.t_thr, n_max=scene.n_max, bg=scene.bg, plane_z=zr, stream=stream)


class _AdamGroup(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("m", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("shadow_bf16", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("lr", ctypes.c_float)]


def adam_step(groups, step, beta1=0.9, beta2=0.99, eps=1e-15, stream=None):
    """Fused Adam step (appendix A).  groups: list of dicts with float32 device
    tensors param, grad, m, v (same size), a learning rate lr and an optional
    bfloat16 tensor shadow that receives the updated values."""
    arr = (_AdamGroup * len(groups))()
    for i, gr in enumerate(groups):
        for k in ("param", "grad", "m", "v"):
            t = gr[k]
            _require_cuda(t, k)
            if t.dtype != torch.float32 or t.numel() != gr["param"].numel():
                raise OmerfError(f"adam group {i}: {k} must be float32 with the param's size")
        sh = gr.get("shadow")
        if sh is not None and (sh.dtype != torch.bfloat16 or sh.numel() != gr["param"].numel()):
            raise OmerfError(f"adam group {i}: shadow must be bfloat16 with the param's size")
        arr[i] = _AdamGroup(gr["param"].data_ptr(), gr["grad"].data_ptr(), gr["m"].data_ptr(), gr["v"].data_ptr(),
                            sh.data_ptr() if sh is not None else None, gr["param"].numel(), float(gr["lr"]))
    _check(lib().omerf_adam_step(arr, len(groups), float(beta1), float(beta2), float(eps), int(step),
                                 _stream(stream)), "omerf_adam_step")


def lr_exponential(lr0, lr1, step, total):
    return float(lib().omerf_lr_exponential(float(lr0), float(lr1), int(step), int(total)))


def lambda_occ(step):
    return float(lib().omerf_lambda_occ(int(step)))


def probe_load_bandwidth(buf: torch.Tensor, bytes_per_cta: int, ctas: int, passes: int, sink=None, stream=None):
    """Launch the load-bandwidth probe over ``buf`` (float32, at least
    ctas * bytes_per_cta bytes); returns the bytes it delivers to registers."""
    _require_cuda(buf, "buf")
    if buf.dtype != torch.float32 or buf.numel() * 4 < int(ctas) * int(bytes_per_cta):
        raise OmerfError("buf must be float32 with at least ctas * bytes_per_cta bytes")
    if sink is None:
        sink = torch.empty(int(ctas) * 256, dtype=torch.float32, device=buf.device)
    _check(lib().omerf_probe_load_bandwidth(_ptr(buf), int(bytes_per_cta), int(ctas), int(passes), _ptr(sink),
                                            _stream(stream)), "omerf_probe_load_bandwidth")
    return int(ctas) * int(bytes_per_cta) * int(passes)


def scene_device_bytes(scene: Scene) -> int:
    """Device bytes the scene handle allocates for its own state (the
    caller's arrays not counted)."""
    n = int(lib().omerf_scene_device_bytes(ctypes.byref(scene._desc)))
    if n < 0:
        raise OmerfError(f"omerf_scene_device_bytes: status {n}")
    return n


def probe_red_bandwidth(buf: torch.Tensor, bytes_per_warp: int, ctas: int, passes: int, stream=None):
    """Launch the reduction-throughput probe over ``buf`` (float32, at least
    ctas * 8 * bytes_per_warp bytes; its contents grow); returns the bytes it
    reduces."""
    _require_cuda(buf, "buf")
    if buf.dtype != torch.float32 or buf.numel() * 4 < int(ctas) * 8 * int(bytes_per_warp):
        raise OmerfError("buf must be float32 with at least ctas * 8 * bytes_per_warp bytes")
    _check(lib().omerf_probe_red_bandwidth(_ptr(buf), int(bytes_per_warp), int(ctas), int(passes), _stream(stream)),
           "omerf_probe_red_bandwidth")
    return int(ctas) * int(bytes_per_warp) * int(passes)


def check_counts(scene: Scene, reset=True, stream=None):
    """The checking build's counters of a scene: (corner reads of unstored
    bricks, feature reads outside the arrays).  Raises in the default build,
    or (status -7) if a read fell outside an array."""
    c = (ctypes.c_uint64 * 2)()
    _check(lib().omerf_check_counts(scene.handle, c, int(bool(reset)), _stream(stream)), "omerf_check_counts")
    return int(c[0]), int(c[1])


def check_totals():
    """The checking build's counters of every scene destroyed so far in this
    process: (corner reads of unstored bricks, feature reads outside the
    arrays); zeros in the default build."""
    c = (ctypes.c_uint64 * 2)()
    lib().omerf_check_totals(c)
    return int(c[0]), int(c[1])


def sync(stream=None, timeout_ms=-1):
    """Bounded wait for a stream (raises OmerfError on timeout or CUDA error)."""
    _check(lib().omerf_sync(_stream(stream), int(timeout_ms)), "omerf_sync")


class TrainStep(torch.autograd.Function):
    """Differentiable loss of Eqs. 5, 9-10, 12 over the scene's parameters.

    Usage: loss = TrainStep.apply(scene, rays, target, smooth_dirs, lam,
    scene.grid, scene.p_xy, scene.p_xz, scene.p_yz, scene.occ, scene.mlp)
    The parameter tensors must be the scene's own tensors (the kernels read
    them through the scene handle); their gradients are float32.
    """

    @staticmethod
    def forward(ctx, scene, rays, target, smooth_dirs, lam, grid, p_xy, p_xz, p_yz, occ, mlp):
        for a, b in ((grid, scene.grid), (p_xy, scene.p_xy), (p_xz, scene.p_xz), (p_yz, scene.p_yz),
                     (occ, scene.occ), (mlp, scene.mlp)):
            if a.data_ptr() != b.data_ptr():
                raise OmerfError("TrainStep parameters must be the scene's own tensors")
        loss, saved, inputs = train_fwd(scene, rays, target, smooth_dirs, lam)
        ctx.scene, ctx.saved, ctx.inputs, ctx.lam = scene, saved, inputs, lam
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out):
        g = train_bwd(ctx.scene, ctx.saved, ctx.inputs, ctx.lam, grad_scale=grad_out.detach().float())
        s = ctx.scene

        def cast(name):
            t = g[name]
            ref = getattr(s, name)
            return t if ref.dtype == torch.float32 else t.to(ref.dtype)

        return (None, None, None, None, None, cast("grid"), cast("p_xy"), cast("p_xz"), cast("p_yz"),
                g["occ"], g["mlp"])


class Trainer:
    """The training loop of appendix A over a scene: one fused forward +
    backward (train_step), the sparsity and entropy terms (Eqs. 13-14) when
    their point and ray sets are given, one fused Adam step over features, occupancy plane
    and MLP with exponentially decaying learning rates, the lambda_7 schedule,
    and a hull update after the occupancy plane moved.  For a BF16 scene the
    optimiser keeps FP32 master copies and writes the rounded features back
    into the scene's tensors.
    """

    def __init__(self, scene: Scene, total_steps=80000, lr=(1e-2, 1e-3), lr_occ=(5e-5, 1e-5), lam_rgb=1.0,
                 lam_smooth=0.1, lam_occ=None, lam_sparsity=0.05, lam_entropy=1e-3, betas=(0.9, 0.99),
                 eps=1e-15, grow_bricks_every=1):
        self.scene = scene
        self.grow_bricks_every = int(grow_bricks_every)
        self.bricks_grown = 0
        self.total = int(total_steps)
        self.lr, self.lr_occ = lr, lr_occ
        self.lam_rgb, self.lam_smooth, self.lam_occ = lam_rgb, lam_smooth, lam_occ
        self.lam_sparsity, self.lam_entropy = lam_sparsity, lam_entropy
        self.betas, self.eps = betas, eps
        self.step_no = 0
        self.grads = zero_grads(scene)
        self.master, self.shadow = {}, {}
        for k in ("grid", "p_xy", "p_xz", "p_yz", "occ", "mlp"):
            t = getattr(scene, k)
            if t.dtype == torch.float32:
                self.master[k], self.shadow[k] = t, None
            else:
                self.master[k], self.shadow[k] = t.float().contiguous(), t
        self.moments = {k: (torch.zeros_like(v), torch.zeros_like(v)) for k, v in self.master.items()}
        self.saved = None

    def step(self, rays, target, smooth_dirs=None, sparsity_points=None, entropy_rays=None):
        """One iteration; the optional point and ray sets add the sparsity
        (Eq. 13) and entropy (Eq. 14) terms to the loss total (slot 0) and the
        gradients before the Adam step."""
        lam7 = lambda_occ(self.step_no) if self.lam_occ is None else self.lam_occ
        lam = (self.lam_rgb, self.lam_smooth, lam7)
        for g in self.grads.values():
            g.zero_()
        n = int(torch.as_tensor(rays).shape[0])
        if self.saved is None or self.saved.numel() < n * saved_bytes_per_ray() // 4:
            self.saved = torch.empty(max(n, 1) * saved_bytes_per_ray() // 4, dtype=torch.float32,
                                     device=self.scene.device)
        res = train_step(self.scene, rays, target, smooth_dirs, lam=lam, grads=self.grads, saved=self.saved)
        total = res["loss"][0:1]
        if sparsity_points is not None and self.lam_sparsity:
            sparsity_loss(self.scene, sparsity_points, lam=self.lam_sparsity, grads=self.grads, loss=total)
        if entropy_rays is not None and self.lam_entropy:
            entropy_loss(self.scene, entropy_rays, lam=self.lam_entropy, grads=self.grads, loss=total)
        lr = lr_exponential(self.lr[0], self.lr[1], self.step_no, self.total)
        lr_o = lr_exponential(self.lr_occ[0], self.lr_occ[1], self.step_no, self.total)
        groups = []
        for k, p in self.master.items():
            m, v = self.moments[k]
            groups.append({"param": p.view(-1), "grad": self.grads[k].view(-1), "m": m.view(-1), "v": v.view(-1),
                           "lr": lr_o if k == "occ" else lr,
                           "shadow": None if self.shadow[k] is None else self.shadow[k].view(-1)})
        self.step_no += 1
        adam_step(groups, self.step_no, beta1=self.betas[0], beta2=self.betas[1], eps=self.eps)
        self.scene.update()
        if self.scene.brick and self.grow_bricks_every > 0 and self.step_no % self.grow_bricks_every == 0:
            self.grow_bricks()
        return res["loss"]

    def grow_bricks(self, stream=None) -> bool:
        """Store the bricks Sec. 4.4's rule now wants for the moved occupancy
        plane (brick scenes): the table grows (no brick is dropped), the FP32
        master grid, both Adam moments and the scene's features are
        re-extracted into the new pool layout (new bricks start at zero) and
        the trainer's scene is rebuilt over them.  One 4-byte readback; returns
        True if the table grew."""
        sc = self.scene
        if not sc.brick:
            return False
        table, n_alloc, missing = grow_brick_table(sc.aabb, sc.grid_res, sc.brick, sc.occ, sc.table, stream)
        if int(missing.item()) == 0:
            return False
        nb = int(n_alloc.item())

        def remap(t):
            return extract_bricks(sc.grid_res, sc.brick, table, t, src_table=sc.table, n_bricks=nb,
                                  src_n_bricks=int(t.shape[0]), stream=stream)

        master = remap(self.master["grid"])
        m, v = (remap(t) for t in self.moments["grid"])
        grid = master if self.shadow["grid"] is None else remap(sc.grid)
        new = Scene(aabb=sc.aabb, grid=grid, table=table, brick=sc.brick, grid_res=sc.grid_res, p_xy=sc.p_xy,
                    p_xz=sc.p_xz, p_yz=sc.p_yz, occ=sc.occ, mlp=sc.mlp, step=sc.step, eps=sc.eps, t_thr=sc.t_thr,
                    n_max=sc.n_max, bg=sc.bg, plane_z=sc.plane_z, stream=stream)
        self.master["grid"] = master
        if self.shadow["grid"] is not None:
            self.shadow["grid"] = grid
        self.moments["grid"] = (m, v)
        self.grads["grid"] = torch.zeros(grid.shape, dtype=torch.float32, device=grid.device)
        self.scene = new
        sc.close()
        self.bricks_grown += 1
        return True

    # ------------------------------------------------------------ checkpointing
    _SETTINGS = ("total", "lr", "lr_occ", "lam_rgb", "lam_smooth", "lam_occ", "lam_sparsity", "lam_entropy",
                 "betas", "eps", "grow_bricks_every")

    def state_dict(self) -> dict:
        """What resuming needs, as host arrays: the FP32 master parameters,
        both Adam moments of every group, the iteration counter and the
        optimiser settings.  (A BF16 scene's features are the rounded master.)"""
        out = {"step_no": np.int64(self.step_no)}
        for k in self._SETTINGS:
            v = getattr(self, k)
            out["setting/" + k] = np.asarray(np.nan if v is None else v, np.float64)
        for k, p in self.master.items():
            m, v = self.moments[k]
            out["param/" + k] = p.detach().cpu().numpy()
            out["m/" + k] = m.cpu().numpy()
            out["v/" + k] = v.cpu().numpy()
        return out

    def load_state_dict(self, state: dict):
        """Restore a state_dict into this trainer's tensors in place (shapes
        must match), rewrite a BF16 scene's features from the master copy and
        recompute the occupancy hull."""
        for k, p in self.master.items():
            for name, dst in (("param/", p), ("m/", self.moments[k][0]), ("v/", self.moments[k][1])):
                src = np.asarray(state[name + k])
                if tuple(src.shape) != tuple(dst.shape):
                    raise OmerfError(f"checkpoint {name + k} has shape {src.shape}, expected {tuple(dst.shape)}")
                dst.copy_(torch.as_tensor(src, dtype=torch.float32))
            if self.shadow[k] is not None:
                self.shadow[k].copy_(p)
        for k in self._SETTINGS:
            if "setting/" + k not in state:
                continue  # a checkpoint written before the setting existed
            v = np.asarray(state["setting/" + k])
            if k == "lam_occ" and np.isnan(v):
                v = None
            elif k in ("total", "grow_bricks_every"):
                v = int(v)
            elif v.ndim:
                v = tuple(float(x) for x in v)
            else:
                v = float(v)
            setattr(self, k, v)
        self.step_no = int(state["step_no"])
        self.scene.update()

    def save(self, path):
        """Write the scene's layout (box, grid and plane sizes, brick table,
        plane z-range, march settings, feature dtype) and the state_dict to
        one .npz file."""
        sc = self.scene
        meta = {"scene/aabb": np.asarray(sc.aabb, np.float32), "scene/grid_res": np.asarray(sc.grid_res, np.int32),
                "scene/brick": np.int32(sc.brick),
                "scene/march": np.asarray([sc.step, sc.eps, sc.t_thr, sc.n_max], np.float64),
                "scene/bg": np.asarray(sc.bg, np.float32),
                "scene/plane_z": np.asarray(sc.plane_z if sc.plane_z is not None else (np.nan, np.nan), np.float32),
                "scene/bf16": np.int32(sc.feat_dtype == torch.bfloat16)}
        if sc.table is not None:
            meta["scene/table"] = sc.table.cpu().numpy()
        np.savez(path, **meta, **self.state_dict())

    @classmethod
    def load(cls, path, device="cuda", stream=None) -> "Trainer":
        """Rebuild the scene and its trainer from a file written by save()."""
        z = np.load(path)
        dev = torch.device(device)
        dt = torch.bfloat16 if int(z["scene/bf16"]) else torch.float32
        feats = {k: torch.as_tensor(z["param/" + k]).to(dev).to(dt).contiguous()
                 for k in ("grid", "p_xy", "p_xz", "p_yz")}
        step, eps, t_thr, n_max = (float(v) for v in z["scene/march"])
        pz = z["scene/plane_z"]
        scene = Scene(aabb=tuple(z["scene/aabb"]), grid=feats["grid"], p_xy=feats["p_xy"], p_xz=feats["p_xz"],
                      p_yz=feats["p_yz"], occ=torch.as_tensor(z["param/occ"]).to(dev).contiguous(),
                      mlp=torch.as_tensor(z["param/mlp"]).to(dev).contiguous(), step=step, eps=eps, t_thr=t_thr,
                      n_max=int(n_max), bg=tuple(z["scene/bg"]),
                      table=torch.as_tensor(z["scene/table"]).to(dev) if "scene/table" in z else None,
                      brick=int(z["scene/brick"]), grid_res=tuple(int(v) for v in z["scene/grid_res"]),
                      plane_z=None if np.isnan(pz).any() else tuple(pz), stream=stream)
        tr = cls(scene)
        tr.load_state_dict(dict(z))
        return tr
