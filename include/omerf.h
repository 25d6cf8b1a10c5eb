/*
 * omerf.h -- C ABI of the GB300 (sm_103a) Oblique-MERF hot path.
 *
 * Oblique-MERF (arXiv 2404.09531) renders a ray by marching through a
 * low-resolution feature grid plus three high-resolution feature planes
 * (Sec. 3, Eq. 2), restricted to the interval [z_min, z_max] that an
 * occupancy plane stores for the nearest (x, y) grid point (Sec. 4.1,
 * Eqs. 6-8), alpha-compositing diffuse colour and specular features front to
 * back (Eq. 1) and shading the pixel with a small deferred MLP (Eq. 4).
 * Training adds a photometric Charbonnier loss (Eq. 12), a view-direction
 * smoothness loss (Eqs. 9-10) and an interval-span loss (Eq. 5).
 *
 * Conventions shared by every entry point
 *   - Pointers named "device" point to CUDA device memory owned by the caller
 *     (for example PyTorch tensors); the library never frees them and never
 *     keeps them beyond the scene handle's lifetime.  Before launching, every
 *     entry point checks on the host (cudaPointerGetAttributes, which
 *     allocates nothing) that each non-NULL device pointer it was given is
 *     device or managed memory, and returns OMERF_EDEVICE naming the argument
 *     otherwise (render outputs may also be page-locked host memory, see
 *     omerf_render); their sizes cannot be checked and are the caller's.
 *     "host" pointers are read before the call returns.
 *   - Layouts are channel-last and x-major:
 *       dense grid   [Lx][Ly][Lz][8]
 *       brick pool   [n_bricks][B][B][B][8] with brick table [nbx][nby][nbz]
 *                    (nb? = ceil(L?/B), entries are pool indices or -1)
 *       planes       XY [Rx][Ry][8], XZ [Rx][Rz][8], YZ [Ry][Rz][8]
 *       occupancy    [M][M][2] = (z_min, z_max), cell (i, j) covers
 *                    x0 + [i, i+1) (x1-x0)/M by y0 + [j, j+1) (y1-y0)/M
 *       MLP          883 floats: W1[16][34] b1[16] W2[16][16] b2[16] W3[3][16] b3[3]
 *                    input = [F (7), d, sin(2^k d), cos(2^k d) for k = 0..3]
 *       rays         [n][6] = (origin, unit direction), float32
 *   - Features are float32 (OMERF_F32) or bfloat16 (OMERF_BF16); every
 *     accumulation, the transmittance and the sample schedule are float32.
 *   - Which lattice samples t_k = k * step (k >= 0) a ray evaluates is
 *     decided in float32 without fused multiply-add: p = o + t_k d, p inside
 *     the box (closed), nearest occupancy cell c = floor((x - x0) * (M /
 *     (x1 - x0))) clamped to [0, M-1] (same for y), z_min(c) < z < z_max(c).
 *     A ray stops after the sample where its transmittance drops below t_thr
 *     (0 disables), or after n_max evaluated samples, and uses lattice
 *     indices k < 2^24 only.
 *   - Every call is asynchronous on the given CUDA stream (NULL = the legacy
 *     default stream).  Errors found on the host (bad sizes, null pointers,
 *     misaligned pointers) return a negative status before anything is
 *     launched; CUDA launch errors return OMERF_ECUDA; errors raised while a
 *     kernel runs surface at the next call or at omerf_sync.
 *   - omerf_last_error() returns a thread-local message for the last failure.
 *   - Calls that share one scene handle must be ordered on one stream: a
 *     render or training launch uses the scene's internal work counters.
 */
#ifndef OMERF_H
#define OMERF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OMERF_OK = 0,
    OMERF_EINVAL = -1,   /* invalid argument (null pointer, bad enum, bad value) */
    OMERF_ESHAPE = -2,   /* inconsistent sizes */
    OMERF_EDEVICE = -3,  /* no usable CUDA device, or a pointer is not device memory */
    OMERF_ECUDA = -4,    /* a CUDA runtime call failed */
    OMERF_ETIMEOUT = -5, /* omerf_sync gave up waiting, or a bounded device-side wait ran out */
    OMERF_ENOMEM = -6,   /* the library could not allocate its own state */
    OMERF_ECHECK = -7    /* the checking build counted feature reads outside the arrays */
} omerf_status;

enum { OMERF_F32 = 0, OMERF_BF16 = 1 };

/* Scene description.  All array pointers are device pointers owned by the
 * caller and must stay valid while the scene handle exists. */
typedef struct {
    float aabb[6];             /* x0, x1, y0, y1, z0, z1 (x1 > x0 etc.) */
    int32_t grid_res[3];       /* grid vertices Lx, Ly, Lz (each >= 2) */
    int32_t brick;             /* brick edge B in vertices (power of two, 2..32), 0 = dense grid */
    int32_t n_bricks;          /* number of pool bricks (brick grids only) */
    int32_t plane_res[3];      /* plane texels Rx, Ry, Rz (each >= 2) */
    int32_t occ_res;           /* occupancy cells per axis M (>= 1) */
    int32_t feat_dtype;        /* OMERF_F32 or OMERF_BF16 (grid and planes) */
    float step;                /* lattice spacing; must be a power of two */
    float eps_occ;             /* ramp width epsilon of Eq. 6 (> 0); q = 2 */
    float t_thr;               /* early-termination threshold on T (>= 0) */
    float bg[3];               /* background colour added as T_N * bg */
    int32_t n_max;             /* maximum evaluated samples per ray (1..65536) */
    const void *grid;          /* device: dense grid or brick pool; 32-byte aligned (float32) or 16 (bfloat16) */
    const int32_t *brick_table;/* device: brick table (brick grids only): [nbx][nby][nbz] int32, pool
                                  index or -1.  Each of a sample's 8 corner vertices is read
                                  through the brick that holds it; a vertex of a brick that is not
                                  stored reads as zero (and receives no gradient).  Any table is
                                  accepted; one from omerf_build_brick_table (Sec. 4.4's rule,
                                  dilated by one voxel) stores every brick an evaluated sample
                                  touches, and omerf_grow_brick_table extends a table after the
                                  occupancy plane has moved. */
    const void *plane_xy;      /* device, aligned like grid */
    const void *plane_xz;      /* device, aligned like grid */
    const void *plane_yz;      /* device, aligned like grid */
    const float *occ;          /* device: [M][M][2], 8-byte aligned */
    const float *mlp;          /* device: 883 float32 weights (always float32) */
    float plane_z[2];          /* z-range spanned by the Rz rows of the XZ and YZ planes (a crop to the
                                  occupancy bounds, Sec. 4.4); plane_z[1] <= plane_z[0], e.g. zeros:
                                  the box's z-range */
} omerf_scene_desc;

/* Pinhole camera (host data, validated: finite pose and intrinsics, non-zero
 * focal lengths and a non-singular R, else OMERF_EINVAL before any launch).
 * c2w is the 3x4 row-major camera-to-world matrix [R | o];
 * the camera looks down its -z axis, image rows go along -y.  The ray of
 * pixel (px, py) has direction normalize(R (u, v, -1)) with
 * u = (px + 0.5 - cx) / fx and v = -(py + 0.5 - cy) / fy, evaluated in
 * float32 left to right without fused operations; ray index py * width + px. */
typedef struct {
    float c2w[12];
    float fx, fy, cx, cy;
    int32_t width, height;
} omerf_camera;

typedef struct omerf_scene omerf_scene;

/* Create a scene handle from a description (validated on the host).  The
 * handle owns small device state only: the occupancy hull and coarse
 * max-pooled occupancy grid used to skip empty space, per-launch work
 * counters and, for a brick grid, one 32-byte neighbour record per brick of
 * the grid (nbx * nby * nbz, stored or not).  It builds
 * that state on `stream`; for a brick grid it then waits for the stream and
 * checks that every table entry is -1 or a valid pool index (OMERF_ESHAPE
 * otherwise).  Texels are addressed with 32-bit element offsets, so the
 * dense grid (or the brick pool) and each plane must hold fewer than 2^31
 * elements (OMERF_ESHAPE otherwise).  Errors: OMERF_EINVAL / OMERF_ESHAPE
 * for bad descriptions, OMERF_ENOMEM / OMERF_ECUDA if its state cannot be
 * allocated. */
omerf_status omerf_scene_create(const omerf_scene_desc *desc, void *stream, omerf_scene **out);

/* Device memory in bytes that omerf_scene_create allocates for this
 * description (the handle's own state listed above; the caller's arrays are
 * not counted), or the negative status omerf_scene_create would return
 * for an invalid description (the same host checks; no pointer is read or
 * queried).  Host only: no CUDA call, no allocation. */
int64_t omerf_scene_device_bytes(const omerf_scene_desc *desc);

/* Recompute the scene's occupancy hull after the caller changed occ in
 * place (for example after an optimiser step on z_min / z_max). */
omerf_status omerf_scene_update(omerf_scene *scene, void *stream);

/* Free the handle's own device state (not the caller's arrays). */
void omerf_scene_destroy(omerf_scene *scene);

/* Occupancy-driven brick allocation (Sec. 4.4: features are stored only
 * where the occupancy plane marks space as occupied).  Brick (bi, bj, bk)
 * of B^3 vertices is allocated iff an occupancy cell overlapping the brick's
 * xy footprint dilated by one voxel has a non-empty [z_min, z_max] meeting
 * the brick's z-range dilated by one voxel (float32 test).  Pool indices
 * are assigned in x-major brick order.
 *   occ      device [M][M][2]
 *   table    device int32 [ceil(Lx/B)][ceil(Ly/B)][ceil(Lz/B)] (output)
 *   n_alloc  device int32 scalar (output): number of allocated bricks
 * The dilation guarantees that no evaluated sample interpolates a vertex of
 * an unallocated brick. */
omerf_status omerf_build_brick_table(const float aabb[6], const int32_t grid_res[3], int32_t brick,
                                     const float *occ, int32_t occ_res, int32_t *table,
                                     int32_t *n_alloc, void *stream);

/* Grow a brick table after the occupancy plane has moved (training moves
 * z_min and z_max, so the bricks Sec. 4.4's rule stores change): table =
 * the bricks old_table stores plus the bricks the rule of
 * omerf_build_brick_table allocates for occ, pool indices reassigned in
 * x-major brick order (re-extract the pool with omerf_extract_bricks from the
 * old pool and old_table).  Bricks are never dropped, so the features
 * trained so far are kept.
 *   old_table  device int32 [nbx][nby][nbz]: entries -1 or >= 0
 *   table      device int32, same shape (output; must not be old_table)
 *   n_alloc    device int32 scalar (output): bricks in table
 *   missing    device int32 scalar (output): bricks the rule allocates that
 *              old_table does not store; 0 means old_table already covers
 *              the rule (table then stores the same bricks)
 * Errors as omerf_build_brick_table.  Two kernel launches and a memset. */
omerf_status omerf_grow_brick_table(const float aabb[6], const int32_t grid_res[3], int32_t brick,
                                    const float *occ, int32_t occ_res, const int32_t *old_table,
                                    int32_t *table, int32_t *n_alloc, int32_t *missing, void *stream);

/* Ray interval (box and occupancy-slab intersection, Sec. 4.4's bounding-box
 * skipping): for each ray, the inclusive lattice index range [k_lo, k_hi]
 * that the march scans.  Every evaluated sample of the ray lies inside it;
 * an empty range has k_lo > k_hi.
 *   cam    host camera (then n must be width * height and rays NULL), or NULL
 *   rays   device [n][6] when cam is NULL
 *   k_range device int32 [n][2] (output) */
omerf_status omerf_ray_interval(const omerf_scene *scene, const omerf_camera *cam, const float *rays,
                                int64_t n, int32_t *k_range, void *stream);

/* Forward render (Eqs. 1-4, 6-8): per ray, composite the evaluated samples
 * and shade with the deferred MLP:
 *     rgb = sum_i w_i c^d_i + G(F, d) + T_N * bg,  F = [sum w c^d, sum w f],
 *     w_i = T_i M_i alpha_i,  T_{i+1} = T_i (1 - M_i alpha_i),
 * and rgb = bg for a ray with no evaluated sample.
 *   cam    host camera (n == width * height, rays NULL), or NULL
 *   rays   device [n][6] float32 when cam is NULL: origin, unit direction
 *          (device data is not validated on the host; a ray with a
 *          non-finite component evaluates no sample and returns bg)
 *   rgb    float32 [n][3] (output): device memory, or page-locked host memory
 *          (cudaHostAlloc / cudaHostRegister), which the kernel writes
 *          directly (on Grace-Blackwell over the coherent chip-to-chip link),
 *          so that no copy follows the render; any other host pointer is
 *          rejected with OMERF_EDEVICE
 *   count  int32 [n] evaluated samples per ray (output, may be NULL), memory
 *          as for rgb
 * The deferred MLP runs in float32 for OMERF_F32 scenes and in bfloat16 on
 * tensor cores with float32 accumulation for OMERF_BF16 scenes. */
omerf_status omerf_render(const omerf_scene *scene, const omerf_camera *cam, const float *rays,
                          int64_t n, float *rgb, int32_t *count, void *stream);

/* Render without allocating (the paper has no counterpart: this is a
 * deployment variant of omerf_render).  For callers that must not allocate
 * device memory -- a host framework that owns all device memory and passes in
 * fixed buffers, or a frame loop that cannot afford cudaMalloc, which may
 * synchronise the device.  It takes the scene description directly (no
 * handle) and keeps its scratch (work counters, occupancy hulls, brick
 * neighbour records) in an 8 MiB static __device__ array that every GPU
 * loading this library holds until the process exits.  Arguments, layouts
 * and results are those of omerf_render.
 *   - The first call on a device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *     The address is kept for the life of the process: do not call this
 *     entry point on a device after cudaDeviceReset on it.
 *   - Pointers are checked as omerf_scene_create and omerf_render check them:
 *     the description's arrays and a ray list must be device memory
 *     (OMERF_EDEVICE otherwise), rgb and count device or page-locked host
 *     memory.
 *   - Scenes whose scratch does not fit are rejected with OMERF_ESHAPE: the
 *     coarse occupancy grid takes 8 bytes per cell (ceil(M / 2^l)^2 cells, l
 *     the smallest level whose cells span a 32-sample lattice window,
 *     rounded up to 256 bytes) and a brick grid 32 bytes per brick of the
 *     grid, stored or not (nbx * nby * nbz); together at most 8,384,256
 *     bytes.
 *   - Every call reuses the same array: calls whose kernels overlap on the GPU
 *     (different streams, or several host threads) race and give wrong
 *     results.  Order them on one stream.
 *   - Unlike omerf_scene_create it does not check the brick table (that
 *     needs a synchronising read): every entry must be -1 or a pool index
 *     below n_bricks.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine. */
omerf_status omerf_render_noalloc(const omerf_scene_desc *desc, const omerf_camera *cam, const float *rays,
                                  int64_t n, float *rgb, int32_t *count, void *stream);

/* Render several cameras in one launch (a step of a multi-view frame set):
 * rgb [sum of width * height][3] and count in camera order, memory as for
 * omerf_render.  The cameras' super-tiles share one persistent launch (up to
 * 16 cameras per launch; more are rendered in groups of 16), so no SM idles
 * at the end of one frame while the next waits.  The camera records are
 * copied to the scene's device state on `stream`, which therefore orders
 * this call with the scene's other calls as usual. */
omerf_status omerf_render_cameras(const omerf_scene *scene, const omerf_camera *cams, int32_t n_cams,
                                  float *rgb, int32_t *count, void *stream);

/* Bytes of per-ray state that omerf_train_fwd writes for omerf_train_bwd. */
int64_t omerf_saved_bytes_per_ray(void);

/* Training forward (Eqs. 5, 9-10, 12), float32 or bfloat16 features:
 *   L = lambda[0] * mean_r sqrt(|C_r - C*_r|^2 + 1e-6)
 *     + lambda[1] * mean_r sum_k S(d, s_k) |G(F, s_k/|s_k|) - G(F, d)|^2
 *     + lambda[2] * sum_cells (z_max - z_min)^2
 * with S the cosine similarity and s_k = d + delta_k supplied by the caller.
 *   rays        device [n][6]       target     device [n][3]
 *   smooth_dirs device [n][K][3] (K in 0..16; may be NULL when K == 0)
 *   lambda      host [3]
 *   saved       device, n * omerf_saved_bytes_per_ray() bytes, 16-byte aligned (output)
 *   loss        device float32 [4] (output): total, rgb, smooth, occ terms */
omerf_status omerf_train_fwd(const omerf_scene *scene, const float *rays, const float *target,
                             const float *smooth_dirs, int64_t n, int32_t K, const float lambda[3],
                             void *saved, float *loss, void *stream);

/* Training backward: recomputes each ray's march (no per-sample storage)
 * and ACCUMULATES (+=) grad_scale * dL/dparam into caller-zeroed float32
 * buffers shaped like the parameters (g_grid like the dense grid or the
 * brick pool).  grad_scale is a device float32 scalar (NULL means 1).
 * The same rays, target, smooth_dirs, K, lambda and saved state as the
 * matching omerf_train_fwd call must be passed; the backward also writes the
 * per-ray dL/dF and dL/dT_N into the second half of each saved record. */
omerf_status omerf_train_bwd(const omerf_scene *scene, const float *rays, const float *target,
                             const float *smooth_dirs, int64_t n, int32_t K, const float lambda[3],
                             void *saved, const float *grad_scale, float *g_grid, float *g_xy,
                             float *g_xz, float *g_yz, float *g_occ, float *g_mlp, void *stream);

/* One fused training step: omerf_train_fwd then omerf_train_bwd with
 * grad_scale 1 (loss written, gradients accumulated). */
omerf_status omerf_train_step(const omerf_scene *scene, const float *rays, const float *target,
                              const float *smooth_dirs, int64_t n, int32_t K, const float lambda[3],
                              void *saved, float *loss, float *g_grid, float *g_xy, float *g_xz,
                              float *g_yz, float *g_occ, float *g_mlp, void *stream);

/* Sparsity loss (Sec. 4.3, Eq. 13): L = lambda / n * sum_i alpha(p_i) with
 * alpha = 1 - exp(-tau(p) * step), tau = exp of the density channel of Eq. 2,
 * over n caller-chosen points (the paper draws them in the occupied space).
 *   points  device float32 [n][3]
 *   loss    device float32 [1] or NULL: L is ADDED (+=) to *loss
 *   g_*     caller-owned float32 gradient buffers shaped like the parameters
 *           (g_grid like the dense grid or the brick pool), each may be NULL:
 *           grad_scale * dL/dparam is ADDED; only channel 0 is touched
 *   grad_scale  device float32 scalar or NULL (1)
 * Float32 or bfloat16 features.  One kernel launch. */
omerf_status omerf_sparsity_loss(const omerf_scene *scene, const float *points, int64_t n, float lambda,
                                 const float *grad_scale, float *loss, float *g_grid, float *g_xy,
                                 float *g_xz, float *g_yz, void *stream);

/* Entropy loss (Sec. 4.3, Eq. 14) over n rays (the paper casts them from high
 * altitude towards the ground): for each ray, a_i = M_i alpha_i over its
 * evaluated samples (the sample rule of Eq. 7 with no early termination, at
 * most n_max samples), p_i = a_i / sum_j a_j, L_r = -sum_i p_i log p_i;
 * L = lambda / n * sum_r L_r.  Rays with no sample add nothing.  The gradient
 * reaches channel 0 of the features and, through the occupancy ramps of
 * Eq. 6, both z bounds of the occupancy plane (g_occ [M][M][2], 8-byte
 * aligned).  Arguments otherwise as omerf_sparsity_loss; rays device float32
 * [n][6] (origin, unit direction).  One kernel launch. */
omerf_status omerf_entropy_loss(const omerf_scene *scene, const float *rays, int64_t n, float lambda,
                                const float *grad_scale, float *loss, float *g_grid, float *g_xy,
                                float *g_xz, float *g_yz, float *g_occ, void *stream);

/* ---- extraction after training (Sec. 4.4, Sec. 5.3) ------------------ */

/* 3D occupancy grid of N[0] x N[1] x N[2] voxels over the box, derived from
 * the occupancy plane alone (the paper extracts one after training and
 * reports its occupancy ratio, Sec. 5.3).  Voxel (i, j, k) covers
 * [x0 + i hx, x0 + (i+1) hx) x [y0 + j hy, ...) x [z0 + k hz, z0 + (k+1) hz)
 * and is occupied iff an occupancy cell a, b overlapping its xy footprint
 * (a / M < (i + 1) / Nx and (a + 1) / M > i / Nx, same for b; exact integer
 * arithmetic) has z_min < z_max, z_min < z_hi and z_max > z_lo, with z_lo =
 * z0 + k hz, z_hi = z0 + (k + 1) hz and hz = (z1 - z0) / Nz in float32
 * without fused operations: exactly the voxels holding a point the sample
 * rule could evaluate.
 *   aabb   host [6]; only z0, z1 and the occupancy cell layout matter
 *   occ    device [M][M][2]
 *   bits   device uint32 [Nx][Ny][ceil(Nz / 32)] (output): bit t of word w is
 *          voxel k = 32 w + t; unused high bits of the last word are 0
 *   count  device uint64 or NULL: the number of occupied voxels is ADDED
 * One kernel launch. */
omerf_status omerf_occupancy_grid(const float aabb[6], const float *occ, int32_t M, const int32_t N[3],
                                  uint32_t *bits, unsigned long long *count, void *stream);

/* Brick pool for a brick table (Sec. 4.4: the grid is stored as sparse
 * bricks where the occupancy plane marks space as occupied; build the table
 * with omerf_build_brick_table).  Brick b = table[bi][bj][bk] >= 0 receives
 * vertices (bi B + li, bj B + lj, bk B + lk) of the source, which is a dense
 * grid [Lx][Ly][Lz][8] (src_table NULL) or an older brick pool with table
 * src_table (same grid_res and B; re-extraction after the occupancy plane
 * changed).  Vertices beyond the grid, or in a brick the source does not
 * hold, are 0.  Table entries >= n_bricks (and source entries >=
 * src_n_bricks) are skipped.
 *   table, src_table  device int32 [nbx][nby][nbz]
 *   src, pool         device, feat_dtype elements, 16-byte aligned; pool holds
 *                     n_bricks x B^3 x 8 values (output; must not overlap src)
 * One kernel launch. */
omerf_status omerf_extract_bricks(const int32_t grid_res[3], int32_t brick, const int32_t *table, int32_t n_bricks,
                                  const void *src, const int32_t *src_table, int32_t src_n_bricks,
                                  int32_t feat_dtype, void *pool, void *stream);

/* 1 if the driver provides tensor-map encoding, so that omerf_extract_bricks
 * copies bricks of up to 32 KB from a dense grid with tiled tensor-memory-
 * accelerator loads (an (8, B, B, B) box of the grid per brick, zeros beyond
 * its end) and bulk stores; 0 if it falls back to plain loads.  Host-only. */
int32_t omerf_tma_available(void);

/* Rows [k0, k1] of the XZ and YZ planes that any evaluated sample can read
 * (Sec. 4.4: the planes' z-resolution follows the occupancy plane's bounds).
 * Samples lie strictly inside (lo, hi), the hull of the non-empty cells;
 * the stencil reads rows floor(u) and floor(u) + 1 with u = (z - plane_z[0])
 * (Rz - 1) / (plane_z[1] - plane_z[0]) in float32; one row of margin on each
 * side, clamped to [0, Rz - 1], at least two rows.
 *   plane_z  host [2]: the z-range the current Rz rows span (the box's
 *            z-range for uncropped planes)
 *   rows     device int32 [2] (output): k0, k1, or -1, -1 if no cell is occupied
 *   z_range  device float [2] (output): plane_z[0] + k (plane_z[1] -
 *            plane_z[0]) / (Rz - 1) for k0 and k1, the cropped planes' plane_z
 * One single-block kernel launch; the caller reads rows back to size the
 * cropped planes. */
omerf_status omerf_plane_crop_rows(const float plane_z[2], int32_t Rz, const float *occ, int32_t M,
                                   int32_t *rows, float *z_range, void *stream);

/* Copy rows [k0, k1] of a plane [n_outer][Rz][8] into [n_outer][k1-k0+1][8]
 * (XZ: n_outer = Rx; YZ: n_outer = Ry).  src and dst device, feat_dtype
 * elements, 16-byte aligned, not overlapping.  One kernel launch. */
omerf_status omerf_crop_planes(const void *src, int64_t n_outer, int32_t Rz, int32_t k0, int32_t k1,
                               int32_t feat_dtype, void *dst, void *stream);

/* One parameter group of an Adam step: float32 master values, gradient and
 * moments (device, n values each, updated in place; moments start at zero),
 * an optional bfloat16 copy written after the update (the feature tensor a
 * BF16 scene renders from), and the group's learning rate. */
typedef struct {
    float *param;
    const float *grad;
    float *m;
    float *v;
    void *shadow_bf16;  /* device bfloat16 [n] or NULL */
    int64_t n;
    float lr;
} omerf_adam_group;

/* Fused Adam step over up to 8 groups in one launch (appendix A trains with
 * Adam, beta1 = 0.9, beta2 = 0.99, eps = 1e-15; Kingma and Ba's update with
 * bias correction): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).  step >= 1
 * counts from 1.  After changing the occupancy plane call omerf_scene_update. */
omerf_status omerf_adam_step(const omerf_adam_group *groups, int32_t n_groups, float beta1, float beta2,
                             float eps, int64_t step, void *stream);

/* Learning-rate decay of appendix A: lr0 at step 0 to lr1 at step total,
 * exponential in between (1e-2 -> 1e-3 for features and MLP, 5e-5 -> 1e-5
 * for the occupancy plane).  Host-only. */
float omerf_lr_exponential(float lr0, float lr1, int64_t step, int64_t total);

/* Occupancy-loss weight lambda_7 of appendix A: 0 before iteration 10,000,
 * then 1e-4 multiplied by 1.5 every 2,000 iterations, at most 0.2.  Host-only. */
float omerf_lambda_occ(int64_t step);

/* Load-bandwidth probe (the paper has no counterpart: a measurement tool
 * for the roofline of the march, whose feature gather is served from L1 and
 * L2).  ctas CTAs of 256 threads each read their own bytes_per_cta-byte
 * slice of buf `passes` times with the gather's 256-bit read-only load, a
 * warp's load covering 1 KB contiguous; bytes delivered to registers =
 * ctas * bytes_per_cta * passes.  A slice that fits in L1 (with the CTAs
 * resident on one SM) measures L1's load bandwidth, a larger one inside L2
 * measures L2's.
 *   buf   device float32, ctas * bytes_per_cta bytes, 32-byte aligned
 *   bytes_per_cta  a positive multiple of 8192, at most 2^30
 *   sink  device float32 [ctas * 256] (output: per-thread sums, so that the
 *         loads are not removed)
 * One kernel launch. */
omerf_status omerf_probe_load_bandwidth(const float *buf, int64_t bytes_per_cta, int32_t ctas, int32_t passes,
                                        float *sink, void *stream);

/* Reduction-throughput probe (no counterpart in the paper: the roofline of
 * the re-march backward, whose gradient scatter of Eqs. 2 and 6-8 adds each
 * sample's 32-byte texel gradients with 16-byte vector FP32 reductions, one
 * lane per sample).  ctas CTAs of 256 threads; every warp reduces into its
 * own bytes_per_warp-byte region of buf, each lane into its own 128-byte
 * line (16 B per lane, 512 B per warp instruction), stepping through the
 * region 4 KB at a time, `passes` times; bytes reduced =
 * ctas * bytes_per_warp * passes.  The caller sizes the regions so that buf
 * stays inside L2 (the scatter's gradient lines are mostly L2 hits).
 *   buf   device float32, ctas * 8 * bytes_per_warp bytes, 16-byte aligned;
 *         every element of each warp's region that a lane hits grows by
 *         1.0 per pass (contents are otherwise unspecified)
 *   bytes_per_warp  a positive multiple of 4096, at most 2^24
 * One kernel launch. */
omerf_status omerf_probe_red_bandwidth(float *buf, int64_t bytes_per_warp, int32_t ctas, int32_t passes,
                                       void *stream);

/* Wait for `stream` with a bounded host-side poll; returns OMERF_ETIMEOUT
 * after timeout_ms milliseconds (< 0 waits without limit), OMERF_ECUDA if
 * the stream reported an error. */
omerf_status omerf_sync(void *stream, int32_t timeout_ms);

/* ---- the checking build (libomerf_check.so) ------------------------------
 * The same sources compiled with OMERF_CHECK=1: every feature read of the
 * march, the training backward and the regularisers is bounds-checked
 * against the arrays' sizes (a read outside is counted and skipped, its
 * gradient write too), and every corner read of a brick the table does not
 * store (read as zero, Eq. 2 with Sec. 4.4's sparse storage) is counted.  A
 * table built by omerf_build_brick_table never causes one for an evaluated
 * sample; both counts are 0 on valid inputs.  The default build has neither
 * check and no counter. */

/* 1 in the checking build, 0 otherwise.  Host-only. */
int32_t omerf_check_build(void);

/* The scene's counters since creation or the last reset: counts[0] corner
 * reads of unstored bricks, counts[1] reads outside a feature array.  Waits
 * for `stream`; reset != 0 zeroes them afterwards (on `stream`).  Returns
 * OMERF_ECHECK if counts[1] > 0, OMERF_EINVAL in the default build (counts 0). */
omerf_status omerf_check_counts(const omerf_scene *scene, uint64_t counts[2], int32_t reset, void *stream);

/* The counters of every scene destroyed so far in this process, summed
 * (read back when each is destroyed; counts reset by omerf_check_counts are
 * not included); zeros in the default build.  Host-only. */
void omerf_check_totals(uint64_t totals[2]);

/* Thread-local description of the last failure in this thread. */
const char *omerf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OMERF_H */
