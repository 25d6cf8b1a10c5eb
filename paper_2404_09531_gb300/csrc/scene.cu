// scene.cu -- C ABI: scene handles, validation, small setup kernels
// (occupancy hull, brick table, ray interval, L_occ) and launches.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>

#include "internal.h"

namespace omerf {

static thread_local char g_err[512] = "";
// checking build: counts of the scenes destroyed so far in this process
static std::atomic<unsigned long long> g_check_total[2];

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

unsigned* next_counter(const omerf_scene* s, cudaStream_t stream) {
  unsigned slot = s->seq.fetch_add(1u) % kCounterSlots;
  unsigned* c = s->counters + slot;
  cudaMemsetAsync(c, 0, sizeof(unsigned), stream);
  return c;
}

// ---------------------------------------------------------------------------
// occupancy hull: min z_min and max z_max over the non-empty cells
// ---------------------------------------------------------------------------
__global__ void hull_kernel(const float2* __restrict__ occ, long cells, float* __restrict__ hull) {
  __shared__ float slo[32], shi[32];
  float lo = __int_as_float(0x7f800000), hi = -lo;
  for (long i = threadIdx.x; i < cells; i += blockDim.x) {
    float2 z = occ[i];
    if (z.x <= z.y) {
      lo = fminf(lo, z.x);
      hi = fmaxf(hi, z.y);
    }
  }
  for (int s = 16; s > 0; s >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(kFull, lo, s));
    hi = fmaxf(hi, __shfl_xor_sync(kFull, hi, s));
  }
  if ((threadIdx.x & 31) == 0) {
    slo[threadIdx.x >> 5] = lo;
    shi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
      lo = fminf(lo, slo[w]);
      hi = fmaxf(hi, shi[w]);
    }
    hull[0] = lo;
    hull[1] = hi;
  }
}

// Coarse max-pooled occupancy grid (Sec. 4.4: 2D max pooling of the occupancy
// plane for empty-space skipping): cell (X, Y) holds the min z_min and max
// z_max over the non-empty occupancy cells it covers, (+inf, -inf) if none.
__global__ void coarse_hull_kernel(const float2* __restrict__ occ, int M, int clog2, int Mc,
                                   float2* __restrict__ chull) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= Mc * Mc) return;
  const int X = id / Mc, Y = id % Mc;
  float lo = __int_as_float(0x7f800000), hi = -lo;
  const int i1 = min((X + 1) << clog2, M), j1 = min((Y + 1) << clog2, M);
  for (int i = X << clog2; i < i1; i++)
    for (int j = Y << clog2; j < j1; j++) {
      const float2 z = occ[i * M + j];
      if (z.x <= z.y) {
        lo = fminf(lo, z.x);
        hi = fmaxf(hi, z.y);
      }
    }
  chull[id] = make_float2(lo, hi);
}

// ---------------------------------------------------------------------------
// brick allocation (Sec. 4.4)
// ---------------------------------------------------------------------------
__device__ __forceinline__ long floor_div(long a, long b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

struct BrickArgs {
  float z0, vz;
  int L[3], B, M, nb[3];
  const float2* occ;
  int* table;
  const int* old_table;  // growing: bricks already stored are kept (NULL otherwise)
  int* missing;          // growing: count of bricks the rule adds
};

__global__ void brick_flag_kernel(const BrickArgs a, long total) {
  long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= total) return;
  const int bk = (int)(id % a.nb[2]);
  const int bj = (int)((id / a.nb[2]) % a.nb[1]);
  const int bi = (int)(id / ((long)a.nb[2] * a.nb[1]));
  long lo[2], hi[2];
  const int bb[2] = {bi, bj};
  for (int ax = 0; ax < 2; ax++) {
    const long v0 = (long)bb[ax] * a.B, den = a.L[ax] - 1;
    lo[ax] = -floor_div(-((v0 - 1) * (long)a.M), den) - 1;
    hi[ax] = floor_div((v0 + a.B) * (long)a.M, den);
    lo[ax] = lo[ax] < 0 ? 0 : lo[ax];
    hi[ax] = hi[ax] > a.M - 1 ? a.M - 1 : hi[ax];
  }
  const float zlo = __fadd_rn(a.z0, __fmul_rn((float)(bk * a.B - 1), a.vz));
  const float zhi = __fadd_rn(a.z0, __fmul_rn((float)(bk * a.B + a.B), a.vz));
  int hit = 0;
  for (long i = lo[0]; i <= hi[0] && !hit; i++)
    for (long j = lo[1]; j <= hi[1] && !hit; j++) {
      const float2 z = a.occ[i * a.M + j];
      if (z.x <= z.y && z.y >= zlo && z.x <= zhi) hit = 1;
    }
  if (a.old_table) {
    const int kept = a.old_table[id] >= 0;
    if (hit && !kept) atomicAdd(a.missing, 1);
    hit |= kept;
  }
  a.table[id] = hit;
}

// Neighbour records of a brick grid, one per brick of the grid (stored or
// not): nbr[id][dx*4 + dy*2 + dz] is the element offset in the pool
// (pool index << shift, shift = log2 of a brick's B^3 x 8 elements) of the
// brick at (bi + dx, bj + dy, bk + dz), -2^shift if it is not stored or
// outside the grid, so that the brick offset plus any local offset (less
// than 2^shift) stays negative (slot 0 is the brick's own table entry).  A sample whose cell reaches
// into neighbour bricks finds the brick of each of its 8 corners in the
// record of its lowest corner's brick, with one 256-bit load.
__global__ void brick_neighbor_kernel(const int* __restrict__ table, int nbx, int nby, int nbz, int n_bricks,
                                      int shift, int* __restrict__ nbr) {
  const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long)nbx * nby * nbz) return;
  const int bk = (int)(id % nbz), bj = (int)((id / nbz) % nby), bi = (int)(id / ((long)nbz * nby));
  int v[8];
#pragma unroll
  for (int c = 0; c < 8; c++) {
    const int x = bi + ((c >> 2) & 1), y = bj + ((c >> 1) & 1), z = bk + (c & 1);
    int b = -1;
    if (x < nbx && y < nby && z < nbz) b = table[((long)x * nby + y) * nbz + z];
    v[c] = ((b >= 0 && b < n_bricks) ? b : -1) << shift;
  }
  int4* out = reinterpret_cast<int4*>(nbr + 8l * id);
  out[0] = make_int4(v[0], v[1], v[2], v[3]);
  out[1] = make_int4(v[4], v[5], v[6], v[7]);
}

// Count brick-table entries that are neither -1 nor a pool index.
__global__ void brick_table_check_kernel(const int* __restrict__ table, long total, int n_bricks,
                                         unsigned* __restrict__ bad) {
  const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= total) return;
  const int b = table[id];
  if (b < -1 || b >= n_bricks) atomicAdd(bad, 1u);
}

// In-place exclusive scan of the 0/1 flags into pool indices (-1 = empty),
// one CTA, each thread owning a contiguous segment (x-major brick order).
__global__ void brick_scan_kernel(int* table, long total, int* n_alloc) {
  __shared__ int sums[1024];
  const long per = (total + blockDim.x - 1) / blockDim.x;
  const long beg = threadIdx.x * per, end = beg + per < total ? beg + per : total;
  int local = 0;
  for (long i = beg; i < end; i++) local += table[i];
  sums[threadIdx.x] = local;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    int v = threadIdx.x >= (unsigned)off ? sums[threadIdx.x - off] : 0;
    __syncthreads();
    sums[threadIdx.x] += v;
    __syncthreads();
  }
  int run = sums[threadIdx.x] - local;
  for (long i = beg; i < end; i++) {
    const int f = table[i];
    table[i] = f ? run : -1;
    run += f;
  }
  if (threadIdx.x == blockDim.x - 1) *n_alloc = sums[threadIdx.x];
}

// ---------------------------------------------------------------------------
// ray interval (exposed for inspection; the march computes the same range)
// ---------------------------------------------------------------------------
__global__ void interval_kernel(const Geo g, Cam cam, int use_cam, const float* __restrict__ rays, long n,
                                int2* __restrict__ out) {
  long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n) return;
  float o[3], d[3];
  if (use_cam) {
    camera_ray(cam, (int)(id % cam.width), (int)(id / cam.width), o, d);
  } else {
    for (int c = 0; c < 3; c++) {
      o[c] = rays[6 * id + c];
      d[c] = rays[6 * id + 3 + c];
    }
  }
  int klo = 1, khi = 0;
  if (!lattice_range(g, o, d, klo, khi)) {
    klo = 1;
    khi = 0;
  }
  out[id] = make_int2(klo, khi);
}

// ---------------------------------------------------------------------------
// L_occ = sum over cells of (z_max - z_min)^2 (Eq. 5) and its gradient
// ---------------------------------------------------------------------------
__global__ void occ_loss_kernel(const float2* __restrict__ occ, long cells, float lam, const float* grad_scale,
                                float* loss, float2* g_occ) {
  __shared__ float part[32];
  const float gs = grad_scale ? *grad_scale : 1.0f;
  float acc = 0.0f;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (long)gridDim.x * blockDim.x) {
    const float2 z = occ[i];
    const float span = z.y - z.x;
    acc = fmaf(span, span, acc);
    if (g_occ) {
      const float g = gs * lam * 2.0f * span;
      float2 cur = g_occ[i];
      cur.x -= g;
      cur.y += g;
      g_occ[i] = cur;
    }
  }
  if (!loss) return;
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += part[w];
    atomicAdd(loss + 3, lam * s);
    atomicAdd(loss + 0, lam * s);
  }
}

}  // namespace omerf

using namespace omerf;

// ---------------------------------------------------------------------------
// validation helpers
// ---------------------------------------------------------------------------
static bool is_pow2_float(float x) {
  if (!(x > 0.0f) || !std::isfinite(x)) return false;
  int e;
  return std::frexp(x, &e) == 0.5f;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

omerf_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return OMERF_ECUDA;
}

omerf_status validate_desc(const omerf_scene_desc* d) {
  if (!d) { set_error("scene description is NULL"); return OMERF_EINVAL; }
  for (int a = 0; a < 3; a++) {
    if (!(d->aabb[2 * a] < d->aabb[2 * a + 1]) || !std::isfinite(d->aabb[2 * a]) || !std::isfinite(d->aabb[2 * a + 1])) {
      set_error("aabb axis %d is empty or not finite", a);
      return OMERF_EINVAL;
    }
    if (d->grid_res[a] < 2 || d->plane_res[a] < 2) {
      set_error("grid and plane resolutions must be >= 2");
      return OMERF_ESHAPE;
    }
  }
  if (d->occ_res < 1) { set_error("occ_res must be >= 1"); return OMERF_ESHAPE; }
  if (d->feat_dtype != OMERF_F32 && d->feat_dtype != OMERF_BF16) { set_error("feat_dtype must be OMERF_F32 or OMERF_BF16"); return OMERF_EINVAL; }
  if (!is_pow2_float(d->step)) { set_error("step must be a positive power of two"); return OMERF_EINVAL; }
  if (!(d->eps_occ > 0.0f) || !std::isfinite(d->eps_occ)) { set_error("eps_occ must be > 0"); return OMERF_EINVAL; }
  if (!(d->t_thr >= 0.0f) || !(d->t_thr < 1.0f)) { set_error("t_thr must be in [0, 1)"); return OMERF_EINVAL; }
  if (d->n_max < 1 || d->n_max > 65536) { set_error("n_max must be in 1..65536"); return OMERF_EINVAL; }
  for (int j = 0; j < 3; j++)
    if (!std::isfinite(d->bg[j])) { set_error("bg must be finite"); return OMERF_EINVAL; }
  if (!std::isfinite(d->plane_z[0]) || !std::isfinite(d->plane_z[1])) { set_error("plane_z must be finite"); return OMERF_EINVAL; }
  if (d->brick != 0) {
    if (d->brick < 2 || d->brick > 32 || (d->brick & (d->brick - 1))) { set_error("brick must be 0 or a power of two in 2..32"); return OMERF_EINVAL; }
    if (!d->brick_table) { set_error("brick_table is NULL for a brick grid"); return OMERF_EINVAL; }
    if (d->n_bricks < 0) { set_error("n_bricks must be >= 0"); return OMERF_ESHAPE; }
  }
  // the kernels address texels with 32-bit element offsets
  const long long B3 = d->brick ? (long long)d->brick * d->brick * d->brick : 0;
  const long long grid_elems =
      (d->brick ? (long long)d->n_bricks * B3 : (long long)d->grid_res[0] * d->grid_res[1] * d->grid_res[2]) * kNch;
  const long long plane_elems[3] = {(long long)d->plane_res[0] * d->plane_res[1] * kNch,
                                    (long long)d->plane_res[0] * d->plane_res[2] * kNch,
                                    (long long)d->plane_res[1] * d->plane_res[2] * kNch};
  if (grid_elems > 0x7fffffffLL || plane_elems[0] > 0x7fffffffLL || plane_elems[1] > 0x7fffffffLL ||
      plane_elems[2] > 0x7fffffffLL) {
    set_error("a feature array holds 2^31 or more elements (grid or pool %lld, planes %lld / %lld / %lld)",
              grid_elems, plane_elems[0], plane_elems[1], plane_elems[2]);
    return OMERF_ESHAPE;
  }
  if (!d->grid || !d->plane_xy || !d->plane_xz || !d->plane_yz || !d->occ || !d->mlp) {
    set_error("a scene array pointer is NULL");
    return OMERF_EINVAL;
  }
  // one texel (8 channels) is read with a single 256-bit (float32) or 128-bit (bfloat16) load
  const size_t fa = d->feat_dtype == OMERF_F32 ? 32 : 16;
  if (!aligned(d->grid, fa) || !aligned(d->plane_xy, fa) || !aligned(d->plane_xz, fa) || !aligned(d->plane_yz, fa)) {
    set_error("feature arrays must be %zu-byte aligned", fa);
    return OMERF_EINVAL;
  }
  if (!aligned(d->occ, 8) || !aligned(d->mlp, 4)) { set_error("occ must be 8-byte aligned"); return OMERF_EINVAL; }
  return OMERF_OK;
}

omerf_status check_device_ptrs(std::initializer_list<std::pair<const void*, const char*>> ptrs) {
  for (const auto& pn : ptrs) {
    const omerf_status st = check_device_ptr(pn.first, pn.second);
    if (st != OMERF_OK) return st;
  }
  return OMERF_OK;
}

omerf_status check_device_ptr(const void* p, const char* name) {
  if (!p) return OMERF_OK;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("%s: cannot query pointer (%s)", name, cudaGetErrorString(e));
    return OMERF_EDEVICE;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) {
    set_error("%s is not device memory", name);
    return OMERF_EDEVICE;
  }
  return OMERF_OK;
}

void fill_geo(omerf_scene* s) {
  const omerf_scene_desc& d = s->desc;
  Geo& g = s->geo;
  for (int a = 0; a < 3; a++) {
    g.lo[a] = d.aabb[2 * a];
    g.hi[a] = d.aabb[2 * a + 1];
    g.L[a] = d.grid_res[a];
    g.R[a] = d.plane_res[a];
    g.gs[a] = (float)(d.grid_res[a] - 1) / (g.hi[a] - g.lo[a]);
    g.ps[a] = (float)(d.plane_res[a] - 1) / (g.hi[a] - g.lo[a]);
  }
  g.pzoff = 0.0f;
  if (d.plane_z[1] > d.plane_z[0]) {
    g.ps[2] = (float)(d.plane_res[2] - 1) / (d.plane_z[1] - d.plane_z[0]);
    g.pzoff = (d.plane_z[0] - g.lo[2]) * g.ps[2];
  }
  // the decision rule's cell scale: float32 M / (x1 - x0)
  g.osx = (float)d.occ_res / (g.hi[0] - g.lo[0]);
  g.osy = (float)d.occ_res / (g.hi[1] - g.lo[1]);
  g.M = d.occ_res;
  g.step = d.step;
  g.inv_eps = 1.0f / d.eps_occ;
  g.t_thr = d.t_thr;
  for (int j = 0; j < 3; j++) g.bg[j] = d.bg[j];
  g.n_max = d.n_max;
  g.blog2 = 0;
  if (d.brick) {
    while ((1 << g.blog2) < d.brick) g.blog2++;
    for (int a = 0; a < 3; a++) g.nb[a] = (d.grid_res[a] + d.brick - 1) / d.brick;
  } else {
    g.nb[0] = g.nb[1] = g.nb[2] = 0;
  }
  g.grid = d.grid;
  g.table = d.brick_table;
  g.pxy = d.plane_xy;
  g.pxz = d.plane_xz;
  g.pyz = d.plane_yz;
  g.occ = reinterpret_cast<const float2*>(d.occ);
  g.mlp = d.mlp;
  g.hull = s->state;
  g.chull = s->chull;
  g.nbr = s->nbr;
  g.clog2 = s->clog2;
  g.Mc = s->Mc;
  const long long B3 = (long long)d.brick * d.brick * d.brick;
  g.lim[0] = (d.brick ? (long long)d.n_bricks * B3 : (long long)d.grid_res[0] * d.grid_res[1] * d.grid_res[2]) * kNch;
  g.lim[1] = (long long)d.plane_res[0] * d.plane_res[1] * kNch;
  g.lim[2] = (long long)d.plane_res[0] * d.plane_res[2] * kNch;
  g.lim[3] = (long long)d.plane_res[1] * d.plane_res[2] * kNch;
  g.check = s->check;
}

size_t brick_records_bytes(const omerf_scene_desc* d) {
  if (!d->brick) return 0;
  size_t n = 8 * sizeof(int);
  for (int a = 0; a < 3; a++) n *= (size_t)((d->grid_res[a] + d->brick - 1) / d->brick);
  return n;
}

omerf_status build_brick_neighbors(omerf_scene* s, cudaStream_t stream) {
  const Geo& g = s->geo;
  const long total = (long)g.nb[0] * g.nb[1] * g.nb[2];
  if (total > 0)
    brick_neighbor_kernel<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(s->desc.brick_table, g.nb[0], g.nb[1],
                                                                              g.nb[2], s->desc.n_bricks,
                                                                              3 * g.blog2 + 3, s->nbr);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "neighbour record kernel");
}

// Coarse level: the smallest power-of-two block of occupancy cells whose side
// is at least one 32-sample lattice window, so a window meets at most a few
// coarse cells.
void choose_coarse_level(omerf_scene* s) {
  const omerf_scene_desc& d = s->desc;
  const float cw = std::min((d.aabb[1] - d.aabb[0]) / d.occ_res, (d.aabb[3] - d.aabb[2]) / d.occ_res);
  int l = 0;
  while (l < 20 && cw * (float)(1 << l) < 32.0f * d.step && (1 << l) < d.occ_res) l++;
  s->clog2 = l;
  s->Mc = (d.occ_res + (1 << l) - 1) >> l;
}

// Device bytes of a scene handle's own state, in the order omerf_scene_create
// allocates it: hull state, work counters, coarse occupancy grid, camera
// records, brick neighbour records, the checking build's counters.
static void scene_alloc_bytes(const omerf_scene_desc* d, int Mc, size_t out[6]) {
  out[0] = 64 * sizeof(float);
  out[1] = kCounterSlots * sizeof(unsigned);
  out[2] = (size_t)Mc * Mc * sizeof(float2);
  out[3] = kMaxCams * sizeof(CamRec);
  out[4] = d->brick ? brick_records_bytes(d) : 0;
  out[5] = OMERF_CHECK ? 2 * sizeof(unsigned long long) : 0;
}

omerf_status validate_camera(const omerf_camera* c, int64_t n) {
  if (c->width < 1 || c->height < 1 || (int64_t)c->width * c->height != n) {
    set_error("camera size %d x %d does not match n = %lld", c->width, c->height, (long long)n);
    return OMERF_ESHAPE;
  }
  if (c->width > (1 << 20) || c->height > (1 << 20)) { set_error("camera too large"); return OMERF_ESHAPE; }
  if (!(c->fx != 0.0f) || !(c->fy != 0.0f)) { set_error("camera focal lengths must be non-zero"); return OMERF_EINVAL; }
  bool finite = std::isfinite(c->fx) && std::isfinite(c->fy) && std::isfinite(c->cx) && std::isfinite(c->cy);
  for (int i = 0; i < 12; i++) finite = finite && std::isfinite(c->c2w[i]);
  if (!finite) { set_error("camera pose and intrinsics must be finite"); return OMERF_EINVAL; }
  // a pixel's direction R (u, v, -1) is zero-length only if R is singular
  const float* m = c->c2w;
  const double det = (double)m[0] * ((double)m[5] * m[10] - (double)m[6] * m[9]) -
                     (double)m[1] * ((double)m[4] * m[10] - (double)m[6] * m[8]) +
                     (double)m[2] * ((double)m[4] * m[9] - (double)m[5] * m[8]);
  if (!(std::fabs(det) > 1e-12)) { set_error("camera rotation is singular: rays would have no direction"); return OMERF_EINVAL; }
  return OMERF_OK;
}

Cam to_cam(const omerf_camera* c) {
  Cam k;
  std::memcpy(k.c2w, c->c2w, sizeof(k.c2w));
  k.fx = c->fx;
  k.fy = c->fy;
  k.cx = c->cx;
  k.cy = c->cy;
  k.width = c->width;
  k.height = c->height;
  return k;
}

// An output buffer of the render: device memory, or page-locked host memory
// the device addresses directly (the pointer the device uses is returned).
omerf_status output_ptr(void* p, void** dev, const char* name) {
  *dev = p;
  if (!p) return OMERF_OK;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    set_error("%s: not a CUDA-accessible pointer", name);
    return OMERF_EDEVICE;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return OMERF_OK;
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    *dev = at.devicePointer;
    return OMERF_OK;
  }
  set_error("%s must be device memory or page-locked host memory", name);
  return OMERF_EDEVICE;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

omerf_status omerf_scene_create(const omerf_scene_desc* desc, void* stream, omerf_scene** out) {
  OMERF_API_RANGE();
  if (!out) { set_error("out is NULL"); return OMERF_EINVAL; }
  *out = nullptr;
  omerf_status st = validate_desc(desc);
  if (st != OMERF_OK) return st;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { cudaGetLastError(); set_error("no CUDA device: %s", cudaGetErrorString(e)); return OMERF_EDEVICE; }
  const void* ptrs[] = {desc->grid, desc->brick_table, desc->plane_xy, desc->plane_xz, desc->plane_yz, desc->occ, desc->mlp};
  const char* names[] = {"grid", "brick_table", "plane_xy", "plane_xz", "plane_yz", "occ", "mlp"};
  for (int i = 0; i < 7; i++)
    if ((st = check_device_ptr(ptrs[i], names[i])) != OMERF_OK) return st;
  omerf_scene* s = new (std::nothrow) omerf_scene;
  if (!s) { set_error("out of host memory"); return OMERF_ENOMEM; }
  s->desc = *desc;
  s->device = dev;
  cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (s->num_sms < 1) s->num_sms = 1;
  // OMERF_FAULT=alloc: the handle's first allocation fails (tests of the path)
  choose_coarse_level(s);
  size_t bytes[6];
  scene_alloc_bytes(desc, s->Mc, bytes);
  e = fault_injected("alloc") ? cudaErrorMemoryAllocation : cudaMalloc(&s->state, bytes[0]);
  if (e != cudaSuccess) { cudaGetLastError(); delete s; set_error("cudaMalloc: %s", cudaGetErrorString(e)); return OMERF_ENOMEM; }
  e = cudaMalloc(&s->counters, bytes[1]);
  if (e != cudaSuccess) { cudaGetLastError(); cudaFree(s->state); delete s; set_error("cudaMalloc: %s", cudaGetErrorString(e)); return OMERF_ENOMEM; }
  e = cudaMalloc(&s->chull, bytes[2]);
  if (e == cudaSuccess) e = cudaMalloc(&s->cams, bytes[3]);
  if (e == cudaSuccess && bytes[4]) e = cudaMalloc(&s->nbr, bytes[4]);
  if (e == cudaSuccess && bytes[5]) {
    e = cudaMalloc(&s->check, bytes[5]);
    if (e == cudaSuccess) e = cudaMemset(s->check, 0, bytes[5]);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    omerf_scene_destroy(s);
    set_error("cudaMalloc: %s", cudaGetErrorString(e));
    return OMERF_ENOMEM;
  }
  fill_geo(s);
  if (desc->brick) {
    // a table entry outside the pool would make the march read outside it
    const long total = (long)s->geo.nb[0] * s->geo.nb[1] * s->geo.nb[2];
    unsigned* bad = s->counters;  // counter slot 0 doubles as the check result
    cudaStream_t cs = (cudaStream_t)stream;
    unsigned nbad = 0;
    e = cudaMemsetAsync(bad, 0, sizeof(unsigned), cs);
    if (e == cudaSuccess && total > 0) {
      brick_table_check_kernel<<<(unsigned)((total + 255) / 256), 256, 0, cs>>>(desc->brick_table, total,
                                                                                desc->n_bricks, bad);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
      omerf_scene_destroy(s);
      return cuda_fail(e, "brick table check");
    }
    if (nbad) {
      omerf_scene_destroy(s);
      set_error("the brick table holds %u entries outside [-1, n_bricks = %d)", nbad, desc->n_bricks);
      return OMERF_ESHAPE;
    }
    if ((st = build_brick_neighbors(s, cs)) != OMERF_OK) {
      omerf_scene_destroy(s);
      return st;
    }
  }
  st = omerf_scene_update(s, stream);
  if (st != OMERF_OK) { omerf_scene_destroy(s); return st; }
  *out = s;
  return OMERF_OK;
}

int64_t omerf_scene_device_bytes(const omerf_scene_desc* desc) {
  const omerf_status st = validate_desc(desc);
  if (st != OMERF_OK) return st;
  omerf_scene s;
  s.desc = *desc;
  choose_coarse_level(&s);
  size_t bytes[6];
  scene_alloc_bytes(desc, s.Mc, bytes);
  size_t total = 0;
  for (size_t b : bytes) total += b;
  return (int64_t)total;
}

omerf_status omerf_scene_update(omerf_scene* s, void* stream) {
  OMERF_API_RANGE();
  if (!s) { set_error("scene is NULL"); return OMERF_EINVAL; }
  const long cells = (long)s->desc.occ_res * s->desc.occ_res;
  OMERF_LAUNCH_FAULT();
  hull_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(s->geo.occ, cells, s->state);
  const int nc = s->Mc * s->Mc;
  coarse_hull_kernel<<<(nc + 255) / 256, 256, 0, (cudaStream_t)stream>>>(s->geo.occ, s->desc.occ_res, s->clog2,
                                                                         s->Mc, s->chull);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "hull kernel");
}

void omerf_scene_destroy(omerf_scene* s) {
  OMERF_API_RANGE();
  if (!s) return;
  if (s->check) {
    // the checking build keeps the counts of destroyed scenes (omerf_check_totals)
    unsigned long long h[2] = {0, 0};
    if (cudaMemcpy(h, s->check, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess) {
      g_check_total[0].fetch_add(h[0]);
      g_check_total[1].fetch_add(h[1]);
    } else {
      cudaGetLastError();
    }
  }
  cudaFree(s->state);
  cudaFree(s->counters);
  cudaFree(s->chull);
  cudaFree(s->nbr);
  cudaFree(s->cams);
  cudaFree(s->check);
  delete s;
}

// Shared by omerf_build_brick_table and omerf_grow_brick_table.
static omerf_status brick_table_impl(const float aabb[6], const int32_t grid_res[3], int32_t brick, const float* occ,
                                     int32_t occ_res, const int32_t* old_table, int32_t* table, int32_t* n_alloc,
                                     int32_t* missing, void* stream, const char* entry) {
  if (!aabb || !grid_res || !occ || !table || !n_alloc) { set_error("NULL argument"); return OMERF_EINVAL; }
  if (brick < 2 || brick > 32 || (brick & (brick - 1))) { set_error("brick must be a power of two in 2..32"); return OMERF_EINVAL; }
  if (occ_res < 1) { set_error("occ_res must be >= 1"); return OMERF_ESHAPE; }
  for (int a = 0; a < 3; a++) {
    if (grid_res[a] < 2) { set_error("grid_res must be >= 2"); return OMERF_ESHAPE; }
    if (!(aabb[2 * a] < aabb[2 * a + 1])) { set_error("aabb axis %d is empty", a); return OMERF_EINVAL; }
  }
  if (!aligned(occ, 8)) { set_error("occ must be 8-byte aligned"); return OMERF_EINVAL; }
  BrickArgs a;
  a.z0 = aabb[4];
  a.vz = (aabb[5] - aabb[4]) / (float)(grid_res[2] - 1);
  a.B = brick;
  a.M = occ_res;
  for (int i = 0; i < 3; i++) {
    a.L[i] = grid_res[i];
    a.nb[i] = (grid_res[i] + brick - 1) / brick;
  }
  a.occ = reinterpret_cast<const float2*>(occ);
  a.table = table;
  a.old_table = old_table;
  a.missing = missing;
  const long total = (long)a.nb[0] * a.nb[1] * a.nb[2];
  if (total > (1l << 31)) { set_error("too many bricks"); return OMERF_ESHAPE; }
  cudaStream_t s = (cudaStream_t)stream;
  if (fault_injected("launch")) return injected_launch_failure(entry);
  omerf_status st = check_device_ptrs({{occ, "occ"}, {table, "table"}, {n_alloc, "n_alloc"},
                                       {old_table, "old_table"}, {missing, "missing"}});
  if (st != OMERF_OK) return st;
  if (missing) {
    cudaError_t e = cudaMemsetAsync(missing, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "brick table memset");
  }
  brick_flag_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(a, total);
  brick_scan_kernel<<<1, 1024, 0, s>>>(table, total, n_alloc);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "brick table kernels");
}

omerf_status omerf_build_brick_table(const float aabb[6], const int32_t grid_res[3], int32_t brick, const float* occ,
                                     int32_t occ_res, int32_t* table, int32_t* n_alloc, void* stream) {
  OMERF_API_RANGE();
  return brick_table_impl(aabb, grid_res, brick, occ, occ_res, nullptr, table, n_alloc, nullptr, stream, __func__);
}

omerf_status omerf_grow_brick_table(const float aabb[6], const int32_t grid_res[3], int32_t brick, const float* occ,
                                    int32_t occ_res, const int32_t* old_table, int32_t* table, int32_t* n_alloc,
                                    int32_t* missing, void* stream) {
  OMERF_API_RANGE();
  if (!old_table || !missing) { set_error("NULL argument"); return OMERF_EINVAL; }
  if (old_table == table) { set_error("table must not be old_table"); return OMERF_EINVAL; }
  return brick_table_impl(aabb, grid_res, brick, occ, occ_res, old_table, table, n_alloc, missing, stream, __func__);
}

omerf_status omerf_ray_interval(const omerf_scene* s, const omerf_camera* cam, const float* rays, int64_t n,
                                int32_t* k_range, void* stream) {
  OMERF_API_RANGE();
  if (!s || (!k_range && n > 0)) { set_error("NULL argument"); return OMERF_EINVAL; }
  if (n < 0) { set_error("n must be >= 0"); return OMERF_ESHAPE; }
  omerf_status st;
  Cam k{};
  if (cam) {
    if ((st = validate_camera(cam, n)) != OMERF_OK) return st;
    k = to_cam(cam);
  } else if (!rays && n > 0) {
    set_error("rays is NULL and no camera given");
    return OMERF_EINVAL;
  }
  if (n == 0) return OMERF_OK;
  OMERF_LAUNCH_FAULT();
  if ((st = check_device_ptrs({{cam ? nullptr : rays, "rays"}, {k_range, "k_range"}})) != OMERF_OK) return st;
  interval_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(s->geo, k, cam ? 1 : 0, rays, n,
                                                                                  reinterpret_cast<int2*>(k_range));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "interval kernel");
}

omerf_status omerf_render(const omerf_scene* s, const omerf_camera* cam, const float* rays, int64_t n, float* rgb,
                          int32_t* count, void* stream) {
  OMERF_API_RANGE();
  if (!s || (!rgb && n > 0)) { set_error("NULL argument"); return OMERF_EINVAL; }
  if (n < 0) { set_error("n must be >= 0"); return OMERF_ESHAPE; }
  omerf_status st;
  Cam k{};
  if (cam) {
    if ((st = validate_camera(cam, n)) != OMERF_OK) return st;
    k = to_cam(cam);
  } else if (!rays && n > 0) {
    set_error("rays is NULL and no camera given");
    return OMERF_EINVAL;
  }
  if (n > 0) {
    void *rd = nullptr, *cd = nullptr;
    if ((st = output_ptr(rgb, &rd, "rgb")) != OMERF_OK) return st;
    if ((st = output_ptr(count, &cd, "count")) != OMERF_OK) return st;
    rgb = static_cast<float*>(rd);
    count = static_cast<int32_t*>(cd);
  }
  if (n == 0) return OMERF_OK;
  OMERF_LAUNCH_FAULT();
  if ((st = check_device_ptr(cam ? nullptr : rays, "rays")) != OMERF_OK) return st;
  cudaError_t e = launch_march_fwd(s, cam ? &k : nullptr, rays, n, rgb, count, nullptr, nullptr, 0, nullptr,
                                   nullptr, nullptr, (cudaStream_t)stream);
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "render launch");
}

omerf_status omerf_render_cameras(const omerf_scene* s, const omerf_camera* cams, int32_t n_cams, float* rgb,
                                  int32_t* count, void* stream) {
  OMERF_API_RANGE();
  if (!s || (!cams && n_cams > 0)) { set_error("NULL argument"); return OMERF_EINVAL; }
  if (n_cams < 0) { set_error("n_cams must be >= 0"); return OMERF_ESHAPE; }
  if (n_cams == 0) return OMERF_OK;
  if (!rgb) { set_error("rgb is NULL"); return OMERF_EINVAL; }
  omerf_status st;
  for (int c = 0; c < n_cams; c++)
    if ((st = validate_camera(&cams[c], (int64_t)cams[c].width * cams[c].height)) != OMERF_OK) return st;
  void *rd = nullptr, *cd = nullptr;
  if ((st = output_ptr(rgb, &rd, "rgb")) != OMERF_OK) return st;
  if ((st = output_ptr(count, &cd, "count")) != OMERF_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  long ray0 = 0;
  for (int c0 = 0; c0 < n_cams; c0 += kMaxCams) {
    const int m = std::min(kMaxCams, n_cams - c0);
    CamRec rec[kMaxCams];
    long supers = 0, rays = 0;
    for (int c = 0; c < m; c++) {
      const omerf_camera& k = cams[c0 + c];
      rec[c].cam = to_cam(&k);
      rec[c].super_x = (k.width + 15) / 16;
      rec[c].super_start = supers;
      rec[c].ray_start = rays;
      rec[c].pad = 0;
      supers += (long)rec[c].super_x * ((k.height + 15) / 16);
      rays += (long)k.width * k.height;
    }
    OMERF_LAUNCH_FAULT();
    // pageable source: the copy is staged before the call returns
    cudaError_t e = cudaMemcpyAsync(s->cams, rec, m * sizeof(CamRec), cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "camera upload");
    e = launch_march_fwd_cams(s, s->cams, m, supers, rays, static_cast<float*>(rd) + 3 * ray0,
                              cd ? static_cast<int32_t*>(cd) + ray0 : nullptr, cs);
    if (e != cudaSuccess) return cuda_fail(e, "render launch");
    ray0 += rays;
  }
  return OMERF_OK;
}

int64_t omerf_saved_bytes_per_ray(void) { return (int64_t)kSavedFloats * sizeof(float); }

static omerf_status check_train_args(const omerf_scene* s, const float* rays, const float* target,
                                     const float* dirs, int64_t n, int32_t K, const float lambda[3],
                                     const void* saved) {
  if (!s || !lambda) { set_error("NULL argument"); return OMERF_EINVAL; }
  if (n < 0) { set_error("n must be >= 0"); return OMERF_ESHAPE; }
  if (K < 0 || K > 16) { set_error("K must be in 0..16"); return OMERF_EINVAL; }
  if (n > 0 && (!rays || !target || !saved || (K > 0 && !dirs))) { set_error("NULL array argument"); return OMERF_EINVAL; }
  if (saved && !aligned(saved, 16)) { set_error("saved must be 16-byte aligned"); return OMERF_EINVAL; }
  for (int i = 0; i < 3; i++)
    if (!std::isfinite(lambda[i])) { set_error("lambda must be finite"); return OMERF_EINVAL; }
  return OMERF_OK;
}

// The arrays of a training call, checked to be device memory.
static omerf_status check_train_ptrs(const float* rays, const float* target, const float* dirs, const void* saved,
                                     const float* loss, const float* grad_scale, std::initializer_list<const float*> g) {
  omerf_status st = check_device_ptrs({{rays, "rays"}, {target, "target"}, {dirs, "smooth_dirs"}, {saved, "saved"},
                                       {loss, "loss"}, {grad_scale, "grad_scale"}});
  if (st != OMERF_OK) return st;
  for (const float* p : g)
    if ((st = check_device_ptr(p, "gradient buffer")) != OMERF_OK) return st;
  return OMERF_OK;
}

omerf_status omerf_train_fwd(const omerf_scene* s, const float* rays, const float* target, const float* smooth_dirs,
                             int64_t n, int32_t K, const float lambda[3], void* saved, float* loss, void* stream) {
  OMERF_API_RANGE();
  omerf_status st = check_train_args(s, rays, target, smooth_dirs, n, K, lambda, saved);
  if (st != OMERF_OK) return st;
  if (!loss) { set_error("loss is NULL"); return OMERF_EINVAL; }
  OMERF_LAUNCH_FAULT();
  if ((st = check_train_ptrs(rays, target, smooth_dirs, saved, loss, nullptr, {})) != OMERF_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(loss, 0, 4 * sizeof(float), cs);
  if (e != cudaSuccess) return cuda_fail(e, "loss memset");
  if (n > 0) {
    e = launch_march_fwd(s, nullptr, rays, n, nullptr, nullptr, target, smooth_dirs, K, lambda,
                         static_cast<float*>(saved), loss, cs);
    if (e != cudaSuccess) return cuda_fail(e, "train forward launch");
  }
  const long cells = (long)s->desc.occ_res * s->desc.occ_res;
  occ_loss_kernel<<<(unsigned)std::min<long>((cells + 255) / 256, 1024), 256, 0, cs>>>(s->geo.occ, cells, lambda[2],
                                                                                       nullptr, loss, nullptr);
  e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "occupancy loss launch");
}

omerf_status omerf_train_bwd(const omerf_scene* s, const float* rays, const float* target, const float* smooth_dirs,
                             int64_t n, int32_t K, const float lambda[3], void* saved, const float* grad_scale,
                             float* g_grid, float* g_xy, float* g_xz, float* g_yz, float* g_occ, float* g_mlp,
                             void* stream) {
  OMERF_API_RANGE();
  omerf_status st = check_train_args(s, rays, target, smooth_dirs, n, K, lambda, saved);
  if (st != OMERF_OK) return st;
  const void* gps[] = {g_grid, g_xy, g_xz, g_yz};
  for (const void* p : gps)
    if (p && !aligned(p, 16)) { set_error("gradient buffers must be 16-byte aligned"); return OMERF_EINVAL; }
  if (g_occ && !aligned(g_occ, 8)) { set_error("g_occ must be 8-byte aligned"); return OMERF_EINVAL; }
  OMERF_LAUNCH_FAULT();
  if ((st = check_train_ptrs(rays, target, smooth_dirs, saved, nullptr, grad_scale,
                             {g_grid, g_xy, g_xz, g_yz, g_occ, g_mlp})) != OMERF_OK)
    return st;
  cudaStream_t cs = (cudaStream_t)stream;
  cudaError_t e;
  if (n > 0) {
    e = launch_march_bwd(s, rays, target, smooth_dirs, n, K, lambda, static_cast<float*>(saved), grad_scale,
                         g_grid, g_xy, g_xz, g_yz, g_occ, g_mlp, nullptr, cs);
    if (e != cudaSuccess) return cuda_fail(e, "train backward launch");
  }
  if (g_occ) {
    const long cells = (long)s->desc.occ_res * s->desc.occ_res;
    occ_loss_kernel<<<(unsigned)std::min<long>((cells + 255) / 256, 1024), 256, 0, cs>>>(
        s->geo.occ, cells, lambda[2], grad_scale, nullptr, reinterpret_cast<float2*>(g_occ));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "occupancy gradient launch");
  }
  return OMERF_OK;
}

omerf_status omerf_train_step(const omerf_scene* s, const float* rays, const float* target, const float* smooth_dirs,
                              int64_t n, int32_t K, const float lambda[3], void* saved, float* loss, float* g_grid,
                              float* g_xy, float* g_xz, float* g_yz, float* g_occ, float* g_mlp, void* stream) {
  OMERF_API_RANGE();
  // The forward only marches and saves the per-ray state; the MLP backward,
  // which evaluates the deferred MLP anyway, adds the Charbonnier and
  // smoothness terms to the loss, and one L_occ launch adds its loss and
  // gradient.
  omerf_status st = check_train_args(s, rays, target, smooth_dirs, n, K, lambda, saved);
  if (st != OMERF_OK) return st;
  if (!loss) { set_error("loss is NULL"); return OMERF_EINVAL; }
  const void* gps[] = {g_grid, g_xy, g_xz, g_yz};
  for (const void* p : gps)
    if (p && !aligned(p, 16)) { set_error("gradient buffers must be 16-byte aligned"); return OMERF_EINVAL; }
  if (g_occ && !aligned(g_occ, 8)) { set_error("g_occ must be 8-byte aligned"); return OMERF_EINVAL; }
  OMERF_LAUNCH_FAULT();
  if ((st = check_train_ptrs(rays, target, smooth_dirs, saved, loss, nullptr,
                             {g_grid, g_xy, g_xz, g_yz, g_occ, g_mlp})) != OMERF_OK)
    return st;
  cudaStream_t cs = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(loss, 0, 4 * sizeof(float), cs);
  if (e != cudaSuccess) return cuda_fail(e, "loss memset");
  if (n > 0) {
    e = launch_march_fwd(s, nullptr, rays, n, nullptr, nullptr, target, smooth_dirs, K, lambda,
                         static_cast<float*>(saved), nullptr, cs);
    if (e != cudaSuccess) return cuda_fail(e, "train forward launch");
    e = launch_march_bwd(s, rays, target, smooth_dirs, n, K, lambda, static_cast<float*>(saved), nullptr, g_grid,
                         g_xy, g_xz, g_yz, g_occ, g_mlp, loss, cs);
    if (e != cudaSuccess) return cuda_fail(e, "train backward launch");
  }
  const long cells = (long)s->desc.occ_res * s->desc.occ_res;
  occ_loss_kernel<<<(unsigned)std::min<long>((cells + 255) / 256, 1024), 256, 0, cs>>>(
      s->geo.occ, cells, lambda[2], nullptr, loss, reinterpret_cast<float2*>(g_occ));
  e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "occupancy loss launch");
}

omerf_status omerf_sync(void* stream, int32_t timeout_ms) {
  OMERF_API_RANGE();
  cudaStream_t cs = (cudaStream_t)stream;
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(cs);
    if (e == cudaSuccess) return take_device_error();
    if (e != cudaErrorNotReady) return cuda_fail(e, "stream");
    if (timeout_ms >= 0) {
      auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
      if (ms >= timeout_ms) {
        set_error("stream still busy after %d ms", timeout_ms);
        return OMERF_ETIMEOUT;
      }
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int32_t omerf_check_build(void) { return OMERF_CHECK ? 1 : 0; }

void omerf_check_totals(uint64_t totals[2]) {
  if (!totals) return;
  totals[0] = g_check_total[0].load();
  totals[1] = g_check_total[1].load();
}

omerf_status omerf_check_counts(const omerf_scene* s, uint64_t counts[2], int32_t reset, void* stream) {
  OMERF_API_RANGE();
  if (!s || !counts) { set_error("NULL argument"); return OMERF_EINVAL; }
  counts[0] = counts[1] = 0;
  if (!s->check) { set_error("the library was built without OMERF_CHECK: nothing is counted"); return OMERF_EINVAL; }
  cudaStream_t cs = (cudaStream_t)stream;
  unsigned long long h[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(h, s->check, sizeof(h), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(s->check, 0, sizeof(h), cs);
  if (e != cudaSuccess) return cuda_fail(e, "check counters");
  counts[0] = h[0];
  counts[1] = h[1];
  if (h[1]) {
    set_error("%llu feature reads fell outside the arrays (skipped by the checking build)", h[1]);
    return OMERF_ECHECK;
  }
  return OMERF_OK;
}

const char* omerf_last_error(void) { return g_err; }

}  // extern "C"
