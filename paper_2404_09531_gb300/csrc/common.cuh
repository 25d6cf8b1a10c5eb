// common.cuh -- device building blocks of the Oblique-MERF march (sm_103a).
//
// Oblique-MERF (arXiv 2404.09531):
//   feature field   t(p) = V(p) + P_xy + P_xz + P_yz          Sec. 3, Eq. 2
//   activations     tau = exp, c^d / f = sigmoid               Eq. 3
//   occupancy       M(z), q = 2 power ramps, nearest cell       Sec. 4.1, Eqs. 6-7
//   compositing     w_i = T_i M_i alpha_i                       Eqs. 1, 8
//   deferred MLP    G(F, d), 34 -> 16 -> 16 -> 3                Eq. 4, appendix A
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#ifndef OMERF_CHECK
#define OMERF_CHECK 0  // 1 in the checking build (libomerf_check.so): bounds and brick counters
#endif

namespace omerf {

constexpr int kNch = 8;
constexpr int kMlpParams = 883;
constexpr int kOffW1 = 0, kOffB1 = 544, kOffW2 = 560, kOffB2 = 816, kOffW3 = 832, kOffB3 = 880;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxLattice = (1 << 24) - 1;  // t_k = k * step is exact below 2^24
// per-ray training state: F[7], T_N, count, k_lo, k_hi, pad | dL/dF[7], dL/dT_N  (80 B)
constexpr int kSavedFloats = 20;

// Kernel-uniform scene description (passed by value, lives in the constant bank).
struct Geo {
  float lo[3], hi[3];      // box
  float gs[3];             // grid: (L - 1) / (hi - lo)
  float ps[3];             // planes: (R - 1) / (plane extent)
  int L[3], R[3];
  float osx, osy;          // occupancy cells: M / (hi - lo), float32 as in the decision rule
  int M;
  float step, inv_eps, t_thr;
  float bg[3];
  int n_max;
  int blog2;               // log2 of the brick edge (brick grids)
  int nb[3];               // brick grid dimensions
  const void* grid;
  const int* table;
  const void* pxy;
  const void* pxz;
  const void* pyz;
  const float2* occ;
  const float* mlp;
  const float* hull;       // device [2]: min z_min, max z_max over non-empty cells
  const int* nbr;          // device [nbx * nby * nbz][8]: pool element offset of the (+dx, +dy, +dz) neighbours
  const float2* chull;     // device [Mc][Mc]: coarse max-pooled (min z_min, max z_max)
  int clog2;               // coarse cell = 2^clog2 x 2^clog2 occupancy cells
  int Mc;                  // coarse cells per axis
  // planes: texel offset of a z-range cropped to the occupancy bounds,
  // (z0' - z0) ps[2] (last, so that the fields above keep their offsets)
  float pzoff;
  // elements of the grid (or pool) and of the XY, XZ, YZ planes, and the
  // checking build's counters [2] (unallocated corner reads, reads outside
  // an array); the default build reads neither
  long long lim[4];
  unsigned long long* check;
};

struct Cam {
  float c2w[12];
  float fx, fy, cx, cy;
  int width, height;
};

// One camera of a multi-camera render: its first super-tile and first ray
// in the launch's numbering, and its super-tiles per row.
struct CamRec {
  Cam cam;
  long long super_start, ray_start;
  int super_x, pad;
};
constexpr int kMaxCams = 16;  // cameras per multi-camera launch

// ---------------------------------------------------------------------------
// rays
// ---------------------------------------------------------------------------

// Pinhole ray of pixel (px, py): float32, left to right, no fused operations.
__device__ __forceinline__ void camera_ray(const Cam& c, int px, int py, float o[3], float d[3]) {
  float ux = __fdiv_rn(__fsub_rn(__fadd_rn((float)px, 0.5f), c.cx), c.fx);
  float uy = -__fdiv_rn(__fsub_rn(__fadd_rn((float)py, 0.5f), c.cy), c.fy);
  float uz = -1.0f;
  float dc[3];
#pragma unroll
  for (int a = 0; a < 3; a++)
    dc[a] = __fadd_rn(__fadd_rn(__fmul_rn(c.c2w[4 * a + 0], ux), __fmul_rn(c.c2w[4 * a + 1], uy)),
                      __fmul_rn(c.c2w[4 * a + 2], uz));
  float nn = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(dc[0], dc[0]), __fmul_rn(dc[1], dc[1])),
                                  __fmul_rn(dc[2], dc[2])));
#pragma unroll
  for (int a = 0; a < 3; a++) {
    d[a] = __fdiv_rn(dc[a], nn);
    o[a] = c.c2w[4 * a + 3];
  }
}

// Conservative lattice range [klo, khi] of a ray: the box, with z narrowed to
// the occupancy hull, each axis padded by more than the float32 error of the
// sample positions, plus two lattice steps.  Returns false when empty.
__device__ __forceinline__ bool lattice_range(const Geo& g, const float o[3], const float d[3], int& klo,
                                              int& khi) {
  // a ray with a non-finite component evaluates no sample (every position
  // test fails): skip its lattice scan
  if (!(isfinite(o[0]) && isfinite(o[1]) && isfinite(o[2]) && isfinite(d[0]) && isfinite(d[1]) && isfinite(d[2])))
    return false;
  float tin = 0.0f, tout = __int_as_float(0x7f800000);
#pragma unroll
  for (int a = 0; a < 3; a++) {
    float lo = g.lo[a], hi = g.hi[a];
    if (a == 2) {
      lo = fmaxf(lo, g.hull[0]);
      hi = fminf(hi, g.hull[1]);
      if (!(lo <= hi)) return false;
    }
    if (d[a] == 0.0f) {
      if (o[a] < lo || o[a] > hi) return false;
      continue;
    }
    float inv = 1.0f / d[a];
    float ta = (lo - o[a]) * inv, tb = (hi - o[a]) * inv;
    if (ta > tb) { float s = ta; ta = tb; tb = s; }
    float pad = 1e-6f * (fmaxf(fabsf(ta), fabsf(tb)) + (fabsf(o[a]) + 1.0f) * fabsf(inv));
    tin = fmaxf(tin, ta - pad);
    tout = fminf(tout, tb + pad);
  }
  if (!(tin <= tout)) return false;
  float kl = floorf(tin / g.step) - 2.0f;
  float kh = ceilf(tout / g.step) + 2.0f;
  kl = fmaxf(kl, 0.0f);
  kh = fminf(kh, (float)kMaxLattice);
  if (kl > kh) return false;
  klo = (int)kl;
  khi = (int)kh;
  return true;
}

// The sample decision for lattice index k (float32, no fused operations):
// inside the closed box and strictly inside the nearest cell's interval.
__device__ __forceinline__ bool lattice_test(const Geo& g, const float o[3], const float d[3], int k,
                                             float p[3], float2& zb, int& cell) {
  float t = __fmul_rn((float)k, g.step);
#pragma unroll
  for (int a = 0; a < 3; a++) p[a] = __fadd_rn(o[a], __fmul_rn(t, d[a]));
  if (!(p[0] >= g.lo[0] && p[0] <= g.hi[0] && p[1] >= g.lo[1] && p[1] <= g.hi[1] && p[2] >= g.lo[2] &&
        p[2] <= g.hi[2]))
    return false;
  int cx = (int)floorf(__fmul_rn(__fsub_rn(p[0], g.lo[0]), g.osx));
  int cy = (int)floorf(__fmul_rn(__fsub_rn(p[1], g.lo[1]), g.osy));
  cx = min(max(cx, 0), g.M - 1);
  cy = min(max(cy, 0), g.M - 1);
  cell = cx * g.M + cy;
  zb = __ldg(g.occ + cell);
  return zb.x < p[2] && p[2] < zb.y;
}

// Empty-space skipping (Sec. 4.4: max-pooled occupancy planes and box tests).
// Lane j reports whether lattice window [kb + 32 j, kb + 32 j + 31] (clipped
// to kh) may hold an evaluated sample: the window's sample positions lie in
// the bounding box of its two end points (padded far beyond float32
// rounding); the decision rule's cell index is monotone in x and y, so the
// cells of those samples lie in the cell range of the padded box, and a
// sample can pass only if its z meets the max-pooled interval of a coarse
// cell in that range.  Windows outside the box or missing every interval
// are culled; the survivors are still tested sample by sample.
__device__ __forceinline__ unsigned window_mask(const Geo& g, const float o[3], const float d[3], int kb, int kh,
                                                int lane) {
  const int ka = kb + 32 * lane;
  bool maybe = false;
  if (ka <= kh) {
    const int kz = min(ka + 31, kh);
    const float ta = __fmul_rn((float)ka, g.step), tb = __fmul_rn((float)kz, g.step);
    float lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const float pa = __fadd_rn(o[a], __fmul_rn(ta, d[a])), pb = __fadd_rn(o[a], __fmul_rn(tb, d[a]));
      const float pad = 1e-5f * (1.0f + fmaxf(fabsf(pa), fabsf(pb)));
      lo[a] = fminf(pa, pb) - pad;
      hi[a] = fmaxf(pa, pb) + pad;
    }
    const bool in_box = hi[0] >= g.lo[0] && lo[0] <= g.hi[0] && hi[1] >= g.lo[1] && lo[1] <= g.hi[1] &&
                        hi[2] >= g.lo[2] && lo[2] <= g.hi[2];
    if (in_box) {
      const int cx0 = min(max((int)floorf(__fmul_rn(__fsub_rn(fmaxf(lo[0], g.lo[0]), g.lo[0]), g.osx)), 0), g.M - 1);
      const int cx1 = min(max((int)floorf(__fmul_rn(__fsub_rn(fminf(hi[0], g.hi[0]), g.lo[0]), g.osx)), 0), g.M - 1);
      const int cy0 = min(max((int)floorf(__fmul_rn(__fsub_rn(fmaxf(lo[1], g.lo[1]), g.lo[1]), g.osy)), 0), g.M - 1);
      const int cy1 = min(max((int)floorf(__fmul_rn(__fsub_rn(fminf(hi[1], g.hi[1]), g.lo[1]), g.osy)), 0), g.M - 1);
      const int X0 = cx0 >> g.clog2, X1 = cx1 >> g.clog2, Y0 = cy0 >> g.clog2, Y1 = cy1 >> g.clog2;
      if (X1 - X0 <= 1 && Y1 - Y0 <= 1) {
        // the common case: at most 2 x 2 coarse cells, read independently
        const float2 h00 = __ldg(g.chull + X0 * g.Mc + Y0), h01 = __ldg(g.chull + X0 * g.Mc + Y1);
        const float2 h10 = __ldg(g.chull + X1 * g.Mc + Y0), h11 = __ldg(g.chull + X1 * g.Mc + Y1);
        const float zl = fminf(fminf(h00.x, h01.x), fminf(h10.x, h11.x));
        const float zh = fmaxf(fmaxf(h00.y, h01.y), fmaxf(h10.y, h11.y));
        maybe = zl <= hi[2] && zh >= lo[2];
      } else if ((X1 - X0 + 1) * (Y1 - Y0 + 1) > 16) {
        maybe = true;  // unusually long window in cell units: keep it
      } else {
        for (int X = X0; X <= X1 && !maybe; X++)
          for (int Y = Y0; Y <= Y1 && !maybe; Y++) {
            const float2 h = __ldg(g.chull + X * g.Mc + Y);
            maybe = h.x <= hi[2] && h.y >= lo[2];
          }
      }
    }
  }
  return __ballot_sync(kFull, maybe);
}

// Eq. 6 with q = 2; overlapping ramps take the smaller value.  branch: 0 flat,
// 1 lower ramp (r = (z - z_min)/eps), 2 upper ramp (r = (z_max - z)/eps).
__device__ __forceinline__ float occupancy(const Geo& g, float z, float2 zb, int& branch, float& r) {
  float rl = (z - zb.x) * g.inv_eps, rh = (zb.y - z) * g.inv_eps;
  float ml = rl * rl, mh = rh * rh;
  if (ml < 1.0f && ml <= mh) { branch = 1; r = rl; return ml; }
  if (mh < 1.0f) { branch = 2; r = rh; return mh; }
  branch = 0;
  r = 0.0f;
  return 1.0f;
}

// ---------------------------------------------------------------------------
// feature gather (Eq. 2): 8 grid corners + 3 x 4 plane texels, 8 channels each
// ---------------------------------------------------------------------------

__device__ __forceinline__ void axis_coord(float x, float lo, float s, int L, int& i, float& w, float off = 0.0f) {
  float u = fmaf(x - lo, s, -off);
  u = fminf(fmaxf(u, 0.0f), (float)(L - 1));
  i = min((int)u, L - 2);
  w = u - (float)i;
}

template <class FT>
struct Texel;

template <>
struct Texel<float> {
  static constexpr int kBytes = 32;
  // one 256-bit read-only load per texel (sm_100+ vector width)
  __device__ __forceinline__ static void load(const void* base, int elem, float v[8]) {
    const float* q = static_cast<const float*>(base) + elem;
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(q));
  }
};

template <>
struct Texel<__nv_bfloat16> {
  static constexpr int kBytes = 16;
  __device__ __forceinline__ static void load(const void* base, int elem, float v[8]) {
    const uint4* q = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(base) + elem);
    uint4 a = __ldg(q);
    unsigned w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int i = 0; i < 4; i++) {
      v[2 * i] = __uint_as_float(w[i] << 16);
      v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
};

// t += w v over the 8 channels of a texel, two channels per packed FP32 FMA
// (sm_100+; each half is one fused multiply-add rounded to nearest, exactly
// as fmaf).  Used where the march is issue-bound (BF16 features); with FP32
// features the scalar form keeps fewer registers live.
__device__ __forceinline__ void fma8x2(float2 t[4], float w, const float v[8]) {
  const float2 ww = make_float2(w, w);
#pragma unroll
  for (int j = 0; j < 4; j++) t[j] = __ffma2_rn(make_float2(v[2 * j], v[2 * j + 1]), ww, t[j]);
}
template <class FT>
struct Packed {
  static constexpr bool value = false;
};
template <>
struct Packed<__nv_bfloat16> {
  static constexpr bool value = true;
};

// Checking build: count the corners of a stencil whose brick is not stored
// (they read as zero); the default build does nothing.
__device__ __forceinline__ void check_unallocated(const Geo& g, const int off[8]) {
#if OMERF_CHECK
  int n = 0;
#pragma unroll
  for (int c = 0; c < 8; c++) n += off[c] < 0;
  if (n && g.check) atomicAdd(g.check, (unsigned long long)n);
#endif
}

// Checking build: whether the 8 channels at element offset off lie inside
// feature array q (0 grid or pool, 1..3 the XY, XZ, YZ planes); a read
// outside is counted and skipped.  The default build always reads.
__device__ __forceinline__ bool check_range(const Geo& g, int q, int off) {
#if OMERF_CHECK
  if (off >= 0 && (long long)off + kNch <= g.lim[q]) return true;
  if (g.check) atomicAdd(g.check + 1, 1ull);
  return false;
#else
  return true;
#endif
}

// The same test without counting (for writes at offsets already checked).
__device__ __forceinline__ bool in_range(const Geo& g, int q, int off) {
#if OMERF_CHECK
  return off >= 0 && (long long)off + kNch <= g.lim[q];
#else
  return true;
#endif
}

// Element offsets of the 8 grid corners (negative for an unallocated brick) and
// their trilinear weights, corner order (dx, dy, dz) with dz fastest.
template <bool SPARSE>
__device__ __forceinline__ void grid_stencil(const Geo& g, const float p[3], int off[8], float w[8]) {
  int i[3];
  float f[3];
#pragma unroll
  for (int a = 0; a < 3; a++) axis_coord(p[a], g.lo[a], g.gs[a], g.L[a], i[a], f[a]);
#pragma unroll
  for (int c = 0; c < 8; c++) {
    int da = (c >> 2) & 1, db = (c >> 1) & 1, dc = c & 1;
    w[c] = (da ? f[0] : 1.0f - f[0]) * (db ? f[1] : 1.0f - f[1]) * (dc ? f[2] : 1.0f - f[2]);
  }
  if (!SPARSE) {
    const int base = ((i[0] * g.L[1] + i[1]) * g.L[2] + i[2]) * kNch;
    const int sz = kNch, sy = g.L[2] * kNch, sx = g.L[1] * g.L[2] * kNch;
#pragma unroll
    for (int c = 0; c < 8; c++) off[c] = base + ((c >> 2) & 1) * sx + ((c >> 1) & 1) * sy + (c & 1) * sz;
  } else {
    // brick grid: a cell inside its brick reads all corners from the brick's
    // table entry; a cell reaching into neighbour bricks reads the record of
    // its lowest corner's brick (one 256-bit load: the pool element offset
    // of the brick of every corner, stored or not), so every corner is read
    // through its own brick without branching on which ones are stored.  A
    // corner's offset is its brick's offset plus per-axis local offsets.
    const int s = g.blog2, m = (1 << s) - 1;
    const int lin = ((i[0] >> s) * g.nb[1] + (i[1] >> s)) * g.nb[2] + (i[2] >> s);
    const int cx = (i[0] & m) == m, cy = (i[1] & m) == m, cz = (i[2] & m) == m;
    int nb[8];
    if (cx | cy | cz) {
      asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(nb[0]), "=r"(nb[1]), "=r"(nb[2]), "=r"(nb[3]), "=r"(nb[4]), "=r"(nb[5]), "=r"(nb[6]),
                     "=r"(nb[7])
                   : "l"(g.nbr + 8 * lin));
    } else {
      // a table entry of -1 (not stored) shifts to -2^(3s+3), below minus
      // any local offset, so the corner offsets through it stay negative
      const int o0 = __ldg(g.table + lin) << (3 * s + 3);
#pragma unroll
      for (int c = 0; c < 8; c++) nb[c] = o0;
    }
    const int lx[2] = {(i[0] & m) << (2 * s + 3), ((i[0] + 1) & m) << (2 * s + 3)};
    const int ly[2] = {(i[1] & m) << (s + 3), ((i[1] + 1) & m) << (s + 3)};
    const int lz[2] = {(i[2] & m) << 3, ((i[2] + 1) & m) << 3};
#pragma unroll
    for (int c = 0; c < 8; c++) {
      const int dx = (c >> 2) & 1, dy = (c >> 1) & 1, dz = c & 1;
      // neighbour slot: the axes on which this corner leaves the base brick
      const int kx = dx & cx, ky = dy & cy, kz = dz & cz;
      const int z0 = kz ? nb[1] : nb[0], z1 = kz ? nb[3] : nb[2], z2 = kz ? nb[5] : nb[4], z3 = kz ? nb[7] : nb[6];
      const int y0 = ky ? z1 : z0, y1 = ky ? z3 : z2;
      const int b = kx ? y1 : y0;
      off[c] = b + lx[dx] + ly[dy] + lz[dz];  // negative through an unstored brick
    }
    check_unallocated(g, off);
  }
}

// Element offsets and bilinear weights of the 12 plane texels: XY, XZ, YZ.
__device__ __forceinline__ void plane_stencil(const Geo& g, const float p[3], int off[12], float w[12]) {
  int i[3];
  float f[3];
#pragma unroll
  // (x - x0) is shared with the grid stencil; z counts from a cropped range
  for (int a = 0; a < 3; a++) axis_coord(p[a], g.lo[a], g.ps[a], g.R[a], i[a], f[a], a == 2 ? g.pzoff : 0.0f);
  const int U[3] = {0, 0, 1}, V[3] = {1, 2, 2};
#pragma unroll
  for (int q = 0; q < 3; q++) {
    int u = U[q], v = V[q];
    const int base = (i[u] * g.R[v] + i[v]) * kNch;
    const int su = g.R[v] * kNch;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      int da = (c >> 1) & 1, db = c & 1;
      off[4 * q + c] = base + da * su + db * kNch;
      w[4 * q + c] = (da ? f[u] : 1.0f - f[u]) * (db ? f[v] : 1.0f - f[v]);
    }
  }
}

__device__ __forceinline__ const void* plane_base(const Geo& g, int q) {
  return q == 0 ? g.pxy : (q == 1 ? g.pxz : g.pyz);
}

// The weighted sum of Eq. 2 over the 8 grid corners and 12 plane texels of
// a stencil (a corner with offset -1 reads zero).
template <class FT>
__device__ __forceinline__ void gather_texels(const Geo& g, const int goff[8], const float gw[8], const int poff[12],
                                              const float pw[12], float t[8]) {
  if constexpr (Packed<FT>::value) {
    float2 t2[4];
#pragma unroll
    for (int j = 0; j < 4; j++) t2[j] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int c = 0; c < 8; c++) {
      float v[8];
      if (goff[c] >= 0 && check_range(g, 0, goff[c])) {
        Texel<FT>::load(g.grid, goff[c], v);
        fma8x2(t2, gw[c], v);
      }
    }
#pragma unroll
    for (int q = 0; q < 3; q++) {
      const void* P = plane_base(g, q);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        float v[8];
        if (!check_range(g, 1 + q, poff[4 * q + c])) continue;
        Texel<FT>::load(P, poff[4 * q + c], v);
        fma8x2(t2, pw[4 * q + c], v);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      t[2 * j] = t2[j].x;
      t[2 * j + 1] = t2[j].y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 8; c++) t[c] = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
      float v[8];
      if (goff[c] >= 0 && check_range(g, 0, goff[c])) {
        Texel<FT>::load(g.grid, goff[c], v);
#pragma unroll
        for (int ch = 0; ch < 8; ch++) t[ch] = fmaf(gw[c], v[ch], t[ch]);
      }
    }
#pragma unroll
    for (int q = 0; q < 3; q++) {
      const void* P = plane_base(g, q);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        float v[8];
        if (!check_range(g, 1 + q, poff[4 * q + c])) continue;
        Texel<FT>::load(P, poff[4 * q + c], v);
#pragma unroll
        for (int ch = 0; ch < 8; ch++) t[ch] = fmaf(pw[4 * q + c], v[ch], t[ch]);
      }
    }
  }
}

template <class FT, bool SPARSE>
__device__ __forceinline__ void gather_features(const Geo& g, const float p[3], float t[8]) {
  int goff[8], poff[12];
  float gw[8], pw[12];
  grid_stencil<SPARSE>(g, p, goff, gw);
  plane_stencil(g, p, poff, pw);
  gather_texels<FT>(g, goff, gw, poff, pw, t);
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }
// Sigmoid of the per-sample activations from the hardware exponential and
// the hardware's approximate reciprocal (one instruction each; relative error
// ~1e-6 together).  An IEEE-rounded reciprocal here cost the issue-bound BF16
// render 6 % and the training step 3 %.
__device__ __forceinline__ float sigmoid_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + __expf(-x)));
  return r;
}

// Eq. 3 and the opacity of Eq. 1 for one evaluated sample.
struct SampleAct {
  float Mv, sigma, alpha, ah;
  float x[7];
  int branch;
  float r;
};

__device__ __forceinline__ void activate(const Geo& g, const float t[8], float z, float2 zb, SampleAct& s) {
  s.Mv = occupancy(g, z, zb, s.branch, s.r);
  const float tau = __expf(t[0]);
  s.sigma = tau * g.step;
  // 1 - exp(-sigma): series for small sigma keeps the relative accuracy of alpha
  s.alpha = s.sigma < 1e-3f ? s.sigma * (1.0f - 0.5f * s.sigma * (1.0f - s.sigma * (1.0f / 3.0f)))
                            : 1.0f - __expf(-s.sigma);
  s.ah = s.Mv * s.alpha;
#pragma unroll
  for (int c = 0; c < 7; c++) s.x[c] = sigmoid_fast(t[c + 1]);
}

// ---------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(kFull, v, s);
  return v;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__device__ __forceinline__ unsigned lanemask_le() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------------------
// deferred MLP G(F, d) in float32 (thread per ray), weights in shared memory
// ---------------------------------------------------------------------------
struct MlpCache {
  float x[34];
  float a1[16], a2[16];
  float y[3];
};

__device__ __forceinline__ void view_encoding(const float d[3], float* x) {
  x[0] = d[0];
  x[1] = d[1];
  x[2] = d[2];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    float f = (float)(1 << k);
#pragma unroll
    for (int a = 0; a < 3; a++) {
      float s, c;
      sincosf(f * d[a], &s, &c);
      x[3 + 6 * k + a] = s;
      x[3 + 6 * k + 3 + a] = c;
    }
  }
}

// Shared-memory copy of the MLP with 16-byte aligned rows (W1 rows padded to
// 36) so that every layer is read with 128-bit broadcast loads.
constexpr int kSW1 = 0, kSB1 = 576, kSW2 = 592, kSB2 = 848, kSW3 = 864, kSB3 = 912, kSmemMlp = 916;

__device__ __forceinline__ void load_mlp_padded(const float* __restrict__ gw, float* __restrict__ sw) {
  for (int i = threadIdx.x; i < kSmemMlp; i += blockDim.x) {
    float v = 0.0f;
    if (i < kSB1) {
      const int j = i / 36, c = i % 36;
      v = c < 34 ? gw[kOffW1 + j * 34 + c] : 0.0f;
    } else if (i < kSW2) {
      v = gw[kOffB1 + i - kSB1];
    } else if (i < kSB2) {
      v = gw[kOffW2 + i - kSW2];
    } else if (i < kSW3) {
      v = gw[kOffB2 + i - kSB2];
    } else if (i < kSB3) {
      v = gw[kOffW3 + i - kSW3];
    } else if (i < kSB3 + 3) {
      v = gw[kOffB3 + i - kSB3];
    }
    sw[i] = v;
  }
}

__device__ __forceinline__ float dot4(float4 w, float a, float b, float c, float d, float acc) {
  return fmaf(w.w, d, fmaf(w.z, c, fmaf(w.y, b, fmaf(w.x, a, acc))));
}

// G(F, d) -> y with the padded shared-memory weights (thread per ray).
__device__ __forceinline__ void mlp_forward_padded(const float* __restrict__ W, const float F[7], const float d[3],
                                                   float y[3]) {
  float x[36];
#pragma unroll
  for (int i = 0; i < 7; i++) x[i] = F[i];
  view_encoding(d, x + 7);
  x[34] = 0.0f;
  x[35] = 0.0f;
  float h1[16];
#pragma unroll
  for (int j = 0; j < 16; j++) {
    const float4* w = reinterpret_cast<const float4*>(W + kSW1 + 36 * j);
    float a = W[kSB1 + j];
#pragma unroll
    for (int q = 0; q < 9; q++) a = dot4(w[q], x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3], a);
    h1[j] = fmaxf(a, 0.0f);
  }
  float h2[16];
#pragma unroll
  for (int j = 0; j < 16; j++) {
    const float4* w = reinterpret_cast<const float4*>(W + kSW2 + 16 * j);
    float a = W[kSB2 + j];
#pragma unroll
    for (int q = 0; q < 4; q++) a = dot4(w[q], h1[4 * q], h1[4 * q + 1], h1[4 * q + 2], h1[4 * q + 3], a);
    h2[j] = fmaxf(a, 0.0f);
  }
#pragma unroll
  for (int j = 0; j < 3; j++) {
    const float4* w = reinterpret_cast<const float4*>(W + kSW3 + 16 * j);
    float a = W[kSB3 + j];
#pragma unroll
    for (int q = 0; q < 4; q++) a = dot4(w[q], h2[4 * q], h2[4 * q + 1], h2[4 * q + 2], h2[4 * q + 3], a);
    y[j] = sigmoidf_(a);
  }
}

__device__ __forceinline__ void mlp_forward(const float* __restrict__ W, const float F[7], const float d[3],
                                            MlpCache& c) {
#pragma unroll
  for (int i = 0; i < 7; i++) c.x[i] = F[i];
  view_encoding(d, c.x + 7);
#pragma unroll
  for (int j = 0; j < 16; j++) {
    float a = W[kOffB1 + j];
#pragma unroll
    for (int i = 0; i < 34; i++) a = fmaf(W[kOffW1 + j * 34 + i], c.x[i], a);
    c.a1[j] = a;
  }
#pragma unroll
  for (int j = 0; j < 16; j++) {
    float a = W[kOffB2 + j];
#pragma unroll
    for (int i = 0; i < 16; i++) a = fmaf(W[kOffW2 + j * 16 + i], fmaxf(c.a1[i], 0.0f), a);
    c.a2[j] = a;
  }
#pragma unroll
  for (int j = 0; j < 3; j++) {
    float a = W[kOffB3 + j];
#pragma unroll
    for (int i = 0; i < 16; i++) a = fmaf(W[kOffW3 + j * 16 + i], fmaxf(c.a2[i], 0.0f), a);
    c.y[j] = sigmoidf_(a);
  }
}

}  // namespace omerf
