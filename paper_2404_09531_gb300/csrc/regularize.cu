// regularize.cu -- the two density regularisers of Sec. 4.3, each one kernel
// that computes the loss and scatters its gradient in the same pass over the
// feature field (float32 or bfloat16 features, float32 gradient buffers shaped
// like the parameters, as for the training backward).
//
//   sparsity  L = lam / |P| sum_{p in P} alpha(p)                      Eq. 13
//             alpha(p) = 1 - exp(-tau(p) delta), delta the lattice step,
//             over caller-chosen points P in the occupied space
//   entropy   L = lam / |R| sum_r -sum_i p_i log p_i,                  Eq. 14
//             p_i = a_i / S, a_i = M_i alpha_i, S = sum_i a_i, over each
//             ray's evaluated samples (the march of Eq. 7 without early
//             termination; at most n_max samples); dL_r/da_k = -(log p_k + L_r)/S
//
// Only the density channel (channel 0 of Eq. 2's sum) enters either loss, so
// both kernels read and scatter that one channel of the 8 grid corners and
// 12 plane texels.  The entropy kernel gives one warp to a ray: the lanes
// test 32 consecutive lattice indices at a time with the exact FP32 decision
// rule, the warp sums S and sum a log a, and a second scan recomputes each
// sample to scatter dL/dt_0 and, through the occupancy ramps of Eq. 6,
// dL/dz_min and dL/dz_max.
#include <cmath>

#include "internal.h"

namespace omerf {

namespace {

// 1 - exp(-sigma), with a series below 1e-3 (the same form as the march).
__device__ __forceinline__ float opacity_of(float sigma) {
  return sigma < 1e-3f ? sigma * (1.0f - 0.5f * sigma * (1.0f - sigma * (1.0f / 3.0f))) : 1.0f - __expf(-sigma);
}

__device__ __forceinline__ float load1(const float* base, int elem) { return __ldg(base + elem); }
__device__ __forceinline__ float load1(const __nv_bfloat16* base, int elem) {
  return __bfloat162float(__ldg(base + elem));
}

// Density channel t_0 at p and the stencil that produced it.
template <class FT, bool SPARSE>
__device__ __forceinline__ float density_at(const Geo& g, const float p[3], int goff[8], float gw[8], int poff[12],
                                            float pw[12]) {
  grid_stencil<SPARSE>(g, p, goff, gw);
  plane_stencil(g, p, poff, pw);
  const FT* grid = static_cast<const FT*>(g.grid);
  float t0 = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; c++)
    if (goff[c] >= 0 && check_range(g, 0, goff[c])) t0 = fmaf(gw[c], load1(grid, goff[c]), t0);
#pragma unroll
  for (int q = 0; q < 3; q++) {
    const FT* P = static_cast<const FT*>(plane_base(g, q));
#pragma unroll
    for (int c = 0; c < 4; c++)
      if (check_range(g, 1 + q, poff[4 * q + c])) t0 = fmaf(pw[4 * q + c], load1(P, poff[4 * q + c]), t0);
  }
  return t0;
}

struct RegGrads {
  float* grid;
  float* plane[3];
  float2* occ;
};

// Scatter dL/dt_0 into channel 0 of the stencil's texels.
__device__ __forceinline__ void scatter_density(const Geo& g, const RegGrads& G, float dt0, const int goff[8],
                                                const float gw[8], const int poff[12], const float pw[12]) {
  if (G.grid) {
#pragma unroll
    for (int c = 0; c < 8; c++)
      if (goff[c] >= 0 && gw[c] != 0.0f && in_range(g, 0, goff[c])) atomicAdd(G.grid + goff[c], gw[c] * dt0);
  }
#pragma unroll
  for (int q = 0; q < 3; q++) {
    if (!G.plane[q]) continue;
#pragma unroll
    for (int c = 0; c < 4; c++)
      if (pw[4 * q + c] != 0.0f && in_range(g, 1 + q, poff[4 * q + c]))
        atomicAdd(G.plane[q] + poff[4 * q + c], pw[4 * q + c] * dt0);
  }
}

// Block sum of v added to *out (v already weighted).
__device__ __forceinline__ void block_add(float v, float* out) {
  __shared__ float part[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) part[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += part[w];
    atomicAdd(out, s);
  }
}

}  // namespace

// Eq. 13: thread per point.
template <class FT, bool SPARSE>
__global__ void __launch_bounds__(kThreads) sparsity_kernel(const Geo g, const float* __restrict__ pts, long n,
                                                            float lam_n, const float* grad_scale, float* loss,
                                                            RegGrads G) {
  const float c = lam_n * (grad_scale ? __ldg(grad_scale) : 1.0f);
  const bool grads = G.grid || G.plane[0] || G.plane[1] || G.plane[2];
  float acc = 0.0f;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float p[3] = {__ldg(pts + 3 * i), __ldg(pts + 3 * i + 1), __ldg(pts + 3 * i + 2)};
    int goff[8], poff[12];
    float gw[8], pw[12];
    const float t0 = density_at<FT, SPARSE>(g, p, goff, gw, poff, pw);
    const float sigma = __expf(t0) * g.step;
    const float alpha = opacity_of(sigma);
    acc += alpha;
    if (grads) scatter_density(g, G, c * (1.0f - alpha) * sigma, goff, gw, poff, pw);
  }
  if (loss) block_add(lam_n * acc, loss);
}

// Eq. 14: one warp per ray, two scans of the ray's lattice range.
template <class FT, bool SPARSE>
__global__ void __launch_bounds__(kThreads) entropy_kernel(const Geo g, const float* __restrict__ rays, long n,
                                                           float lam_n, const float* grad_scale, float* loss,
                                                           RegGrads G) {
  const int lane = threadIdx.x & 31;
  const long warp0 = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
  const float c = lam_n * (grad_scale ? __ldg(grad_scale) : 1.0f);
  const bool grads = G.grid || G.plane[0] || G.plane[1] || G.plane[2] || G.occ;
  float lacc = 0.0f;
  for (long r = warp0; r < n; r += nwarps) {
    float o[3], d[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      o[a] = __ldg(rays + 6 * r + a);
      d[a] = __ldg(rays + 6 * r + 3 + a);
    }
    int klo, khi;
    if (!lattice_range(g, o, d, klo, khi)) continue;
    // scan 1: S = sum a_i, Q = sum a_i log a_i
    float S = 0.0f, Q = 0.0f;
    int seen = 0;
    for (int kb = klo; kb <= khi && seen < g.n_max; kb += 32) {
      const int k = kb + lane;
      float p[3];
      float2 zb;
      int cell;
      bool ev = k <= khi && lattice_test(g, o, d, k, p, zb, cell);
      const unsigned m = __ballot_sync(kFull, ev);
      ev = ev && seen + __popc(m & lanemask_lt()) < g.n_max;
      seen += __popc(m);
      if (ev) {
        int br;
        float rr;
        const float Mv = occupancy(g, p[2], zb, br, rr);
        int goff[8], poff[12];
        float gw[8], pw[12];
        const float t0 = density_at<FT, SPARSE>(g, p, goff, gw, poff, pw);
        const float a = Mv * opacity_of(__expf(t0) * g.step);
        if (a > 0.0f) {
          S += a;
          Q = fmaf(a, logf(a), Q);
        }
      }
    }
    S = warp_sum(S);
    Q = warp_sum(Q);
    if (!(S > 0.0f)) continue;
    const float logS = logf(S);
    const float L = logS - Q / S;
    lacc += L;
    if (!grads) continue;
    // scan 2: recompute every sample, scatter dL/da_k = -(log a_k - log S + L) / S
    const float cS = c / S;
    seen = 0;
    for (int kb = klo; kb <= khi && seen < g.n_max; kb += 32) {
      const int k = kb + lane;
      float p[3];
      float2 zb;
      int cell;
      bool ev = k <= khi && lattice_test(g, o, d, k, p, zb, cell);
      const unsigned m = __ballot_sync(kFull, ev);
      ev = ev && seen + __popc(m & lanemask_lt()) < g.n_max;
      seen += __popc(m);
      if (!ev) continue;
      int br;
      float rr;
      const float Mv = occupancy(g, p[2], zb, br, rr);
      int goff[8], poff[12];
      float gw[8], pw[12];
      const float t0 = density_at<FT, SPARSE>(g, p, goff, gw, poff, pw);
      const float sigma = __expf(t0) * g.step;
      const float alpha = opacity_of(sigma);
      const float a = Mv * alpha;
      if (!(a > 0.0f)) continue;
      const float da = -cS * (logf(a) - logS + L);
      scatter_density(g, G, da * Mv * (1.0f - alpha) * sigma, goff, gw, poff, pw);
      if (G.occ && br != 0) {
        // M = r^2 on a ramp: dM/dz_min = -2 r / eps (lower), dM/dz_max = 2 r / eps (upper)
        const float dM = da * alpha * 2.0f * rr * g.inv_eps;
        if (br == 1) atomicAdd(&G.occ[cell].x, -dM);
        else atomicAdd(&G.occ[cell].y, dM);
      }
    }
  }
  if (loss) {
    if (lane != 0) lacc = 0.0f;
    block_add(lam_n * lacc, loss);
  }
}

}  // namespace omerf

using namespace omerf;

namespace {

omerf_status check_reg_args(const omerf_scene* s, const void* in, int64_t n, float lambda, const float* loss,
                            const float* const* gp, int ngp, const float* g_occ) {
  if (!s) { set_error("NULL scene"); return OMERF_EINVAL; }
  if (n < 0) { set_error("n must be >= 0"); return OMERF_ESHAPE; }
  if (n > 0 && !in) { set_error("NULL array argument"); return OMERF_EINVAL; }
  if (!std::isfinite(lambda)) { set_error("lambda must be finite"); return OMERF_EINVAL; }
  if (loss && !aligned(loss, 4)) { set_error("loss must be 4-byte aligned"); return OMERF_EINVAL; }
  for (int i = 0; i < ngp; i++)
    if (gp[i] && !aligned(gp[i], 4)) { set_error("gradient buffers must be 4-byte aligned"); return OMERF_EINVAL; }
  if (g_occ && !aligned(g_occ, 8)) { set_error("g_occ must be 8-byte aligned"); return OMERF_EINVAL; }
  return OMERF_OK;
}

// The arrays of a regulariser call, checked to be device memory.
omerf_status check_reg_ptrs(const void* in, const float* grad_scale, const float* loss, const float* const* gp,
                            int ngp, const float* g_occ) {
  omerf_status st =
      check_device_ptrs({{in, "points / rays"}, {grad_scale, "grad_scale"}, {loss, "loss"}, {g_occ, "g_occ"}});
  for (int i = 0; i < ngp && st == OMERF_OK; i++) st = check_device_ptr(gp[i], "gradient buffer");
  return st;
}

template <class K>
int reg_grid(K kern, long units_per_block, long n, int num_sms) {
  static std::atomic<int> per_sm[64];  // per device: resident CTAs of this kernel
  int dev = 0;
  cudaGetDevice(&dev);
  dev &= 63;
  int b = per_sm[dev].load(std::memory_order_relaxed);
  if (b == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kThreads, 0) != cudaSuccess || b < 1) b = 1;
    per_sm[dev].store(b, std::memory_order_relaxed);
  }
  const long want = (n + units_per_block - 1) / units_per_block;
  const long cap = (long)b * num_sms;
  return (int)std::max(1L, std::min(want, cap));
}

}  // namespace

omerf_status omerf_sparsity_loss(const omerf_scene* s, const float* points, int64_t n, float lambda,
                                 const float* grad_scale, float* loss, float* g_grid, float* g_xy, float* g_xz,
                                 float* g_yz, void* stream) {
  OMERF_API_RANGE();
  const float* gp[4] = {g_grid, g_xy, g_xz, g_yz};
  omerf_status st = check_reg_args(s, points, n, lambda, loss, gp, 4, nullptr);
  if (st != OMERF_OK) return st;
  if (n == 0) return OMERF_OK;
  RegGrads G{g_grid, {g_xy, g_xz, g_yz}, nullptr};
  cudaStream_t cs = (cudaStream_t)stream;
  const float lam_n = (float)((double)lambda / (double)n);
  const bool bf16 = s->desc.feat_dtype == OMERF_BF16, sparse = s->desc.brick > 0;
  auto k = bf16 ? (sparse ? sparsity_kernel<__nv_bfloat16, true> : sparsity_kernel<__nv_bfloat16, false>)
                : (sparse ? sparsity_kernel<float, true> : sparsity_kernel<float, false>);
  OMERF_LAUNCH_FAULT();
  if ((st = check_reg_ptrs(points, grad_scale, loss, gp, 4, nullptr)) != OMERF_OK) return st;
  k<<<reg_grid(k, kThreads, n, s->num_sms), kThreads, 0, cs>>>(s->geo, points, n, lam_n, grad_scale, loss, G);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "sparsity loss launch");
}

omerf_status omerf_entropy_loss(const omerf_scene* s, const float* rays, int64_t n, float lambda,
                                const float* grad_scale, float* loss, float* g_grid, float* g_xy, float* g_xz,
                                float* g_yz, float* g_occ, void* stream) {
  OMERF_API_RANGE();
  const float* gp[4] = {g_grid, g_xy, g_xz, g_yz};
  omerf_status st = check_reg_args(s, rays, n, lambda, loss, gp, 4, g_occ);
  if (st != OMERF_OK) return st;
  if (n == 0) return OMERF_OK;
  RegGrads G{g_grid, {g_xy, g_xz, g_yz}, reinterpret_cast<float2*>(g_occ)};
  cudaStream_t cs = (cudaStream_t)stream;
  const float lam_n = (float)((double)lambda / (double)n);
  const long rays_per_block = kThreads / 32;
  const bool bf16 = s->desc.feat_dtype == OMERF_BF16, sparse = s->desc.brick > 0;
  auto k = bf16 ? (sparse ? entropy_kernel<__nv_bfloat16, true> : entropy_kernel<__nv_bfloat16, false>)
                : (sparse ? entropy_kernel<float, true> : entropy_kernel<float, false>);
  OMERF_LAUNCH_FAULT();
  if ((st = check_reg_ptrs(rays, grad_scale, loss, gp, 4, g_occ)) != OMERF_OK) return st;
  k<<<reg_grid(k, rays_per_block, n, s->num_sms), kThreads, 0, cs>>>(s->geo, rays, n, lam_n, grad_scale, loss, G);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "entropy loss launch");
}
