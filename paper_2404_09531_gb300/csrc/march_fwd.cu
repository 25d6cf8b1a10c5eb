// march_fwd.cu -- forward march: render and training forward (sm_103a).
//
// Persistent kernel of 8 warps per CTA.  A CTA takes a super-tile of 8
// bundles from an atomic work counter (16 x 16 pixels of a camera, or 256
// consecutive rays of a ray list) so that its warps share L1 lines; a warp
// owns a bundle of 32 rays (an 8 x 4 pixel tile).  The warp walks its rays
// in order and packs their evaluated samples (Sec. 4.1: only samples inside
// the occupancy interval are evaluated) into a 32-entry queue that may span
// rays (packed.cuh); the 32 queued samples are gathered and activated in
// parallel, composited with segmented lane scans (Eq. 1: a product scan of
// 1 - M alpha per ray) and early termination is resolved per ray.  After
// the bundle each lane shades its ray with the deferred MLP (Eq. 4): FP32 on
// CUDA cores, or BF16 on tensor cores for a BF16 scene.
//
// Modes: render (pixels and sample counts); training forward with the loss
// (per-ray state for the backward, MLP, Charbonnier and smoothness terms);
// training forward without the loss (per-ray state only: the fused training
// step lets the MLP backward, which evaluates the MLP anyway, add the loss).
#include <cstdio>

#include <type_traits>

#include "internal.h"
#include "mlp_mma.cuh"
#include "packed.cuh"

namespace omerf {

// Per-warp shared state of the packed march of one bundle of 32 rays.
struct MarchState {
  WarpQueue q;
  float F[32][8];    // per-ray accumulated [sum w c^d, sum w f]
  float T[32];       // per-ray transmittance so far
  int cnt[32];       // per-ray evaluated samples
};
// With the tensor-core MLP the whole march state doubles as the MLP staging
// area: the epilogue copies each ray's F, T and count to registers before it
// stages the MLP rows, and the next bundle starts after a CTA barrier.  The
// smaller per-warp footprint lets the BF16 render take a smaller
// shared-memory carveout, leaving more of the SM's SRAM to L1.
template <bool MMA>
struct WarpMarch {
  MarchState s;
};
template <>
struct WarpMarch<true> {
  union {
    MarchState s;
    MlpStage m;
  };
};

// March the 32 rays of a bundle (lane r owns ray r: o, d, [klo, khi]).
//
// fill:    evaluated samples of consecutive rays are queued, 32 at a time
//          (packed.cuh);
// process: the 32 queued samples are gathered and activated in parallel;
//          compositing is a segmented lane scan (segments = rays) of
//          1 - alpha_hat, early termination is resolved per segment, and
//          the weighted features are summed per segment into the ray's
//          accumulator.
// On return ws.s.F / ws.s.T / ws.s.cnt hold every ray's F, T_N and sample count.
template <class FT, bool SPARSE, class WS>
__device__ __forceinline__ void march_bundle(const Geo& g, int lane, const float o[3], const float d[3], int klo,
                                             int khi, bool any, WS& ws) {
#pragma unroll
  for (int c = 0; c < 8; c++) ws.s.F[lane][c] = 0.0f;
  ws.s.T[lane] = 1.0f;
  ws.s.cnt[lane] = 0;
  ws.s.q.ro[lane] = make_float4(o[0], o[1], o[2], __int_as_float(klo));
  ws.s.q.rd[lane] = make_float4(d[0], d[1], d[2], __int_as_float(khi));
  ws.s.q.cap[lane] = g.n_max;
  unsigned pend = __ballot_sync(kFull, any);
  FillState f;
  __syncwarp();
  while (pend) {
    const int nq = fill_queue(g, lane, pend, f, ws.s.q);
    if (nq == 0) break;
    const bool act = lane < nq;
    const float4 qa = ws.s.q.a[lane], qb = ws.s.q.b[lane];
    const int r = act ? __float_as_int(qb.y) : 32;
    SampleAct s;
    s.ah = 0.0f;
#pragma unroll
    for (int c = 0; c < 7; c++) s.x[c] = 0.0f;
    if (act) {
      const float p[3] = {qa.x, qa.y, qa.z};
      float t[8];
      gather_features<FT, SPARSE>(g, p, t);
      activate(g, t, p[2], make_float2(qa.w, qb.x), s);
    }
    bool head;
    const int segstart = segment_start(lane, r, head);
    // transmittance: segmented inclusive product scan of (1 - alpha_hat)
    const float P = seg_prod_scan(1.0f - s.ah, lane, segstart);
    float Pex = __shfl_up_sync(kFull, P, 1);
    if (head) Pex = 1.0f;
    const float Tprev = act ? ws.s.T[r] : 1.0f;
    const float Ti = Tprev * Pex, Tn = Tprev * P;
    // early termination: the first sample of a segment whose T drops below t_thr ends the ray
    const bool term = act && Tn < g.t_thr;
    const unsigned tm = __ballot_sync(kFull, term);
    const unsigned seglt = lanemask_lt() & ~((1u << segstart) - 1u);
    const bool dropped = (tm & seglt) != 0u;
    const bool ok = act && !dropped;
    const float w = ok ? Ti * s.ah : 0.0f;
    float wx[7];
#pragma unroll
    for (int c = 0; c < 7; c++) wx[c] = w * s.x[c];
    seg_sum_scan7(wx, lane, segstart);
    const unsigned okm = __ballot_sync(kFull, ok);
    const int rnext = __shfl_down_sync(kFull, r, 1);
    const bool tail = act && (lane == 31 || rnext != r);
    const unsigned segle = lanemask_le() & ~((1u << segstart) - 1u);
    if (tail) {
#pragma unroll
      for (int c = 0; c < 7; c++) ws.s.F[r][c] += wx[c];
      ws.s.cnt[r] += __popc(okm & segle);
      if (!(tm & segle)) ws.s.T[r] = Tn;
    }
    const bool first_term = term && !dropped;
    if (first_term) ws.s.T[r] = Tn;
    pend &= ~__reduce_or_sync(kFull, first_term ? (1u << r) : 0u);
    __syncwarp();
  }
}

struct FwdArgs {
  Cam cam;
  int use_cam, super_x;
  const float* rays;
  long n, n_super;
  float* rgb;
  int* count;
  // training
  const float* target;
  const float* dirs;
  int K;
  float lam_rgb, lam_smooth;  // already divided by n
  float* saved;
  float* loss;
  unsigned* counter;
  // multi-camera render (n_cams > 0): device camera records, super-tiles in
  // camera order
  const CamRec* cams;
  int n_cams;
};

#ifndef OMERF_FWD_MINB
#define OMERF_FWD_MINB 3  // resident CTAs per SM the register budget is sized for
#endif

// TRAIN: write the per-ray state the backward needs instead of pixels; with
// LOSS also evaluate the deferred MLP and the loss terms (a fused training
// step leaves the loss to the MLP backward, which evaluates the MLP anyway).
template <class FT, bool SPARSE, bool TRAIN, bool LOSS>
__global__ void __launch_bounds__(kThreads, OMERF_FWD_MINB) march_fwd_kernel(const Geo g, const FwdArgs a) {
  // BF16 render: deferred MLP on tensor cores; otherwise FP32 on CUDA cores
  constexpr bool kMMA = std::is_same<FT, __nv_bfloat16>::value && !TRAIN;
  __shared__ __align__(16) float sW[kMMA ? 4 : kSmemMlp];
  __shared__ typename std::conditional<kMMA, MlpFrags, int>::type sFrag;
  __shared__ float sLoss[2][kThreads / 32];
  __shared__ WarpMarch<kMMA> sMarch[kThreads / 32];
  if constexpr (kMMA) {
    build_mlp_frags(g.mlp, sFrag);
  } else {
    load_mlp_padded(g.mlp, sW);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  WarpMarch<kMMA>& ws = sMarch[threadIdx.x >> 5];
  float l_rgb = 0.0f, l_smooth = 0.0f;

  // The CTA takes work in units of 8 bundles so that its 8 warps march
  // neighbouring rays together and share L1 lines: a camera super-tile of
  // 2 x 4 tiles of 8 x 4 pixels (16 x 16 pixels), or 256 consecutive rays.
  __shared__ unsigned sWork;
  const int warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) sWork = atomicAdd(a.counter, 1u);
    __syncthreads();
    const unsigned sb = sWork;
    __syncthreads();
    if (sb >= a.n_super) break;

    long rid;
    bool valid;
    float o[3] = {0.0f, 0.0f, 0.0f}, d[3] = {0.0f, 0.0f, 1.0f};
    if (a.n_cams > 0) {
      int c = 0;
      while (c + 1 < a.n_cams && (long long)sb >= a.cams[c + 1].super_start) c++;
      const CamRec& cr = a.cams[c];
      const unsigned lsb = (unsigned)((long long)sb - cr.super_start);
      const int sx = (int)(lsb % (unsigned)cr.super_x), sy = (int)(lsb / (unsigned)cr.super_x);
      const int tx = 2 * sx + (warp & 1), ty = 4 * sy + (warp >> 1);
      const int px = tx * 8 + (lane & 7), py = ty * 4 + (lane >> 3);
      valid = px < cr.cam.width && py < cr.cam.height;
      rid = (long)cr.ray_start + (long)py * cr.cam.width + px;
      if (valid) camera_ray(cr.cam, px, py, o, d);
    } else if (a.use_cam) {
      const int sx = (int)(sb % (unsigned)a.super_x), sy = (int)(sb / (unsigned)a.super_x);
      const int tx = 2 * sx + (warp & 1), ty = 4 * sy + (warp >> 1);
      const int px = tx * 8 + (lane & 7), py = ty * 4 + (lane >> 3);
      valid = px < a.cam.width && py < a.cam.height;
      rid = (long)py * a.cam.width + px;
      if (valid) camera_ray(a.cam, px, py, o, d);
    } else {
      rid = ((long)sb * 8 + warp) * 32 + lane;
      valid = rid < a.n;
      if (valid) {
        const float* r = a.rays + 6 * rid;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          o[c] = __ldg(r + c);
          d[c] = __ldg(r + 3 + c);
        }
      }
    }
    int klo = 0, khi = -1;
    const bool any = valid && lattice_range(g, o, d, klo, khi);
    march_bundle<FT, SPARSE>(g, lane, o, d, klo, khi, any, ws);
    float F[7];
#pragma unroll
    for (int c = 0; c < 7; c++) F[c] = ws.s.F[lane][c];
    const float T = ws.s.T[lane];
    const int cnt = ws.s.cnt[lane];
    __syncwarp();

    float yd_mma[3] = {0.0f, 0.0f, 0.0f};
    if constexpr (kMMA) {
      mlp_stage_row(ws.m, lane, valid && cnt > 0, F, d);
      mlp_bf16_warp(sFrag, ws.m, lane, yd_mma);
    }
    if (valid && (!TRAIN || LOSS)) {
      float out[3], yd[3] = {0.0f, 0.0f, 0.0f};
      if (cnt == 0) {
#pragma unroll
        for (int j = 0; j < 3; j++) out[j] = g.bg[j];
      } else {
        if constexpr (kMMA) {
#pragma unroll
          for (int j = 0; j < 3; j++) yd[j] = yd_mma[j];
        } else {
          mlp_forward_padded(sW, F, d, yd);
        }
#pragma unroll
        for (int j = 0; j < 3; j++) out[j] = F[j] + yd[j] + T * g.bg[j];
      }
      if (!TRAIN) {
#pragma unroll
        for (int j = 0; j < 3; j++) a.rgb[3 * rid + j] = out[j];
        if (a.count) a.count[rid] = cnt;
      } else {
        float e2 = 0.0f;
#pragma unroll
        for (int j = 0; j < 3; j++) {
          const float e = out[j] - __ldg(a.target + 3 * rid + j);
          e2 = fmaf(e, e, e2);
        }
        l_rgb += sqrtf(e2 + 1e-6f);
        if (cnt > 0) {
          const float dn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
          for (int k = 0; k < a.K; k++) {
            const float* sp = a.dirs + 3 * ((long)rid * a.K + k);
            float sv[3] = {__ldg(sp), __ldg(sp + 1), __ldg(sp + 2)};
            const float sn = sqrtf(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
            const float S = (d[0] * sv[0] + d[1] * sv[1] + d[2] * sv[2]) / (dn * sn);
            float sh[3] = {sv[0] / sn, sv[1] / sn, sv[2] / sn};
            float ys[3];
            mlp_forward_padded(sW, F, sh, ys);
            float q = 0.0f;
#pragma unroll
            for (int j = 0; j < 3; j++) q = fmaf(ys[j] - yd[j], ys[j] - yd[j], q);
            l_smooth = fmaf(S, q, l_smooth);
          }
        }
      }
    }
    if (TRAIN && valid) {
      float4* sv = reinterpret_cast<float4*>(a.saved + (long)kSavedFloats * rid);
      sv[0] = make_float4(F[0], F[1], F[2], F[3]);
      sv[1] = make_float4(F[4], F[5], F[6], T);
      sv[2] = make_float4(__int_as_float(cnt), __int_as_float(klo), __int_as_float(khi), 0.0f);
    }
  }

  if (TRAIN && LOSS) {
    l_rgb = warp_sum(l_rgb);
    l_smooth = warp_sum(l_smooth);
    if (lane == 0) {
      sLoss[0][threadIdx.x >> 5] = l_rgb;
      sLoss[1][threadIdx.x >> 5] = l_smooth;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float s0 = 0.0f, s1 = 0.0f;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
        s0 += sLoss[0][w];
        s1 += sLoss[1][w];
      }
      s0 *= a.lam_rgb;
      s1 *= a.lam_smooth;
      atomicAdd(a.loss + 1, s0);
      atomicAdd(a.loss + 2, s1);
      atomicAdd(a.loss + 0, s0 + s1);
    }
  }
}

#ifndef OMERF_CARVEOUT
#define OMERF_CARVEOUT 1
#endif
int persistent_blocks(const void* kernel, int threads, size_t smem, int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
#if OMERF_CARVEOUT
  // The marches' gathers are served from L1, which shares each SM's SRAM
  // with shared memory: ask for the smallest shared-memory carveout that
  // still holds per_sm blocks (with the driver's 1 KB per block), leaving
  // the rest to L1; keep it only if the occupancy still holds.
  cudaFuncAttributes fa;
  int dev = 0, max_smem = 0;
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
      max_smem > 0) {
    const size_t need = (fa.sharedSizeBytes + smem + 1024) * (size_t)per_sm;
    const int pct = (int)((need * 100 + (size_t)max_smem - 1) / (size_t)max_smem);
    if (pct < 100 && cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct) == cudaSuccess) {
      int again = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&again, kernel, threads, smem) != cudaSuccess ||
          again < per_sm)
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutDefault);
    }
  }
  cudaGetLastError();  // a refused hint is not an error of the launch
#endif
  return per_sm * num_sms;
}

template <class FT, bool SPARSE, bool TRAIN, bool LOSS = TRAIN>
static cudaError_t launch_variant(const omerf_scene* s, const FwdArgs& a, cudaStream_t stream) {
  auto kern = march_fwd_kernel<FT, SPARSE, TRAIN, LOSS>;
  static std::atomic<int> blocks[64];  // per device: resident CTAs of this variant
  const int dev = s->device & 63;
  int nb = blocks[dev].load(std::memory_order_relaxed);
  if (nb == 0) {
    nb = persistent_blocks((const void*)kern, kThreads, 0, s->num_sms);
    blocks[dev].store(nb, std::memory_order_relaxed);
  }
  long want = a.n_super;
  int grid = (int)(want < nb ? want : nb);
  if (grid < 1) grid = 1;
  kern<<<grid, kThreads, 0, stream>>>(s->geo, a);
  return cudaGetLastError();
}

cudaError_t launch_march_fwd(const omerf_scene* s, const Cam* cam, const float* rays, long n, float* rgb,
                             int* count, const float* target, const float* dirs, int K, const float lam[3],
                             float* saved, float* loss, cudaStream_t stream) {
  FwdArgs a{};
  const bool train = saved != nullptr;
  if (cam) {
    a.cam = *cam;
    a.use_cam = 1;
    a.super_x = (cam->width + 15) / 16;
    a.n_super = (long)a.super_x * ((cam->height + 15) / 16);
  } else {
    a.use_cam = 0;
    a.n_super = (n + 255) / 256;
  }
  a.rays = rays;
  a.n = n;
  a.rgb = rgb;
  a.count = count;
  a.target = target;
  a.dirs = dirs;
  a.K = K;
  if (train) {
    a.lam_rgb = n > 0 ? lam[0] / (float)n : 0.0f;
    a.lam_smooth = n > 0 ? lam[1] / (float)n : 0.0f;
  }
  a.saved = saved;
  a.loss = loss;
  if (a.n_super == 0) return cudaSuccess;
  a.counter = next_counter(s, stream);
  const bool bf16 = s->desc.feat_dtype == OMERF_BF16;
  const bool sparse = s->desc.brick > 0;
  if (train && loss) {
    if (bf16) return sparse ? launch_variant<__nv_bfloat16, true, true>(s, a, stream)
                            : launch_variant<__nv_bfloat16, false, true>(s, a, stream);
    return sparse ? launch_variant<float, true, true>(s, a, stream) : launch_variant<float, false, true>(s, a, stream);
  }
  if (train) {
    if (bf16) return sparse ? launch_variant<__nv_bfloat16, true, true, false>(s, a, stream)
                            : launch_variant<__nv_bfloat16, false, true, false>(s, a, stream);
    return sparse ? launch_variant<float, true, true, false>(s, a, stream)
                  : launch_variant<float, false, true, false>(s, a, stream);
  }
  if (bf16) return sparse ? launch_variant<__nv_bfloat16, true, false>(s, a, stream)
                          : launch_variant<__nv_bfloat16, false, false>(s, a, stream);
  return sparse ? launch_variant<float, true, false>(s, a, stream) : launch_variant<float, false, false>(s, a, stream);
}


cudaError_t launch_march_fwd_cams(const omerf_scene* s, const CamRec* cams, int n_cams, long n_super, long n,
                                  float* rgb, int* count, cudaStream_t stream) {
  FwdArgs a{};
  a.use_cam = 1;
  a.cams = cams;
  a.n_cams = n_cams;
  a.n_super = n_super;
  a.n = n;
  a.rgb = rgb;
  a.count = count;
  if (a.n_super == 0) return cudaSuccess;
  a.counter = next_counter(s, stream);
  const bool bf16 = s->desc.feat_dtype == OMERF_BF16;
  const bool sparse = s->desc.brick > 0;
  if (bf16) return sparse ? launch_variant<__nv_bfloat16, true, false>(s, a, stream)
                          : launch_variant<__nv_bfloat16, false, false>(s, a, stream);
  return sparse ? launch_variant<float, true, false>(s, a, stream) : launch_variant<float, false, false>(s, a, stream);
}

}  // namespace omerf
