// march_fwd.cu -- forward march: render and training forward (sm_103a).
//
// Persistent kernel, one warp per bundle of 32 rays (an 8x4 pixel tile for a
// camera, 32 consecutive rays for a ray list), bundles taken from an atomic
// work counter.  The warp marches the bundle's rays one after another with
// its 32 lanes on 32 consecutive lattice samples of the ray (Sec. 4.1: only
// samples inside the occupancy interval are evaluated; Eq. 1 compositing is a
// lane-parallel product scan of 1 - M*alpha).  Consecutive samples of one ray
// touch neighbouring texels, so one gather instruction of the warp hits few
// cache lines.  After the bundle each lane shades its own ray with the
// deferred MLP (Eq. 4).
#include <cstdio>

#include "internal.h"

namespace omerf {

// March one ray with the whole warp.  acc receives this lane's share of
// F = [sum w c^d, sum w f]; T and cnt are warp-uniform on return.
template <class FT, bool SPARSE>
__device__ __forceinline__ void march_ray(const Geo& g, const float o[3], const float d[3], int klo, int khi,
                                          int lane, float acc[7], float& T, int& cnt) {
  T = 1.0f;
  cnt = 0;
  for (int k = klo; k <= khi; k += 32) {
    const int kk = k + lane;
    float p[3];
    float2 zb = make_float2(0.0f, 0.0f);
    int cell = 0;
    bool ok = kk <= khi && lattice_test(g, o, d, kk, p, zb, cell);
    unsigned m = __ballot_sync(kFull, ok);
    if (m == 0u) continue;
    const int room = g.n_max - cnt;
    if (__popc(m) > room) {
      if (ok && __popc(m & lanemask_lt()) >= room) ok = false;
      m = __ballot_sync(kFull, ok);
    }
    SampleAct s;
    s.ah = 0.0f;
    if (ok) {
      float t[8];
      gather_features<FT, SPARSE>(g, p, t);
      activate(g, t, p[2], zb, s);
    }
    // transmittance: inclusive product scan of (1 - alpha_hat) over the lanes
    float P = 1.0f - s.ah;
#pragma unroll
    for (int sh = 1; sh < 32; sh <<= 1) {
      float v = __shfl_up_sync(kFull, P, sh);
      if (lane >= sh) P *= v;
    }
    float Pex = __shfl_up_sync(kFull, P, 1);
    if (lane == 0) Pex = 1.0f;
    const float Ti = T * Pex, Tn = T * P;
    const unsigned tm = __ballot_sync(kFull, ok && Tn < g.t_thr);
    if (tm) {
      if (lane > __ffs(tm) - 1) ok = false;
      m = __ballot_sync(kFull, ok);
    }
    if (ok) {
      const float w = Ti * s.ah;
#pragma unroll
      for (int c = 0; c < 7; c++) acc[c] = fmaf(w, s.x[c], acc[c]);
    }
    T = __shfl_sync(kFull, Tn, 31 - __clz(m));
    cnt += __popc(m);
    if (tm || cnt >= g.n_max) break;
  }
}

struct FwdArgs {
  Cam cam;
  int use_cam, tiles_x;
  const float* rays;
  long n, n_bundles;
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
};

template <class FT, bool SPARSE, bool TRAIN>
__global__ void __launch_bounds__(kThreads) march_fwd_kernel(const Geo g, const FwdArgs a) {
  __shared__ float sW[kMlpParams];
  __shared__ float sLoss[2][kThreads / 32];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sW[i] = g.mlp[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  float l_rgb = 0.0f, l_smooth = 0.0f;

  for (;;) {
    unsigned b = 0;
    if (lane == 0) b = atomicAdd(a.counter, 1u);
    b = __shfl_sync(kFull, b, 0);
    if (b >= a.n_bundles) break;

    long rid;
    bool valid;
    float o[3] = {0.0f, 0.0f, 0.0f}, d[3] = {0.0f, 0.0f, 1.0f};
    if (a.use_cam) {
      const int tx = (int)(b % (unsigned)a.tiles_x), ty = (int)(b / (unsigned)a.tiles_x);
      const int px = tx * 8 + (lane & 7), py = ty * 4 + (lane >> 3);
      valid = px < a.cam.width && py < a.cam.height;
      rid = (long)py * a.cam.width + px;
      if (valid) camera_ray(a.cam, px, py, o, d);
    } else {
      rid = (long)b * 32 + lane;
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

    float F[7] = {0, 0, 0, 0, 0, 0, 0};
    float T = 1.0f;
    int cnt = 0;
    unsigned todo = __ballot_sync(kFull, any);
    while (todo) {
      const int r = __ffs(todo) - 1;
      todo &= todo - 1;
      float ro[3], rd[3];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        ro[c] = __shfl_sync(kFull, o[c], r);
        rd[c] = __shfl_sync(kFull, d[c], r);
      }
      const int rklo = __shfl_sync(kFull, klo, r), rkhi = __shfl_sync(kFull, khi, r);
      float acc[7] = {0, 0, 0, 0, 0, 0, 0};
      float rT;
      int rc;
      march_ray<FT, SPARSE>(g, ro, rd, rklo, rkhi, lane, acc, rT, rc);
#pragma unroll
      for (int c = 0; c < 7; c++) {
        const float v = warp_sum(acc[c]);
        if (lane == r) F[c] = v;
      }
      if (lane == r) {
        T = rT;
        cnt = rc;
      }
    }

    if (valid) {
      float out[3], yd[3] = {0.0f, 0.0f, 0.0f};
      if (cnt == 0) {
#pragma unroll
        for (int j = 0; j < 3; j++) out[j] = g.bg[j];
      } else {
        MlpCache mc;
        mlp_forward(sW, F, d, mc);
#pragma unroll
        for (int j = 0; j < 3; j++) {
          yd[j] = mc.y[j];
          out[j] = F[j] + mc.y[j] + T * g.bg[j];
        }
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
            MlpCache ms;
            mlp_forward(sW, F, sh, ms);
            float q = 0.0f;
#pragma unroll
            for (int j = 0; j < 3; j++) q = fmaf(ms.y[j] - yd[j], ms.y[j] - yd[j], q);
            l_smooth = fmaf(S, q, l_smooth);
          }
        }
        float4* sv = reinterpret_cast<float4*>(a.saved + (long)kSavedFloats * rid);
        sv[0] = make_float4(F[0], F[1], F[2], F[3]);
        sv[1] = make_float4(F[4], F[5], F[6], T);
        sv[2] = make_float4(__int_as_float(cnt), __int_as_float(klo), __int_as_float(khi), 0.0f);
      }
    }
  }

  if (TRAIN) {
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

int persistent_blocks(const void* kernel, int threads, size_t smem, int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return per_sm * num_sms;
}

template <class FT, bool SPARSE, bool TRAIN>
static cudaError_t launch_variant(const omerf_scene* s, const FwdArgs& a, cudaStream_t stream) {
  auto kern = march_fwd_kernel<FT, SPARSE, TRAIN>;
  static int blocks[64] = {0};
  const int dev = s->device & 63;
  if (blocks[dev] == 0) blocks[dev] = persistent_blocks((const void*)kern, kThreads, 0, s->num_sms);
  long want = (a.n_bundles + (kThreads / 32) - 1) / (kThreads / 32);
  int grid = (int)(want < blocks[dev] ? want : blocks[dev]);
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
    a.tiles_x = (cam->width + 7) / 8;
    a.n_bundles = (long)a.tiles_x * ((cam->height + 3) / 4);
  } else {
    a.use_cam = 0;
    a.n_bundles = (n + 31) / 32;
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
  if (a.n_bundles == 0) return cudaSuccess;
  a.counter = next_counter(s, stream);
  const bool bf16 = s->desc.feat_dtype == OMERF_BF16;
  const bool sparse = s->desc.brick > 0;
  if (train) {
    if (bf16) return sparse ? launch_variant<__nv_bfloat16, true, true>(s, a, stream)
                            : launch_variant<__nv_bfloat16, false, true>(s, a, stream);
    return sparse ? launch_variant<float, true, true>(s, a, stream) : launch_variant<float, false, true>(s, a, stream);
  }
  if (bf16) return sparse ? launch_variant<__nv_bfloat16, true, false>(s, a, stream)
                          : launch_variant<__nv_bfloat16, false, false>(s, a, stream);
  return sparse ? launch_variant<float, true, false>(s, a, stream) : launch_variant<float, false, false>(s, a, stream);
}

}  // namespace omerf
