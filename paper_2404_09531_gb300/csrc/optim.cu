// optim.cu -- fused Adam step over the scene's parameter groups and the
// training schedules of Oblique-MERF (appendix A).
//
// One launch updates every group: the threads walk the concatenation of the
// groups (at most 8), each element reading p, g, m, v and writing p, m, v and,
// for a group with a BF16 shadow (BF16 features with an FP32 master copy),
// the rounded value.  HBM-bound: 28 B per element (30 B with a shadow).
#include <cmath>

#include "internal.h"

namespace omerf {

constexpr int kMaxGroups = 8;

struct AdamArgs {
  float* p[kMaxGroups];
  const float* g[kMaxGroups];
  float* m[kMaxGroups];
  float* v[kMaxGroups];
  __nv_bfloat16* shadow[kMaxGroups];
  long end[kMaxGroups];  // inclusive prefix of group sizes
  float lr_c[kMaxGroups];  // lr / (1 - beta1^t)
  int n_groups;
  long total;
  float b1, b2, inv_bc2, eps;
};

__global__ void adam_kernel(const AdamArgs a) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < a.total; i += (long)gridDim.x * blockDim.x) {
    int q = 0;
    while (q < a.n_groups - 1 && i >= a.end[q]) q++;
    const long j = i - (q ? a.end[q - 1] : 0);
    const float g = a.g[q][j];
    const float m = a.b1 * a.m[q][j] + (1.0f - a.b1) * g;
    const float v = a.b2 * a.v[q][j] + (1.0f - a.b2) * g * g;
    a.m[q][j] = m;
    a.v[q][j] = v;
    const float p = a.p[q][j] - a.lr_c[q] * m / (sqrtf(v * a.inv_bc2) + a.eps);
    a.p[q][j] = p;
    if (a.shadow[q]) a.shadow[q][j] = __float2bfloat16_rn(p);
  }
}

}  // namespace omerf

using namespace omerf;

extern "C" {

omerf_status omerf_adam_step(const omerf_adam_group* groups, int32_t n_groups, float beta1, float beta2, float eps,
                             int64_t step, void* stream) {
  OMERF_API_RANGE();
  if (!groups || n_groups < 1 || n_groups > kMaxGroups) {
    set_error("n_groups must be in 1..%d", kMaxGroups);
    return OMERF_EINVAL;
  }
  if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f) || step < 1) {
    set_error("need 0 <= beta < 1, eps >= 0 and step >= 1");
    return OMERF_EINVAL;
  }
  AdamArgs a{};
  long total = 0;
  for (int q = 0; q < n_groups; q++) {
    const omerf_adam_group& gr = groups[q];
    if (gr.n < 0 || (gr.n > 0 && (!gr.param || !gr.grad || !gr.m || !gr.v)) || !std::isfinite(gr.lr)) {
      set_error("adam group %d: null array or bad size / learning rate", q);
      return OMERF_EINVAL;
    }
    a.p[q] = gr.param;
    a.g[q] = gr.grad;
    a.m[q] = gr.m;
    a.v[q] = gr.v;
    a.shadow[q] = static_cast<__nv_bfloat16*>(gr.shadow_bf16);
    total += gr.n;
    a.end[q] = total;
    // bias corrections in double on the host, applied as FP32 constants
    a.lr_c[q] = (float)((double)gr.lr / (1.0 - std::pow((double)beta1, (double)step)));
  }
  a.n_groups = n_groups;
  a.total = total;
  a.b1 = beta1;
  a.b2 = beta2;
  a.inv_bc2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)step)));
  a.eps = eps;
  if (total == 0) return OMERF_OK;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long want = (total + 255) / 256;
  const int grid = (int)(want < 8L * sms ? want : 8L * sms);
  OMERF_LAUNCH_FAULT();
  for (int q = 0; q < n_groups; q++) {
    const omerf_adam_group& gr = groups[q];
    const omerf_status st = check_device_ptrs(
        {{gr.param, "param"}, {gr.grad, "grad"}, {gr.m, "m"}, {gr.v, "v"}, {gr.shadow_bf16, "shadow_bf16"}});
    if (st != OMERF_OK) return st;
  }
  adam_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(a);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "adam kernel");
}

float omerf_lr_exponential(float lr0, float lr1, int64_t step, int64_t total) {
  if (total <= 0) return lr1;
  const double s = (double)(step < 0 ? 0 : (step > total ? total : step)) / (double)total;
  return (float)((double)lr0 * std::pow((double)lr1 / (double)lr0, s));
}

float omerf_lambda_occ(int64_t step) {
  if (step < 10000) return 0.0f;
  const int64_t k = (step - 10000) / 2000;
  if (k >= 20) return 0.2f;
  const double v = 1e-4 * std::pow(1.5, (double)k);
  return (float)(v < 0.2 ? v : 0.2);
}

}  // extern "C"
