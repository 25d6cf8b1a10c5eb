// probe.cu -- bandwidth probes: the roofline denominators of the marches.
//
// The march's feature gather (Eq. 2: 8 grid corners and 12 plane texels per
// sample) is served from L1 and L2, not from DRAM, so the bandwidth that
// bounds it is the rate at which an SM's L1 returns 256-bit read-only loads
// to registers.  This kernel measures that rate with the gather's own
// instruction (ld.global.nc.v8.f32, 32 B per lane), in the march's launch
// shape (256-thread CTAs, several per SM): each CTA streams its own slice of
// a buffer, a warp's load covering 1 KB contiguous (the best case, 8
// wavefronts per instruction).  A slice that fits in L1 measures L1; one
// larger than L1 (but the whole buffer inside L2) measures L2.
//
// The re-march backward scatters each sample's gradient into its 20 texels
// with 16-byte vector FP32 reductions (red.global.add.v4.f32), one lane per
// sample, the lanes of a warp on different texels.  The second probe
// measures the rate of that instruction in the re-march's launch shape:
// every warp reduces into its own region, each lane into its own 128-byte
// line, 512 bytes per warp instruction.
#include "internal.h"

namespace omerf {

__global__ void __launch_bounds__(256) load_probe_kernel(const float* __restrict__ buf, long long per_cta,
                                                        int passes, float* __restrict__ sink) {
  const float* base = buf + (long long)blockIdx.x * per_cta;
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int p = 0; p < passes; p++) {
#pragma unroll 4
    for (long long i = (long long)threadIdx.x * 8; i < per_cta; i += 256 * 8) {
      float v[8];
      Texel<float>::load(base, (int)i, v);
#pragma unroll
      for (int c = 0; c < 8; c++) acc[c] += v[c];
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; c++) s += acc[c];
  sink[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) red_probe_kernel(float* __restrict__ buf, long long per_warp, int passes) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  float* base = buf + warp * per_warp + lane * 32;
  const long long steps = per_warp / 1024;  // 32 lines (4 KB) per step
  for (int p = 0; p < passes; p++)
    for (long long st = 0; st < steps; st++)
      asm volatile("red.global.add.v4.f32 [%0], {%1, %1, %1, %1};" ::"l"(base + st * 1024), "f"(1.0f) : "memory");
}

}  // namespace omerf

using namespace omerf;

extern "C" omerf_status omerf_probe_load_bandwidth(const float* buf, int64_t bytes_per_cta, int32_t ctas,
                                                   int32_t passes, float* sink, void* stream) {
  OMERF_API_RANGE();
  if (!buf || !sink) { set_error("NULL argument"); return OMERF_EINVAL; }
  if (ctas < 1 || passes < 1) { set_error("ctas and passes must be >= 1"); return OMERF_ESHAPE; }
  if (bytes_per_cta < 8192 || bytes_per_cta % 8192 || bytes_per_cta > (1LL << 30)) {
    set_error("bytes_per_cta must be a positive multiple of 8192 (256 threads x 32 B), at most 1 GiB");
    return OMERF_ESHAPE;
  }
  if (!aligned(buf, 32) || !aligned(sink, 4)) { set_error("buf must be 32-byte aligned"); return OMERF_EINVAL; }
  OMERF_LAUNCH_FAULT();
  const omerf_status st = check_device_ptrs({{buf, "buf"}, {sink, "sink"}});
  if (st != OMERF_OK) return st;
  load_probe_kernel<<<ctas, 256, 0, (cudaStream_t)stream>>>(buf, bytes_per_cta / 4, passes, sink);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "load probe launch");
}

extern "C" omerf_status omerf_probe_red_bandwidth(float* buf, int64_t bytes_per_warp, int32_t ctas, int32_t passes,
                                                  void* stream) {
  OMERF_API_RANGE();
  if (!buf) { set_error("NULL argument"); return OMERF_EINVAL; }
  if (ctas < 1 || passes < 1) { set_error("ctas and passes must be >= 1"); return OMERF_ESHAPE; }
  if (bytes_per_warp < 4096 || bytes_per_warp % 4096 || bytes_per_warp > (1LL << 24)) {
    set_error("bytes_per_warp must be a positive multiple of 4096 (32 lines of 128 B), at most 16 MiB");
    return OMERF_ESHAPE;
  }
  if (!aligned(buf, 16)) { set_error("buf must be 16-byte aligned"); return OMERF_EINVAL; }
  OMERF_LAUNCH_FAULT();
  const omerf_status st = check_device_ptr(buf, "buf");
  if (st != OMERF_OK) return st;
  red_probe_kernel<<<ctas, 256, 0, (cudaStream_t)stream>>>(buf, bytes_per_warp / 4, passes);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "reduction probe launch");
}
