// probe.cu -- load-bandwidth probe: the roofline denominator of the march.
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
  load_probe_kernel<<<ctas, 256, 0, (cudaStream_t)stream>>>(buf, bytes_per_cta / 4, passes, sink);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "load probe launch");
}
