// noalloc.cu -- render entry point that allocates no memory.
//
// omerf_render creates nothing per call, but its scene handle owns device
// state that omerf_scene_create obtains with cudaMalloc: the work counters
// of the persistent march kernel and the occupancy hulls used for
// empty-space skipping.  Some callers cannot allocate: a host framework that
// owns all device memory and hands the renderer fixed buffers, or a frame
// loop that must never call cudaMalloc (it can synchronise the device and
// stall the frame).  omerf_render_noalloc renders from a scene description
// alone; its scratch memory is a file-scope __device__ array that every GPU
// loading this library holds until the process exits.
#include <mutex>

#include "internal.h"

namespace omerf {

// Scratch layout: work counters | occupancy hull (2 floats) | coarse grid |
// brick neighbour records (brick grids).
constexpr size_t kNoAllocCounterBytes = kCounterSlots * sizeof(unsigned);
constexpr size_t kNoAllocHullOffset = kNoAllocCounterBytes;
constexpr size_t kNoAllocCoarseOffset = kNoAllocHullOffset + 256;
constexpr size_t kNoAllocScratchBytes = 8u << 20;  // 8 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array, looked up once per device (with that
// device current) by the first call made on it.
constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mutex;

static omerf_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d is out of range for the no-allocation render", dev);
    return OMERF_EDEVICE;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("cudaGetSymbolAddress of the no-allocation scratch failed: %s", cudaGetErrorString(e));
      return OMERF_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return OMERF_OK;
}

}  // namespace omerf

using namespace omerf;

extern "C" omerf_status omerf_render_noalloc(const omerf_scene_desc* desc, const omerf_camera* cam, const float* rays,
                                             int64_t n, float* rgb, int32_t* count, void* stream) {
  OMERF_API_RANGE();
  omerf_status st = validate_desc(desc);
  if (st != OMERF_OK) return st;
  if (!rgb && n > 0) {
    set_error("rgb is NULL");
    return OMERF_EINVAL;
  }
  if (n < 0) {
    set_error("n must be >= 0");
    return OMERF_ESHAPE;
  }
  Cam k{};
  if (cam) {
    if ((st = validate_camera(cam, n)) != OMERF_OK) return st;
    k = to_cam(cam);
  } else if (!rays && n > 0) {
    set_error("rays is NULL and no camera given");
    return OMERF_EINVAL;
  }
  // The same pointer checks as omerf_scene_create and omerf_render (none of
  // them allocates): the description's arrays and a ray list must be device
  // memory, the outputs device or page-locked host memory, written through its
  // device alias.
  const void* ptrs[] = {desc->grid, desc->brick_table, desc->plane_xy, desc->plane_xz, desc->plane_yz, desc->occ,
                        desc->mlp};
  const char* names[] = {"grid", "brick_table", "plane_xy", "plane_xz", "plane_yz", "occ", "mlp"};
  for (int i = 0; i < 7; i++)
    if ((st = check_device_ptr(ptrs[i], names[i])) != OMERF_OK) return st;
  if (n > 0 && !cam && (st = check_device_ptr(rays, "rays")) != OMERF_OK) return st;
  if (n > 0) {
    void *rd = nullptr, *cd = nullptr;
    if ((st = output_ptr(rgb, &rd, "rgb")) != OMERF_OK) return st;
    if ((st = output_ptr(count, &cd, "count")) != OMERF_OK) return st;
    rgb = static_cast<float*>(rd);
    count = static_cast<int32_t*>(cd);
  }
  // A scene on the stack: the same description and geometry as a handle,
  // with its device state placed in the static scratch array.
  omerf_scene s;
  s.desc = *desc;
  choose_coarse_level(&s);
  const size_t cells = (size_t)s.Mc * (size_t)s.Mc;
  const size_t coarse_bytes = (cells * sizeof(float2) + 255) / 256 * 256;
  const size_t nbr_offset = kNoAllocCoarseOffset + coarse_bytes;
  const size_t nbr_bytes = brick_records_bytes(desc);
  if (nbr_offset + nbr_bytes > kNoAllocScratchBytes) {
    set_error("a %d x %d occupancy plane (%zu-byte coarse grid) with %zu bytes of brick neighbour records needs "
              "more than the %zu bytes the no-allocation render reserves",
              desc->occ_res, desc->occ_res, coarse_bytes, nbr_bytes, kNoAllocScratchBytes - kNoAllocCoarseOffset);
    return OMERF_ESHAPE;
  }
  cudaError_t e = cudaGetDevice(&s.device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("no CUDA device: %s", cudaGetErrorString(e));
    return OMERF_EDEVICE;
  }
  unsigned char* scratch = nullptr;
  if ((st = scratch_address(s.device, &scratch)) != OMERF_OK) return st;
  cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, s.device);
  if (s.num_sms < 1) s.num_sms = 1;
  s.counters = reinterpret_cast<unsigned*>(scratch);
  s.state = reinterpret_cast<float*>(scratch + kNoAllocHullOffset);
  s.chull = reinterpret_cast<float2*>(scratch + kNoAllocCoarseOffset);
  s.nbr = nbr_bytes ? reinterpret_cast<int*>(scratch + nbr_offset) : nullptr;
  fill_geo(&s);
  if (n == 0) return OMERF_OK;
  // Every call rebuilds the hulls and neighbour records: the array keeps
  // whatever the previous call (of any scene) left in it.  The work counter
  // is zeroed by the launch.
  cudaStream_t cs = (cudaStream_t)stream;
  const long occ_cells = (long)desc->occ_res * desc->occ_res;
  OMERF_LAUNCH_FAULT();
  hull_kernel<<<1, 1024, 0, cs>>>(s.geo.occ, occ_cells, s.state);
  coarse_hull_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, cs>>>(s.geo.occ, desc->occ_res, s.clog2, s.Mc,
                                                                      s.chull);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "no-allocation hull kernels");
  if (nbr_bytes && (st = build_brick_neighbors(&s, cs)) != OMERF_OK) return st;
  e = launch_march_fwd(&s, cam ? &k : nullptr, rays, n, rgb, count, nullptr, nullptr, 0, nullptr, nullptr, nullptr,
                       cs);
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "no-allocation render launch");
}
