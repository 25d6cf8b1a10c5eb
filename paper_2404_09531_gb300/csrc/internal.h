// internal.h -- host-side state and launch entry points shared by the .cu files.
#pragma once

#include <atomic>
#include <initializer_list>
#include <utility>

#include "common.cuh"
#include "omerf.h"

struct omerf_scene {
  omerf_scene_desc desc;
  omerf::Geo geo;
  float* state = nullptr;          // device: [0..1] occupancy hull (min z_min, max z_max)
  unsigned* counters = nullptr;    // device: per-launch work counters
  float2* chull = nullptr;         // device: coarse max-pooled occupancy grid [Mc][Mc]
  int* nbr = nullptr;              // device: brick neighbour records [nbx * nby * nbz][8] (brick grids)
  omerf::CamRec* cams = nullptr;   // device: camera records of a multi-camera render [kMaxCams]
  unsigned long long* check = nullptr;  // device [2]: the checking build's counters (NULL otherwise)
  int clog2 = 0, Mc = 1;
  mutable std::atomic<unsigned> seq{0};
  int device = 0;
  int num_sms = 0;
};

namespace omerf {

constexpr int kThreads = 256;      // 8 warps per CTA
constexpr int kCounterSlots = 1024;

// Next work counter of a scene, zeroed on `stream` before the launch that uses it.
unsigned* next_counter(const omerf_scene* s, cudaStream_t stream);

void set_error(const char* fmt, ...);

// runtime.cu: device error word, fault injection, profiler ranges.
constexpr unsigned kErrExtractWait = 1u;   // brick extraction: a tensor load did not complete in time
constexpr unsigned kErrExtractDrain = 2u;  // ... nor the copy in flight when the CTA gave up
constexpr unsigned kErrMlpWait = 4u;       // MLP backward: a tensor-core product did not complete in time
// Device alias of the process-wide error word (page-locked, mapped host
// memory; allocated by the first call), or NULL if it could not be allocated.
unsigned* device_error_word();
// OMERF_ETIMEOUT (with a message) if a kernel reported a bounded wait that
// ran out since the last call, clearing the word; OMERF_OK otherwise.
omerf_status take_device_error();
// True if the comma-separated list in the OMERF_FAULT environment variable
// names `site` (host fault injection for tests).
bool fault_injected(const char* site);
// The status an entry point returns when OMERF_FAULT=launch stands in for a
// failed kernel launch (nothing is launched).
omerf_status injected_launch_failure(const char* entry);
// NVTX range over an entry point's host code.
struct ApiRange {
  explicit ApiRange(const char* name);
  ~ApiRange();
  ApiRange(const ApiRange&) = delete;
  ApiRange& operator=(const ApiRange&) = delete;
};
#define OMERF_API_RANGE() omerf::ApiRange omerf_api_range_(__func__)
// First statement before an entry point's first launch: OMERF_FAULT=launch
// makes the entry point fail there as if the launch had failed.
#define OMERF_LAUNCH_FAULT() \
  do { \
    if (omerf::fault_injected("launch")) return omerf::injected_launch_failure(__func__); \
  } while (0)

cudaError_t launch_march_fwd(const omerf_scene* s, const Cam* cam, const float* rays, long n, float* rgb,
                             int* count, const float* target, const float* dirs, int K, const float lam[3],
                             float* saved, float* loss, cudaStream_t stream);

cudaError_t launch_march_bwd(const omerf_scene* s, const float* rays, const float* target, const float* dirs,
                             long n, int K, const float lam[3], float* saved, const float* grad_scale,
                             float* g_grid, float* g_xy, float* g_xz, float* g_yz, float* g_occ,
                             float* g_mlp, float* loss, cudaStream_t stream);

cudaError_t launch_march_fwd_cams(const omerf_scene* s, const CamRec* cams, int n_cams, long n_super, long n,
                                  float* rgb, int* count, cudaStream_t stream);

int persistent_blocks(const void* kernel, int threads, size_t smem, int num_sms);

}  // namespace omerf

// Host helpers shared by the entry points (scene.cu).
bool aligned(const void* p, size_t a);
omerf_status cuda_fail(cudaError_t e, const char* what);
omerf_status validate_desc(const omerf_scene_desc* d);
void fill_geo(omerf_scene* s);
void choose_coarse_level(omerf_scene* s);
// Bytes of the neighbour records of a brick grid: 32 per brick of the grid.
size_t brick_records_bytes(const omerf_scene_desc* d);
omerf_status build_brick_neighbors(omerf_scene* s, cudaStream_t stream);
omerf_status validate_camera(const omerf_camera* c, int64_t n);
// OMERF_EDEVICE unless p is NULL, device or managed memory.
omerf_status check_device_ptr(const void* p, const char* name);
// The same for every (pointer, name) of a list: the arrays an entry point
// hands to its kernels are checked on the host before anything is launched,
// since a host address read or written by a kernel would fault the device.
omerf_status check_device_ptrs(std::initializer_list<std::pair<const void*, const char*>> ptrs);
// A render output: device memory, or page-locked host memory whose device
// alias is returned in *dev; anything else is OMERF_EDEVICE.
omerf_status output_ptr(void* p, void** dev, const char* name);
omerf::Cam to_cam(const omerf_camera* c);

namespace omerf {
__global__ void hull_kernel(const float2* __restrict__ occ, long cells, float* __restrict__ hull);
__global__ void coarse_hull_kernel(const float2* __restrict__ occ, int M, int clog2, int Mc, float2* __restrict__ chull);
}  // namespace omerf
