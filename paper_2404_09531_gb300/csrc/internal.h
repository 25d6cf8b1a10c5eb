// internal.h -- host-side state and launch entry points shared by the .cu files.
#pragma once

#include <atomic>

#include "common.cuh"
#include "omerf.h"

struct omerf_scene {
  omerf_scene_desc desc;
  omerf::Geo geo;
  float* state = nullptr;          // device: [0..1] occupancy hull (min z_min, max z_max)
  unsigned* counters = nullptr;    // device: per-launch work counters
  float2* chull = nullptr;         // device: coarse max-pooled occupancy grid [Mc][Mc]
  int* nbr = nullptr;              // device: brick neighbour records [n_bricks][8] (brick grids)
  omerf::CamRec* cams = nullptr;   // device: camera records of a multi-camera render [kMaxCams]
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
omerf_status build_brick_neighbors(omerf_scene* s, cudaStream_t stream);
omerf_status validate_camera(const omerf_camera* c, int64_t n);
omerf::Cam to_cam(const omerf_camera* c);

namespace omerf {
__global__ void hull_kernel(const float2* __restrict__ occ, long cells, float* __restrict__ hull);
__global__ void coarse_hull_kernel(const float2* __restrict__ occ, int M, int clog2, int Mc, float2* __restrict__ chull);
}  // namespace omerf
