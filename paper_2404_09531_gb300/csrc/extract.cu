// extract.cu -- the extraction step after training (Sec. 4.4 and Sec. 5.3):
// everything the real-time scene needs is derived from the trained
// occupancy plane on the device, instead of rendering the training views or
// evaluating densities on a dense grid.
//
//   occupancy grid   voxel (i, j, k) occupied iff some point in it would be
//                    evaluated by the sample rule (Sec. 4.1): an occupancy
//                    cell overlapping its xy footprint has a non-empty
//                    interval meeting the voxel's z-range        Sec. 5.3
//   brick pool       the features of the bricks an occupancy-driven table
//                    allocates, from a dense grid or an older pool Sec. 4.4
//   plane crop       the XZ / YZ plane rows that any evaluated sample can
//                    reach, from the occupancy bounds              Sec. 4.4
#include <cmath>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.h"

namespace omerf {

// One thread per (i, j, 32-voxel word along z).  Bit b of word w is voxel
// k = 32 w + b.  The z edges are FP32 without fused operations, as in the
// definition; cell ranges are exact integer arithmetic.
__global__ void __launch_bounds__(256) occupancy_grid_kernel(const float2* __restrict__ occ, int M, int Nx, int Ny,
                                                            int Nz, float z0, float hz, uint32_t* __restrict__ bits,
                                                            unsigned long long* count) {
  const int W = (Nz + 31) >> 5;
  const long long total = (long long)Nx * Ny * W;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned pop = 0;
  if (id < total) {
    const int w = (int)(id % W);
    const long long ij = id / W;
    const int j = (int)(ij % Ny), i = (int)(ij / Ny);
    const int alo = (int)((long long)i * M / Nx), ahi = (int)(((long long)(i + 1) * M + Nx - 1) / Nx) - 1;
    const int blo = (int)((long long)j * M / Ny), bhi = (int)(((long long)(j + 1) * M + Ny - 1) / Ny) - 1;
    const int k0 = 32 * w, nk = min(32, Nz - k0);
    uint32_t word = 0;
    for (int a = alo; a <= ahi; a++)
      for (int b = blo; b <= bhi; b++) {
        const float2 z = __ldg(occ + (long long)a * M + b);
        if (!(z.x < z.y)) continue;
        for (int t = 0; t < nk; t++) {
          const float zl = __fadd_rn(z0, __fmul_rn((float)(k0 + t), hz));
          const float zh = __fadd_rn(z0, __fmul_rn((float)(k0 + t + 1), hz));
          if (z.x < zh && z.y > zl) word |= 1u << t;
        }
      }
    bits[id] = word;
    pop = __popc(word);
  }
  if (count) {
    for (int s = 16; s > 0; s >>= 1) pop += __shfl_xor_sync(kFull, pop, s);
    if ((threadIdx.x & 31) == 0 && pop) atomicAdd(count, (unsigned long long)pop);
  }
}

// One block per table entry (grid-stride): copies the brick's B^3 texels
// (16-byte words: 2 per float32 texel, 1 per bfloat16 texel).
__global__ void __launch_bounds__(256) extract_bricks_kernel(int Lx, int Ly, int Lz, int B, int nbx, int nby, int nbz,
                                                            const int* __restrict__ table, int n_bricks,
                                                            const uint4* __restrict__ src,
                                                            const int* __restrict__ src_table, int src_n_bricks,
                                                            int words, uint4* __restrict__ pool) {
  const long long entries = (long long)nbx * nby * nbz;
  const int per_brick = B * B * B * words;
  for (long long t = blockIdx.x; t < entries; t += gridDim.x) {
    const int b = __ldg(table + t);
    if (b < 0 || b >= n_bricks) continue;
    const int bk = (int)(t % nbz), bj = (int)((t / nbz) % nby), bi = (int)(t / ((long long)nbz * nby));
    int sb = -1;
    if (src_table) {
      sb = __ldg(src_table + t);
      if (sb >= src_n_bricks) sb = -1;
    }
    uint4* dst = pool + (long long)b * per_brick;
    for (int e = threadIdx.x; e < per_brick; e += blockDim.x) {
      const int q = e % words, v = e / words;
      const int lk = v % B, lj = (v / B) % B, li = v / (B * B);
      const int i = bi * B + li, j = bj * B + lj, k = bk * B + lk;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (i < Lx && j < Ly && k < Lz) {
        if (!src_table) val = __ldg(src + (((long long)i * Ly + j) * Lz + k) * words + q);
        else if (sb >= 0) val = __ldg(src + (long long)sb * per_brick + e);
      }
      dst[e] = val;
    }
  }
}

// Bricks from a dense grid with the tensor memory accelerator: the grid is a
// 4-D tensor (8 channels, z, y, x) whose (8, B, B, B) boxes are exactly the
// pool's bricks ([B][B][B][8], x-major), so one tiled load brings a brick
// into shared memory (vertices beyond the grid arrive as zeros) and one bulk
// store writes it to its pool slot.  One thread per CTA drives the copies
// through two buffers: the store of one brick overlaps the load of the
// next.  Every wait on the load's mbarrier is bounded: a CTA whose wait runs
// out of tries (wait_tries, 2^20 normally) ORs kErrExtractWait into the
// error word, waits (again bounded) for the load still in flight so that no
// copy lands in the shared memory of a finished CTA, and stops; the host
// reports the word as OMERF_ETIMEOUT.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// Poll an mbarrier phase at most `tries` times; true once it has completed.
__device__ __forceinline__ bool wait_parity(unsigned bar, unsigned phase, int tries) {
  for (int t = 0; t < tries; t++) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__global__ void __launch_bounds__(32) extract_bricks_tma_kernel(const __grid_constant__ CUtensorMap src, int nbx,
                                                               int nby, int nbz, int B,
                                                               const int* __restrict__ table, int n_bricks,
                                                               unsigned char* __restrict__ pool,
                                                               unsigned brick_bytes, int wait_tries,
                                                               unsigned* err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar[2];
  if (threadIdx.x != 0) return;
  // tiled copies land on 128-byte aligned buffers (the launch adds the slack)
  unsigned char* buf = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  const unsigned b0 = smem_addr(&bar[0]), b1 = smem_addr(&bar[1]);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0));
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b1));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  unsigned phase[2] = {0u, 0u};
  int slot = 0;
  const long long entries = (long long)nbx * nby * nbz;
  for (long long t = blockIdx.x; t < entries; t += gridDim.x) {
    const int b = __ldg(table + t);
    if (b < 0 || b >= n_bricks) continue;
    const int bk = (int)(t % nbz), bj = (int)((t / nbz) % nby), bi = (int)(t / ((long long)nbz * nby));
    const unsigned bar_s = slot ? b1 : b0;
    const unsigned dst = smem_addr(buf + (size_t)slot * brick_bytes);
    // the bulk store that last read this buffer has finished reading it
    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_s), "r"(brick_bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(&src), "r"(0), "r"(bk * B), "r"(bj * B), "r"(bi * B), "r"(bar_s)
        : "memory");
    if (!wait_parity(bar_s, phase[slot], wait_tries)) {
      // give up on this brick: report, let the load in flight land, stop
      const bool drained = wait_parity(bar_s, phase[slot], 1 << 20);
      if (err) {
        atomicOr_system(err, kErrExtractWait | (drained ? 0u : kErrExtractDrain));
        __threadfence_system();
      }
      break;
    }
    phase[slot] ^= 1u;
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(pool + (size_t)b * brick_bytes),
                 "r"(dst), "r"(brick_bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    slot ^= 1;
  }
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Hull of the non-empty cells (z_min < z_max strictly: a sample needs
// z_min < z < z_max) and the crop rule, in one block.
__global__ void plane_crop_kernel(const float2* __restrict__ occ, long long cells, float pz0, float pz1, int Rz,
                                  int* __restrict__ rows, float* __restrict__ zr) {
  __shared__ float slo[32], shi[32];
  float lo = __int_as_float(0x7f800000), hi = -lo;
  for (long long c = threadIdx.x; c < cells; c += blockDim.x) {
    const float2 z = occ[c];
    if (z.x < z.y) {
      lo = fminf(lo, z.x);
      hi = fmaxf(hi, z.y);
    }
  }
  for (int s = 16; s > 0; s >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(kFull, lo, s));
    hi = fmaxf(hi, __shfl_xor_sync(kFull, hi, s));
  }
  if ((threadIdx.x & 31) == 0) {
    slo[threadIdx.x >> 5] = lo;
    shi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
    lo = fminf(lo, slo[w]);
    hi = fmaxf(hi, shi[w]);
  }
  if (!(lo < hi)) {
    rows[0] = rows[1] = -1;
    zr[0] = zr[1] = 0.0f;
    return;
  }
  // samples lie in (lo, hi); the bilinear stencil reads rows floor(u) and
  // floor(u) + 1, u = (z - pz0) (Rz - 1) / (pz1 - pz0); one row of margin
  const float sc = __fdiv_rn((float)(Rz - 1), __fsub_rn(pz1, pz0));
  const float ulo = __fmul_rn(__fsub_rn(lo, pz0), sc), uhi = __fmul_rn(__fsub_rn(hi, pz0), sc);
  long long k0 = (long long)floorf(ulo) - 1, k1 = (long long)floorf(uhi) + 2;
  k0 = k0 < 0 ? 0 : k0;
  k1 = k1 > Rz - 1 ? Rz - 1 : k1;
  k0 = k0 > Rz - 2 ? Rz - 2 : k0;
  k1 = k1 < k0 + 1 ? k0 + 1 : k1;
  rows[0] = (int)k0;
  rows[1] = (int)k1;
  const float h = __fdiv_rn(__fsub_rn(pz1, pz0), (float)(Rz - 1));
  zr[0] = __fadd_rn(pz0, __fmul_rn((float)k0, h));
  zr[1] = __fadd_rn(pz0, __fmul_rn((float)k1, h));
}

// rows [k0, k1] of an [n_outer][Rz][8] plane -> [n_outer][k1 - k0 + 1][8]
__global__ void __launch_bounds__(256) crop_rows_kernel(const uint4* __restrict__ src, long long n_outer, int Rz,
                                                       int k0, int rows, int words, uint4* __restrict__ dst) {
  const long long total = n_outer * rows * words;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e % words);
    const long long r = (e / words) % rows, o = e / ((long long)words * rows);
    dst[e] = __ldg(src + ((o * Rz + k0 + r) * words + q));
  }
}

}  // namespace omerf

using namespace omerf;

namespace {

int grid_for(long long units, int threads, int cap_blocks) {
  long long g = (units + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap_blocks) g = cap_blocks;
  return (int)g;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  // a function-local static: initialised once, thread-safely
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
    return nullptr;
  }();
  return fn;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  return n;
}

}  // namespace

omerf_status omerf_occupancy_grid(const float aabb[6], const float* occ, int32_t M, const int32_t N[3],
                                  uint32_t* bits, unsigned long long* count, void* stream) {
  OMERF_API_RANGE();
  if (!aabb || !N || !occ || !bits) { set_error("NULL argument"); return OMERF_EINVAL; }
  if (M < 1 || N[0] < 1 || N[1] < 1 || N[2] < 1) { set_error("M and N must be >= 1"); return OMERF_ESHAPE; }
  if (!(aabb[4] < aabb[5]) || !std::isfinite(aabb[4]) || !std::isfinite(aabb[5])) {
    set_error("aabb z-range is empty or not finite");
    return OMERF_EINVAL;
  }
  if (!aligned(occ, 8) || !aligned(bits, 4) || (count && !aligned(count, 8))) {
    set_error("occ must be 8-byte, bits 4-byte, count 8-byte aligned");
    return OMERF_EINVAL;
  }
  const long long words = (long long)N[0] * N[1] * ((N[2] + 31) / 32);
  if (words > (1LL << 40)) { set_error("occupancy grid too large"); return OMERF_ESHAPE; }
  const float hz = (aabb[5] - aabb[4]) / (float)N[2];
  const long long blocks = (words + 255) / 256;
  if (blocks > 0x7fffffffLL) { set_error("occupancy grid too large"); return OMERF_ESHAPE; }
  OMERF_LAUNCH_FAULT();
  omerf_status st = check_device_ptrs({{occ, "occ"}, {bits, "bits"}, {count, "count"}});
  if (st != OMERF_OK) return st;
  occupancy_grid_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const float2*>(occ), M, N[0], N[1], N[2], aabb[4], hz, bits, count);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "occupancy grid launch");
}

omerf_status omerf_extract_bricks(const int32_t grid_res[3], int32_t brick, const int32_t* table, int32_t n_bricks,
                                  const void* src, const int32_t* src_table, int32_t src_n_bricks, int32_t feat_dtype,
                                  void* pool, void* stream) {
  OMERF_API_RANGE();
  if (!grid_res || !table || !src || !pool) { set_error("NULL argument"); return OMERF_EINVAL; }
  // a bounded wait of an earlier extraction that ran out is reported here
  // (if omerf_sync has not reported it already)
  omerf_status prev = take_device_error();
  if (prev != OMERF_OK) return prev;
  if (brick < 2 || brick > 32 || (brick & (brick - 1))) { set_error("brick must be a power of two in 2..32"); return OMERF_EINVAL; }
  for (int a = 0; a < 3; a++)
    if (grid_res[a] < 2) { set_error("grid resolutions must be >= 2"); return OMERF_ESHAPE; }
  if (n_bricks < 0 || src_n_bricks < 0) { set_error("brick counts must be >= 0"); return OMERF_ESHAPE; }
  if (feat_dtype != OMERF_F32 && feat_dtype != OMERF_BF16) { set_error("feat_dtype must be OMERF_F32 or OMERF_BF16"); return OMERF_EINVAL; }
  if (!aligned(src, 16) || !aligned(pool, 16) || !aligned(table, 4) || (src_table && !aligned(src_table, 4))) {
    set_error("feature arrays must be 16-byte aligned");
    return OMERF_EINVAL;
  }
  int nb[3];
  for (int a = 0; a < 3; a++) nb[a] = (grid_res[a] + brick - 1) / brick;
  const long long entries = (long long)nb[0] * nb[1] * nb[2];
  const int words = feat_dtype == OMERF_F32 ? 2 : 1;
  const size_t esize = feat_dtype == OMERF_F32 ? 4 : 2;
  const size_t brick_bytes = (size_t)brick * brick * brick * 8 * esize;
  PFN_cuTensorMapEncodeTiled_v12000 encode = src_table ? nullptr : tensor_map_encoder();
  if (encode && brick_bytes <= 32768 && n_bricks > 0) {
    // a dense source: tiled tensor-memory-accelerator copies
    CUtensorMap map;
    const cuuint64_t dims[4] = {8, (cuuint64_t)grid_res[2], (cuuint64_t)grid_res[1], (cuuint64_t)grid_res[0]};
    const cuuint64_t strides[3] = {8 * esize, (cuuint64_t)grid_res[2] * 8 * esize,
                                   (cuuint64_t)grid_res[1] * grid_res[2] * 8 * esize};
    const cuuint32_t box[4] = {8, (cuuint32_t)brick, (cuuint32_t)brick, (cuuint32_t)brick};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(&map, feat_dtype == OMERF_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                             : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                              4, const_cast<void*>(src), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS) {
      const size_t smem = 2 * brick_bytes + 128;
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(extract_bricks_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      const int blocks = grid_for(entries, 1, 6 * sm_count());
      // OMERF_FAULT=extract_wait: every CTA's first wait gives up at once
      // (the load still completes and is waited for), for tests of the report
      const int tries = fault_injected("extract_wait") ? 0 : (1 << 20);
      OMERF_LAUNCH_FAULT();
      const omerf_status st = check_device_ptrs({{table, "table"}, {src, "src"}, {pool, "pool"}});
      if (st != OMERF_OK) return st;
      extract_bricks_tma_kernel<<<blocks, 32, smem, (cudaStream_t)stream>>>(
          map, nb[0], nb[1], nb[2], brick, table, n_bricks, static_cast<unsigned char*>(pool), (unsigned)brick_bytes,
          tries, device_error_word());
      cudaError_t e = cudaGetLastError();
      return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "brick extraction launch");
    }
  }
  OMERF_LAUNCH_FAULT();
  const omerf_status st = check_device_ptrs({{table, "table"}, {src, "src"}, {src_table, "src_table"}, {pool, "pool"}});
  if (st != OMERF_OK) return st;
  const int blocks = grid_for(entries, 1, 16 * sm_count());
  extract_bricks_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(
      grid_res[0], grid_res[1], grid_res[2], brick, nb[0], nb[1], nb[2], table, n_bricks,
      static_cast<const uint4*>(src), src_table, src_n_bricks, words, static_cast<uint4*>(pool));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "brick extraction launch");
}

int32_t omerf_tma_available(void) { return tensor_map_encoder() != nullptr ? 1 : 0; }

omerf_status omerf_plane_crop_rows(const float plane_z[2], int32_t Rz, const float* occ, int32_t M, int32_t* rows,
                                   float* z_range, void* stream) {
  OMERF_API_RANGE();
  if (!plane_z || !occ || !rows || !z_range) { set_error("NULL argument"); return OMERF_EINVAL; }
  if (Rz < 2 || M < 1) { set_error("Rz must be >= 2 and M >= 1"); return OMERF_ESHAPE; }
  if (!(plane_z[0] < plane_z[1]) || !std::isfinite(plane_z[0]) || !std::isfinite(plane_z[1])) {
    set_error("plane_z is empty or not finite");
    return OMERF_EINVAL;
  }
  if (!aligned(occ, 8) || !aligned(rows, 4) || !aligned(z_range, 4)) { set_error("misaligned argument"); return OMERF_EINVAL; }
  OMERF_LAUNCH_FAULT();
  omerf_status st = check_device_ptrs({{occ, "occ"}, {rows, "rows"}, {z_range, "z_range"}});
  if (st != OMERF_OK) return st;
  plane_crop_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(reinterpret_cast<const float2*>(occ), (long long)M * M,
                                                          plane_z[0], plane_z[1], Rz, rows, z_range);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "plane crop launch");
}

omerf_status omerf_crop_planes(const void* src, int64_t n_outer, int32_t Rz, int32_t k0, int32_t k1,
                               int32_t feat_dtype, void* dst, void* stream) {
  OMERF_API_RANGE();
  if (!src || !dst) { set_error("NULL argument"); return OMERF_EINVAL; }
  if (n_outer < 1 || Rz < 2 || k0 < 0 || k1 <= k0 || k1 > Rz - 1) {
    set_error("need n_outer >= 1 and 0 <= k0 < k1 <= Rz - 1");
    return OMERF_ESHAPE;
  }
  if (feat_dtype != OMERF_F32 && feat_dtype != OMERF_BF16) { set_error("feat_dtype must be OMERF_F32 or OMERF_BF16"); return OMERF_EINVAL; }
  if (!aligned(src, 16) || !aligned(dst, 16)) { set_error("planes must be 16-byte aligned"); return OMERF_EINVAL; }
  const int words = feat_dtype == OMERF_F32 ? 2 : 1;
  const long long total = (long long)n_outer * (k1 - k0 + 1) * words;
  OMERF_LAUNCH_FAULT();
  omerf_status st = check_device_ptrs({{src, "src"}, {dst, "dst"}});
  if (st != OMERF_OK) return st;
  crop_rows_kernel<<<grid_for(total, 256, 8 * sm_count()), 256, 0, (cudaStream_t)stream>>>(
      static_cast<const uint4*>(src), (long long)n_outer, Rz, k0, k1 - k0 + 1, words, static_cast<uint4*>(dst));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OMERF_OK : cuda_fail(e, "plane crop launch");
}
