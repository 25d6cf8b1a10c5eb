// packed.cuh -- the fill phase shared by the forward and backward marches.
//
// A warp owns a bundle of 32 rays (lane r owns ray r).  The fill phase walks
// the bundle's rays in order and appends their evaluated lattice samples
// (Sec. 4.1: samples outside the nearest cell's [z_min, z_max] are not
// evaluated) to a 32-entry shared-memory queue that may span several rays.
// Windows of 32 candidates that the coarse occupancy grid proves empty are
// skipped (Sec. 4.4); the remaining candidates are decided one by one with
// the float32 rule of lattice_test, so the queued samples of every ray are
// exactly its first `cap` evaluated samples, in lattice order.
#pragma once

#include "common.cuh"

namespace omerf {

// One queued sample: position, occupancy interval, ray slot, occupancy cell;
// plus the bundle's rays (kept in shared memory, not registers).
struct WarpQueue {
  float4 a[32];   // p.x, p.y, p.z, z_min
  float4 b[32];   // z_max, ray slot (int bits), cell (int bits), unused
  float4 ro[32];  // ray origin, first lattice index (int bits)
  float4 rd[32];  // ray direction, last lattice index (int bits)
  int cap[32];    // maximum samples of the ray
};

// Warp-uniform state of the ray currently being filled.
struct FillState {
  int cur = -1;
  float o[3], d[3];
  int kn, kh, qc, cap;
  int wbase;
  unsigned wmask;
};

// Append evaluated samples to the queue until it holds 32 or no pending ray
// is left.  pend: bitmask of rays with candidates left (the lowest is filled
// first; callers clear bits of rays that stop early).  The rays (origin,
// direction, lattice range, sample cap) are read from q.ro / q.rd / q.cap.
// Returns the number of queued samples.
__device__ __forceinline__ int fill_queue(const Geo& g, int lane, unsigned& pend, FillState& f, WarpQueue& q) {
  int nq = 0;
  while (nq < 32 && pend) {
    const int nxt = __ffs(pend) - 1;
    if (f.cur != nxt) {
      f.cur = nxt;
      const float4 ro = q.ro[nxt], rd = q.rd[nxt];
      f.o[0] = ro.x;
      f.o[1] = ro.y;
      f.o[2] = ro.z;
      f.d[0] = rd.x;
      f.d[1] = rd.y;
      f.d[2] = rd.z;
      f.kn = __float_as_int(ro.w);
      f.kh = __float_as_int(rd.w);
      f.cap = q.cap[nxt];
      f.qc = 0;
      f.wbase = f.kn;
      f.wmask = window_mask(g, f.o, f.d, f.wbase, f.kh, lane);
    }
    // move kn to the next window the coarse grid cannot rule out
    bool have = true;
    for (;;) {
      if (f.kn > f.kh) {
        have = false;
        break;
      }
      int off = f.kn - f.wbase;
      if (off >= 1024) {
        f.wbase = f.kn;
        f.wmask = window_mask(g, f.o, f.d, f.wbase, f.kh, lane);
        off = 0;
      }
      const unsigned rem = f.wmask & (~0u << (off >> 5));
      if (!rem) {
        f.kn = f.wbase + 1024;
        continue;
      }
      const int jn = __ffs(rem) - 1;
      if (jn > (off >> 5)) f.kn = f.wbase + 32 * jn;
      break;
    }
    if (!have || f.qc >= f.cap) {
      pend &= ~(1u << f.cur);
      continue;
    }
    // decide the 32 candidates [kn, kn + 31] of the current ray
    const int kk = f.kn + lane;
    float p[3];
    float2 zb = make_float2(0.0f, 0.0f);
    int cell = 0;
    const bool ok = kk <= f.kh && lattice_test(g, f.o, f.d, kk, p, zb, cell);
    const unsigned m = __ballot_sync(kFull, ok);
    const int take = min(__popc(m), min(f.cap - f.qc, 32 - nq));
    const int rank = __popc(m & lanemask_lt());
    const bool sel = ok && rank < take;
    if (sel) {
      const int pos = nq + rank;
      q.a[pos] = make_float4(p[0], p[1], p[2], zb.x);
      q.b[pos] = make_float4(zb.y, __int_as_float(f.cur), __int_as_float(cell), 0.0f);
    }
    const unsigned rest = m & ~__ballot_sync(kFull, sel);
    nq += take;
    f.qc += take;
    if (f.qc >= f.cap) {
      pend &= ~(1u << f.cur);  // sample cap reached
    } else if (rest) {
      f.kn += __ffs(rest) - 1;  // queue full: resume at the first sample not taken
    } else {
      f.kn += 32;
    }
  }
  __syncwarp();
  return nq;
}

// Segment bookkeeping of a processed queue: lanes with the same ray slot are
// contiguous; segstart is the first lane of this lane's segment.
__device__ __forceinline__ int segment_start(int lane, int r, bool& head) {
  const int rprev = __shfl_up_sync(kFull, r, 1);
  head = lane == 0 || rprev != r;
  const unsigned H = __ballot_sync(kFull, head);
  return 31 - __clz(H & lanemask_le());
}

// Segmented inclusive product scan over the lanes.
__device__ __forceinline__ float seg_prod_scan(float v, int lane, int segstart) {
#pragma unroll
  for (int sh = 1; sh < 32; sh <<= 1) {
    const float u = __shfl_up_sync(kFull, v, sh);
    if (lane - sh >= segstart) v *= u;
  }
  return v;
}

// Segmented inclusive sum scan of 7 channels over the lanes.
__device__ __forceinline__ void seg_sum_scan7(float v[7], int lane, int segstart) {
#pragma unroll
  for (int sh = 1; sh < 32; sh <<= 1) {
#pragma unroll
    for (int c = 0; c < 7; c++) {
      const float u = __shfl_up_sync(kFull, v[c], sh);
      if (lane - sh >= segstart) v[c] += u;
    }
  }
}

}  // namespace omerf
