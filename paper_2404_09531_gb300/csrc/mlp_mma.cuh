// mlp_mma.cuh -- deferred MLP G(F, d) (Eq. 4) on tensor cores, one warp per
// 32 rays: BF16 operands, FP32 accumulation (mma.sync m16n8k16).
//
// Rows are rays (two 16-row tiles), columns are units.  Layer 1 is
// [32 x 48] x [48 x 16] (the 34 inputs padded to 48), layers 2 and 3 take
// the previous layer's accumulators, ReLU'd and rounded to BF16, directly
// as their A fragments (the m16n8 accumulator layout of two adjacent column
// tiles is the m16k16 A layout), so only the input rows and the 3 outputs
// per ray pass through shared memory.
#pragma once

#include "common.cuh"

namespace omerf {

// Per-lane B fragments (B = W^T, k x n) of the three layers, packed BF16x2,
// plus the biases: built once per CTA from the FP32 weights.
struct MlpFrags {
  uint32_t b[32][18];  // [lane][ 0..11 layer 1 (ks, nt, half) | 12..15 layer 2 | 16..17 layer 3 ]
  float bias1[16], bias2[16], bias3[8];
};

// Per-warp staging: input rows (BF16, 48 used columns, 56-wide rows so that
// the fragment loads of the 32 lanes hit 32 different banks), then outputs.
union MlpStage {
  uint32_t X[32][28];
  float Y[32][8];
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Build the fragments from the 883 FP32 weights (all threads of the CTA).
__device__ __forceinline__ void build_mlp_frags(const float* __restrict__ gw, MlpFrags& f) {
  for (int idx = threadIdx.x; idx < 32 * 18; idx += blockDim.x) {
    const int lane = idx / 18, r = idx % 18;
    const int g = lane >> 2, t = lane & 3;
    int layer, nt, half, ks;
    if (r < 12) {
      layer = 1;
      ks = r >> 2;
      nt = (r >> 1) & 1;
      half = r & 1;
    } else if (r < 16) {
      layer = 2;
      ks = 0;
      nt = (r - 12) >> 1;
      half = (r - 12) & 1;
    } else {
      layer = 3;
      ks = 0;
      nt = 0;
      half = r - 16;
    }
    const int n = 8 * nt + g;
    const int k = 16 * ks + 2 * t + 8 * half;
    float lo = 0.0f, hi = 0.0f;
    if (layer == 1) {
      if (k < 34) lo = gw[kOffW1 + n * 34 + k];
      if (k + 1 < 34) hi = gw[kOffW1 + n * 34 + k + 1];
    } else if (layer == 2) {
      lo = gw[kOffW2 + n * 16 + k];
      hi = gw[kOffW2 + n * 16 + k + 1];
    } else if (n < 3) {
      lo = gw[kOffW3 + n * 16 + k];
      hi = gw[kOffW3 + n * 16 + k + 1];
    }
    f.b[lane][r] = pack_bf16x2(lo, hi);
  }
  for (int i = threadIdx.x; i < 40; i += blockDim.x) {
    if (i < 16) f.bias1[i] = gw[kOffB1 + i];
    else if (i < 32) f.bias2[i - 16] = gw[kOffB2 + i - 16];
    else f.bias3[i - 32] = i - 32 < 3 ? gw[kOffB3 + i - 32] : 0.0f;
  }
}

// Stage this lane's MLP input row [F, view encoding] (zeros if !live).
__device__ __forceinline__ void mlp_stage_row(MlpStage& st, int lane, bool live, const float F[7],
                                              const float d[3]) {
  float x[48];
#pragma unroll
  for (int i = 0; i < 48; i++) x[i] = 0.0f;
  if (live) {
#pragma unroll
    for (int i = 0; i < 7; i++) x[i] = F[i];
    view_encoding(d, x + 7);
  }
#pragma unroll
  for (int j = 0; j < 24; j++) st.X[lane][j] = pack_bf16x2(x[2 * j], x[2 * j + 1]);
}

// G for the warp's 32 staged rows; returns this lane's (row = lane) outputs
// after the sigmoid.  All 32 lanes must call it.
__device__ __forceinline__ void mlp_bf16_warp(const MlpFrags& f, MlpStage& st, int lane, float y[3]) {
  __syncwarp();
  const int g = lane >> 2, t = lane & 3;
  float h[2][2][4];
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
      const float b0 = f.bias1[8 * nt + 2 * t], b1 = f.bias1[8 * nt + 2 * t + 1];
      h[mt][nt][0] = b0;
      h[mt][nt][1] = b1;
      h[mt][nt][2] = b0;
      h[mt][nt][3] = b1;
    }
#pragma unroll
  for (int mt = 0; mt < 2; mt++) {
    const int r0 = 16 * mt + g, r1 = r0 + 8;
#pragma unroll
    for (int ks = 0; ks < 3; ks++) {
      const uint32_t a0 = st.X[r0][8 * ks + t], a1 = st.X[r1][8 * ks + t];
      const uint32_t a2 = st.X[r0][8 * ks + 4 + t], a3 = st.X[r1][8 * ks + 4 + t];
#pragma unroll
      for (int nt = 0; nt < 2; nt++)
        mma_bf16_16816(h[mt][nt], a0, a1, a2, a3, f.b[lane][4 * ks + 2 * nt], f.b[lane][4 * ks + 2 * nt + 1]);
    }
  }
  // layer 2: ReLU'd layer-1 accumulators are the A fragments
  float h2[2][2][4];
#pragma unroll
  for (int mt = 0; mt < 2; mt++) {
    const uint32_t a0 = pack_bf16x2(fmaxf(h[mt][0][0], 0.0f), fmaxf(h[mt][0][1], 0.0f));
    const uint32_t a1 = pack_bf16x2(fmaxf(h[mt][0][2], 0.0f), fmaxf(h[mt][0][3], 0.0f));
    const uint32_t a2 = pack_bf16x2(fmaxf(h[mt][1][0], 0.0f), fmaxf(h[mt][1][1], 0.0f));
    const uint32_t a3 = pack_bf16x2(fmaxf(h[mt][1][2], 0.0f), fmaxf(h[mt][1][3], 0.0f));
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
      const float b0 = f.bias2[8 * nt + 2 * t], b1 = f.bias2[8 * nt + 2 * t + 1];
      h2[mt][nt][0] = b0;
      h2[mt][nt][1] = b1;
      h2[mt][nt][2] = b0;
      h2[mt][nt][3] = b1;
      mma_bf16_16816(h2[mt][nt], a0, a1, a2, a3, f.b[lane][12 + 2 * nt], f.b[lane][13 + 2 * nt]);
    }
  }
  // layer 3 (3 of 8 columns used)
  float o[2][4];
#pragma unroll
  for (int mt = 0; mt < 2; mt++) {
    const uint32_t a0 = pack_bf16x2(fmaxf(h2[mt][0][0], 0.0f), fmaxf(h2[mt][0][1], 0.0f));
    const uint32_t a1 = pack_bf16x2(fmaxf(h2[mt][0][2], 0.0f), fmaxf(h2[mt][0][3], 0.0f));
    const uint32_t a2 = pack_bf16x2(fmaxf(h2[mt][1][0], 0.0f), fmaxf(h2[mt][1][1], 0.0f));
    const uint32_t a3 = pack_bf16x2(fmaxf(h2[mt][1][2], 0.0f), fmaxf(h2[mt][1][3], 0.0f));
    const float b0 = f.bias3[2 * t], b1 = f.bias3[2 * t + 1];
    o[mt][0] = b0;
    o[mt][1] = b1;
    o[mt][2] = b0;
    o[mt][3] = b1;
    mma_bf16_16816(o[mt], a0, a1, a2, a3, f.b[lane][16], f.b[lane][17]);
  }
  __syncwarp();  // every lane has read its input rows: the staging becomes the output
#pragma unroll
  for (int mt = 0; mt < 2; mt++) {
    const int r0 = 16 * mt + g;
    st.Y[r0][2 * t] = o[mt][0];
    st.Y[r0][2 * t + 1] = o[mt][1];
    st.Y[r0 + 8][2 * t] = o[mt][2];
    st.Y[r0 + 8][2 * t + 1] = o[mt][3];
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 3; j++) y[j] = sigmoidf_(st.Y[lane][j]);
  __syncwarp();
}

}  // namespace omerf
