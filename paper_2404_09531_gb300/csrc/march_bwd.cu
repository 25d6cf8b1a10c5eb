// march_bwd.cu -- training backward: deferred-MLP backward and the
// recompute-in-backward march (sm_103a).
//
// Per bundle of 32 consecutive rays (one warp):
//  1. the warp recomputes the deferred MLP G(F, d) (Eq. 4) and the
//     smoothness evaluations G(F, s_k) (Eqs. 9-10) of its 32 rays, forms
//     dL/dC of the Charbonnier loss (Eq. 12) and backpropagates to dL/dF,
//     dL/dT_N and the MLP weights; every MLP product is a warp-level
//     tensor-core product over the 32 rays (mma.sync TF32 with split
//     operands), the weight gradient accumulating in registers; in a fused
//     training step it also adds the Charbonnier and smoothness loss terms;
//  2. the warp re-marches every ray of the bundle exactly like the forward
//     (same lattice windows, same product scan) for its saved sample count,
//     and converts dL/dF into per-sample gradients:
//        dL/d(alpha_hat_i) = T_i g.x_i - [g.(F - A_<=i) + g_T T_N] / (1 - alpha_hat_i)
//     (A_<=i = prefix sum of w x, by a lane scan), then chains through Eq. 3
//     and Eq. 6 and scatter-adds into the grid, planes and z-bounds with
//     vector float atomics.  No per-sample state is stored between passes.
#include "internal.h"
#include "mma_tf32.cuh"
#include "packed.cuh"

namespace omerf {

constexpr int kBwdThreads = 128;   // 4 warps per CTA
#ifndef OMERF_FOLD
#define OMERF_FOLD 3       // lanes folded into one reduction
#endif
constexpr int kRow = 101;          // staged floats per ray: x 34, h1 16, h2 16, g1 16, g2 16, g3 3

struct BwdArgs {
  const float* rays;
  const float* target;
  const float* dirs;
  int K;
  long n, n_bundles;
  float lam_rgb, lam_smooth;  // divided by n
  float* saved;
  const float* grad_scale;
  float* g_grid;
  float* g_xy;
  float* g_xz;
  float* g_yz;
  float* g_occ;
  float* g_mlp;
  float* loss;  // device [4] or NULL: the Charbonnier and smoothness terms are added (fused step)
  unsigned* counter;
};

// ---------------------------------------------------------------------------
// The per-ray deferred MLP of the backward, forward and backward, as
// warp-level products on tensor cores: the warp's 32 rays are the rows of
// every product (two m16 tiles), so each layer is one [32 x K] x [K x N]
// product, run as mma.sync m16n8k8 TF32 with split operands (about FP32
// accurate, see mma3).  Activations and deltas pass between layers through
// the staged rows, which the weight-gradient products read afterwards.
//
// B fragments of the weights, per lane (b0, b1) = (B[t][g], B[t + 4][g]) of
// each k8 x n8 block, g = lane / 4, t = lane % 4:
//   L1  [input][unit]  = W1[unit][input]    5 k-blocks x 2 n-blocks
//   L2  [unit1][unit2] = W2[unit2][unit1]   2 x 2
//   B2  [unit2][unit1] = W2[unit2][unit1]   2 x 2   (g1 = G2 . W2)
//   B1  [unit1][input] = W1[unit1][input]   2 x 1   (dL/dF = G1 . W1[:, :7])
// W3 (3 x 16) is read from a compact copy.
constexpr int kFragL1 = 0, kFragL2 = 10, kFragB2 = 14, kFragB1 = 18, kFrags = 20;

struct MlpBwdShared {
  float2 frag[kFrags][32];
  float w3[48];
  float b1[16], b2[16], b3[4];
};

__device__ __forceinline__ void build_bwd_frags(const float* __restrict__ gw, MlpBwdShared& S) {
  for (int i = threadIdx.x; i < kFrags * 32; i += blockDim.x) {
    const int f = i >> 5, l = i & 31, g = l >> 2, t = l & 3;
    float v0, v1;
    if (f < kFragL2) {
      const int s = f >> 1, j = f & 1, u = 8 * j + g, c0 = 8 * s + t, c1 = c0 + 4;
      v0 = c0 < 34 ? gw[kOffW1 + u * 34 + c0] : 0.0f;
      v1 = c1 < 34 ? gw[kOffW1 + u * 34 + c1] : 0.0f;
    } else if (f < kFragB2) {
      const int s = (f - kFragL2) >> 1, j = (f - kFragL2) & 1, u2 = 8 * j + g;
      v0 = gw[kOffW2 + u2 * 16 + 8 * s + t];
      v1 = gw[kOffW2 + u2 * 16 + 8 * s + t + 4];
    } else if (f < kFragB1) {
      const int s = (f - kFragB2) >> 1, j = (f - kFragB2) & 1, u1 = 8 * j + g;
      v0 = gw[kOffW2 + (8 * s + t) * 16 + u1];
      v1 = gw[kOffW2 + (8 * s + t + 4) * 16 + u1];
    } else {
      const int s = f - kFragB1;
      v0 = g < 7 ? gw[kOffW1 + (8 * s + t) * 34 + g] : 0.0f;
      v1 = g < 7 ? gw[kOffW1 + (8 * s + t + 4) * 34 + g] : 0.0f;
    }
    S.frag[f][l] = make_float2(v0, v1);
  }
  for (int i = threadIdx.x; i < 48 + 36; i += blockDim.x) {
    if (i < 48) S.w3[i] = gw[kOffW3 + i];
    else if (i < 64) S.b1[i - 48] = gw[kOffB1 + i - 48];
    else if (i < 80) S.b2[i - 64] = gw[kOffB2 + i - 64];
    else S.b3[i - 80] = i - 80 < 3 ? gw[kOffB3 + i - 80] : 0.0f;
  }
}

// This lane's staged input row [F (7), view encoding (27)], zeros if !live.
__device__ __forceinline__ void stage_x(float* __restrict__ row, bool live, const float F[7], const float d[3]) {
  float x[34];
#pragma unroll
  for (int i = 0; i < 34; i++) x[i] = 0.0f;
  if (live) {
#pragma unroll
    for (int i = 0; i < 7; i++) x[i] = F[i];
    view_encoding(d, x + 7);
  }
#pragma unroll
  for (int i = 0; i < 34; i++) row[i] = x[i];
}

// ---------------------------------------------------------------------------
// Weight-gradient accumulation on tensor cores.  The MLP weight gradient of a
// warp's 32 staged rows is three small GEMMs whose reduction dimension is the
// rays:  [dW1 | db1] (16 x 35) += G1^T [16 x 32] . [X | 1] [32 x 35],
//        [dW2 | db2] (16 x 17) += G2^T . [H1 | 1],
//        [dW3 | db3]^T (17 x 3) += [H2 | 1]^T . G3.
// They run as mma.sync m16n8k8 TF32 with each operand split into a TF32 part
// and a TF32 residual (three products, hi.hi + hi.lo + lo.hi), about FP32
// accurate; the FP32 accumulators stay in registers for the whole persistent
// loop, in the m16n8 accumulator layout (c0: row g, col 2t; c1: row g, col
// 2t+1; c2, c3: row g + 8), g = lane / 4, t = lane % 4.
struct DwAcc {
  float w1[5][4];  // units x (34 inputs, bias, pad): 5 column tiles of 8
  float w2[3][4];  // units x (16 inputs, bias, pad)
  float w3[2][4];  // (16 inputs, bias, pad) x (3 outputs, pad): 2 row tiles
};

__device__ __forceinline__ void zero_acc(DwAcc& acc) {
#pragma unroll
  for (int i = 0; i < 4; i++) {
#pragma unroll
    for (int j = 0; j < 5; j++) acc.w1[j][i] = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; j++) acc.w2[j][i] = 0.0f;
#pragma unroll
    for (int j = 0; j < 2; j++) acc.w3[j][i] = 0.0f;
  }
}

// Add the warp's 32 staged rows (x 0..33, h1 34..49, h2 50..65, g1 66..81,
// g2 82..97, g3 98..100) to the accumulators.  All 32 lanes must call it.
__device__ __forceinline__ void accumulate_mma(const float* __restrict__ rows, int lane, DwAcc& acc) {
  __syncwarp();
  const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
  for (int s = 0; s < 4; s++) {  // rays 8 s .. 8 s + 7 (the k dimension)
    const float* r0 = rows + (8 * s + t) * kRow;
    const float* r1 = rows + (8 * s + t + 4) * kRow;
    uint32_t ah[4], al[4];
    // layer 1: A = G1^T (unit x ray), B = [X | 1] (ray x input)
    split_tf32(r0[66 + g], ah[0], al[0]);
    split_tf32(r0[74 + g], ah[1], al[1]);
    split_tf32(r1[66 + g], ah[2], al[2]);
    split_tf32(r1[74 + g], ah[3], al[3]);
#pragma unroll
    for (int j = 0; j < 5; j++) {
      const int c = 8 * j + g;
      const float b0 = c < 34 ? r0[c] : (c == 34 ? 1.0f : 0.0f);
      const float b1 = c < 34 ? r1[c] : (c == 34 ? 1.0f : 0.0f);
      mma3(acc.w1[j], ah, al, b0, b1);
    }
    // layer 2: A = G2^T, B = [H1 | 1]
    split_tf32(r0[82 + g], ah[0], al[0]);
    split_tf32(r0[90 + g], ah[1], al[1]);
    split_tf32(r1[82 + g], ah[2], al[2]);
    split_tf32(r1[90 + g], ah[3], al[3]);
#pragma unroll
    for (int j = 0; j < 3; j++) {
      const int c = 8 * j + g;
      const float b0 = c < 16 ? r0[34 + c] : (c == 16 ? 1.0f : 0.0f);
      const float b1 = c < 16 ? r1[34 + c] : (c == 16 ? 1.0f : 0.0f);
      mma3(acc.w2[j], ah, al, b0, b1);
    }
    // layer 3 (transposed): A = [H2 | 1]^T (input x ray), B = G3 (ray x output)
    const float b0 = g < 3 ? r0[98 + g] : 0.0f;
    const float b1 = g < 3 ? r1[98 + g] : 0.0f;
#pragma unroll
    for (int mt = 0; mt < 2; mt++) {
      const int i0 = 16 * mt + g, i1 = i0 + 8;
      split_tf32(i0 < 16 ? r0[50 + i0] : (i0 == 16 ? 1.0f : 0.0f), ah[0], al[0]);
      split_tf32(i1 < 16 ? r0[50 + i1] : (i1 == 16 ? 1.0f : 0.0f), ah[1], al[1]);
      split_tf32(i0 < 16 ? r1[50 + i0] : (i0 == 16 ? 1.0f : 0.0f), ah[2], al[2]);
      split_tf32(i1 < 16 ? r1[50 + i1] : (i1 == 16 ? 1.0f : 0.0f), ah[3], al[3]);
      mma3(acc.w3[mt], ah, al, b0, b1);
    }
  }
  __syncwarp();
}

// Store the accumulators as weight-gradient sums indexed like the 883
// parameters (every parameter is held by exactly one lane and element).
__device__ __forceinline__ void store_acc(const DwAcc& acc, int lane, float* __restrict__ dW) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const int r = g + 8 * (e >> 1), cc = 2 * t + (e & 1);
#pragma unroll
    for (int j = 0; j < 5; j++) {
      const int c = 8 * j + cc;  // unit r, input c
      if (c < 34) dW[kOffW1 + r * 34 + c] = acc.w1[j][e];
      else if (c == 34) dW[kOffB1 + r] = acc.w1[j][e];
    }
#pragma unroll
    for (int j = 0; j < 3; j++) {
      const int c = 8 * j + cc;
      if (c < 16) dW[kOffW2 + r * 16 + c] = acc.w2[j][e];
      else if (c == 16) dW[kOffB2 + r] = acc.w2[j][e];
    }
#pragma unroll
    for (int mt = 0; mt < 2; mt++) {
      const int i = 16 * mt + r;  // input i, output cc
      if (cc < 3) {
        if (i < 16) dW[kOffW3 + cc * 16 + i] = acc.w3[mt][e];
        else if (i == 16) dW[kOffB3 + cc] = acc.w3[mt][e];
      }
    }
  }
}

// G for the warp's 32 staged rows (x in columns 0..33): writes h1 (34..49),
// h2 (50..65) and this lane's sigmoid outputs y.  All 32 lanes call it.
__device__ __forceinline__ void warp_mlp_forward(float* __restrict__ rows, const MlpBwdShared& S, int lane,
                                                 float y[3]) {
  __syncwarp();
  const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
  for (int mt = 0; mt < 2; mt++) {
    float* r0 = rows + (16 * mt + g) * kRow;
    float* r1 = r0 + 8 * kRow;
    float c[2][4];
#pragma unroll
    for (int j = 0; j < 2; j++) {
      c[j][0] = c[j][2] = S.b1[8 * j + 2 * t];
      c[j][1] = c[j][3] = S.b1[8 * j + 2 * t + 1];
    }
#pragma unroll
    for (int s = 0; s < 5; s++) {
      uint32_t ah[4], al[4];
      load_a(r0, r1, 8 * s + t, 8 * s + t < 34, 8 * s + t + 4 < 34, ah, al);
#pragma unroll
      for (int j = 0; j < 2; j++) {
        const float2 b = S.frag[kFragL1 + 2 * s + j][lane];
        mma3(c[j], ah, al, b.x, b.y);
      }
    }
#pragma unroll
    for (int j = 0; j < 2; j++) {
      const int u = 34 + 8 * j + 2 * t;
      r0[u] = fmaxf(c[j][0], 0.0f);
      r0[u + 1] = fmaxf(c[j][1], 0.0f);
      r1[u] = fmaxf(c[j][2], 0.0f);
      r1[u + 1] = fmaxf(c[j][3], 0.0f);
    }
  }
  __syncwarp();
#pragma unroll 1
  for (int mt = 0; mt < 2; mt++) {
    float* r0 = rows + (16 * mt + g) * kRow;
    float* r1 = r0 + 8 * kRow;
    float c[2][4];
#pragma unroll
    for (int j = 0; j < 2; j++) {
      c[j][0] = c[j][2] = S.b2[8 * j + 2 * t];
      c[j][1] = c[j][3] = S.b2[8 * j + 2 * t + 1];
    }
#pragma unroll
    for (int s = 0; s < 2; s++) {
      uint32_t ah[4], al[4];
      load_a(r0, r1, 34 + 8 * s + t, true, true, ah, al);
#pragma unroll
      for (int j = 0; j < 2; j++) {
        const float2 b = S.frag[kFragL2 + 2 * s + j][lane];
        mma3(c[j], ah, al, b.x, b.y);
      }
    }
#pragma unroll
    for (int j = 0; j < 2; j++) {
      const int u = 50 + 8 * j + 2 * t;
      r0[u] = fmaxf(c[j][0], 0.0f);
      r0[u + 1] = fmaxf(c[j][1], 0.0f);
      r1[u] = fmaxf(c[j][2], 0.0f);
      r1[u + 1] = fmaxf(c[j][3], 0.0f);
    }
  }
  __syncwarp();
  // layer 3: B[k = unit2][n = output] = W3[output][unit2], outputs 0..2 of 8
#pragma unroll 1
  for (int mt = 0; mt < 2; mt++) {
    float* r0 = rows + (16 * mt + g) * kRow;
    float* r1 = r0 + 8 * kRow;
    float c[4];
    c[0] = c[2] = 2 * t < 3 ? S.b3[2 * t] : 0.0f;
    c[1] = c[3] = 2 * t + 1 < 3 ? S.b3[2 * t + 1] : 0.0f;
#pragma unroll
    for (int s = 0; s < 2; s++) {
      uint32_t ah[4], al[4];
      load_a(r0, r1, 50 + 8 * s + t, true, true, ah, al);
      const float b0 = g < 3 ? S.w3[g * 16 + 8 * s + t] : 0.0f;
      const float b1 = g < 3 ? S.w3[g * 16 + 8 * s + t + 4] : 0.0f;
      mma3(c, ah, al, b0, b1);
    }
    // pre-activations into the g3 columns (this lane's row is read back below)
    if (2 * t < 3) {
      r0[98 + 2 * t] = c[0];
      r1[98 + 2 * t] = c[2];
    }
    if (2 * t + 1 < 3) {
      r0[98 + 2 * t + 1] = c[1];
      r1[98 + 2 * t + 1] = c[3];
    }
  }
  __syncwarp();
  const float* row = rows + lane * kRow;
#pragma unroll
  for (int j = 0; j < 3; j++) y[j] = sigmoidf_(row[98 + j]);
}

// Backpropagate this lane's gy through the staged evaluation: writes the
// deltas g3 (98..100), g2 (82..97) and g1 (66..81).  A ReLU unit is active
// iff its staged output is positive.  All 32 lanes call it.
__device__ __forceinline__ void warp_mlp_backward(float* __restrict__ rows, const MlpBwdShared& S, int lane,
                                                  const float y[3], const float gy[3]) {
  const int g = lane >> 2, t = lane & 3;
  {
    float* row = rows + lane * kRow;
#pragma unroll
    for (int j = 0; j < 3; j++) row[98 + j] = gy[j] * y[j] * (1.0f - y[j]);
  }
  __syncwarp();
  // g2 = (G3 . W3) masked: K = 3 outputs (one k8 block, rows t < 3)
#pragma unroll 1
  for (int mt = 0; mt < 2; mt++) {
    float* r0 = rows + (16 * mt + g) * kRow;
    float* r1 = r0 + 8 * kRow;
    uint32_t ah[4], al[4];
    load_a(r0, r1, 98 + t, t < 3, false, ah, al);
#pragma unroll
    for (int j = 0; j < 2; j++) {
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      const float b0 = t < 3 ? S.w3[t * 16 + 8 * j + g] : 0.0f;
      mma3(c, ah, al, b0, 0.0f);
      const int u = 8 * j + 2 * t;
      r0[82 + u] = r0[50 + u] > 0.0f ? c[0] : 0.0f;
      r0[83 + u] = r0[51 + u] > 0.0f ? c[1] : 0.0f;
      r1[82 + u] = r1[50 + u] > 0.0f ? c[2] : 0.0f;
      r1[83 + u] = r1[51 + u] > 0.0f ? c[3] : 0.0f;
    }
  }
  __syncwarp();
  // g1 = (G2 . W2) masked
#pragma unroll 1
  for (int mt = 0; mt < 2; mt++) {
    float* r0 = rows + (16 * mt + g) * kRow;
    float* r1 = r0 + 8 * kRow;
    float c[2][4] = {{0.0f, 0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f, 0.0f}};
#pragma unroll
    for (int s = 0; s < 2; s++) {
      uint32_t ah[4], al[4];
      load_a(r0, r1, 82 + 8 * s + t, true, true, ah, al);
#pragma unroll
      for (int j = 0; j < 2; j++) {
        const float2 b = S.frag[kFragB2 + 2 * s + j][lane];
        mma3(c[j], ah, al, b.x, b.y);
      }
    }
#pragma unroll
    for (int j = 0; j < 2; j++) {
      const int u = 8 * j + 2 * t;
      r0[66 + u] = r0[34 + u] > 0.0f ? c[j][0] : 0.0f;
      r0[67 + u] = r0[35 + u] > 0.0f ? c[j][1] : 0.0f;
      r1[66 + u] = r1[34 + u] > 0.0f ? c[j][2] : 0.0f;
      r1[67 + u] = r1[35 + u] > 0.0f ? c[j][3] : 0.0f;
    }
  }
  __syncwarp();
}

// dL/dF = G1 . W1[:, :7] for the warp's rows, added into this lane's gF.
// Uses the x columns 0..6 as scratch: call after the weight-gradient products.
__device__ __forceinline__ void warp_mlp_input_grad(float* __restrict__ rows, const MlpBwdShared& S, int lane,
                                                    float gF[7]) {
  __syncwarp();
  const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
  for (int mt = 0; mt < 2; mt++) {
    float* r0 = rows + (16 * mt + g) * kRow;
    float* r1 = r0 + 8 * kRow;
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int s = 0; s < 2; s++) {
      uint32_t ah[4], al[4];
      load_a(r0, r1, 66 + 8 * s + t, true, true, ah, al);
      const float2 b = S.frag[kFragB1 + s][lane];
      mma3(c, ah, al, b.x, b.y);
    }
    __syncwarp();  // every lane has read its g1 columns of these rows
    if (2 * t < 7) {
      r0[2 * t] = c[0];
      r1[2 * t] = c[2];
    }
    if (2 * t + 1 < 7) {
      r0[2 * t + 1] = c[1];
      r1[2 * t + 1] = c[3];
    }
  }
  __syncwarp();
  const float* row = rows + lane * kRow;
#pragma unroll
  for (int i = 0; i < 7; i++) gF[i] += row[i];
}

// Pair folding by stencil: lanes whose samples share the key (the base grid
// vertex, or a plane's base texel) share every texel of that stencil, so a
// lane at an even position of a run of equal keys adds its right neighbour's
// contribution and the neighbour issues nothing.
__device__ __forceinline__ void pair_fold_info(int key, int lane, bool& emit, int& nfold) {
  const int kprev = __shfl_up_sync(kFull, key, 1);
  const unsigned H = __ballot_sync(kFull, lane == 0 || kprev != key);
  const int runstart = 31 - __clz(H & lanemask_le());
  const unsigned later = H & ~lanemask_le();
  const int runend = later ? __ffs(later) - 1 : 32;
  emit = ((lane - runstart) % OMERF_FOLD) == 0;
  nfold = emit ? min(OMERF_FOLD, runend - lane) : 0;  // lanes [lane, lane + nfold) share the stencil
}

__device__ __forceinline__ void red8(float* base, int off, const float v[8]) {
  float4* q = reinterpret_cast<float4*>(base + off);
  atomicAdd(q, make_float4(v[0], v[1], v[2], v[3]));
  atomicAdd(q + 1, make_float4(v[4], v[5], v[6], v[7]));
}

// Per-warp shared state of the packed backward re-march of 32 rays.
struct WarpBwd {
  WarpQueue q;
  float F[32][8];    // per-ray F (7)
  float G[32][8];    // per-ray dL/dF (7), dL/dT_N
  float A[32][8];    // per-ray running prefix of w x
  float T[32];       // per-ray transmittance so far
  float TN[32];
  int cnt[32];       // per-ray sample count of the forward
  int done[32];      // per-ray samples already processed
};

// Re-march a bundle exactly like the forward (same lattice candidates, same
// decisions, the first `count` evaluated samples of each ray) and scatter the
// per-sample gradients.  Lane r owns ray r of the bundle.
template <class FT, bool SPARSE>
__device__ __forceinline__ void march_bundle_bwd(const Geo& g, const BwdArgs& a, int lane, const float o[3],
                                                 const float d[3], int klo, int khi, bool live, WarpBwd& ws) {
  ws.q.ro[lane] = make_float4(o[0], o[1], o[2], __int_as_float(klo));
  ws.q.rd[lane] = make_float4(d[0], d[1], d[2], __int_as_float(khi));
  ws.q.cap[lane] = ws.cnt[lane];
  unsigned pend = __ballot_sync(kFull, live);
  FillState f;
  __syncwarp();
  while (pend) {
    const int nq = fill_queue(g, lane, pend, f, ws.q);
    if (nq == 0) break;
    const bool act = lane < nq;
    const float4 qa = ws.q.a[lane], qb = ws.q.b[lane];
    const int r = act ? __float_as_int(qb.y) : 32;
    SampleAct s;
    s.ah = 0.0f;
    s.alpha = 0.0f;
    s.branch = 0;
#pragma unroll
    for (int c = 0; c < 7; c++) s.x[c] = 0.0f;
    int goff[8], poff[12];
    float gw[8], pw[12];
    if (act) {
      const float p[3] = {qa.x, qa.y, qa.z};
      grid_stencil<SPARSE>(g, p, goff, gw);
      plane_stencil(g, p, poff, pw);
      float t[8];
#pragma unroll
      for (int c = 0; c < 8; c++) t[c] = 0.0f;
#pragma unroll
      for (int c = 0; c < 8; c++) {
        if (goff[c] < 0 || !check_range(g, 0, goff[c])) continue;
        float v[8];
        Texel<FT>::load(g.grid, goff[c], v);
#pragma unroll
        for (int ch = 0; ch < 8; ch++) t[ch] = fmaf(gw[c], v[ch], t[ch]);
      }
#pragma unroll
      for (int q = 0; q < 3; q++) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
          float v[8];
          if (!check_range(g, 1 + q, poff[4 * q + c])) continue;
          Texel<FT>::load(plane_base(g, q), poff[4 * q + c], v);
#pragma unroll
          for (int ch = 0; ch < 8; ch++) t[ch] = fmaf(pw[4 * q + c], v[ch], t[ch]);
        }
      }
      activate(g, t, p[2], make_float2(qa.w, qb.x), s);
    }
    bool head;
    const int segstart = segment_start(lane, r, head);
    const float P = seg_prod_scan(1.0f - s.ah, lane, segstart);
    float Pex = __shfl_up_sync(kFull, P, 1);
    if (head) Pex = 1.0f;
    const float Tprev = act ? ws.T[r] : 1.0f;
    const float Ti = Tprev * Pex, Tn = Tprev * P;
    const float w = act ? Ti * s.ah : 0.0f;
    float Ai[7];
#pragma unroll
    for (int c = 0; c < 7; c++) Ai[c] = w * s.x[c];
    seg_sum_scan7(Ai, lane, segstart);
    float dt[8];
#pragma unroll
    for (int c = 0; c < 8; c++) dt[c] = 0.0f;
    if (act) {
      const int idx = ws.done[r] + (lane - segstart);
      const bool last = idx == ws.cnt[r] - 1;
      const float gT = ws.G[r][7], TN = ws.TN[r];
      float gx = 0.0f, suffix = gT * TN;
#pragma unroll
      for (int c = 0; c < 7; c++) {
        Ai[c] += ws.A[r][c];
        const float gc = ws.G[r][c];
        gx = fmaf(gc, s.x[c], gx);
        suffix = fmaf(gc, ws.F[r][c] - Ai[c], suffix);
      }
      const float dah = last ? Ti * (gx - gT) : Ti * gx - suffix / (1.0f - s.ah);
      const float dsig = dah * s.Mv * (1.0f - s.alpha);
      dt[0] = dsig * s.sigma;
#pragma unroll
      for (int c = 0; c < 7; c++) dt[c + 1] = w * ws.G[r][c] * s.x[c] * (1.0f - s.x[c]);
      if (a.g_occ && s.branch != 0) {
        const float dM = dah * s.alpha;
        const float dz = (s.branch == 1 ? -2.0f : 2.0f) * s.r * g.inv_eps;
        atomicAdd(a.g_occ + 2 * __float_as_int(qb.z) + (s.branch == 1 ? 0 : 1), dM * dz);
      }
    }
    // gradient scatter (all lanes; inactive lanes contribute nothing)
    // neighbours' dL/dt and weights, lanes +1 .. +OMERF_FOLD-1
    float dtn[OMERF_FOLD - 1][8];
#pragma unroll
    for (int j = 1; j < OMERF_FOLD; j++)
#pragma unroll
      for (int c = 0; c < 8; c++) dtn[j - 1][c] = __shfl_down_sync(kFull, dt[c], j);
    if (a.g_grid) {
      bool emit;
      int nfold;
      pair_fold_info(act && goff[0] >= 0 ? goff[0] : -1 - lane, lane, emit, nfold);
#pragma unroll
      for (int c = 0; c < 8; c++) {
        float v[8];
#pragma unroll
        for (int ch = 0; ch < 8; ch++) v[ch] = gw[c] * dt[ch];
#pragma unroll
        for (int j = 1; j < OMERF_FOLD; j++) {
          const float wn = __shfl_down_sync(kFull, gw[c], j);
          if (j < nfold)
#pragma unroll
            for (int ch = 0; ch < 8; ch++) v[ch] = fmaf(wn, dtn[j - 1][ch], v[ch]);
        }
        if (act && emit && goff[c] >= 0 && in_range(g, 0, goff[c])) red8(a.g_grid, goff[c], v);
      }
    }
    {
      float* gp[3] = {a.g_xy, a.g_xz, a.g_yz};
#pragma unroll
      for (int q = 0; q < 3; q++) {
        if (!gp[q]) continue;
        bool emit;
        int nfold;
        pair_fold_info(act ? poff[4 * q] : -1 - lane, lane, emit, nfold);
#pragma unroll
        for (int c = 0; c < 4; c++) {
          float v[8];
#pragma unroll
          for (int ch = 0; ch < 8; ch++) v[ch] = pw[4 * q + c] * dt[ch];
#pragma unroll
          for (int j = 1; j < OMERF_FOLD; j++) {
            const float wn = __shfl_down_sync(kFull, pw[4 * q + c], j);
            if (j < nfold)
#pragma unroll
              for (int ch = 0; ch < 8; ch++) v[ch] = fmaf(wn, dtn[j - 1][ch], v[ch]);
          }
          if (act && emit && in_range(g, 1 + q, poff[4 * q + c])) red8(gp[q], poff[4 * q + c], v);
        }
      }
    }
    const int rnext = __shfl_down_sync(kFull, r, 1);
    const bool tail = act && (lane == 31 || rnext != r);
    __syncwarp();
    if (tail) {
#pragma unroll
      for (int c = 0; c < 7; c++) ws.A[r][c] = Ai[c];
      ws.T[r] = Tn;
      ws.done[r] += lane - segstart + 1;
    }
    __syncwarp();
  }
}

// Kernel 1: per-ray deferred-MLP backward.  Writes dL/dF (7) and dL/dT_N
// into the ray's saved state and adds the MLP weight gradient.
__global__ void __launch_bounds__(kBwdThreads, 4) mlp_bwd_kernel(const Geo g, const BwdArgs a) {
  extern __shared__ float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  MlpBwdShared& S = *reinterpret_cast<MlpBwdShared*>(smem);
  float* rowsAll = smem + sizeof(MlpBwdShared) / sizeof(float);  // 32 staged rows per warp
  float* rows = rowsAll + warp * 32 * kRow;
  build_bwd_frags(g.mlp, S);
  __syncthreads();
  const float gs = a.grad_scale ? __ldg(a.grad_scale) : 1.0f;
  const long nwarps = (long)gridDim.x * (blockDim.x >> 5);
  const bool want_dw = a.g_mlp != nullptr;
  DwAcc acc;
  zero_acc(acc);
  float l_rgb = 0.0f, l_smooth = 0.0f;
  for (long b = (long)blockIdx.x * (blockDim.x >> 5) + warp; b < a.n_bundles; b += nwarps) {
    const long rid = b * 32 + lane;
    const bool valid = rid < a.n;
    float d[3] = {0, 0, 1};
    float F[7] = {0, 0, 0, 0, 0, 0, 0}, TN = 1.0f;
    int cnt = 0;
    if (valid) {
#pragma unroll
      for (int c = 0; c < 3; c++) d[c] = __ldg(a.rays + 6 * rid + 3 + c);
      const float4* sv = reinterpret_cast<const float4*>(a.saved + (long)kSavedFloats * rid);
      const float4 s0 = __ldg(sv), s1 = __ldg(sv + 1), s2 = __ldg(sv + 2);
      F[0] = s0.x; F[1] = s0.y; F[2] = s0.z; F[3] = s0.w;
      F[4] = s1.x; F[5] = s1.y; F[6] = s1.z; TN = s1.w;
      cnt = __float_as_int(s2.x);
    }
    const bool live = valid && cnt > 0;
    float* row = rows + lane * kRow;
    float gF[7] = {0, 0, 0, 0, 0, 0, 0};
    float gC[3] = {0, 0, 0}, yd[3] = {0, 0, 0}, gyd[3] = {0, 0, 0};
    stage_x(row, live, F, d);
    warp_mlp_forward(rows, S, lane, yd);
    if (live) {
      float e[3], e2 = 0.0f;
#pragma unroll
      for (int j = 0; j < 3; j++) {
        e[j] = F[j] + yd[j] + TN * g.bg[j] - __ldg(a.target + 3 * rid + j);
        e2 = fmaf(e[j], e[j], e2);
      }
      const float ell = sqrtf(e2 + 1e-6f);
      const float inv_ell = 1.0f / ell;
      l_rgb += ell;
#pragma unroll
      for (int j = 0; j < 3; j++) {
        gC[j] = gs * a.lam_rgb * e[j] * inv_ell;
        gyd[j] = gC[j];
      }
    } else if (valid && a.loss) {
      // no evaluated sample: the pixel is the background, with no gradient
      float e2 = 0.0f;
#pragma unroll
      for (int j = 0; j < 3; j++) {
        const float e = g.bg[j] - __ldg(a.target + 3 * rid + j);
        e2 = fmaf(e, e, e2);
      }
      l_rgb += sqrtf(e2 + 1e-6f);
    }
    // smoothness evaluations (Eqs. 9-10): each one is backpropagated and staged
    const float dn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < a.K; k++) {
      float sh[3] = {0.0f, 0.0f, 1.0f}, S_cos = 0.0f;
      if (live) {
        const float* sp = a.dirs + 3 * ((long)rid * a.K + k);
        float sv[3] = {__ldg(sp), __ldg(sp + 1), __ldg(sp + 2)};
        const float sn = sqrtf(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
        S_cos = (d[0] * sv[0] + d[1] * sv[1] + d[2] * sv[2]) / (dn * sn);
#pragma unroll
        for (int c = 0; c < 3; c++) sh[c] = sv[c] / sn;
      }
      stage_x(row, live, F, sh);
      float ys[3], gys[3] = {0.0f, 0.0f, 0.0f};
      warp_mlp_forward(rows, S, lane, ys);
      if (live) {
        float q = 0.0f;
#pragma unroll
        for (int j = 0; j < 3; j++) {
          gys[j] = gs * a.lam_smooth * 2.0f * S_cos * (ys[j] - yd[j]);
          gyd[j] -= gys[j];
          q = fmaf(ys[j] - yd[j], ys[j] - yd[j], q);
        }
        l_smooth = fmaf(S_cos, q, l_smooth);
      }
      warp_mlp_backward(rows, S, lane, ys, gys);
      if (want_dw) accumulate_mma(rows, lane, acc);
      warp_mlp_input_grad(rows, S, lane, gF);
    }
    // the evaluation at d, recomputed (the smoothness evaluations reused the rows)
    float y[3];
    stage_x(row, live, F, d);
    warp_mlp_forward(rows, S, lane, y);
    warp_mlp_backward(rows, S, lane, y, gyd);
    if (want_dw) accumulate_mma(rows, lane, acc);
    warp_mlp_input_grad(rows, S, lane, gF);
    if (valid) {
#pragma unroll
      for (int j = 0; j < 3; j++) gF[j] += gC[j];
      const float gT = gC[0] * g.bg[0] + gC[1] * g.bg[1] + gC[2] * g.bg[2];
      float4* sv = reinterpret_cast<float4*>(a.saved + (long)kSavedFloats * rid);
      sv[3] = make_float4(gF[0], gF[1], gF[2], gF[3]);
      sv[4] = make_float4(gF[4], gF[5], gF[6], gT);
    }
  }
  // loss terms of a fused step: warp sums -> CTA sum -> one global add per CTA
  if (a.loss) {
    __shared__ float sL[2][kBwdThreads / 32];
    l_rgb = warp_sum(l_rgb);
    l_smooth = warp_sum(l_smooth);
    if (lane == 0) {
      sL[0][warp] = l_rgb;
      sL[1][warp] = l_smooth;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float s0 = 0.0f, s1 = 0.0f;
      for (int w = 0; w < kBwdThreads / 32; w++) {
        s0 += sL[0][w];
        s1 += sL[1][w];
      }
      s0 *= a.lam_rgb;
      s1 *= a.lam_smooth;
      atomicAdd(a.loss + 1, s0);
      atomicAdd(a.loss + 2, s1);
      atomicAdd(a.loss + 0, s0 + s1);
    }
  }
  // weight gradients: per-warp sums (in the staging area, no longer needed)
  // -> CTA sum -> one global add per CTA
  if (!want_dw) return;
  __syncthreads();
  store_acc(acc, lane, rowsAll + warp * kMlpParams);
  __syncthreads();
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    float v = 0.0f;
    for (int w = 0; w < kBwdThreads / 32; w++) v += rowsAll[w * kMlpParams + i];
    atomicAdd(a.g_mlp + i, v);
  }
}

// Kernel 2: re-march every ray (one warp per bundle of 32 rays, persistent)
// and scatter the per-sample gradients.
#ifndef OMERF_BWD_MINB
#define OMERF_BWD_MINB 2  // resident CTAs per SM the register budget is sized for
#endif

template <class FT, bool SPARSE>
__global__ void __launch_bounds__(kThreads, OMERF_BWD_MINB) march_bwd_kernel(const Geo g, const BwdArgs a) {
  __shared__ WarpBwd sBwd[kThreads / 32];
  const int lane = threadIdx.x & 31;
  WarpBwd& ws = sBwd[threadIdx.x >> 5];
  for (;;) {
    unsigned b = 0;
    if (lane == 0) b = atomicAdd(a.counter, 1u);
    b = __shfl_sync(kFull, b, 0);
    if (b >= a.n_bundles) break;
    const long rid = (long)b * 32 + lane;
    const bool valid = rid < a.n;
    float o[3] = {0, 0, 0}, d[3] = {0, 0, 1};
    int cnt = 0, klo = 0, khi = -1;
    if (valid) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        o[c] = __ldg(a.rays + 6 * rid + c);
        d[c] = __ldg(a.rays + 6 * rid + 3 + c);
      }
      const float4* sv = reinterpret_cast<const float4*>(a.saved + (long)kSavedFloats * rid);
      const float4 s0 = __ldg(sv), s1 = __ldg(sv + 1), s2 = __ldg(sv + 2), s3 = __ldg(sv + 3),
                   s4 = __ldg(sv + 4);
      ws.F[lane][0] = s0.x; ws.F[lane][1] = s0.y; ws.F[lane][2] = s0.z; ws.F[lane][3] = s0.w;
      ws.F[lane][4] = s1.x; ws.F[lane][5] = s1.y; ws.F[lane][6] = s1.z; ws.TN[lane] = s1.w;
      cnt = __float_as_int(s2.x);
      klo = __float_as_int(s2.y);
      khi = __float_as_int(s2.z);
      ws.G[lane][0] = s3.x; ws.G[lane][1] = s3.y; ws.G[lane][2] = s3.z; ws.G[lane][3] = s3.w;
      ws.G[lane][4] = s4.x; ws.G[lane][5] = s4.y; ws.G[lane][6] = s4.z; ws.G[lane][7] = s4.w;
    }
    ws.cnt[lane] = cnt;
    ws.done[lane] = 0;
    ws.T[lane] = 1.0f;
#pragma unroll
    for (int c = 0; c < 8; c++) ws.A[lane][c] = 0.0f;
    __syncwarp();
    march_bundle_bwd<FT, SPARSE>(g, a, lane, o, d, klo, khi, valid && cnt > 0, ws);
    __syncwarp();
  }
}

template <class FT, bool SPARSE>
static cudaError_t launch_bwd_variant(const omerf_scene* s, const BwdArgs& a, cudaStream_t stream) {
  auto kern = march_bwd_kernel<FT, SPARSE>;
  static std::atomic<int> blocks[64];  // per device: resident CTAs of this variant
  const int dev = s->device & 63;
  int nb = blocks[dev].load(std::memory_order_relaxed);
  if (nb == 0) {
    nb = persistent_blocks((const void*)kern, kThreads, 0, s->num_sms);
    blocks[dev].store(nb, std::memory_order_relaxed);
  }
  long want = (a.n_bundles + (kThreads / 32) - 1) / (kThreads / 32);
  int grid = (int)(want < nb ? want : nb);
  if (grid < 1) grid = 1;
  kern<<<grid, kThreads, 0, stream>>>(s->geo, a);
  return cudaGetLastError();
}

static cudaError_t launch_mlp_bwd(const omerf_scene* s, const BwdArgs& a, cudaStream_t stream) {
  const size_t smem = sizeof(MlpBwdShared) + (size_t)(kBwdThreads / 32) * 32 * kRow * sizeof(float);
  static std::atomic<int> blocks[64];  // per device: resident CTAs
  const int dev = s->device & 63;
  int nb = blocks[dev].load(std::memory_order_relaxed);
  if (nb == 0) {
    cudaFuncSetAttribute((const void*)mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    nb = persistent_blocks((const void*)mlp_bwd_kernel, kBwdThreads, smem, s->num_sms);
    blocks[dev].store(nb, std::memory_order_relaxed);
  }
  long want = (a.n_bundles + (kBwdThreads / 32) - 1) / (kBwdThreads / 32);
  int grid = (int)(want < nb ? want : nb);
  if (grid < 1) grid = 1;
  mlp_bwd_kernel<<<grid, kBwdThreads, smem, stream>>>(s->geo, a);
  return cudaGetLastError();
}

cudaError_t launch_march_bwd(const omerf_scene* s, const float* rays, const float* target, const float* dirs,
                             long n, int K, const float lam[3], float* saved, const float* grad_scale,
                             float* g_grid, float* g_xy, float* g_xz, float* g_yz, float* g_occ, float* g_mlp,
                             float* loss, cudaStream_t stream) {
  BwdArgs a{};
  a.loss = loss;
  a.rays = rays;
  a.target = target;
  a.dirs = dirs;
  a.K = K;
  a.n = n;
  a.n_bundles = (n + 31) / 32;
  a.lam_rgb = n > 0 ? lam[0] / (float)n : 0.0f;
  a.lam_smooth = n > 0 ? lam[1] / (float)n : 0.0f;
  a.saved = saved;
  a.grad_scale = grad_scale;
  a.g_grid = g_grid;
  a.g_xy = g_xy;
  a.g_xz = g_xz;
  a.g_yz = g_yz;
  a.g_occ = g_occ;
  a.g_mlp = g_mlp;
  if (a.n_bundles == 0) return cudaSuccess;
  cudaError_t e = launch_mlp_bwd(s, a, stream);
  if (e != cudaSuccess) return e;
  a.counter = next_counter(s, stream);
  const bool bf16 = s->desc.feat_dtype == OMERF_BF16;
  const bool sparse = s->desc.brick > 0;
  if (bf16) return sparse ? launch_bwd_variant<__nv_bfloat16, true>(s, a, stream)
                          : launch_bwd_variant<__nv_bfloat16, false>(s, a, stream);
  return sparse ? launch_bwd_variant<float, true>(s, a, stream) : launch_bwd_variant<float, false>(s, a, stream);
}

}  // namespace omerf
