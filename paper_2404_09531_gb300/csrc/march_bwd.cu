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
#include <cstdlib>
#include <cstring>

#include "internal.h"
#include "mma_tf32.cuh"
#include "packed.cuh"
#include "tc.cuh"

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
  unsigned* err;  // device error word of bounded waits (NULL: not reported)
  int wait_tries; // polls of a bounded mbarrier wait (tcgen05 MLP backward)
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
      gather_texels<FT>(g, goff, gw, poff, pw, t);
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

// ---------------------------------------------------------------------------
// Kernel 1, fifth-generation tensor-core form (tcgen05).  One CTA of 128
// threads per tile of 128 consecutive rays: thread t owns ray t of the tile
// and row t of every product (TMEM lane t).  Each layer of the MLP and of
// its backward is one M = 128 product, D = A B, with A the tile's staged
// rows in shared memory and B a weight matrix; one thread issues it as
// kind::tf32 products with split operands (A_lo B_hi + A_hi B_lo + A_hi B_hi,
// about FP32 accurate, as in the mma.sync form), commits it to an mbarrier,
// and every thread reads its row of the FP32 accumulator from TMEM.  The
// weight gradient sum_rays act (x) delta is one more product per evaluation
// whose reduction dimension is the tile's 128 rays: A = the staged
// activation rows read MN-major, B = the staged delta rows read MN-major,
// accumulating in TMEM for the CTA's whole run, read once at the end.  The
// tensor core takes MN-major operands in 16-bit formats only, so this
// product runs as kind::f16 on BF16 copies split the same way (hi + lo,
// 16 significant bits, three products: relative error ~2^-16, far inside the
// 1e-3 bar of the gradients; the TF32 layers keep the loss FP32 accurate).
//
// Staged rows (the tc.cuh layouts):
//   act   [128][76] TF32 hi / lo: x 0..33 (34..39 zero), h1 40..55, h2 56..71, 1 at 72 (live rays), 73..75 zero
//   delta [128][40] TF32 hi / lo: g1 0..15, g2 16..31, g3 32..34, 35..39 zero
//   actb  [128][80], deltab [128][48]: BF16 hi / lo copies of the same columns (actb 73..79, deltab 35..47 zero)
// Weight operands (K-major B, [N rows][K], TF32 hi / lo):
//   W1B [16 units][40 inputs] = W1        W2B [16][16] = W2     W3B [16 (3 used)][16] = W3
//   W3T [16 u2][8 (3 used)]   = W3^T      W2T [16][16] = W2^T   W1T [16 (7 used)][16 u] = W1[:, :7]^T
// The M = 128 weight-gradient product reads 128 activation columns per ray;
// the columns beyond 80 are the next rays' data and land in accumulator
// rows that are never read.
namespace tcmlp {
constexpr int kRows = 128;
constexpr int kActW = 76, kH1 = 40, kH2 = 56, kOne = 72;
constexpr int kDelW = 40, kG1 = 0, kG2 = 16, kG3 = 32;
constexpr int kActBytes = kRows * kActW * 4, kDelBytes = kRows * kDelW * 4;
constexpr int kW1B = 0, kW2B = kW1B + 16 * 40 * 4, kW3B = kW2B + 16 * 16 * 4, kW3T = kW3B + 16 * 16 * 4,
              kW2T = kW3T + 16 * 8 * 4, kW1T = kW2T + 16 * 16 * 4, kWBytes = kW1T + 16 * 16 * 4;
constexpr int kActBW = 80, kDelBW = 48;
constexpr int kActBBytes = kRows * kActBW * 2, kDelBBytes = kRows * kDelBW * 2;
constexpr int kActHi = 0, kActLo = kActBytes, kDelHi = 2 * kActBytes, kDelLo = kDelHi + kDelBytes,
              kActBHi = kDelLo + kDelBytes, kActBLo = kActBHi + kActBBytes, kDelBHi = kActBLo + kActBBytes,
              kDelBLo = kDelBHi + kDelBBytes, kWHi = kDelBLo + kDelBBytes, kWLo = kWHi + kWBytes,
              kSmem = kWLo + kWBytes;
constexpr uint32_t kTmemCols = 128, kColL = 0, kColW = 64;
constexpr int kTries = 1 << 24;  // bounded mbarrier wait (a product takes well under a microsecond)

// Write v (TF32 hi and lo) at (row, col) of a staged tile of width W.
__device__ __forceinline__ void put(unsigned char* hi, unsigned char* lo, int row, int col, int W, float v) {
  uint32_t h, l;
  split_tf32(v, h, l);
  const uint32_t o = tc::off4(row, col, W);
  *reinterpret_cast<uint32_t*>(hi + o) = h;
  *reinterpret_cast<uint32_t*>(lo + o) = l;
}

// Four consecutive columns (col % 4 == 0) with one 16-byte store per copy.
__device__ __forceinline__ void put4(unsigned char* hi, unsigned char* lo, int row, int col, int W, float v0,
                                     float v1, float v2, float v3) {
  uint32_t h[4], l[4];
  split_tf32(v0, h[0], l[0]);
  split_tf32(v1, h[1], l[1]);
  split_tf32(v2, h[2], l[2]);
  split_tf32(v3, h[3], l[3]);
  const uint32_t o = tc::off4(row, col, W);
  *reinterpret_cast<uint4*>(hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Eight consecutive columns (col % 8 == 0) of a BF16 tile, hi and lo copies.
__device__ __forceinline__ void putb8(unsigned char* hi, unsigned char* lo, int row, int col, int W, const float v[8]) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * i]), h1 = __float2bfloat16_rn(v[2 * i + 1]);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * i] - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * i + 1] - __bfloat162float(h1));
    h[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    l[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
  }
  const uint32_t o = tc::off2(row, col, W);
  *reinterpret_cast<uint4*>(hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
}
}  // namespace tcmlp

__global__ void __launch_bounds__(128, 1) mlp_bwd_tc_kernel(const Geo g, const BwdArgs a) {
  using namespace tcmlp;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ uint32_t tmem_base;
  __shared__ float sL[2][4];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *act_hi = sm + kActHi, *act_lo = sm + kActLo, *del_hi = sm + kDelHi, *del_lo = sm + kDelLo;
  unsigned char *actb_hi = sm + kActBHi, *actb_lo = sm + kActBLo, *delb_hi = sm + kDelBHi, *delb_lo = sm + kDelBLo;
  unsigned char *w_hi = sm + kWHi, *w_lo = sm + kWLo;
  // the BF16 delta columns 35..47 stay zero (only 0..34 are staged)
  for (int i = tid; i < 2 * kDelBBytes / 16; i += kRows)
    reinterpret_cast<uint4*>(delb_hi)[i] = make_uint4(0u, 0u, 0u, 0u);
  const uint32_t s_base = tc::smem_u32(sm), s_bar = tc::smem_u32(&bar);
  const float* W = g.mlp;
  // weight operands (the tile-independent B matrices), TF32 hi / lo
  for (int i = tid; i < 16 * 40; i += kRows) {
    const int u = i / 40, c = i % 40;
    put(w_hi + kW1B, w_lo + kW1B, u, c, 40, c < 34 ? W[kOffW1 + u * 34 + c] : 0.0f);
  }
  for (int i = tid; i < 16 * 16; i += kRows) {
    const int r = i / 16, c = i % 16;
    put(w_hi + kW2B, w_lo + kW2B, r, c, 16, W[kOffW2 + r * 16 + c]);           // W2[u2][u1]
    put(w_hi + kW3B, w_lo + kW3B, r, c, 16, r < 3 ? W[kOffW3 + r * 16 + c] : 0.0f);  // W3[o][u2]
    put(w_hi + kW2T, w_lo + kW2T, r, c, 16, W[kOffW2 + c * 16 + r]);           // [u1][u2] = W2[u2][u1]
    put(w_hi + kW1T, w_lo + kW1T, r, c, 16, r < 7 ? W[kOffW1 + c * 34 + r] : 0.0f);  // [i][u] = W1[u][i]
  }
  for (int i = tid; i < 16 * 8; i += kRows) {
    const int r = i / 8, c = i % 8;
    put(w_hi + kW3T, w_lo + kW3T, r, c, 8, c < 3 ? W[kOffW3 + c * 16 + r] : 0.0f);  // [u2][o] = W3[o][u2]
  }
  float b1[16], b2[16], b3[3];
#pragma unroll
  for (int j = 0; j < 16; j++) {
    b1[j] = __ldg(W + kOffB1 + j);
    b2[j] = __ldg(W + kOffB2 + j);
  }
#pragma unroll
  for (int j = 0; j < 3; j++) b3[j] = __ldg(W + kOffB3 + j);
  if (warp == 0) tc::alloc(&tmem_base, kTmemCols);
  if (tid == 0) tc::mbar_init(s_bar, 1);
  tc::fence_proxy();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t my_lane = tmem + ((uint32_t)(32 * warp) << 16);
  const float gs = a.grad_scale ? __ldg(a.grad_scale) : 1.0f;
  const bool want_dw = a.g_mlp != nullptr;
  const long n_tiles = (a.n + kRows - 1) / kRows;
  uint32_t phase = 0;
  bool dw_started = false, failed = false;
  float l_rgb = 0.0f, l_smooth = 0.0f;

  // Sync the staged rows, let thread 0 issue the products, wait for them.
  // Returns false (on every thread) if the wait ran out: the error word is
  // set and the products still in flight are waited for (bounded).
  auto round_trip = [&](auto issue) -> bool {
    tc::fence_proxy();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      issue();
      tc::commit(s_bar);
    }
    bool ok = tc::mbar_wait(s_bar, phase, a.wait_tries);
    if (__syncthreads_or(!ok)) {
      if (!ok) tc::mbar_wait(s_bar, phase, kTries);
      if (tid == 0 && a.err) {
        atomicOr_system(a.err, kErrMlpWait);
        __threadfence_system();
      }
      failed = true;
      return false;
    }
    phase ^= 1u;
    tc::fence_after();
    return true;
  };
  const uint32_t id16 = tc::idesc(2, 128, 16);
  const uint32_t idw = tc::idesc(1, 128, 48, 1, 1);  // BF16, both operands MN-major
  const int sAct = (kActW / 4) * 128, sDel = (kDelW / 4) * 128;
  // three TF32 products per K-step of K-major operands into accumulator column col
  auto mma3k = [&](uint32_t col, int a_off, int a_sbo, int a_lo_shift, int b_off, int b_sbo, int ksteps,
                   uint32_t id) {
    for (int k = 0; k < ksteps; k++) {
      const uint64_t ah = tc::desc(s_base + a_off + 256 * k, 128, a_sbo);
      const uint64_t al = tc::desc(s_base + a_off + a_lo_shift + 256 * k, 128, a_sbo);
      const uint64_t bh = tc::desc(s_base + kWHi + b_off + 256 * k, 128, b_sbo);
      const uint64_t bl = tc::desc(s_base + kWLo + b_off + 256 * k, 128, b_sbo);
      tc::mma_tf32(tmem + col, al, bh, id, k > 0);
      tc::mma_tf32(tmem + col, ah, bl, id, true);
      tc::mma_tf32(tmem + col, ah, bh, id, true);
    }
  };
  // the weight-gradient product of the staged tile, accumulated in TMEM
  auto mma_dw = [&]() {
    constexpr int lA = (kActBW / 8) * 128, lD = (kDelBW / 8) * 128;  // next 8 rays (K)
    for (int k = 0; k < kRows / 16; k++) {  // 16 rays per product
      const uint64_t ah = tc::desc(s_base + kActBHi + 2 * k * lA, lA, 128);
      const uint64_t al = tc::desc(s_base + kActBLo + 2 * k * lA, lA, 128);
      const uint64_t dh = tc::desc(s_base + kDelBHi + 2 * k * lD, lD, 128);
      const uint64_t dl = tc::desc(s_base + kDelBLo + 2 * k * lD, lD, 128);
      tc::mma_f16(tmem + kColW, al, dh, idw, dw_started || k > 0);
      tc::mma_f16(tmem + kColW, ah, dl, idw, true);
      tc::mma_f16(tmem + kColW, ah, dh, idw, true);
    }
  };
  // staged x row (and the ones column) of this thread's ray
  auto stage_x = [&](bool live, const float F[7], const float dir[3]) {
    float x[40];
#pragma unroll
    for (int i = 0; i < 40; i++) x[i] = 0.0f;
    if (live) {
#pragma unroll
      for (int i = 0; i < 7; i++) x[i] = F[i];
      view_encoding(dir, x + 7);
    }
#pragma unroll
    for (int c = 0; c < 40; c += 4) put4(act_hi, act_lo, tid, c, kActW, x[c], x[c + 1], x[c + 2], x[c + 3]);
#pragma unroll
    for (int c = 0; c < 40; c += 8) putb8(actb_hi, actb_lo, tid, c, kActBW, x + c);
    const float one[8] = {live ? 1.0f : 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    put4(act_hi, act_lo, tid, kOne, kActW, one[0], 0.0f, 0.0f, 0.0f);
    putb8(actb_hi, actb_lo, tid, kOne, kActBW, one);
  };
  // 16 values at column col of the activation (act = true) or delta rows, TF32 and BF16
  auto stage16 = [&](bool act, int col, const float v[16]) {
#pragma unroll
    for (int c = 0; c < 16; c += 4)
      put4(act ? act_hi : del_hi, act ? act_lo : del_lo, tid, col + c, act ? kActW : kDelW, v[c], v[c + 1], v[c + 2],
           v[c + 3]);
    putb8(act ? actb_hi : delb_hi, act ? actb_lo : delb_lo, tid, col, act ? kActBW : kDelBW, v);
    putb8(act ? actb_hi : delb_hi, act ? actb_lo : delb_lo, tid, col + 8, act ? kActBW : kDelBW, v + 8);
  };
  // forward of the staged x: h1, h2 staged and returned, y = G
  auto forward = [&](float h1[16], float h2[16], float y[3]) -> bool {
    float t[16];
    if (!round_trip([&] { mma3k(kColL, kActHi, sAct, kActLo - kActHi, kW1B, 1280, 5, id16); })) return false;
    tc::ld16(my_lane + kColL, t);
#pragma unroll
    for (int j = 0; j < 16; j++) h1[j] = fmaxf(t[j] + b1[j], 0.0f);
    stage16(true, kH1, h1);
    if (!round_trip([&] { mma3k(kColL, kActHi + (kH1 / 4) * 128, sAct, kActLo - kActHi, kW2B, 512, 2, id16); }))
      return false;
    tc::ld16(my_lane + kColL, t);
#pragma unroll
    for (int j = 0; j < 16; j++) h2[j] = fmaxf(t[j] + b2[j], 0.0f);
    stage16(true, kH2, h2);
    if (!round_trip([&] { mma3k(kColL, kActHi + (kH2 / 4) * 128, sAct, kActLo - kActHi, kW3B, 512, 2, id16); }))
      return false;
    tc::ld16(my_lane + kColL, t);
#pragma unroll
    for (int j = 0; j < 3; j++) y[j] = sigmoidf_(t[j] + b3[j]);
    return true;
  };
  // backward of the evaluation whose activations are staged (h1, h2 its ReLU
  // outputs): deltas staged, the weight gradient accumulated, dL/dF added to gF
  auto backward = [&](const float h1[16], const float h2[16], const float y[3], const float gy[3],
                      float gF[7]) -> bool {
    float t[16];
    const float g3[8] = {gy[0] * y[0] * (1.0f - y[0]), gy[1] * y[1] * (1.0f - y[1]), gy[2] * y[2] * (1.0f - y[2]),
                         0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    put4(del_hi, del_lo, tid, kG3, kDelW, g3[0], g3[1], g3[2], 0.0f);
    put4(del_hi, del_lo, tid, kG3 + 4, kDelW, 0.0f, 0.0f, 0.0f, 0.0f);
    putb8(delb_hi, delb_lo, tid, kG3, kDelBW, g3);
    if (!round_trip([&] { mma3k(kColL, kDelHi + (kG3 / 4) * 128, sDel, kDelLo - kDelHi, kW3T, 256, 1, id16); }))
      return false;
    tc::ld16(my_lane + kColL, t);
#pragma unroll
    for (int j = 0; j < 16; j++) t[j] = h2[j] > 0.0f ? t[j] : 0.0f;
    stage16(false, kG2, t);
    if (!round_trip([&] { mma3k(kColL, kDelHi + (kG2 / 4) * 128, sDel, kDelLo - kDelHi, kW2T, 512, 2, id16); }))
      return false;
    tc::ld16(my_lane + kColL, t);
#pragma unroll
    for (int j = 0; j < 16; j++) t[j] = h1[j] > 0.0f ? t[j] : 0.0f;
    stage16(false, kG1, t);
    if (!round_trip([&] {
          mma3k(kColL, kDelHi + (kG1 / 4) * 128, sDel, kDelLo - kDelHi, kW1T, 512, 2, id16);
          if (want_dw) mma_dw();
        }))
      return false;
    dw_started = dw_started || want_dw;
    tc::ld16(my_lane + kColL, t);
#pragma unroll
    for (int i = 0; i < 7; i++) gF[i] += t[i];
    return true;
  };

  for (long tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
    const long rid = tile * kRows + tid;
    const bool valid = rid < a.n;
    float d[3] = {0.0f, 0.0f, 1.0f}, F[7] = {0, 0, 0, 0, 0, 0, 0}, TN = 1.0f;
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
    float gF[7] = {0, 0, 0, 0, 0, 0, 0};
    float gC[3] = {0, 0, 0}, yd[3], gyd[3] = {0, 0, 0}, h1d[16], h2d[16];
    stage_x(live, F, d);
    if (!forward(h1d, h2d, yd)) break;
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
      float e2 = 0.0f;
#pragma unroll
      for (int j = 0; j < 3; j++) {
        const float e = g.bg[j] - __ldg(a.target + 3 * rid + j);
        e2 = fmaf(e, e, e2);
      }
      l_rgb += sqrtf(e2 + 1e-6f);
    }
    // smoothness evaluations (Eqs. 9-10), each backpropagated at once
    const float dn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    bool ok = true;
    for (int k = 0; k < a.K && ok; k++) {
      float sh[3] = {0.0f, 0.0f, 1.0f}, S_cos = 0.0f;
      if (live) {
        const float* sp = a.dirs + 3 * ((long)rid * a.K + k);
        const float sv[3] = {__ldg(sp), __ldg(sp + 1), __ldg(sp + 2)};
        const float sn = sqrtf(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
        S_cos = (d[0] * sv[0] + d[1] * sv[1] + d[2] * sv[2]) / (dn * sn);
#pragma unroll
        for (int c = 0; c < 3; c++) sh[c] = sv[c] / sn;
      }
      float h1[16], h2[16], ys[3], gys[3] = {0.0f, 0.0f, 0.0f};
      stage_x(live, F, sh);
      ok = forward(h1, h2, ys);
      if (!ok) break;
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
      ok = backward(h1, h2, ys, gys, gF);
    }
    if (!ok) break;
    // the evaluation at d: its activations re-staged from registers
    if (a.K > 0) {
      stage_x(live, F, d);
      stage16(true, kH1, h1d);
      stage16(true, kH2, h2d);
    }
    if (!backward(h1d, h2d, yd, gyd, gF)) break;
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
    l_rgb = warp_sum(l_rgb);
    l_smooth = warp_sum(l_smooth);
    if (lane == 0) {
      sL[0][warp] = l_rgb;
      sL[1][warp] = l_smooth;
    }
    __syncthreads();
    if (tid == 0) {
      float s0 = 0.0f, s1 = 0.0f;
      for (int w = 0; w < kRows / 32; w++) {
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
  // weight gradient: accumulator row m = activation column m, column n =
  // delta column n; each thread reads its row and adds the entries that are
  // parameters of Eq. 4's MLP
  if (dw_started && !failed) {
    float v[48];
    tc::ld16(my_lane + kColW, v);
    tc::ld16(my_lane + kColW + 16, v + 16);
    tc::ld16(my_lane + kColW + 32, v + 32);
    const int m = tid;
    float* G = a.g_mlp;
    if (m < 34) {
#pragma unroll
      for (int u = 0; u < 16; u++) atomicAdd(G + kOffW1 + u * 34 + m, v[kG1 + u]);
    } else if (m >= kH1 && m < kH1 + 16) {
#pragma unroll
      for (int u2 = 0; u2 < 16; u2++) atomicAdd(G + kOffW2 + u2 * 16 + (m - kH1), v[kG2 + u2]);
    } else if (m >= kH2 && m < kH2 + 16) {
#pragma unroll
      for (int o = 0; o < 3; o++) atomicAdd(G + kOffW3 + o * 16 + (m - kH2), v[kG3 + o]);
    } else if (m == kOne) {
#pragma unroll
      for (int u = 0; u < 16; u++) {
        atomicAdd(G + kOffB1 + u, v[kG1 + u]);
        atomicAdd(G + kOffB2 + u, v[kG2 + u]);
      }
#pragma unroll
      for (int o = 0; o < 3; o++) atomicAdd(G + kOffB3 + o, v[kG3 + o]);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::dealloc(tmem, kTmemCols);
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

static cudaError_t launch_mlp_bwd_tc(const omerf_scene* s, const BwdArgs& a, cudaStream_t stream) {
  static std::atomic<int> ready[64];  // per device: shared-memory attribute set
  const int dev = s->device & 63;
  if (!ready[dev].load(std::memory_order_relaxed)) {
    cudaFuncSetAttribute((const void*)mlp_bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tcmlp::kSmem);
    ready[dev].store(1, std::memory_order_relaxed);
  }
  const long tiles = (a.n + tcmlp::kRows - 1) / tcmlp::kRows;
  const int grid = (int)(tiles < s->num_sms ? tiles : s->num_sms);
  mlp_bwd_tc_kernel<<<grid < 1 ? 1 : grid, tcmlp::kRows, tcmlp::kSmem, stream>>>(s->geo, a);
  return cudaGetLastError();
}

// The deferred-MLP backward runs as warp-level mma.sync products (16 warps
// per SM keep the small per-ray products busy); OMERF_MLP_BWD=tcgen05 in the
// environment selects the tcgen05 form instead (one 128-ray tile per SM in
// flight: about three times slower on these 16-unit layers, kept as a
// tested alternative).
static bool mlp_bwd_tcgen05() {
  const char* v = std::getenv("OMERF_MLP_BWD");
  return v && std::strcmp(v, "tcgen05") == 0;
}

static cudaError_t launch_mlp_bwd(const omerf_scene* s, const BwdArgs& a, cudaStream_t stream) {
  if (mlp_bwd_tcgen05()) return launch_mlp_bwd_tc(s, a, stream);
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
  a.err = device_error_word();
  // OMERF_FAULT=mlp_wait: the tcgen05 MLP backward's first wait gives up at
  // once (its products still complete and are waited for), for tests
  a.wait_tries = fault_injected("mlp_wait") ? 0 : tcmlp::kTries;
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
