// Learned local smoother: a per-DoF network 16 -> 32 -> 32 -> 1 (ReLU, no
// biases) on the 15-point neighbourhood of s = D^-1 r, evaluated and trained
// on the tensor cores with BF16 operands and FP32 accumulation
// (mma.sync m16n8k16).  The smoothing step is x <- x + omega s + N(s) at
// macro-cell-interior DoFs and x <- x + omega s elsewhere.
//
// Fragment layouts (PTX m16n8k16, g = lane / 4, t = lane % 4):
//   A (16x16, row): r0 = (g, 2t..2t+1), r1 = (g+8, 2t..), r2 = (g, 2t+8..), r3 = (g+8, 2t+8..)
//   B (16x8, col):  r0 = (k=2t..2t+1, n=g), r1 = (k=2t+8.., n=g)
//   C (16x8, f32):  c0,c1 = (g, 2t..2t+1), c2,c3 = (g+8, 2t..2t+1)
// so the C tiles of one layer are the A fragments of the next (two n-tiles
// per 16-wide k-step).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "hg_internal.h"

namespace hg {

namespace {

constexpr int kMlpThreads = 256;
constexpr int kMlpWarps = kMlpThreads / 32;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ void mma16816(float d[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Weights of the network as B fragments (per thread) and w3 entries.
struct WFrag {
  uint32_t w1[4][2];      // layer 1: n-tile j (outputs 8j..8j+7), K = 16 inputs
  uint32_t w2[2][4][2];   // layer 2: k-step ks (inputs 16ks..), n-tile j
  float w3[4][2];         // w3[8j + 2t + {0,1}]
};

// W1 (32x16), W2 (32x32) in FP32 (row = output), w3 (32).
__device__ __forceinline__ void load_wfrag(WFrag& F, const float* __restrict__ W1,
                                           const float* __restrict__ W2,
                                           const float* __restrict__ w3, int lane) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float* r = W1 + (8 * j + g) * 16;
    F.w1[j][0] = pack_bf16(r[2 * t], r[2 * t + 1]);
    F.w1[j][1] = pack_bf16(r[2 * t + 8], r[2 * t + 9]);
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const float* q = W2 + (8 * j + g) * 32 + 16 * ks;
      F.w2[ks][j][0] = pack_bf16(q[2 * t], q[2 * t + 1]);
      F.w2[ks][j][1] = pack_bf16(q[2 * t + 8], q[2 * t + 9]);
    }
    F.w3[j][0] = w3[8 * j + 2 * t];
    F.w3[j][1] = w3[8 * j + 2 * t + 1];
  }
}

// Forward pass of one 16-row tile whose inputs are the bf16 rows X[16][16]
// (row stride 16) in shared memory.  Returns per thread the outputs of rows g
// and g+8; z1/z2 receive the pre-activations (C layout) for backprop.
__device__ __forceinline__ void mlp_tile_forward(const WFrag& F, const __nv_bfloat16* X, int lane,
                                                 float z1[4][4], float z2[4][4], float& out_g,
                                                 float& out_g8) {
  const int g = lane >> 2, t = lane & 3;
  uint32_t a[4];
  const uint32_t* X32 = reinterpret_cast<const uint32_t*>(X);
  a[0] = X32[g * 8 + t];
  a[1] = X32[(g + 8) * 8 + t];
  a[2] = X32[g * 8 + t + 4];
  a[3] = X32[(g + 8) * 8 + t + 4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    z1[j][0] = z1[j][1] = z1[j][2] = z1[j][3] = 0.f;
    mma16816(z1[j], a, F.w1[j]);
  }
  uint32_t h[2][4];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    h[ks][0] = pack_bf16(fmaxf(z1[2 * ks][0], 0.f), fmaxf(z1[2 * ks][1], 0.f));
    h[ks][1] = pack_bf16(fmaxf(z1[2 * ks][2], 0.f), fmaxf(z1[2 * ks][3], 0.f));
    h[ks][2] = pack_bf16(fmaxf(z1[2 * ks + 1][0], 0.f), fmaxf(z1[2 * ks + 1][1], 0.f));
    h[ks][3] = pack_bf16(fmaxf(z1[2 * ks + 1][2], 0.f), fmaxf(z1[2 * ks + 1][3], 0.f));
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    z2[j][0] = z2[j][1] = z2[j][2] = z2[j][3] = 0.f;
    mma16816(z2[j], h[0], F.w2[0][j]);
    mma16816(z2[j], h[1], F.w2[1][j]);
  }
  float o0 = 0.f, o8 = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    o0 += fmaxf(z2[j][0], 0.f) * F.w3[j][0] + fmaxf(z2[j][1], 0.f) * F.w3[j][1];
    o8 += fmaxf(z2[j][2], 0.f) * F.w3[j][0] + fmaxf(z2[j][3], 0.f) * F.w3[j][1];
  }
  o0 += __shfl_xor_sync(0xffffffffu, o0, 1);
  o0 += __shfl_xor_sync(0xffffffffu, o0, 2);
  o8 += __shfl_xor_sync(0xffffffffu, o8, 1);
  o8 += __shfl_xor_sync(0xffffffffu, o8, 2);
  out_g = o0;
  out_g8 = o8;
  (void)t;
}

// ---------------------------------------------------------------- forward
// out[b] = N(X[b]) for N rows of FP32 features (rounded to bf16).
__global__ void __launch_bounds__(kMlpThreads) mlp_forward_kernel(
    const float* __restrict__ X, int64_t N, const float* __restrict__ W1,
    const float* __restrict__ W2, const float* __restrict__ w3, float* __restrict__ out) {
  __shared__ __align__(16) __nv_bfloat16 sX[kMlpWarps][16 * 16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WFrag F;
  load_wfrag(F, W1, W2, w3, lane);
  const int64_t ntile = (N + 15) / 16;
  for (int64_t tile = blockIdx.x * (int64_t)kMlpWarps + warp; tile < ntile;
       tile += (int64_t)gridDim.x * kMlpWarps) {
    for (int e = lane; e < 256; e += 32) {
      const int64_t row = tile * 16 + e / 16;
      sX[warp][e] = __float2bfloat16_rn(row < N ? X[row * 16 + e % 16] : 0.f);
    }
    __syncwarp();
    float z1[4][4], z2[4][4], o0, o8;
    mlp_tile_forward(F, sX[warp], lane, z1, z2, o0, o8);
    const int g = lane >> 2, t = lane & 3;
    if (t == 0) {
      const int64_t r0 = tile * 16 + g, r8 = tile * 16 + g + 8;
      if (r0 < N) out[r0] = o0;
      if (r8 < N) out[r8] = o8;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- training
// Gradient of L = mean_b (N(X_b) - t_b)^2 over N bf16 samples, accumulated
// per block (FP32, tensor-core weight gradients) into partial[block][1568]
// (W1: 512, W2: 1024, w3: 32) and the block's sum of squared residuals into
// lpart[block].  The samples of block b are tiles b*W + warp, b*W + warp + G*W...
__global__ void __launch_bounds__(kMlpThreads) mlp_grad_kernel(
    const __nv_bfloat16* __restrict__ Xs, const float* __restrict__ ts, int64_t N, int64_t first,
    int64_t count, double inv_count, const float* __restrict__ W1, const float* __restrict__ W2,
    const float* __restrict__ w3, float* __restrict__ partial, double* __restrict__ lpart) {
  __shared__ __align__(16) __nv_bfloat16 sX[kMlpWarps][16 * 16];
  __shared__ __align__(16) __nv_bfloat16 sH1[kMlpWarps][16 * 32];
  __shared__ __align__(16) __nv_bfloat16 sD2[kMlpWarps][16 * 32];
  __shared__ __align__(16) __nv_bfloat16 sD1[kMlpWarps][16 * 32];
  __shared__ float red[1568];
  __shared__ double lred[kMlpWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  WFrag F;
  load_wfrag(F, W1, W2, w3, lane);
  // B fragments of W2 for dH1 = dH2 W2: k = output o, n = input h
  uint32_t w2t[2][4][2];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int h = 8 * j + g, o = 16 * ks + 2 * t;
      w2t[ks][j][0] = pack_bf16(W2[o * 32 + h], W2[(o + 1) * 32 + h]);
      w2t[ks][j][1] = pack_bf16(W2[(o + 8) * 32 + h], W2[(o + 9) * 32 + h]);
    }
  float gW2[2][4][4] = {}, gW1[2][2][4] = {}, gw3[4][2] = {};
  double lsum = 0.0;
  const int64_t ntile = (count + 15) / 16;
  for (int64_t tile = blockIdx.x * (int64_t)kMlpWarps + warp; tile < ntile;
       tile += (int64_t)gridDim.x * kMlpWarps) {
    // stage 16 samples (rows beyond `count` are zero: no contribution)
    {
      const int64_t row = tile * 16 + (lane >> 1);
      const int64_t src = first + row;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (row < count && src < N) v = reinterpret_cast<const uint4*>(Xs + src * 16)[lane & 1];
      reinterpret_cast<uint4*>(sX[warp])[lane] = v;
    }
    __syncwarp();
    float z1[4][4], z2[4][4], o0, o8;
    mlp_tile_forward(F, sX[warp], lane, z1, z2, o0, o8);
    const int64_t r0 = tile * 16 + g, r8 = r0 + 8;
    const bool v0 = r0 < count && first + r0 < N, v8 = r8 < count && first + r8 < N;
    const float e0 = v0 ? o0 - ts[first + r0] : 0.f, e8 = v8 ? o8 - ts[first + r8] : 0.f;
    if (t == 0) lsum += (double)e0 * e0 + (double)e8 * e8;
    const float q0 = (float)(2.0 * inv_count) * e0, q8 = (float)(2.0 * inv_count) * e8;
    // dw3 and dH2 = q w3 [z2 > 0]; H1 and dH2 to shared memory (bf16) for the
    // sample-reduction GEMMs
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 8 * j + 2 * t;
      gw3[j][0] += q0 * fmaxf(z2[j][0], 0.f) + q8 * fmaxf(z2[j][2], 0.f);
      gw3[j][1] += q0 * fmaxf(z2[j][1], 0.f) + q8 * fmaxf(z2[j][3], 0.f);
      const float d00 = z2[j][0] > 0.f ? q0 * F.w3[j][0] : 0.f;
      const float d01 = z2[j][1] > 0.f ? q0 * F.w3[j][1] : 0.f;
      const float d80 = z2[j][2] > 0.f ? q8 * F.w3[j][0] : 0.f;
      const float d81 = z2[j][3] > 0.f ? q8 * F.w3[j][1] : 0.f;
      z2[j][0] = d00; z2[j][1] = d01; z2[j][2] = d80; z2[j][3] = d81;   // reuse as dH2
      reinterpret_cast<uint32_t*>(sD2[warp])[(g * 32 + c) / 2] = pack_bf16(d00, d01);
      reinterpret_cast<uint32_t*>(sD2[warp])[((g + 8) * 32 + c) / 2] = pack_bf16(d80, d81);
      reinterpret_cast<uint32_t*>(sH1[warp])[(g * 32 + c) / 2] =
          pack_bf16(fmaxf(z1[j][0], 0.f), fmaxf(z1[j][1], 0.f));
      reinterpret_cast<uint32_t*>(sH1[warp])[((g + 8) * 32 + c) / 2] =
          pack_bf16(fmaxf(z1[j][2], 0.f), fmaxf(z1[j][3], 0.f));
    }
    // dH1 = (dH2 W2) [z1 > 0]
    uint32_t a2[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      a2[ks][0] = pack_bf16(z2[2 * ks][0], z2[2 * ks][1]);
      a2[ks][1] = pack_bf16(z2[2 * ks][2], z2[2 * ks][3]);
      a2[ks][2] = pack_bf16(z2[2 * ks + 1][0], z2[2 * ks + 1][1]);
      a2[ks][3] = pack_bf16(z2[2 * ks + 1][2], z2[2 * ks + 1][3]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      mma16816(d, a2[0], w2t[0][j]);
      mma16816(d, a2[1], w2t[1][j]);
      const int c = 8 * j + 2 * t;
      const float u00 = z1[j][0] > 0.f ? d[0] : 0.f, u01 = z1[j][1] > 0.f ? d[1] : 0.f;
      const float u80 = z1[j][2] > 0.f ? d[2] : 0.f, u81 = z1[j][3] > 0.f ? d[3] : 0.f;
      reinterpret_cast<uint32_t*>(sD1[warp])[(g * 32 + c) / 2] = pack_bf16(u00, u01);
      reinterpret_cast<uint32_t*>(sD1[warp])[((g + 8) * 32 + c) / 2] = pack_bf16(u80, u81);
    }
    __syncwarp();
    // dW2[o][h] += sum_b dH2[b][o] H1[b][h]  (M = o, N = h, K = 16 samples)
    // dW1[o][f] += sum_b dH1[b][o] X[b][f]
    const unsigned short* D2 = reinterpret_cast<const unsigned short*>(sD2[warp]);
    const unsigned short* D1 = reinterpret_cast<const unsigned short*>(sD1[warp]);
    const unsigned short* H1 = reinterpret_cast<const unsigned short*>(sH1[warp]);
    const unsigned short* XX = reinterpret_cast<const unsigned short*>(sX[warp]);
    auto pk = [](unsigned short lo, unsigned short hi) { return (uint32_t)lo | ((uint32_t)hi << 16); };
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int o = 16 * mt + g;
      uint32_t aD2[4], aD1[4];
      aD2[0] = pk(D2[(2 * t) * 32 + o], D2[(2 * t + 1) * 32 + o]);
      aD2[1] = pk(D2[(2 * t) * 32 + o + 8], D2[(2 * t + 1) * 32 + o + 8]);
      aD2[2] = pk(D2[(2 * t + 8) * 32 + o], D2[(2 * t + 9) * 32 + o]);
      aD2[3] = pk(D2[(2 * t + 8) * 32 + o + 8], D2[(2 * t + 9) * 32 + o + 8]);
      aD1[0] = pk(D1[(2 * t) * 32 + o], D1[(2 * t + 1) * 32 + o]);
      aD1[1] = pk(D1[(2 * t) * 32 + o + 8], D1[(2 * t + 1) * 32 + o + 8]);
      aD1[2] = pk(D1[(2 * t + 8) * 32 + o], D1[(2 * t + 9) * 32 + o]);
      aD1[3] = pk(D1[(2 * t + 8) * 32 + o + 8], D1[(2 * t + 9) * 32 + o + 8]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int h = 8 * j + g;
        uint32_t b[2];
        b[0] = pk(H1[(2 * t) * 32 + h], H1[(2 * t + 1) * 32 + h]);
        b[1] = pk(H1[(2 * t + 8) * 32 + h], H1[(2 * t + 9) * 32 + h]);
        mma16816(gW2[mt][j], aD2, b);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int f = 8 * j + g;
        uint32_t b[2];
        b[0] = pk(XX[(2 * t) * 16 + f], XX[(2 * t + 1) * 16 + f]);
        b[1] = pk(XX[(2 * t + 8) * 16 + f], XX[(2 * t + 9) * 16 + f]);
        mma16816(gW1[mt][j], aD1, b);
      }
    }
    __syncwarp();
  }
  // block reduction: the warps add their fragments into one buffer in warp order
  for (int e = threadIdx.x; e < 1568; e += kMlpThreads) red[e] = 0.f;
  // dw3: sum over the 8 groups (lanes with the same t) first
  float w3s[4][2];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float v = gw3[j][q];
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 16);
      w3s[j][q] = v;
    }
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
  if (lane == 0) lred[warp] = lsum;
  __syncthreads();
  for (int wsel = 0; wsel < kMlpWarps; ++wsel) {
    if (warp == wsel) {
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int o = 16 * mt + g, h = 8 * j + 2 * t;
          red[512 + o * 32 + h] += gW2[mt][j][0];
          red[512 + o * 32 + h + 1] += gW2[mt][j][1];
          red[512 + (o + 8) * 32 + h] += gW2[mt][j][2];
          red[512 + (o + 8) * 32 + h + 1] += gW2[mt][j][3];
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int o = 16 * mt + g, f = 8 * j + 2 * t;
          red[o * 16 + f] += gW1[mt][j][0];
          red[o * 16 + f + 1] += gW1[mt][j][1];
          red[(o + 8) * 16 + f] += gW1[mt][j][2];
          red[(o + 8) * 16 + f + 1] += gW1[mt][j][3];
        }
      }
      if (g == 0)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          red[1536 + 8 * j + 2 * t] += w3s[j][0];
          red[1536 + 8 * j + 2 * t + 1] += w3s[j][1];
        }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < 1568; e += kMlpThreads)
    partial[(int64_t)blockIdx.x * 1568 + e] = red[e];
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kMlpWarps; ++w) s += lred[w];
    lpart[blockIdx.x] = s;
  }
}

// Sum the block partials in a fixed order: grad[e] = sum_b partial[b][e].
__global__ void mlp_grad_sum_kernel(const float* __restrict__ partial, int nb,
                                    const double* __restrict__ lpart, float* __restrict__ grad,
                                    double* __restrict__ loss, double inv_count) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < 1568) {
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += partial[(int64_t)b * 1568 + e];
    grad[e] = s;
  }
  if (e == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += lpart[b];
    *loss = s * inv_count;
  }
}

// Adam (Kingma & Ba) on the 1568 FP32 master weights.
__global__ void mlp_adam_kernel(float* __restrict__ p, const float* __restrict__ grad,
                                float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                                float b2, float eps, float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 1568) return;
  const float g = grad[e];
  const float mi = b1 * m[e] + (1.f - b1) * g;
  const float vi = b2 * v[e] + (1.f - b2) * g * g;
  m[e] = mi;
  v[e] = vi;
  p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------ smoother step and samples
// Rows of the level's lattice: row item r -> (cell, j, k), lanes over i.
__device__ __forceinline__ void mlp_row(int w, int r, int& cell, int& j, int& k) {
  const int per = ntri32(w);
  cell = r / per;
  const int rr = r - cell * per;
  const float q = 2.0f * w + 1.0f;
  int kk = (int)floorf((q - sqrtf(fmaxf(q * q - 8.0f * rr, 0.0f))) * 0.5f);
  if (kk < 0) kk = 0;
  while ((kk + 1) * (2 * w - kk) / 2 <= rr) ++kk;
  while (kk * (2 * w - kk + 1) / 2 > rr) --kk;
  k = kk;
  j = rr - kk * (2 * w - kk + 1) / 2;
}

// s = invdiag * r at the 15 neighbours of an interior point (direction order).
__device__ __forceinline__ void s_neighbourhood(const float* __restrict__ r,
                                                const float* __restrict__ inv, int w, int i,
                                                int j, int k, float v[16]) {
  const int L = w - k - j;
  const int r0 = row_start(w, j, k);
  const int rjp = r0 + L, rjm = r0 - (L + 1);
  const int rkp = r0 + ntri32(w - k - 1) + L, rkm = r0 - ntri32(w - k) - (L + 1);
  const int rjmkp = rkp - L, rjpkm = rkm + L + 1;
  const int rows[15] = {r0, r0, r0, rjp, rjm, rkp, rkm, rjp, rjm, rkp, rkm, rjmkp, rjpkm, rjmkp, rjpkm};
#pragma unroll
  for (int d = 0; d < kNDir; ++d) {
    int di, dj, dk;
    dir_offset(d, di, dj, dk);
    const int idx = rows[d] + i + di;
    v[d] = r[idx] * inv[idx];
  }
  v[15] = 0.f;
}

// x_out = x + omega s (+ N(s) at macro-cell-interior DoFs); Dirichlet DoFs
// keep x.  One warp per lattice row (cell, j, k), windows of 30 points: lane
// l holds i = i0 - 1 + l, lanes 1..30 produce outputs and lanes 0 and 31 are
// the i -/+ 1 halo.  In rows that hold cell-interior points (j, k >= 1,
// row length >= 3) every lane forms s = r / D at its i on the seven
// neighbour rows (plane k rows j, j+1, j-1; plane k+1 rows j, j-1; plane k-1
// rows j, j+1, each one coalesced load of r and of 1/D with a warp-uniform
// base) and takes the i +/- 1 neighbours by shuffle; the interior points'
// 15 values go through the network as two 16-row tiles.  Loads of lanes past
// the row's end stay inside the padded cell (at most 30 elements past its
// last point) and feed no output.
__global__ void __launch_bounds__(kMlpThreads) learned_step_kernel(
    int n, int64_t stride, const uint8_t* __restrict__ flags, int n_rows, const float* __restrict__ x,
    const float* __restrict__ r, const float* __restrict__ inv, float omega, const float* W1,
    const float* W2, const float* w3, float* __restrict__ xo) {
  __shared__ __align__(16) __nv_bfloat16 sX[kMlpWarps][32 * 16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w = n + 1;
  const unsigned F = 0xffffffffu;
  WFrag Wf;
  load_wfrag(Wf, W1, W2, w3, lane);
  for (int row = blockIdx.x * kMlpWarps + warp; row < n_rows; row += gridDim.x * kMlpWarps) {
    int cell, j, k;
    mlp_row(w, row, cell, j, k);
    const int64_t base = (int64_t)cell * stride;
    const float* __restrict__ rc = r + base;
    const float* __restrict__ ic = inv + base;
    const int len = w - k - j;
    const int r0 = row_start(w, j, k);
    const uint8_t* fl = flags + cell * 16;
    const bool nbr = j >= 1 && k >= 1 && len >= 3;
    // neighbour row starts (valid only when nbr): j+1, j-1, (k+1, j), (k+1, j-1), (k-1, j), (k-1, j+1)
    const int rjp = r0 + len, rjm = r0 - (len + 1);
    const int rkp = r0 + ntri32(w - k - 1) + len, rkm = r0 - ntri32(w - k) - (len + 1);
    const int rjmkp = rkp - len, rjpkm = rkm + len + 1;
    for (int i0 = 0; i0 < len; i0 += 30) {
      const int i = i0 - 1 + lane;
      const int il = i < 0 ? 0 : i;
      const float s0 = __ldg(rc + r0 + il) * __ldg(ic + r0 + il);
      const bool out = lane >= 1 && lane <= 30 && i <= len - 1;
      const bool interior = nbr && out && i >= 1 && i <= len - 2;
      if (nbr) {
        float sr[7];
        const int rows[7] = {r0, rjp, rjm, rkp, rjmkp, rkm, rjpkm};
        sr[0] = s0;
#pragma unroll
        for (int m = 1; m < 7; ++m) sr[m] = __ldg(rc + rows[m] + il) * __ldg(ic + rows[m] + il);
        // direction order of the network's features (see the header comment)
        float v[16];
        v[0] = sr[0];
        v[1] = __shfl_down_sync(F, sr[0], 1);
        v[2] = __shfl_up_sync(F, sr[0], 1);
        v[3] = sr[1];
        v[4] = sr[2];
        v[5] = sr[3];
        v[6] = sr[5];
        v[7] = __shfl_up_sync(F, sr[1], 1);
        v[8] = __shfl_down_sync(F, sr[2], 1);
        v[9] = __shfl_up_sync(F, sr[3], 1);
        v[10] = __shfl_down_sync(F, sr[5], 1);
        v[11] = sr[4];
        v[12] = sr[6];
        v[13] = __shfl_down_sync(F, sr[4], 1);
        v[14] = __shfl_up_sync(F, sr[6], 1);
        v[15] = 0.f;
#pragma unroll
        for (int d = 0; d < 16; d += 2)
          reinterpret_cast<uint32_t*>(sX[warp])[(lane * 16 + d) / 2] =
              interior ? pack_bf16(v[d], v[d + 1]) : 0u;
        __syncwarp();
      }
      float corr = 0.f;
      if (nbr) {
        float z1[4][4], z2[4][4], oa0, oa8, ob0, ob8;
        mlp_tile_forward(Wf, sX[warp], lane, z1, z2, oa0, oa8);
        mlp_tile_forward(Wf, sX[warp] + 16 * 16, lane, z1, z2, ob0, ob8);
        // rows of the tiles: lane g -> row g (tile a), g+8, 16+g (tile b), 24+g
        const float cand0 = __shfl_sync(F, oa0, (lane & 7) * 4);
        const float cand8 = __shfl_sync(F, oa8, ((lane - 8) & 7) * 4);
        const float cand16 = __shfl_sync(F, ob0, ((lane - 16) & 7) * 4);
        const float cand24 = __shfl_sync(F, ob8, ((lane - 24) & 7) * 4);
        corr = lane < 8 ? cand0 : lane < 16 ? cand8 : lane < 24 ? cand16 : cand24;
        __syncwarp();
      }
      if (out) {
        const int64_t idx = base + r0 + i;
        const int cls = point_class(n, i, j, k);
        const uint8_t f = fl[cls];
        if (f & CF_DIRICHLET) {
          xo[idx] = x[idx];
        } else {
          xo[idx] = x[idx] + omega * s0 + (interior ? corr : 0.f);
        }
      }
    }
  }
}

// Training samples from one (r, e = xstar - x) pair: every `stride`-th
// macro-cell-interior DoF (interior rank q with q % stride == offset) gives
// features s(15 neighbours)/|.| (bf16, padded to 16) and target
// (e - omega s)/|.| at sample slot q / stride.
__global__ void __launch_bounds__(kMlpThreads) sample_kernel(
    int n, int64_t stride, int ncells, const float* __restrict__ r, const float* __restrict__ inv,
    const float* __restrict__ xstar, const float* __restrict__ x, float omega, int sstride,
    int soff, __nv_bfloat16* __restrict__ X, float* __restrict__ t) {
  const int w = n + 1, wi = n - 3;
  const int64_t per = ntet32(wi);
  const int64_t total = per * ncells;
  for (int64_t q = soff + (int64_t)(blockIdx.x * blockDim.x + threadIdx.x) * sstride; q < total;
       q += (int64_t)gridDim.x * blockDim.x * sstride) {
    const int cell = (int)(q / per);
    int rem = (int)(q - cell * per);
    // interior rank -> (i-1, j-1, k-1) in I_tet(wi) (k outer, then j, i)
    int k = 0;
    while (rem >= ntri32(wi - k)) {
      rem -= ntri32(wi - k);
      ++k;
    }
    int j = 0;
    while (rem >= wi - k - j) {
      rem -= wi - k - j;
      ++j;
    }
    const int i = rem + 1;
    ++j;
    ++k;
    const int64_t base = (int64_t)cell * stride;
    float v[16];
    s_neighbourhood(r + base, inv + base, w, i, j, k, v);
    float nrm = 0.f;
#pragma unroll
    for (int d = 0; d < 15; ++d) nrm += v[d] * v[d];
    nrm = sqrtf(nrm);
    const float sc = nrm > 0.f ? 1.f / nrm : 0.f;
    const int64_t idx = base + row_start(w, j, k) + i;
    const int64_t slot = q / sstride;
    for (int d = 0; d < 16; ++d) X[slot * 16 + d] = __float2bfloat16_rn(v[d] * sc);
    t[slot] = (xstar[idx] - x[idx] - omega * v[0]) * sc;
  }
}

}  // namespace

int launch_mlp_forward(const float* X, int64_t N, const float* W1, const float* W2,
                       const float* w3, float* out, cudaStream_t s) {
  const int64_t tiles = (N + 15) / 16;
  const int grid = (int)std::min<int64_t>((tiles + kMlpWarps - 1) / kMlpWarps, 152 * 8);
  mlp_forward_kernel<<<grid > 0 ? grid : 1, kMlpThreads, 0, s>>>(X, N, W1, W2, w3, out);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int mlp_grad_blocks(int64_t count) {
  const int64_t tiles = (count + 15) / 16;
  return (int)std::max<int64_t>(1, std::min<int64_t>((tiles + kMlpWarps - 1) / kMlpWarps, 152 * 2));
}

int launch_mlp_grad(const void* Xs, const float* ts, int64_t N, int64_t first, int64_t count,
                    const float* W1, const float* W2, const float* w3, float* partial,
                    double* lpart, float* grad, double* loss, cudaStream_t s) {
  const int nb = mlp_grad_blocks(count);
  const double inv = count > 0 ? 1.0 / (double)count : 0.0;
  mlp_grad_kernel<<<nb, kMlpThreads, 0, s>>>((const __nv_bfloat16*)Xs, ts, N, first, count, inv,
                                            W1, W2, w3, partial, lpart);
  HG_CUDA(cudaGetLastError());
  mlp_grad_sum_kernel<<<(1568 + 255) / 256, 256, 0, s>>>(partial, nb, lpart, grad, loss, inv);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_mlp_adam(float* p, const float* grad, float* m, float* v, float lr, int step,
                    cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  mlp_adam_kernel<<<(1568 + 255) / 256, 256, 0, s>>>(p, grad, m, v, lr, b1, b2, 1e-8f, c1, c2);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_learned_step(const LevelDev& L, const float* x, const float* r, const float* inv,
                        float omega, const float* params, float* xo, cudaStream_t s) {
  const int n_rows = L.ncells * ntri32(L.w);
  const int grid = std::max(1, std::min((n_rows + kMlpWarps - 1) / kMlpWarps, 152 * 8));
  learned_step_kernel<<<grid, kMlpThreads, 0, s>>>(L.n, L.cell_stride, L.cls_flags, n_rows, x, r,
                                                   inv, omega, params, params + 512,
                                                   params + 1536, xo);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int64_t learned_sample_count(const LevelDev& L, int sstride, int soff) {
  const int64_t total = (int64_t)ntet(L.n - 3) * L.ncells;
  return total > soff ? (total - soff + sstride - 1) / sstride : 0;
}

int launch_learned_sample(const LevelDev& L, const float* r, const float* inv, const float* xstar,
                          const float* x, float omega, int sstride, int soff, void* X, float* t,
                          cudaStream_t s) {
  const int64_t cnt = learned_sample_count(L, sstride, soff);
  if (cnt <= 0) return HG_OK;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((cnt + 255) / 256, 152 * 8));
  sample_kernel<<<grid, 256, 0, s>>>(L.n, L.cell_stride, L.ncells, r, inv, xstar, x, omega,
                                     sstride, soff, (__nv_bfloat16*)X, t);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

}  // namespace hg
