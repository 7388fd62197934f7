// mhd_mlp.cuh -- the thermal surrogate network 4 -> 64 -> 64 -> 1 on the GPU.
//
//   h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = w3 . h2 + b3,
// x = (log10 n_H, log10 T, log10 dt, Z) mapped to [-1, 1] by the training range,
// y = q, the change of log10 T over dt in units of the saturated explicit estimate
// S = th_scale(th_dlin(x)) (mhd_thermal.cuh); the change applied is q S.
//
// The 64x64 layer runs on the tensor cores: BF16 operands (activations h1 and weights W2
// rounded to BF16), FP32 accumulation.  Inference in the thermal step and training both use
// tcgen05.mma with the accumulators in tensor memory (mhd_mlp_tc.cu); the warp-level
// mma.sync m16n8k16 kernels of mhd_mlp.cu compute the same products and serve as the
// cross-check of the tcgen05 ones.  The 4-wide input layer and the 64-wide output layer are
// FP32 FMAs.  Master weights are FP32.
// Parameter block layout (floats): W1[64][4], b1[64], W2[64][64] (row = output), b2[64],
// w3[64], b3[1].
#pragma once
#include <cuda_bf16.h>

#include "mhd_device.cuh"

namespace mhd {

constexpr int kHid = 64;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * 4, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid, kNParam = kOffB3 + 1;  // 4545
constexpr int kMlpRows = 64;  // rows per CTA tile (4 warps x 16)

struct MlpDev {
  const float* p;            // FP32 parameter block
  const __nv_bfloat16* W2h;  // BF16 copy of W2 [64][64]
  float xlo[4], xscale[4];   // x_s = (x - xlo) * xscale - 1
  float qmax;                // fallback when |y| > qmax
  float dmax;                // or when the change |y S| > dmax (or is not finite)
};

// Minibatch row of training step `step`, position r: mix64(seed ^ mix64(step * (2^32 + 1) + r))
// modulo the number of harvested rows, mix64 being the splitmix64 finaliser.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  // splitmix64 finaliser
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// The hidden activation of every surrogate kernel (training and inference, tcgen05 and
// mma.sync alike): the single-instruction hardware approximation tanh.approx.f32.  Its error
// against the exact tanh stays below 1e-3 (a GPU test sweeps it against libm), under the
// BF16 rounding that h1 takes for the tensor cores anyway and an order below the fit error
// of the trained network.
__device__ __forceinline__ float mlp_tanh(float z) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(z));
  return r;
}

__device__ __forceinline__ unsigned pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16_16816(float* c, unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                               unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// c[16x8] += A[16x16] B[16x8]; A element (m, k) at A[m*sm + k*sk], B element (k, n) at
// B[k*tk + n*tn].  Accumulator layout per lane (g = lane/4, t = lane%4):
// c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1).
__device__ __forceinline__ void mma_tile(float* c, const __nv_bfloat16* A, int sm, int sk,
                                         const __nv_bfloat16* B, int tk, int tn) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const unsigned a0 = pack_bf16(A[g * sm + (2 * t) * sk], A[g * sm + (2 * t + 1) * sk]);
  const unsigned a1 = pack_bf16(A[(g + 8) * sm + (2 * t) * sk], A[(g + 8) * sm + (2 * t + 1) * sk]);
  const unsigned a2 = pack_bf16(A[g * sm + (2 * t + 8) * sk], A[g * sm + (2 * t + 9) * sk]);
  const unsigned a3 = pack_bf16(A[(g + 8) * sm + (2 * t + 8) * sk], A[(g + 8) * sm + (2 * t + 9) * sk]);
  const unsigned b0 = pack_bf16(B[(2 * t) * tk + g * tn], B[(2 * t + 1) * tk + g * tn]);
  const unsigned b1 = pack_bf16(B[(2 * t + 8) * tk + g * tn], B[(2 * t + 9) * tk + g * tn]);
  mma_bf16_16816(c, a0, a1, a2, a3, b0, b1);
}

// Shared-memory working set of one CTA (4 warps, 64 rows).
struct MlpSmem {
  __nv_bfloat16 W2[kHid * kHid];   // row = output, col = input
  __nv_bfloat16 h1b[kMlpRows * kHid];
  float h1f[kMlpRows * kHid];
  float x[kMlpRows * 4];
  float W1[kHid * 4], b1[kHid], b2[kHid], w3[kHid], b3;
};

__device__ __forceinline__ void mlp_load_weights(MlpSmem& S, const MlpDev& M) {
  for (int q = threadIdx.x; q < kHid * kHid; q += blockDim.x) S.W2[q] = M.W2h[q];
  for (int q = threadIdx.x; q < kHid * 4; q += blockDim.x) S.W1[q] = M.p[kOffW1 + q];
  for (int q = threadIdx.x; q < kHid; q += blockDim.x) {
    S.b1[q] = M.p[kOffB1 + q];
    S.b2[q] = M.p[kOffB2 + q];
    S.w3[q] = M.p[kOffW3 + q];
  }
  if (threadIdx.x == 0) S.b3 = M.p[kOffB3];
}

// Layer 1 for the warp's 16 rows (x already standardised in S.x): lane covers one row
// (r0 + lane/2) and 32 of its 64 outputs.
__device__ __forceinline__ void mlp_layer1(MlpSmem& S, int r0) {
  const int lane = threadIdx.x & 31;
  const int row = r0 + (lane >> 1), c0 = (lane & 1) * 32;
  const float x0 = S.x[row * 4 + 0], x1 = S.x[row * 4 + 1], x2 = S.x[row * 4 + 2], x3 = S.x[row * 4 + 3];
#pragma unroll 8
  for (int c = c0; c < c0 + 32; ++c) {
    const float z = S.b1[c] + S.W1[c * 4 + 0] * x0 + S.W1[c * 4 + 1] * x1 + S.W1[c * 4 + 2] * x2 +
                    S.W1[c * 4 + 3] * x3;
    const float h = mlp_tanh(z);
    S.h1f[row * kHid + c] = h;
    S.h1b[row * kHid + c] = __float2bfloat16_rn(h);
  }
}

// Layer 2 on the tensor cores for the warp's 16 rows: acc[nt][.] = (h1 W2^T)[16 x 64].
__device__ __forceinline__ void mlp_layer2(const MlpSmem& S, int r0, float acc[8][4]) {
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
      mma_tile(acc[nt], S.h1b + r0 * kHid + ks * 16, kHid, 1, S.W2 + nt * 8 * kHid + ks * 16, 1, kHid);
  }
}

// h2 = tanh(acc + b2) in place and y = w3 . h2 + b3 for rows r0 + g and r0 + g + 8.
__device__ __forceinline__ void mlp_head(const MlpSmem& S, float acc[8][4], float& y_lo, float& y_hi) {
  const int lane = threadIdx.x & 31, t = lane & 3;
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int c = nt * 8 + 2 * t;
    acc[nt][0] = mlp_tanh(acc[nt][0] + S.b2[c]);
    acc[nt][1] = mlp_tanh(acc[nt][1] + S.b2[c + 1]);
    acc[nt][2] = mlp_tanh(acc[nt][2] + S.b2[c]);
    acc[nt][3] = mlp_tanh(acc[nt][3] + S.b2[c + 1]);
    s0 += S.w3[c] * acc[nt][0] + S.w3[c + 1] * acc[nt][1];
    s1 += S.w3[c] * acc[nt][2] + S.w3[c + 1] * acc[nt][3];
  }
  s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
  s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
  y_lo = s0 + S.b3;
  y_hi = s1 + S.b3;
}

__device__ __forceinline__ float mlp_standardize(const MlpDev& M, int f, float v) {
  return (v - M.xlo[f]) * M.xscale[f] - 1.0f;
}

}  // namespace mhd
