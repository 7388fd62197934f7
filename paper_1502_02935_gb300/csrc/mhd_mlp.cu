// mhd_mlp.cu -- training and inference kernels of the thermal surrogate (mhd_mlp.cuh).
//
// Training: each minibatch row is drawn from the harvested set with a counter-based hash
// of (seed, step, row).  k_mlp_grad_tc (mhd_mlp_tc.cu) computes a minibatch's loss and
// gradient on tcgen05; k_mlp_grad below is the same computation on mma.sync (64 rows per
// CTA of 4 warps; dW2 = dz2^T h1 and dh1 = dz2 W2 also on the tensor cores), kept as the
// cross-check.  k_adam_sched then updates the FP32 master weights and the BF16 copy of W2.
//
// Inference (thermal mode SURROGATE): per interior cell, features -> network -> change of
// log10 T (k_thermal_surrogate_tc in mhd_mlp_tc.cu, on tcgen05).  A cell whose standardised
// features leave [-1, 1] or whose predicted change exceeds the stated bound is appended to a
// fallback list that the plain FP64 integrator then handles (k_thermal_fallback below), so
// the divergent fallback stays out of the network kernel.
#include <cuda_bf16.h>

#include "mhd_mlp.cuh"
#include "mhd_mlp_launch.h"
#include "mhd_thermal.cuh"

namespace mhd {

// ------------------------------------------------------------------- forward --
// Unit-level forward: standardised inputs xs[n][4] -> y[n].
__global__ void __launch_bounds__(128) k_mlp_forward(long long n, const float* __restrict__ xs, MlpDev M,
                                                     float* __restrict__ y) {
  __shared__ MlpSmem S;
  mlp_load_weights(S, M);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, r0 = warp * 16;
  for (long long base = (long long)blockIdx.x * kMlpRows; base < n; base += (long long)gridDim.x * kMlpRows) {
    __syncthreads();
    for (int q = threadIdx.x; q < kMlpRows * 4; q += blockDim.x) {
      const long long row = base + q / 4;
      S.x[q] = row < n ? xs[row * 4 + (q & 3)] : 0.f;
    }
    __syncthreads();
    mlp_layer1(S, r0);
    __syncwarp();
    float acc[8][4];
    mlp_layer2(S, r0, acc);
    float ylo, yhi;
    mlp_head(S, acc, ylo, yhi);
    const int g = lane >> 2;
    if ((lane & 3) == 0) {
      const long long a = base + r0 + g, b = base + r0 + g + 8;
      if (a < n) y[a] = ylo;
      if (b < n) y[b] = yhi;
    }
  }
}

// -------------------------------------------------------------- train step --
struct TrainSmem {
  MlpSmem m;
  __nv_bfloat16 dz2[kMlpRows * kHid];
  float t[kMlpRows];
  float red[kHid * 2];
  float gw1[kHid * 4];
  float gb1[kHid];
};

// One minibatch chunk of 64 rows: loss and gradient contributions.  rows == nullptr:
// rows come from the dataset by hash; else they are given (xs, targets) directly.
__global__ void __launch_bounds__(128) k_mlp_grad(MlpDev M, const float* __restrict__ data, long long nrows,
                                                  unsigned long long seed, long long step, int batch,
                                                  float* __restrict__ grad, float* __restrict__ loss_sum) {
  __shared__ TrainSmem T;
  MlpSmem& S = T.m;
  mlp_load_weights(S, M);
  for (int q = threadIdx.x; q < kHid * 4; q += blockDim.x) T.gw1[q] = 0.f;
  for (int q = threadIdx.x; q < kHid; q += blockDim.x) T.gb1[q] = 0.f;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, r0 = warp * 16;
  const int g = lane >> 2, t = lane & 3;
  const long long base = (long long)blockIdx.x * kMlpRows;
  // gather rows and standardise
  for (int q = threadIdx.x; q < kMlpRows; q += blockDim.x) {
    const long long r = base + q;
    long long src = -1;
    if (r < batch) src = seed ? (long long)(mix64(seed ^ mix64((unsigned long long)step * 0x100000001ull + r)) %
                                            (unsigned long long)nrows)
                              : r;
    for (int f = 0; f < 4; ++f) S.x[q * 4 + f] = src >= 0 ? mlp_standardize(M, f, data[src * kHvCols + f]) : 0.f;
    T.t[q] = src >= 0 ? data[src * kHvCols + 4] : 0.f;
  }
  __syncthreads();
  mlp_layer1(S, r0);
  __syncwarp();
  float acc[8][4];
  mlp_layer2(S, r0, acc);
  float ylo, yhi;
  mlp_head(S, acc, ylo, yhi);  // acc now holds h2
  const long long ra = base + r0 + g, rb = ra + 8;
  const float inv_b = 1.0f / (float)batch;
  const float dya = ra < batch ? 2.0f * (ylo - T.t[r0 + g]) * inv_b : 0.f;
  const float dyb = rb < batch ? 2.0f * (yhi - T.t[r0 + g + 8]) * inv_b : 0.f;
  if (t == 0) {
    float l = 0.f;
    if (ra < batch) l += (ylo - T.t[r0 + g]) * (ylo - T.t[r0 + g]);
    if (rb < batch) l += (yhi - T.t[r0 + g + 8]) * (yhi - T.t[r0 + g + 8]);
    if (l != 0.f) atomicAdd(loss_sum, l);
  }
  // output layer: gw3, gb3; dz2 = dy w3 (1 - h2^2)
  float gb2p[16], gw3p[16];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = nt * 8 + 2 * t + h;
      const float h2a = acc[nt][h], h2b = acc[nt][2 + h];
      gw3p[nt * 2 + h] = dya * h2a + dyb * h2b;
      const float dza = dya * S.w3[c] * (1.f - h2a * h2a);
      const float dzb = dyb * S.w3[c] * (1.f - h2b * h2b);
      gb2p[nt * 2 + h] = dza + dzb;
      T.dz2[(r0 + g) * kHid + c] = __float2bfloat16_rn(dza);
      T.dz2[(r0 + g + 8) * kHid + c] = __float2bfloat16_rn(dzb);
    }
  }
  // reduce gw3 / gb2 over the 8 row groups of the warp, then across warps
#pragma unroll
  for (int q = 0; q < 16; ++q) {
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      gw3p[q] += __shfl_xor_sync(0xffffffffu, gw3p[q], o);
      gb2p[q] += __shfl_xor_sync(0xffffffffu, gb2p[q], o);
    }
  }
  for (int q = threadIdx.x; q < 2 * kHid; q += blockDim.x) T.red[q] = 0.f;
  float db3 = t == 0 ? dya + dyb : 0.f;  // the four lanes of a quad hold the same two rows
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) db3 += __shfl_xor_sync(0xffffffffu, db3, o);
  __syncthreads();
  if (g == 0) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        atomicAdd(&T.red[nt * 8 + 2 * t + h], gw3p[nt * 2 + h]);
        atomicAdd(&T.red[kHid + nt * 8 + 2 * t + h], gb2p[nt * 2 + h]);
      }
  }
  if (lane == 0) atomicAdd(grad + kOffB3, db3);
  __syncthreads();
  for (int q = threadIdx.x; q < kHid; q += blockDim.x) {
    atomicAdd(grad + kOffW3 + q, T.red[q]);
    atomicAdd(grad + kOffB2 + q, T.red[kHid + q]);
  }
  // dW2[out][in] = sum_rows dz2[row][out] h1[row][in]: warp w takes outputs 16w..16w+15
  {
    float gacc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      gacc[nt][0] = gacc[nt][1] = gacc[nt][2] = gacc[nt][3] = 0.f;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        mma_tile(gacc[nt], T.dz2 + ks * 16 * kHid + warp * 16, 1, kHid, S.h1b + ks * 16 * kHid + nt * 8, kHid, 1);
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int in = nt * 8 + 2 * t, out = warp * 16 + g;
      atomicAdd(grad + kOffW2 + out * kHid + in, gacc[nt][0]);
      atomicAdd(grad + kOffW2 + out * kHid + in + 1, gacc[nt][1]);
      atomicAdd(grad + kOffW2 + (out + 8) * kHid + in, gacc[nt][2]);
      atomicAdd(grad + kOffW2 + (out + 8) * kHid + in + 1, gacc[nt][3]);
    }
  }
  // dh1 = dz2 W2 for the warp's rows; dz1 = dh1 (1 - h1^2); gW1, gb1
  {
    float dacc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      dacc[nt][0] = dacc[nt][1] = dacc[nt][2] = dacc[nt][3] = 0.f;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        mma_tile(dacc[nt], T.dz2 + r0 * kHid + ks * 16, kHid, 1, S.W2 + ks * 16 * kHid + nt * 8, kHid, 1);
    }
    const float* xa = S.x + (r0 + g) * 4;
    const float* xb = S.x + (r0 + g + 8) * 4;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = nt * 8 + 2 * t + h;
        const float h1a = S.h1f[(r0 + g) * kHid + c], h1b = S.h1f[(r0 + g + 8) * kHid + c];
        const float dza = dacc[nt][h] * (1.f - h1a * h1a);
        const float dzb = dacc[nt][2 + h] * (1.f - h1b * h1b);
        float gb = dza + dzb;
        float gw[4] = {dza * xa[0] + dzb * xb[0], dza * xa[1] + dzb * xb[1], dza * xa[2] + dzb * xb[2],
                       dza * xa[3] + dzb * xb[3]};
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
          gb += __shfl_xor_sync(0xffffffffu, gb, o);
#pragma unroll
          for (int f = 0; f < 4; ++f) gw[f] += __shfl_xor_sync(0xffffffffu, gw[f], o);
        }
        if (g == 0) {
          atomicAdd(&T.gb1[c], gb);
#pragma unroll
          for (int f = 0; f < 4; ++f) atomicAdd(&T.gw1[c * 4 + f], gw[f]);
        }
      }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kHid * 4; q += blockDim.x) atomicAdd(grad + kOffW1 + q, T.gw1[q]);
  for (int q = threadIdx.x; q < kHid; q += blockDim.x) atomicAdd(grad + kOffB1 + q, T.gb1[q]);
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) on parameter q; b1c, b2c the bias corrections.
__device__ __forceinline__ void adam_param(int q, float* __restrict__ p, float gq, float* __restrict__ m,
                                           float* __restrict__ v, float lr, float b1c, float b2c,
                                           __nv_bfloat16* __restrict__ W2h) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float mq = b1 * m[q] + (1.f - b1) * gq;
  const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
  m[q] = mq;
  v[q] = vq;
  const float pq = p[q] - lr * (mq / b1c) / (sqrtf(vq / b2c) + eps);
  p[q] = pq;
  if (q >= kOffW2 && q < kOffW2 + kHid * kHid) W2h[q - kOffW2] = __float2bfloat16_rn(pq);
}

// The Adam step of a training run replayed as a graph: the step index comes from device
// memory, the learning rate follows the cosine decay from lr0 to lr0/20 over `total` steps,
// the gradient block is cleared for the next step and the index advanced.  One CTA.
__global__ void __launch_bounds__(1024) k_adam_sched(float* __restrict__ p, float* __restrict__ grad,
                                                     float* __restrict__ m, float* __restrict__ v, double lr0,
                                                     long long total, long long* __restrict__ step_dev,
                                                     __nv_bfloat16* __restrict__ W2h) {
  __shared__ float sched[3];
  const long long stp = *step_dev;
  if (threadIdx.x == 0) {  // one thread: FP64 is slow on this part
    const double pi = 3.14159265358979323846;
    sched[0] = (float)(lr0 * (0.05 + 0.95 * 0.5 * (1.0 + cos(pi * (double)stp / (double)total))));
    sched[1] = 1.f - powf(0.9f, (float)(stp + 1));
    sched[2] = 1.f - powf(0.999f, (float)(stp + 1));
  }
  __syncthreads();
  const float lr = sched[0], b1c = sched[1], b2c = sched[2];
  for (int q = threadIdx.x; q < kNParam; q += blockDim.x) {
    adam_param(q, p, grad[q], m, v, lr, b1c, b2c, W2h);
    grad[q] = 0.f;
  }
  __syncthreads();
  if (threadIdx.x == 0) *step_dev = stp + 1;
}

__global__ void k_refresh_w2h(const float* __restrict__ p, __nv_bfloat16* __restrict__ W2h) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < kHid * kHid) W2h[q] = __float2bfloat16_rn(p[kOffW2 + q]);
}

// -------------------------------------------------------- surrogate thermal --
// Plain FP64 integrator on the listed cells (grid-stride over the device-side count); with
// Wst, each cell's W and the CFL limit as in k_thermal_surrogate_tc.
__global__ void __launch_bounds__(256) k_thermal_fallback(PatchDev P, ThermalDev th, const int* __restrict__ fb_list,
                                                          const unsigned long long* __restrict__ fb_count,
                                                          float* __restrict__ Wst) {
  const long long n = (long long)*fb_count;
  float lim = INFINITY;
  const double dt = *P.dt_used;
  const double cef = th_cef(P, th);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const long long c = fb_list[q];
    const int i = (int)(c % P.n[0]);
    const long long r = c / P.n[0];
    const int j = (int)(r % P.n[1]), k = (int)(r / P.n[1]);
    double T, nh, ce;
    th_cell(P, th, P.Un, i, j, k, cef, T, nh, ce);
    int st, nsub;
    const double T1 = th_integrate(T, nh, ce, dt, th, &st, &nsub);
    P.Un[EN * P.FS + sidx(P, i, j, k)] += ce * (T1 - T);
    if (Wst) lim = fminf(lim, prim_point<float>(P, P.Un, Wst, i, j, k, true, true));
    if (st & (TST_SUBSTEP_CAP | TST_NEWTON_CAP)) atomicAdd(th.stats + 2, 1ull);
    atomicAdd(th.stats + 1, (unsigned long long)nsub);
  }
  if (Wst) block_min_atomic(lim, P.cfl_min);
}

// ------------------------------------------------------------ host side ----
int mlp_forward(long long n, const float* xs, const MlpDev& M, float* y, cudaStream_t s) {
  if (n <= 0) return 0;
  long long blocks = (n + kMlpRows - 1) / kMlpRows;
  if (blocks > 65535) blocks = 65535;
  k_mlp_forward<<<(unsigned)blocks, 128, 0, s>>>(n, xs, M, y);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mlp_grad(const MlpDev& M, const float* data, long long nrows, unsigned long long seed, long long step, int batch,
             float* grad, float* loss_sum, cudaStream_t s) {
  const int blocks = (batch + kMlpRows - 1) / kMlpRows;
  k_mlp_grad<<<blocks, 128, 0, s>>>(M, data, nrows, seed, step, batch, grad, loss_sum);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mlp_adam_sched(float* p, float* grad, float* m, float* v, double lr0, long long total, long long* step_dev,
                   __nv_bfloat16* W2h, cudaStream_t s) {
  k_adam_sched<<<1, 1024, 0, s>>>(p, grad, m, v, lr0, total, step_dev, W2h);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mlp_refresh(const float* p, __nv_bfloat16* W2h, cudaStream_t s) {
  k_refresh_w2h<<<(kHid * kHid + 255) / 256, 256, 0, s>>>(p, W2h);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int issue_surrogate(const PatchDev& P, const ThermalDev& th, const MlpDev& M, int* fb_list,
                    unsigned long long* fb_count, float* Wst, int sms, cudaStream_t s, long long* launches) {
  if (cudaMemsetAsync(fb_count, 0, sizeof(unsigned long long), s) != cudaSuccess) return -1;
  if (issue_surrogate_tc(P, th, M, fb_list, fb_count, Wst, sms, s, launches)) return -1;
  k_thermal_fallback<<<(unsigned)(sms * 4), 256, 0, s>>>(P, th, fb_list, fb_count, Wst);
  *launches += 1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace mhd
