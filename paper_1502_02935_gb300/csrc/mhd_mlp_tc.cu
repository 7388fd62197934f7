// mhd_mlp_tc.cu -- the surrogate's 64x64 layer on the 5th-generation tensor cores
// (tcgen05.mma with the accumulator in tensor memory).
//
// One CTA of 128 threads takes 128 rows.  Each thread computes its row of h1 =
// tanh(W1 x + b1) in FP32 and stores it as BF16 into shared memory in the canonical
// K-major layout without swizzle: 8-row x 16-byte core matrices, the two core matrices
// of one 16-wide K chunk 128 bytes apart (leading byte offset) and consecutive 8-row
// groups 1024 bytes apart (stride byte offset).  W2 (N = 64 outputs x K = 64 inputs,
// K-major) sits in the same layout.  One thread issues four tcgen05.mma (M = 128, N = 64,
// K = 16 each, BF16 x BF16 -> FP32) into 64 TMEM columns and commits them to an mbarrier;
// every thread waits on it (bounded by the global timer), then reads its own row of the
// accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31), applies tanh(. + b2),
// and the 64-wide output layer y = w3 . h2 + b3 in FP32.
#include <cuda_bf16.h>
#include <stdint.h>

#include "mhd_mlp.cuh"
#include "mhd_mlp_launch.h"
#include "mhd_thermal.cuh"

namespace mhd {

constexpr int kTcRows = 128;
constexpr unsigned long long kTcWaitNs = 200000000ull;  // 0.2 s bound on the MMA wait

struct TcSmem {
  alignas(1024) __nv_bfloat16 A[kTcRows * kHid];  // h1, core-matrix layout
  alignas(1024) __nv_bfloat16 B[kHid * kHid];     // W2, core-matrix layout
  alignas(8) unsigned long long mbar;
  uint32_t taddr;
  int timed_out;
  float W1[kHid * 4], b1[kHid], b2[kHid], w3[kHid], b3;
};

// byte offset of element (row r, k) in the K-major no-swizzle core-matrix layout with K = 64
__device__ __forceinline__ uint32_t cm_offset(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start address, leading / stride byte offsets (>> 4),
// descriptor version 1 (bits 46-47), no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tc_tanh(float z) { return tanhf(z); }

__device__ __forceinline__ unsigned long long tc_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Load the weights, set up the mbarrier and allocate 64 TMEM columns (warp 0).
__device__ __forceinline__ uint32_t tc_setup(TcSmem& S, const float* __restrict__ p,
                                             const __nv_bfloat16* __restrict__ W2h) {
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int q = tid; q < kHid * kHid; q += blockDim.x) {
    const int nrow = q >> 6, k = q & 63;
    *(__nv_bfloat16*)((char*)S.B + cm_offset(nrow, k)) = W2h[q];
  }
  for (int q = tid; q < kHid * 4; q += blockDim.x) S.W1[q] = p[kOffW1 + q];
  for (int q = tid; q < kHid; q += blockDim.x) {
    S.b1[q] = p[kOffB1 + q];
    S.b2[q] = p[kOffB2 + q];
    S.w3[q] = p[kOffW3 + q];
  }
  if (tid == 0) {
    S.b3 = p[kOffB3];
    S.timed_out = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.taddr)),
                 "r"(64));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return S.taddr;
}

// Layer 1 of this thread's row (x already standardised) into the A tile.
__device__ __forceinline__ void tc_layer1(TcSmem& S, float x0, float x1, float x2, float x3) {
  const int tid = threadIdx.x;
#pragma unroll 8
  for (int c = 0; c < kHid; ++c) {
    const float z = S.b1[c] + S.W1[c * 4] * x0 + S.W1[c * 4 + 1] * x1 + S.W1[c * 4 + 2] * x2 + S.W1[c * 4 + 3] * x3;
    *(__nv_bfloat16*)((char*)S.A + cm_offset(tid, c)) = __float2bfloat16_rn(tc_tanh(z));
  }
}

// h1 W2^T for the 128-row tile on the tensor cores; returns this thread's output y.
// *ok = false (for every thread) if the bounded wait for the MMA ran out.
__device__ __forceinline__ float tc_tile(TcSmem& S, uint32_t taddr, uint32_t& phase, bool* ok) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t idesc = idesc_bf16(kTcRows, kHid);
  // make the generic-proxy stores of the A tile visible to the tensor cores' async proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t a0 = smem_u32(S.A), b0 = smem_u32(S.B);
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      const uint64_t ad = smem_desc(a0 + kc * 256, 128, 1024);
      const uint64_t bd = smem_desc(b0 + kc * 256, 128, 1024);
      const uint32_t acc = kc > 0 ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
          "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&S.mbar))
                 : "memory");
  }
  {
    const unsigned long long t0 = tc_ns();
    uint32_t done = 0;
    while (!done) {
      asm volatile(
          "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}\n"
          : "=r"(done)
          : "r"(smem_u32(&S.mbar)), "r"(phase)
          : "memory");
      if (!done && tc_ns() - t0 > kTcWaitNs) {
        S.timed_out = 1;
        break;
      }
    }
    phase ^= 1u;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (S.timed_out) {
    *ok = false;
    return 0.f;
  }
  float out = S.b3;
#pragma unroll
  for (int c0 = 0; c0 < kHid; c0 += 16) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) out += S.w3[c0 + q] * tc_tanh(__uint_as_float(r[q]) + S.b2[c0 + q]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();  // the A tile and the accumulator are reused by the next tile
  *ok = true;
  return out;
}

__device__ __forceinline__ void tc_teardown(uint32_t taddr) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(64));
}

__global__ void __launch_bounds__(128) k_mlp_forward_tc(long long n, const float* __restrict__ xs,
                                                        const float* __restrict__ p,
                                                        const __nv_bfloat16* __restrict__ W2h,
                                                        float* __restrict__ y, int* __restrict__ err) {
  __shared__ TcSmem S;
  const uint32_t taddr = tc_setup(S, p, W2h);
  uint32_t phase = 0;
  for (long long base = (long long)blockIdx.x * kTcRows; base < n; base += (long long)gridDim.x * kTcRows) {
    const long long row = base + threadIdx.x;
    float x[4] = {0.f, 0.f, 0.f, 0.f};
    if (row < n)
      for (int f = 0; f < 4; ++f) x[f] = xs[row * 4 + f];
    tc_layer1(S, x[0], x[1], x[2], x[3]);
    bool ok;
    const float out = tc_tile(S, taddr, phase, &ok);
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
      break;
    }
    if (row < n) y[row] = out;
  }
  tc_teardown(taddr);
}

// Surrogate thermal step, one interior cell per thread, 128 cells per tile; cells outside
// the training range or over the bound go to the fallback list (see mhd_mlp.cu).
__global__ void __launch_bounds__(128) k_thermal_surrogate_tc(PatchDev P, ThermalDev th, MlpDev M,
                                                              int* __restrict__ fb_list,
                                                              unsigned long long* __restrict__ fb_count) {
  __shared__ TcSmem S;
  const uint32_t taddr = tc_setup(S, M.p, M.W2h);
  uint32_t phase = 0;
  const long long nc = (long long)P.n[0] * P.n[1] * P.n[2];
  const double dt = *P.dt_used;
  const float ldt = log10f((float)dt);
  const DlinConst dc = th_dlin_const(th, P.gm1);
  const double cef = th_cef(P, th);
  const float zf = (float)th.z;
  for (long long base = (long long)blockIdx.x * kTcRows; base < nc; base += (long long)gridDim.x * kTcRows) {
    const long long c = base + threadIdx.x;
    int i = 0, j = 0, k = 0;
    bool inrange = false;
    double T = 0.0, nh = 0.0, ce = 0.0;
    float x[4] = {0.f, 0.f, 0.f, 0.f}, dl = 0.f;
    if (c < nc) {
      i = (int)(c % P.n[0]);
      const long long r = c / P.n[0];
      j = (int)(r % P.n[1]);
      k = (int)(r / P.n[1]);
      th_cell(P, th, P.Un, i, j, k, cef, T, nh, ce);
      // features in FP32 (integer-pipe conversions; the clamp lets a NaN through to fall back)
      const float tf = d2f_alu(T);
      const float raw[4] = {log10f(d2f_alu(nh)), log10f(tf < 10.0f ? 10.0f : (tf > 1e8f ? 1e8f : tf)), ldt, zf};
      dl = th_scale(th_dlin(dc, raw[0], raw[1], raw[2]));
      inrange = true;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        x[f] = mlp_standardize(M, f, raw[f]);
        inrange = inrange && x[f] >= -1.0f && x[f] <= 1.0f;
      }
    }
    tc_layer1(S, x[0], x[1], x[2], x[3]);
    bool ok;
    const float y = tc_tile(S, taddr, phase, &ok);
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(P.err, ERR_TIMEOUT);
      break;
    }
    int fb = 0, live = 0;
    if (c < nc) {
      live = 1;
      const float d = y * dl;  // predicted change of log10 T
      if (inrange && fabsf(y) <= M.qmax && fabsf(d) <= M.dmax) {
        const double T0 = th_clamp(T);
        const double T1 = th_clamp(T0 * f2d_alu(exp10f(d)));
        P.Un[EN * P.FS + sidx(P, i, j, k)] += ce * (T1 - T);
      } else {
        fb_list[atomicAdd(fb_count, 1ull)] = (int)c;
        fb = 1;
      }
    }
    const unsigned nfb = __reduce_add_sync(0xffffffffu, (unsigned)fb);
    const unsigned nlive = __reduce_add_sync(0xffffffffu, (unsigned)live);
    if ((threadIdx.x & 31) == 0) {
      if (nfb) atomicAdd(th.stats + 3, (unsigned long long)nfb);
      if (nlive) atomicAdd(th.stats + 0, (unsigned long long)nlive);
    }
  }
  tc_teardown(taddr);
}

int mlp_forward_tc(long long n, const float* xs, const float* p, const __nv_bfloat16* W2h, float* y, int* err,
                   int sms, cudaStream_t s) {
  if (n <= 0) return 0;
  long long blocks = (n + kTcRows - 1) / kTcRows;
  if (blocks > (long long)sms * 4) blocks = (long long)sms * 4;
  k_mlp_forward_tc<<<(unsigned)blocks, 128, 0, s>>>(n, xs, p, W2h, y, err);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace mhd

namespace mhd {
int issue_surrogate_tc(const PatchDev& P, const ThermalDev& th, const MlpDev& M, int* fb_list,
                       unsigned long long* fb_count, int sms, cudaStream_t s, long long* launches) {
  const long long nc = (long long)P.n[0] * P.n[1] * P.n[2];
  long long blocks = (nc + kTcRows - 1) / kTcRows;
  if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
  k_thermal_surrogate_tc<<<(unsigned)blocks, 128, 0, s>>>(P, th, M, fb_list, fb_count);
  *launches += 1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
}  // namespace mhd
