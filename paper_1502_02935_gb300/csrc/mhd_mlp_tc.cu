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

__global__ void __launch_bounds__(128) k_mlp_forward_tc(long long n, const float* __restrict__ xs,
                                                        const float* __restrict__ p,
                                                        const __nv_bfloat16* __restrict__ W2h,
                                                        float* __restrict__ y, int* __restrict__ err) {
  __shared__ TcSmem S;
  const int tid = threadIdx.x, warp = tid >> 5;
  // weights: W2 into the core-matrix layout, the FP32 layers into shared memory
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
  const uint32_t taddr = S.taddr;
  const uint32_t idesc = idesc_bf16(kTcRows, kHid);
  uint32_t phase = 0;
  for (long long base = (long long)blockIdx.x * kTcRows; base < n; base += (long long)gridDim.x * kTcRows) {
    // layer 1 for this thread's row
    const long long row = base + tid;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f, x3 = 0.f;
    if (row < n) {
      x0 = xs[row * 4 + 0];
      x1 = xs[row * 4 + 1];
      x2 = xs[row * 4 + 2];
      x3 = xs[row * 4 + 3];
    }
#pragma unroll 8
    for (int c = 0; c < kHid; ++c) {
      const float z = S.b1[c] + S.W1[c * 4] * x0 + S.W1[c * 4 + 1] * x1 + S.W1[c * 4 + 2] * x2 + S.W1[c * 4 + 3] * x3;
      *(__nv_bfloat16*)((char*)S.A + cm_offset(tid, c)) = __float2bfloat16_rn(tc_tanh(z));
    }
    // make the generic-proxy stores visible to the tensor cores' async proxy
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
    // wait for the MMAs (bounded)
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
      if (tid == 0) atomicOr(err, ERR_TIMEOUT);
      break;
    }
    // accumulator row of this thread: TMEM lane 32*warp + lane, columns 0..63
    float h2[kHid];
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
      for (int q = 0; q < 16; ++q) h2[c0 + q] = __uint_as_float(r[q]);
    }
    float out = S.b3;
#pragma unroll
    for (int c = 0; c < kHid; ++c) out += S.w3[c] * tc_tanh(h2[c] + S.b2[c]);
    if (row < n) y[row] = out;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // A and the accumulator are reused by the next tile
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(64));
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
