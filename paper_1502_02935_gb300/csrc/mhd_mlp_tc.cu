// mhd_mlp_tc.cu -- the surrogate's 64-wide products on the 5th-generation tensor cores
// (tcgen05.mma with the accumulators in tensor memory): inference (k_mlp_forward_tc, and
// k_thermal_surrogate_tc in the thermal step) and training (k_mlp_grad_tc, further down).
//
// Inference: one CTA of 128 threads takes 128 rows.  Each thread computes its row of h1 =
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

__device__ __forceinline__ float tc_tanh(float z) { return mlp_tanh(z); }

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
// the training range or over the bound go to the fallback list (see mhd_mlp.cu).  With Wst,
// each updated cell also stores its W (the recovery of the new state) there and the block's
// CFL limit goes into the patch's (reset) slot: the recovery that would otherwise start the
// next step.
__global__ void __launch_bounds__(128, 8) k_thermal_surrogate_tc(PatchDev P, ThermalDev th, MlpDev M,
                                                              int* __restrict__ fb_list,
                                                              unsigned long long* __restrict__ fb_count,
                                                              float* __restrict__ Wst) {
  __shared__ TcSmem S;
  const uint32_t taddr = tc_setup(S, M.p, M.W2h);
  uint32_t phase = 0;
  const long long nc = (long long)P.n[0] * P.n[1] * P.n[2];
  const double dt = *P.dt_used;
  const float ldt = log10f((float)dt);
  const DlinConst dc = th_dlin_const(th, P.gm1);
  // FP32 copies: only the pressure needs FP64 (the cancellation in E - kinetic - magnetic);
  // T and n_H feed FP32 features, and the energy change is an FP32 increment added to the
  // FP64 energy, as the fluxes of the step are
  const float cef = (float)th_cef(P, th), tpp = (float)th.t_per_pr, npr = (float)th.nh_per_rho;
  const float zf = (float)th.z;
  const float kLn10 = 2.302585093f;
  float lim = INFINITY;
  const long long FS = P.FS;
  for (long long base = (long long)blockIdx.x * kTcRows; base < nc; base += (long long)gridDim.x * kTcRows) {
    const long long c = base + threadIdx.x;
    int i = 0, j = 0, k = 0;
    bool inrange = false;
    float tf = 0.f, rf = 0.f;
    float x[4] = {0.f, 0.f, 0.f, 0.f}, dl = 0.f;
    long long cs = 0;
    // The recovery's terms that the isochoric change of E leaves alone, computed once: the
    // FP64 ones for T here and for the new pressure below, the bulk-type velocity and field
    // for the new W (prim_core's arithmetic, so W is what a recovery pass would store).
    double rho = 1.0, e0 = 0.0;
    RecoveryTerms rt{1.0, 0.0, 0.0};
    float vx = 0.f, vy = 0.f, vz = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
    if (c < nc) {
      i = (int)(c % P.n[0]);
      const long long r = c / P.n[0];
      j = (int)(r % P.n[1]);
      k = (int)(r / P.n[1]);
      cs = sidx(P, i, j, k);
      rho = P.Un[cs];
      const double mx = P.Un[MX * FS + cs], my = P.Un[MY * FS + cs], mz = P.Un[MZ * FS + cs];
      e0 = P.Un[EN * FS + cs];
      const double sbx = P.Un[BXF * FS + cs] + P.Un[BXF * FS + sidx(P, fmap(P, 0, i + 1), j, k)];
      const double sby = P.Un[BYF * FS + cs] + P.Un[BYF * FS + sidx(P, i, fmap(P, 1, j + 1), k)];
      const double sbz = P.Un[BZF * FS + cs] + P.Un[BZF * FS + sidx(P, i, j, fmap(P, 2, k + 1))];
      rt = recovery_terms<float>(rho, mx, my, mz, sbx, sby, sbz);
      const double p = recovery_pressure(P, rt, e0);
      const double irho = rt.irho;
      const float rirho = d2f_alu(irho);
      vx = __fmul_rn(d2f_alu(mx), rirho), vy = __fmul_rn(d2f_alu(my), rirho), vz = __fmul_rn(d2f_alu(mz), rirho);
      bx = d2f_alu(sbx) * 0.5f, by = d2f_alu(sby) * 0.5f, bz = d2f_alu(sbz) * 0.5f;
      // T and n_H in FP32 (integer-pipe conversions); the clamp lets a NaN through to fall back
      rf = d2f_alu(rho);
      tf = tpp * d2f_alu(p) * d2f_alu(irho);
      const float raw[4] = {log10f(npr * rf), log10f(tf < 10.0f ? 10.0f : (tf > 1e8f ? 1e8f : tf)), ldt, zf};
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
        // T1 = clamp(clamp(T) 10^d); the change T1 - T without cancellation when no clamp
        // acts (T0 (10^d - 1) = T0 expm1(d ln 10))
        const float T0 = tf < 10.0f ? 10.0f : (tf > 1e8f ? 1e8f : tf);
        const float T1 = T0 * exp10f(d);
        const float dT = (T0 != tf || !(T1 >= 10.0f && T1 <= 1e8f))
                             ? (T1 < 10.0f ? 10.0f : (T1 > 1e8f ? 1e8f : T1)) - tf
                             : T0 * expm1f(d * kLn10);
        const double e1 = e0 + f2d_alu(cef * rf * dT);
        P.Un[EN * FS + cs] = e1;
        if (Wst) {
          // (the floors' FP64 comparisons only where the FP32 pre-check cannot decide them)
          if (P.floors && !surely_above(rf, P.rho_floor_f) && rho < P.rho_floor) {
            // the recovery floors the density (not after the step's own floors): in full
            lim = fminf(lim, prim_point<float>(P, P.Un, Wst, i, j, k, true, true));
          } else {
            double p1 = recovery_pressure(P, rt, e1);
            float pr = d2f_alu(p1);
            if (P.floors && !surely_inside(pr, rf * P.pr_floor_f, rf * P.pr_ceil_f)) {
              const double lo = rho * P.pr_floor, hi = rho * P.pr_ceil;
              p1 = p1 < lo ? lo : (p1 > hi ? hi : p1);
              pr = d2f_alu(p1);
            }
            lim = fminf(lim, prim_store<float>(P, rf, vx, vy, vz, bx, by, bz, pr, finite_d(e1), Wst,
                                               qidx(P, i, j, k), true, true));
          }
        }
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
  if (Wst) block_min_atomic(lim, P.cfl_min);
  tc_teardown(taddr);
}

// ------------------------------------------------------------- training --
// Loss and gradient contributions of one minibatch on the tensor cores, 128 rows per CTA.
// Three tcgen05.mma (M = 128, N = 64, BF16 x BF16 -> FP32 in TMEM):
//   Z2  = H1 W2^T   K = 64 inputs:  A = H1 [row][in],     B = W2 [out][in]     columns   0-63
//   dH1 = dZ2 W2    K = 64 outputs: A = dZ2 [row][out],   B = W2^T [in][out]   columns  64-127
//   dW2 = dZ2^T H1  K = 128 rows:   A = dZ2^T [out][row] (rows 64-127 zero),
//                                   B = H1^T [in][row]                        columns 128-191
// all operands K-major in the no-swizzle core-matrix layout.  The FP32 parts (layer 1, the
// head, the tanh derivatives and the small W1, b1, b2, w3, b3 gradients) run on four
// threads per row, 16 columns each: warp w reads TMEM lanes 32 (w mod 4) and up (its rows)
// at columns 16 (w / 4) and up.  Sums over rows are warp reduce-scatters followed by a
// four-way shared-memory sum.
constexpr int kTrRows = 128;
constexpr int kTrSlices = 4;                     // threads per row
constexpr int kTrThreads = kTrRows * kTrSlices;  // 512
constexpr int kTrCols16 = kHid / kTrSlices;      // columns per thread
constexpr unsigned kTrCols = 256;                // TMEM columns allocated (three 64-wide accumulators)

struct TrainTcSmem {
  alignas(1024) __nv_bfloat16 Ah1[kTrRows * kHid];      // H1     [row][in]  K = 64
  alignas(1024) __nv_bfloat16 Bw2[kHid * kHid];         // W2     [out][in]  K = 64
  alignas(1024) __nv_bfloat16 Bw2t[kHid * kHid];        // W2^T   [in][out]  K = 64
  alignas(1024) __nv_bfloat16 Adz[kTrRows * kHid];      // dZ2    [row][out] K = 64
  alignas(1024) __nv_bfloat16 Adzt[kTrRows * kTrRows];  // dZ2^T  [out][row] K = 128
  alignas(1024) __nv_bfloat16 Bh1t[kHid * kTrRows];     // H1^T   [in][row]  K = 128
  alignas(8) unsigned long long mbar;
  uint32_t taddr;
  int timed_out;
  float W1[kHid * 4], b1[kHid], b2[kHid], w3[kHid], b3;
  float ypart[kTrSlices][kTrRows];  // the four partial sums w3 . h2 of each row
  float red[7 * kHid];              // gw3 | gb2 | gb1 | gW1 [64][4]
};

// byte offset of (row r, k) in the K-major no-swizzle core-matrix layout of a K-wide operand
__device__ __forceinline__ uint32_t cm_off(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (16 * K) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void put_bf16(void* base, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(static_cast<char*>(base) + off) = __float2bfloat16_rn(v);
}

// D (+)= A B^T over `ksteps` K = 16 chunks; A and B share the stride byte offset `sbo`
// (16 x their K in bytes).
__device__ __forceinline__ void tc_mma_k(uint32_t d, uint32_t a0, uint32_t b0, uint32_t sbo, int ksteps) {
  constexpr uint32_t idesc = idesc_bf16(kTrRows, kHid);
  for (int kc = 0; kc < ksteps; ++kc) {
    const uint64_t ad = smem_desc(a0 + kc * 256, 128, sbo);
    const uint64_t bd = smem_desc(b0 + kc * 256, 128, sbo);
    const uint32_t acc = kc > 0 ? 1u : 0u;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Every thread waits (bounded by the global timer) for the MMAs committed to the barrier;
// returns false, for every thread, if the wait ran out.
__device__ __forceinline__ bool tc_wait_all(TrainTcSmem& S, uint32_t& phase) {
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
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  return S.timed_out == 0;
}

// 16 FP32 values of TMEM lane (32 (warp mod 4) + lane) from column col.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t col, float (&v)[kTrCols16]) {
  const uint32_t lane_base = (uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16;
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr + lane_base + col));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// Sum of a 16-vector over the warp's 32 lanes: recursive halving over lane bits 2, 1, 0,
// then a butterfly over bits 3 and 4.  Lane l ends with the totals of entries 2 (l mod 8)
// and 2 (l mod 8) + 1 in v[0] and v[1] (18 shuffles instead of 80).
__device__ __forceinline__ void warp_reduce_scatter16(float (&v)[kTrCols16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = kTrCols16 / 2; h >= 2; h >>= 1) {
    const bool up = (lane & (h >> 1)) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = up ? v[i] : v[i + h];
      const float keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h >> 1);
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    v[i] += __shfl_xor_sync(0xffffffffu, v[i], 8);
    v[i] += __shfl_xor_sync(0xffffffffu, v[i], 16);
  }
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// step_dev != nullptr: the step index is read from device memory (a training run replayed
// as a graph); the squared errors are added to *loss_sum from step loss_from on.
__global__ void __launch_bounds__(kTrThreads) k_mlp_grad_tc(MlpDev M, const float* __restrict__ data,
                                                            long long nrows, unsigned long long seed, long long step,
                                                            const long long* __restrict__ step_dev,
                                                            long long loss_from, int batch, float* __restrict__ grad,
                                                            float* __restrict__ loss_sum, int* __restrict__ err) {
  if (step_dev) step = *step_dev;
  const bool want_loss = step >= loss_from;
  extern __shared__ unsigned char tr_raw[];
  TrainTcSmem& S = *reinterpret_cast<TrainTcSmem*>(((uintptr_t)tr_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = (warp & 3) * 32 + lane, sl = warp >> 2, c0 = sl * kTrCols16;
  // weights: W2 in both layouts and the FP32 vectors; rows 64-127 of dZ2^T zeroed
  for (int q = tid; q < kHid * kHid; q += blockDim.x) {
    const int o = q >> 6, i = q & 63;
    const __nv_bfloat16 w = M.W2h[q];
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(S.Bw2) + cm_off(o, i, kHid)) = w;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(S.Bw2t) + cm_off(i, o, kHid)) = w;
  }
  {
    uint4* z = reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.Adzt) + cm_off(kHid, 0, kTrRows));
    for (int q = tid; q < kHid * kTrRows * 2 / 16; q += blockDim.x) z[q] = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int q = tid; q < kHid * 4; q += blockDim.x) S.W1[q] = M.p[kOffW1 + q];
  for (int q = tid; q < kHid; q += blockDim.x) {
    S.b1[q] = M.p[kOffB1 + q];
    S.b2[q] = M.p[kOffB2 + q];
    S.w3[q] = M.p[kOffW3 + q];
  }
  for (int q = tid; q < 7 * kHid; q += blockDim.x) S.red[q] = 0.f;
  if (tid == 0) {
    S.b3 = M.p[kOffB3];
    S.timed_out = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.taddr)),
                 "r"(kTrCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // this thread's row: drawn by the counter-based hash of (seed, step, row), or given in
  // order when seed == 0; standardised
  const long long r = (long long)blockIdx.x * kTrRows + row;
  long long src = -1;
  if (r < batch)
    src = seed ? (long long)(mix64(seed ^ mix64((unsigned long long)step * 0x100000001ull + r)) %
                             (unsigned long long)nrows)
               : r;
  float x[4], target = 0.f;
#pragma unroll
  for (int f = 0; f < 4; ++f) x[f] = src >= 0 ? mlp_standardize(M, f, data[src * kHvCols + f]) : 0.f;
  if (src >= 0) target = data[src * kHvCols + 4];
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = S.taddr;
  // layer 1: this thread's 16 columns of H1 = tanh(W1 x + b1), into both operand layouts;
  // the FP32 values stay in registers for the derivative of the backward pass
  float h1[kTrCols16];
#pragma unroll
  for (int q = 0; q < kTrCols16; ++q) {
    const int c = c0 + q;
    const float z = S.b1[c] + S.W1[c * 4] * x[0] + S.W1[c * 4 + 1] * x[1] + S.W1[c * 4 + 2] * x[2] +
                    S.W1[c * 4 + 3] * x[3];
    h1[q] = tc_tanh(z);
    put_bf16(S.Ah1, cm_off(row, c, kHid), h1[q]);
    put_bf16(S.Bh1t, cm_off(c, row, kTrRows), h1[q]);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  uint32_t phase = 0;
  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tc_mma_k(taddr, smem_u32(S.Ah1), smem_u32(S.Bw2), 16 * kHid, kHid / 16);
    tc_commit(&S.mbar);
  }
  bool ok = tc_wait_all(S, phase);
  float v[kTrCols16], t[kTrCols16];
  if (ok) {
    // head: h2 = tanh(z2 + b2); the four partial sums of w3 . h2 meet in shared memory
    tc_ld16(taddr, (uint32_t)c0, v);
    float yp = 0.f;
#pragma unroll
    for (int q = 0; q < kTrCols16; ++q) {
      v[q] = tc_tanh(v[q] + S.b2[c0 + q]);
      yp += S.w3[c0 + q] * v[q];
    }
    S.ypart[sl][row] = yp;
  }
  __syncthreads();
  if (ok) {
    // y = w3 . h2 + b3; loss (y - target)^2, dy = 2 (y - target) / B
    const float y = S.b3 + S.ypart[0][row] + S.ypart[1][row] + S.ypart[2][row] + S.ypart[3][row];
    const float e = src >= 0 ? y - target : 0.f;
    const float dy = 2.f * e / (float)batch;
    if (sl == 0) {
      const float l = warp_sum(e * e), db3 = warp_sum(dy);
      if (lane == 0 && l != 0.f && want_loss) atomicAdd(loss_sum, l);
      if (lane == 0 && db3 != 0.f) atomicAdd(grad + kOffB3, db3);
    }
    const int cr = c0 + 2 * (lane & 7);  // the two columns this lane holds after a reduce-scatter
    const bool adds = lane < 8;
    // gw3 = sum dy h2
#pragma unroll
    for (int q = 0; q < kTrCols16; ++q) t[q] = dy * v[q];
    warp_reduce_scatter16(t);
    if (adds) {
      atomicAdd(&S.red[cr], t[0]);
      atomicAdd(&S.red[cr + 1], t[1]);
    }
    // dz2 = dy w3 (1 - h2^2): BF16 operands of the backward products, FP32 sum for gb2
#pragma unroll
    for (int q = 0; q < kTrCols16; ++q) {
      const int c = c0 + q;
      t[q] = dy * S.w3[c] * (1.f - v[q] * v[q]);
      put_bf16(S.Adz, cm_off(row, c, kHid), t[q]);
      put_bf16(S.Adzt, cm_off(c, row, kTrRows), t[q]);
    }
    warp_reduce_scatter16(t);
    if (adds) {
      atomicAdd(&S.red[kHid + cr], t[0]);
      atomicAdd(&S.red[kHid + cr + 1], t[1]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (ok && tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tc_mma_k(taddr + kHid, smem_u32(S.Adz), smem_u32(S.Bw2t), 16 * kHid, kHid / 16);
    tc_mma_k(taddr + 2 * kHid, smem_u32(S.Adzt), smem_u32(S.Bh1t), 16 * kTrRows, kTrRows / 16);
    tc_commit(&S.mbar);
  }
  if (ok) ok = tc_wait_all(S, phase);
  if (ok) {
    // dz1 = dh1 (1 - h1^2) with the FP32 h1; gb1 = sum dz1, gW1 = sum dz1 x^T
    tc_ld16(taddr, (uint32_t)(kHid + c0), v);
#pragma unroll
    for (int q = 0; q < kTrCols16; ++q) {
      v[q] *= 1.f - h1[q] * h1[q];
      t[q] = v[q];
    }
    const int cr = c0 + 2 * (lane & 7);
    const bool adds = lane < 8;
    warp_reduce_scatter16(t);
    if (adds) {
      atomicAdd(&S.red[2 * kHid + cr], t[0]);
      atomicAdd(&S.red[2 * kHid + cr + 1], t[1]);
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
#pragma unroll
      for (int q = 0; q < kTrCols16; ++q) t[q] = v[q] * x[f];
      warp_reduce_scatter16(t);
      if (adds) {
        atomicAdd(&S.red[3 * kHid + cr * 4 + f], t[0]);
        atomicAdd(&S.red[3 * kHid + (cr + 1) * 4 + f], t[1]);
      }
    }
    // dW2: TMEM lanes 0-63 of the third accumulator (warps with w mod 4 < 2); the load is
    // warp-collective, lanes 64-127 hold the zero padding and are not added
    tc_ld16(taddr, (uint32_t)(2 * kHid + c0), v);
    if ((warp & 3) < 2) {
#pragma unroll
      for (int q = 0; q < kTrCols16; ++q) atomicAdd(grad + kOffW2 + row * kHid + c0 + q, v[q]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (ok) {
    for (int q = tid; q < kHid; q += blockDim.x) {
      atomicAdd(grad + kOffW3 + q, S.red[q]);
      atomicAdd(grad + kOffB2 + q, S.red[kHid + q]);
      atomicAdd(grad + kOffB1 + q, S.red[2 * kHid + q]);
    }
    for (int q = tid; q < 4 * kHid; q += blockDim.x) atomicAdd(grad + kOffW1 + q, S.red[3 * kHid + q]);
  } else if (tid == 0) {
    atomicOr(err, ERR_TIMEOUT);
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTrCols));
}

int mlp_grad_tc_setup() {
  static bool done = false;
  if (done) return 0;
  const int smem = (int)(sizeof(TrainTcSmem) + 1024);
  if (cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return -1;
  done = true;
  return 0;
}

int mlp_grad_tc(const MlpDev& M, const float* data, long long nrows, unsigned long long seed, long long step,
                const long long* step_dev, long long loss_from, int batch, float* grad, float* loss_sum, int* err,
                cudaStream_t s) {
  if (mlp_grad_tc_setup()) return -1;
  const size_t smem = sizeof(TrainTcSmem) + 1024;
  const int blocks = (batch + kTrRows - 1) / kTrRows;
  k_mlp_grad_tc<<<blocks, kTrThreads, smem, s>>>(M, data, nrows, seed, step, step_dev, loss_from, batch, grad,
                                               loss_sum, err);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
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
                       unsigned long long* fb_count, float* Wst, int sms, cudaStream_t s, long long* launches) {
  const long long nc = (long long)P.n[0] * P.n[1] * P.n[2];
  long long blocks = (nc + kTcRows - 1) / kTcRows;
  if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
  k_thermal_surrogate_tc<<<(unsigned)blocks, 128, 0, s>>>(P, th, M, fb_list, fb_count, Wst);
  *launches += 1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
}  // namespace mhd
