// mhd_persistent.cuh -- one persistent launch per van Leer step for a batch of
// independent patches of uneven size.
//
// The launch is cooperative (all CTAs co-resident).  It runs the eight phases of a step
// (recovery+CFL, fluxes, corner EMFs, update; twice) over the work list of every patch,
// with a grid-wide barrier between phases.  Work items are tiles of TX x TY points of one
// z-plane of a phase's index box; each CTA takes a contiguous range of the phase's tiles,
// so that it rarely changes patch (a strided assignment reloaded the patch descriptor at
// almost every tile of the small patches).  Patches are listed largest first.  Each patch
// keeps its own CFL time step.  (The update fused with the recovery, which the per-phase
// launches use, is slower here: it needs more resident warps than this single kernel has.)
//
// The barrier's wait is bounded by the GPU global timer: a CTA that waits longer than the
// limit sets ERR_TIMEOUT in the device error word and every CTA returns at its next
// barrier, so a failed or non-resident grid ends the kernel instead of hanging it.
#pragma once
#include "mhd_device.cuh"

namespace mhd {

struct BoxDev {
  int lo[3];
  int ext[3];
  int ntx, nty;
  long long count;  // tiles in this box: ntx * nty * ext[2]
};

enum { BOX_PRIM = 0, BOX_FLUX0 = 1, BOX_EDGE = 4, NBOX = 5 };

struct PersistentArgs {
  const PatchDev* P;          // [np], largest patch first
  const BoxDev* box;          // [np][NBOX]
  const long long* pre_prim;  // [np + 1] tile prefix sums per phase
  const long long* pre_flux;
  const long long* pre_edge;
  int np;
  int TX, TY;
  double dt_host;  // > 0: that dt for every patch; else cfl * the patch's own CFL limit
  double cfl;
  SourceDev src;
  unsigned int* bar;  // [0] arrivals, [1] generation
  int* err;
  unsigned long long limit_ns;  // longest wait at one barrier
  int phantom;                  // extra arrivals the barrier waits for (0; > 0 only to test the timeout)
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier with a bounded wait.  Returns false (for the whole CTA) once any
// CTA has timed out.
__device__ __forceinline__ bool grid_barrier(const PersistentArgs& A) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* vgen = A.bar + 1;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int target = gridDim.x + (unsigned)A.phantom;
    const unsigned int arrived = atomicAdd(A.bar, 1u) + 1u;
    if (arrived == target) {
      atomicExch(A.bar, 0u);
      __threadfence();
      atomicAdd(A.bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*vgen == g) {
        if (global_ns() - t0 > A.limit_ns) {
          atomicOr(A.err, ERR_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int*)A.err & ERR_TIMEOUT) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// block-wide minimum (any blockDim up to 1024), one ordered-bits atomicMin
__device__ __forceinline__ void tile_min_atomic(double v, unsigned long long* slot) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)((blockDim.x + 31) >> 5) ? red[lane] : INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w < v ? w : v;
    }
    if (lane == 0 && v < INFINITY) atomicMin(slot, dbits(v));
  }
  __syncthreads();
}

enum { PH_PRIM = 0, PH_FLUX = 1, PH_EMF = 2, PH_UPDATE = 3 };

template <class R, int PH>
__device__ __forceinline__ void persistent_phase(const PersistentArgs& A, int stage, PatchDev& sP,
                                                 int& cur) {
  const long long* pre = PH == PH_PRIM ? A.pre_prim : (PH == PH_FLUX ? A.pre_flux : A.pre_edge);
  const long long total = pre[A.np];
  // this CTA's contiguous share of the phase's tiles
  const long long t0 = total * blockIdx.x / gridDim.x, t1 = total * (blockIdx.x + 1) / gridDim.x;
  if (t0 >= t1) return;
  int p = 0;  // last patch with pre[p] <= t0
  {
    int lo = 0, hi = A.np - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pre[mid] <= t0) lo = mid;
      else hi = mid - 1;
    }
    p = lo;
  }
  for (long long t = t0; t < t1; ++t) {
    while (t >= pre[p + 1]) ++p;
    if (p != cur) {
      __syncthreads();
      const int* src = (const int*)(A.P + p);
      int* dst = (int*)&sP;
      for (int w = threadIdx.x; w < (int)(sizeof(PatchDev) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
      __syncthreads();
      if (threadIdx.x == 0) cur = p;
      __syncthreads();
    }
    long long lt = t - pre[p];
    int bi = PH == PH_PRIM ? BOX_PRIM : (PH == PH_FLUX ? BOX_FLUX0 : BOX_EDGE);
    if (PH == PH_FLUX) {
      while (bi < BOX_FLUX0 + 2 && lt >= A.box[p * NBOX + bi].count) {
        lt -= A.box[p * NBOX + bi].count;
        ++bi;
      }
    }
    const BoxDev B = A.box[p * NBOX + bi];
    const int tx = (int)(lt % B.ntx);
    const long long r = lt / B.ntx;
    const int ty = (int)(r % B.nty);
    const int z = (int)(r / B.nty);
    const int i = B.lo[0] + tx * A.TX + (int)(threadIdx.x % A.TX);
    const int j = B.lo[1] + ty * A.TY + (int)(threadIdx.x / A.TX);
    const int k = B.lo[2] + z;
    const bool in = i < B.lo[0] + B.ext[0] && j < B.lo[1] + B.ext[1];
    const double* Usrc = stage == 0 ? sP.Un : sP.Uh;
    if (PH == PH_PRIM) {
      double lim = INFINITY;
      if (in) {
        const bool interior = stage == 0 && i >= 0 && i < sP.n[0] && j >= 0 && j < sP.n[1] && k >= 0 &&
                              k < sP.n[2];
        lim = Ar<R>::to_d(prim_point<R>(sP, Usrc, (R*)sP.W, i, j, k, true, interior));
      }
      if (stage == 0) tile_min_atomic(lim, sP.cfl_min);
    } else if (PH == PH_FLUX) {
      if (in) {
        const int d = bi - BOX_FLUX0;
        if (stage == 0) {
          if (d == 0) flux_point<R, 0, 1>(sP, (const R*)sP.W, Usrc, (R*)sP.F[0], i, j, k, sP.riemann);
          else if (d == 1) flux_point<R, 1, 1>(sP, (const R*)sP.W, Usrc, (R*)sP.F[1], i, j, k, sP.riemann);
          else flux_point<R, 2, 1>(sP, (const R*)sP.W, Usrc, (R*)sP.F[2], i, j, k, sP.riemann);
        } else {
          if (d == 0) flux_point<R, 0, 2>(sP, (const R*)sP.W, Usrc, (R*)sP.F[0], i, j, k, sP.riemann);
          else if (d == 1) flux_point<R, 1, 2>(sP, (const R*)sP.W, Usrc, (R*)sP.F[1], i, j, k, sP.riemann);
          else flux_point<R, 2, 2>(sP, (const R*)sP.W, Usrc, (R*)sP.F[2], i, j, k, sP.riemann);
        }
      }
    } else if (PH == PH_EMF) {
      if (in) emf_point<R>(sP, (const R*)sP.W, (R*)sP.E, i, j, k);
    } else {
      const double dt = A.dt_host > 0.0 ? A.dt_host : A.cfl * __longlong_as_double((long long)*sP.cfl_min);
      const R h = Ar<R>::from_d(stage == 0 ? 0.5 * dt : dt);
      if (stage == 1 && lt == 0 && threadIdx.x == 0) *sP.dt_used = dt;
      if (in) update_point<R>(sP, sP.Un, Usrc, stage == 0 ? sP.Uh : sP.Un, (const R*)sP.E, h, A.src, i, j, k);
    }
  }
}

template <class R>
__global__ void __launch_bounds__(512) k_persistent(PersistentArgs A) {
  __shared__ PatchDev sP;
  __shared__ int cur;
  if (threadIdx.x == 0) cur = -1;
  __syncthreads();
  for (int stage = 0; stage < 2; ++stage) {
    persistent_phase<R, PH_PRIM>(A, stage, sP, cur);
    if (!grid_barrier(A)) return;
    persistent_phase<R, PH_FLUX>(A, stage, sP, cur);
    if (!grid_barrier(A)) return;
    persistent_phase<R, PH_EMF>(A, stage, sP, cur);
    if (!grid_barrier(A)) return;
    persistent_phase<R, PH_UPDATE>(A, stage, sP, cur);
    if (stage == 0 && !grid_barrier(A)) return;
  }
}

template <class R>
static int issue_persistent(const PersistentArgs& A, int blocks, cudaStream_t s, long long* launches) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks, 1, 1);
  cfg.blockDim = dim3((unsigned)(A.TX * A.TY), 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  *launches += 1;
  return cudaLaunchKernelEx(&cfg, k_persistent<R>, A) == cudaSuccess ? 0 : -1;
}

template <class R>
static int persistent_occupancy(int block, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_persistent<R>, block, 0) == cudaSuccess
             ? 0
             : -1;
}

}  // namespace mhd
