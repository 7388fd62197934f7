// mhd_kernels.cuh -- CUDA kernels of the MHD step (one kernel per phase, grid over the
// phase's index box) and the host-side launch sequence of one van Leer step.
// Included by one translation unit per precision, which exports a Backend table.
#pragma once
#include "mhd_backend.h"
#include "mhd_device.cuh"
#include "mhd_persistent.cuh"

namespace mhd {

constexpr int kBlock = 256;

// index box [lo, lo + ext) per axis; the kernel grid is (ceil(ex*ey/kBlock), ez)
struct Range {
  int lo[3];
  int ext[3];
};

__device__ __forceinline__ bool range_point(const Range& rg, int& i, int& j, int& k) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long plane = (long long)rg.ext[0] * rg.ext[1];
  if (r >= plane) return false;
  const int jj = (int)(r / rg.ext[0]);
  i = rg.lo[0] + (int)(r - (long long)jj * rg.ext[0]);
  j = rg.lo[1] + jj;
  k = rg.lo[2] + (int)blockIdx.y;
  return true;
}

// Block minimum of v in its own type (FP32 compares on the mixed path), then one
// ordered-bits atomicMin of its exact double value per block (deterministic).
template <class T>
__device__ __forceinline__ void block_min_atomic(T v, unsigned long long* slot) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  __shared__ T red[kBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : T(INFINITY);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w < v ? w : v;
    }
    if (lane == 0 && v < T(INFINITY)) atomicMin(slot, dbits(Ar<T>::to_d(v)));
  }
}

template <class R>
__global__ void __launch_bounds__(kBlock) k_prim(PatchDev P, const double* __restrict__ U, Range rg,
                                                 int store, int want_cfl) {
  int i, j, k;
  R lim = R(INFINITY);
  if (range_point(rg, i, j, k)) {
    const bool interior = want_cfl && i >= 0 && i < P.n[0] && j >= 0 && j < P.n[1] && k >= 0 &&
                          k < P.n[2];
    lim = prim_point<R>(P, U, (R*)P.W, i, j, k, store != 0, interior);
  }
  if (want_cfl) block_min_atomic(lim, P.cfl_min);
}

template <class R, int D, int ORDER>
__global__ void __launch_bounds__(kBlock) k_flux(PatchDev P, const double* __restrict__ Ub, Range rg) {
  int i, j, k;
  if (!range_point(rg, i, j, k)) return;
  flux_point<R, D, ORDER>(P, (const R*)P.W, Ub, (R*)P.F[D], i, j, k);
}

// corner EMFs: memory-latency bound; eight resident blocks per SM (measured)
template <class R>
__global__ void __launch_bounds__(kBlock, 8) k_emf(PatchDev P, Range rg) {
  int i, j, k;
  if (!range_point(rg, i, j, k)) return;
  emf_point<R>(P, (const R*)P.W, (R*)P.E, i, j, k);
}

// Stage update fused with the recovery of the new state (see update_fused_point).  Its FP64
// arithmetic is the bound; six resident blocks per SM (40 registers, a few spills to L1)
// hide the memory latency better than fewer blocks without spills (measured).  The
// predictor takes dt from the host or the CFL slot and records it; the corrector reuses the
// recorded dt and accumulates the CFL limit of the new state into the (reset) slot.
template <class R>
__global__ void __launch_bounds__(kBlock, 6) k_update_fused(PatchDev P, const double* __restrict__ Ub,
                                                         const double* __restrict__ Us,
                                                         double* __restrict__ Uo, Range rg, StageArgs a) {
  // dt and h once per block
  __shared__ R sh;
  if (threadIdx.x == 0) {
    double dt;
    if (a.stage == 0) {
      dt = a.dt_host > 0.0 ? a.dt_host : a.cfl * __longlong_as_double((long long)*P.cfl_min);
      if (blockIdx.x == 0 && blockIdx.y == 0) *P.dt_used = dt;
    } else {
      dt = *P.dt_used;
    }
    sh = Ar<R>::from_d(a.stage == 0 ? 0.5 * dt : dt);
  }
  __syncthreads();
  const R h = sh;
  int i, j, k, nfl = 0;
  R lim = R(INFINITY);
  if (range_point(rg, i, j, k))
    lim = update_fused_point<R>(P, Ub, Us, Uo, (const R*)P.E, h, a.src, i, j, k, a.stage == 1, &nfl);
  if (a.stage == 1) {
    if (P.floors) {
      const unsigned tot = __reduce_add_sync(0xffffffffu, (unsigned)nfl);
      if ((threadIdx.x & 31) == 0 && tot) atomicAdd(P.floored, (unsigned long long)tot);
    }
    block_min_atomic(lim, P.cfl_min);
  }
}

// W of the ghost shell from the interior W and U of the current state (see ghost_point).
template <class R>
__global__ void __launch_bounds__(kBlock) k_ghost(PatchDev P, const double* __restrict__ U) {
  const long long n = ghost_count(P);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    if (ghost_index(P, t, i, j, k)) ghost_point<R>(P, U, i, j, k);
  }
}

template <class R>
__global__ void k_hlld(int n, const double* __restrict__ wl, const double* __restrict__ wr,
                       const double* __restrict__ bn, double gam, double* __restrict__ flux) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  R a[7], b[7], f[8];
  const int src[7] = {0, 1, 2, 3, 4, 6, 7};
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    a[m] = (R)wl[8 * q + src[m]];
    b[m] = (R)wr[8 * q + src[m]];
  }
  hlld<R>(a, b, (R)bn[q], (R)gam, f);
#pragma unroll
  for (int m = 0; m < 7; ++m) flux[8 * q + src[m]] = (double)f[m];
  flux[8 * q + 5] = 0.0;
}

// ------------------------------------------------------------- host side ----

static inline dim3 grid_of(const Range& rg) {
  const long long plane = (long long)rg.ext[0] * rg.ext[1];
  return dim3((unsigned)((plane + kBlock - 1) / kBlock), (unsigned)rg.ext[2], 1);
}

static inline Range prim_range(const PatchDev& P) {
  Range r;
  for (int a = 0; a < 3; ++a) {
    r.lo[a] = -P.g2[a];
    r.ext[a] = P.n[a] + 2 * P.g2[a];
  }
  return r;
}

static inline Range interior_range(const PatchDev& P) {
  Range r;
  for (int a = 0; a < 3; ++a) {
    r.lo[a] = 0;
    r.ext[a] = P.n[a];
  }
  return r;
}

static inline Range flux_range(const PatchDev& P, int d) {
  Range r;
  for (int a = 0; a < 3; ++a) {
    if (a == d) {
      r.lo[a] = 0;
      r.ext[a] = P.n[a] + 1;
    } else if (P.act[a]) {
      r.lo[a] = -1;
      r.ext[a] = P.n[a] + 2;
    } else {
      r.lo[a] = 0;
      r.ext[a] = 1;
    }
  }
  return r;
}

static inline Range edge_range(const PatchDev& P) {
  Range r;
  for (int a = 0; a < 3; ++a) {
    r.lo[a] = 0;
    r.ext[a] = P.act[a] ? P.n[a] + 1 : 1;
  }
  return r;
}

// per-direction flux kernels and the corner-EMF kernel of one stage
template <class R>
static int issue_fluxes(const PatchDev& P, const StageArgs& a, const double* Usrc, cudaStream_t s, ProfRec* prof) {
  int nl = 0;
  for (int d = 0; d < 3; ++d) {
    if (!P.act[d]) continue;
    const Range fr = flux_range(P, d);
    ProfScope ps(prof, (a.stage == 0 ? KC_FLUX1 : KC_FLUX2) + d, s);
    if (a.stage == 0) {
      if (d == 0) k_flux<R, 0, 1><<<grid_of(fr), kBlock, 0, s>>>(P, Usrc, fr);
      if (d == 1) k_flux<R, 1, 1><<<grid_of(fr), kBlock, 0, s>>>(P, Usrc, fr);
      if (d == 2) k_flux<R, 2, 1><<<grid_of(fr), kBlock, 0, s>>>(P, Usrc, fr);
    } else {
      if (d == 0) k_flux<R, 0, 2><<<grid_of(fr), kBlock, 0, s>>>(P, Usrc, fr);
      if (d == 1) k_flux<R, 1, 2><<<grid_of(fr), kBlock, 0, s>>>(P, Usrc, fr);
      if (d == 2) k_flux<R, 2, 2><<<grid_of(fr), kBlock, 0, s>>>(P, Usrc, fr);
    }
    ++nl;
  }
  const Range er = edge_range(P);
  ProfScope ps(prof, KC_EMF, s);
  k_emf<R><<<grid_of(er), kBlock, 0, s>>>(P, er);
  return nl + 1;
}

// One stage of the step for one patch: per-direction fluxes and the corner EMFs from the
// stored W, then the fused update + recovery and the ghost shell of W.  The predictor writes U^{n+1/2} into Uh; the corrector, whose base is U^n and whose
// source term is evaluated at U^{n+1/2}, writes U^{n+1} into Uh as well (each cell's
// U^{n+1/2} is read by the thread that overwrites it, and no kernel of the stage reads the
// faces of Uh after the fluxes), so the caller swaps Un and Uh after the corrector.
template <class R>
static int issue_stage(const PatchDev& P, const StageArgs& a, cudaStream_t s, long long* launches,
                       ProfRec* prof) {
  const double* Usrc = a.stage == 0 ? P.Un : P.Uh;  // state the fluxes and S are built from
  int nl = issue_fluxes<R>(P, a, Usrc, s, prof);
  const Range er = edge_range(P);
  {
    ProfScope ps(prof, KC_UPDATE, s);
    k_update_fused<R><<<grid_of(er), kBlock, 0, s>>>(P, P.Un, Usrc, P.Uh, er, a);
    ++nl;
  }
  {
    ProfScope ps(prof, KC_GHOST, s);
    const long long ng = ghost_count(P);
    if (ng > 0) {
      long long blocks = (ng + kBlock - 1) / kBlock;
      if (blocks > 65535) blocks = 65535;
      k_ghost<R><<<(unsigned)blocks, kBlock, 0, s>>>(P, P.Uh);
      ++nl;
    }
  }
  *launches += nl;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// W of the current state over the padded box, and its CFL limit into the patch's slot
// (which the caller resets): the recovery that starts a step when W is not already that of
// the current state.
template <class R>
static int issue_prim(const PatchDev& P, cudaStream_t s, long long* launches, ProfRec* prof) {
  const Range pr = prim_range(P);
  ProfScope ps(prof, KC_PRIM, s);
  k_prim<R><<<grid_of(pr), kBlock, 0, s>>>(P, P.Un, pr, 1, 1);
  *launches += 1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class R>
static int issue_cfl(const PatchDev& P, cudaStream_t s, long long* launches) {
  const Range r = interior_range(P);
  k_prim<R><<<grid_of(r), kBlock, 0, s>>>(P, P.Un, r, 0, 1);
  *launches += 1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class R>
static int issue_hlld(int n, const double* wl, const double* wr, const double* bn, double gam,
                      double* flux, cudaStream_t s) {
  if (n <= 0) return 0;
  k_hlld<R><<<(n + 127) / 128, 128, 0, s>>>(n, wl, wr, bn, gam, flux);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class R> Backend make_backend() {
  Backend b;
  b.scratch_elem = sizeof(R);
  b.stage = &issue_stage<R>;
  b.prim = &issue_prim<R>;
  b.cfl = &issue_cfl<R>;
  b.hlld = &issue_hlld<R>;
  b.persistent = &issue_persistent<R>;
  b.occupancy = &persistent_occupancy<R>;
  return b;
}

}  // namespace mhd
