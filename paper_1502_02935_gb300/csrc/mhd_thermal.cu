// mhd_thermal.cu -- kernels of the thermal source term: the plain FP64 integrator per cell
// (see mhd_thermal.cuh).
#include "mhd_thermal.cuh"
#include "mhd_thermal_launch.h"

namespace mhd {

__device__ __forceinline__ void warp_add(unsigned long long* slot, unsigned long long v) {
  const unsigned long long tot = __reduce_add_sync(0xffffffffu, (unsigned)v);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(slot, tot);
}

__global__ void __launch_bounds__(256) k_thermal_plain(PatchDev P, ThermalDev th) {
  const long long nc = (long long)P.n[0] * P.n[1] * P.n[2];
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double dt = *P.dt_used;
  int nsub = 0, capped = 0, live = 0;
  if (c < nc) {
    const int i = (int)(c % P.n[0]);
    const long long r = c / P.n[0];
    const int j = (int)(r % P.n[1]);
    const int k = (int)(r / P.n[1]);
    double T, nh, ce;
    th_cell(P, th, P.Un, i, j, k, T, nh, ce);
    int st;
    const double T1 = th_integrate(T, nh, ce, dt, th, &st, &nsub);
    P.Un[EN * P.FS + sidx(P, i, j, k)] += ce * (T1 - T);
    capped = (st & (TST_SUBSTEP_CAP | TST_NEWTON_CAP)) != 0;
    live = 1;
    if (th.hv_data) {
      // sampled cells: a hash of the cell index salted by this step's dt
      const unsigned long long salt = (unsigned long long)__double_as_longlong(dt);
      unsigned long long h = (unsigned long long)c * 0x9E3779B97F4A7C15ull ^ salt;
      h ^= h >> 29;
      h *= 0xBF58476D1CE4E5B9ull;
      h ^= h >> 32;
      if (h % (unsigned long long)th.hv_stride == 0) {
        // the step's pair plus pairs for dt/3 and 3 dt from the same integrator, so that the
        // training set spans half a decade of dt around the steps it was harvested from
        const unsigned long long row0 = atomicAdd(th.hv_count, 3ull);
        const double Tc = th_clamp(T);
        const double fac[3] = {1.0, 1.0 / 3.0, 3.0};
#pragma unroll 1
        for (int v = 0; v < 3; ++v) {
          int st2, ns2;
          const double Th = v == 0 ? T1 : th_integrate(T, nh, ce, dt * fac[v], th, &st2, &ns2);
          float* o = th.hv_data + ((row0 + v) % (unsigned long long)th.hv_cap) * 5;
          o[0] = (float)log10(nh);
          o[1] = (float)log10(Tc);
          o[2] = (float)log10(dt * fac[v]);
          o[3] = (float)th.z;
          o[4] = (float)(log10(Th) - log10(Tc));
        }
      }
    }
  }
  warp_add(th.stats + 0, (unsigned long long)live);
  warp_add(th.stats + 1, (unsigned long long)nsub);
  warp_add(th.stats + 2, (unsigned long long)capped);
}

__global__ void __launch_bounds__(256) k_thermal_cells(long long n, const double* __restrict__ T0,
                                                       const double* __restrict__ nh, const double* __restrict__ ce,
                                                       const double* __restrict__ dt, ThermalDev th,
                                                       double* __restrict__ T_out, int* __restrict__ status) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  int st, nsub;
  T_out[q] = th_integrate(T0[q], nh[q], ce[q], dt[q], th, &st, &nsub);
  if (status) status[q] = st;
}

int issue_thermal_cells(long long n, const double* T0, const double* nh, const double* ce, const double* dt,
                        const ThermalDev& th, double* T_out, int* status, cudaStream_t s) {
  if (n <= 0) return 0;
  k_thermal_cells<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, T0, nh, ce, dt, th, T_out, status);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int issue_thermal(const PatchDev& P, const ThermalDev& th, cudaStream_t s, long long* launches) {
  const long long nc = (long long)P.n[0] * P.n[1] * P.n[2];
  if (th.mode == TH_PLAIN) {
    k_thermal_plain<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(P, th);
    *launches += 1;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace mhd
