// mhd_thermal.cu -- kernels of the thermal source term: the plain FP64 integrator per cell
// (see mhd_thermal.cuh).
#include "mhd_thermal.cuh"
#include "mhd_thermal_launch.h"

namespace mhd {

// splitmix64 finaliser (Steele, Lea and Flood 2014): a counter-based hash for sampling
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

constexpr int kHvJitter = 3;         // jittered pairs per sampled cell
constexpr double kHvWidth = 0.5;     // offsets uniform in [-kHvWidth, kHvWidth] decades

// uniform offset in [-kHvWidth, kHvWidth] from the low 21 bits of u
__device__ __forceinline__ double hv_offset(unsigned long long u) {
  return kHvWidth * (2.0 * (double)(u & 0x1FFFFFull) / 2097151.0 - 1.0);
}

__device__ __forceinline__ void warp_add(unsigned long long* slot, unsigned long long v) {
  const unsigned long long tot = __reduce_add_sync(0xffffffffu, (unsigned)v);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(slot, tot);
}

__global__ void __launch_bounds__(256) k_thermal_plain(PatchDev P, ThermalDev th) {
  const long long nc = (long long)P.n[0] * P.n[1] * P.n[2];
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double dt = *P.dt_used;
  const double cef = th_cef(P, th);
  int nsub = 0, capped = 0, live = 0;
  if (c < nc) {
    const int i = (int)(c % P.n[0]);
    const long long r = c / P.n[0];
    const int j = (int)(r % P.n[1]);
    const int k = (int)(r / P.n[1]);
    double T, nh, ce;
    th_cell(P, th, P.Un, i, j, k, cef, T, nh, ce);
    int st;
    const double T1 = th_integrate(T, nh, ce, dt, th, &st, &nsub);
    P.Un[EN * P.FS + sidx(P, i, j, k)] += ce * (T1 - T);
    capped = (st & (TST_SUBSTEP_CAP | TST_NEWTON_CAP)) != 0;
    live = 1;
    if (th.hv_data) {
      // sampled cells: a hash of the cell index salted by this step's dt
      const unsigned long long salt = (unsigned long long)__double_as_longlong(dt);
      const unsigned long long h = mix64((unsigned long long)c * 0x9E3779B97F4A7C15ull ^ salt);
      if (h % (unsigned long long)th.hv_stride == 0) {
        // the step's own pair plus kHvJitter pairs from the same integrator at inputs shifted
        // by independent uniform offsets of up to kHvWidth decades in n_H (with c_e, which is
        // proportional to it), T and dt, so that the training set covers a neighbourhood of
        // the visited states rather than only the states themselves
        const unsigned long long row0 = atomicAdd(th.hv_count, (unsigned long long)(1 + kHvJitter));
        const double Tc = th_clamp(T);
        const DlinConst dc = th_dlin_const(th, P.gm1);
#pragma unroll 1
        for (int v = 0; v <= kHvJitter; ++v) {
          double nv = nh, cv = ce, Tv = Tc, dv = dt, Th = T1;
          if (v > 0) {
            unsigned long long u = mix64(h + 0xD1B54A32D192ED03ull * (unsigned long long)v);
            const double off[3] = {hv_offset(u), hv_offset(u >> 21), hv_offset(u >> 42)};
            const double sn = exp10(off[0]);
            nv = nh * sn;
            cv = ce * sn;
            Tv = th_clamp(Tc * exp10(off[1]));
            dv = dt * exp10(off[2]);
            int st2, ns2;
            Th = th_integrate(Tv, nv, cv, dv, th, &st2, &ns2);
          }
          // features as the surrogate computes them, the label q = change / S at those
          // features, and the change itself
          const float f0 = log10f((float)nv), f1 = log10f((float)Tv), f2 = log10f((float)dv);
          const float sc = th_scale(th_dlin(dc, f0, f1, f2));
          const double d = log10(Th) - log10(Tv);
          float q = (sc != 0.0f && isfinite(sc)) ? (float)(d / (double)sc) : 1.0f;
          q = fminf(fmaxf(q, -kQClip), kQClip);
          float* o = th.hv_data + ((row0 + v) % (unsigned long long)th.hv_cap) * kHvCols;
          o[0] = f0;
          o[1] = f1;
          o[2] = f2;
          o[3] = (float)th.z;
          o[4] = q;
          o[5] = (float)d;
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
