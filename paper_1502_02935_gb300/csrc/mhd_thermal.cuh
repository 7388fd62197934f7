// mhd_thermal.cuh -- thermal source term (heating/cooling in S of Eq. 2, Section 3.10 of
// arXiv:1502.02935), applied operator-split after each MHD step, in FP64.
//
// Isochoric update of each interior cell over the step's dt:
//   e = c_e T,  de/dt = (n_H Gamma - n_H^2 Lambda(T, Z)) / rate_unit,
// with T = t_per_pr p/rho, n_H = nh_per_rho rho, c_e = rho/(t_per_pr (gamma-1)), by
// backward Euler in T on sub-steps whose explicit change is capped at cap*T, each solved
// by Newton's method with a bisection safeguard (<= 30 iterations, relative tolerance
// 1e-12), T clamped to [10, 1e8] K, at most 4096 sub-steps.  Caps that are hit are
// counted, never looped on.
//
// Lambda(T, Z) is a stand-in for the paper's (unavailable) tables: a piecewise power law
// between knots (log10 T, log10 Lambda) over 10 K .. 1e8 K, scaled by (0.2 + 0.8 Z/0.02).
#pragma once
#include "mhd_device.cuh"

namespace mhd {

enum { TH_OFF = 0, TH_PLAIN = 1, TH_SURROGATE = 2 };
enum { TST_SUBSTEP_CAP = 1, TST_NEWTON_CAP = 2, TST_NO_BRACKET = 4 };

struct ThermalDev {
  int mode;
  double gamma_heat, z, rate_unit, cap, nh_per_rho, t_per_pr;
  unsigned long long* stats;  // [0] cells, [1] sub-steps, [2] capped cells, [3] surrogate fallbacks
  // harvesting of training pairs during plain steps (hv_data == nullptr: off): rows of
  // (log10 n_H, log10 T, log10 dt, Z, log10 T_new - log10 T) into a ring of hv_cap rows
  float* hv_data;
  unsigned long long* hv_count;
  long long hv_cap;
  int hv_stride;
};

constexpr int kKnots = 11;
static __constant__ double kLT[kKnots] = {1.0, 2.0, 3.0, 3.8, 4.0, 4.2, 5.0, 5.4, 6.0, 7.0, 8.0};
static __constant__ double kLL[kKnots] = {-28.5, -27.0, -26.2, -25.9, -23.5, -21.8, -21.3, -21.2, -22.0, -22.7, -22.6};
constexpr double kTmin = 10.0, kTmax = 1e8;
constexpr int kMaxSub = 4096, kMaxNewton = 30;

__device__ __forceinline__ double th_cooling(double T, double z, double* slope) {
  const double lt = log10(T);
  int k = 0;
#pragma unroll 1
  while (k < kKnots - 2 && lt >= kLT[k + 1]) ++k;
  const double a = (kLL[k + 1] - kLL[k]) / (kLT[k + 1] - kLT[k]);
  const double ll = kLL[k] + a * (lt - kLT[k]);
  if (slope) *slope = a;
  return pow(10.0, ll) * (0.2 + 0.8 * z / 0.02);
}

__device__ __forceinline__ double th_rate(double T, double nh, double ce, const ThermalDev& P, double* dfdT) {
  double a;
  const double lam = th_cooling(T, P.z, &a);
  const double f = (nh * P.gamma_heat - nh * nh * lam) / (P.rate_unit * ce);
  if (dfdT) *dfdT = -(nh * nh * lam * a / T) / (P.rate_unit * ce);
  return f;
}

__device__ __forceinline__ double th_clamp(double T) { return T < kTmin ? kTmin : (T > kTmax ? kTmax : T); }

static __device__ double th_integrate(double T0, double nh, double ce, double dt, const ThermalDev& P, int* st,
                               int* nsub_out) {
  double T = th_clamp(T0), t = 0.0;
  int nsub = 0;
  *st = 0;
  while (t < dt) {
    if (nsub == kMaxSub) {
      *st |= TST_SUBSTEP_CAP;
      break;
    }
    const double r = th_rate(T, nh, ce, P, nullptr);
    double h = dt - t;
    if (fabs(r) * h > P.cap * T) h = P.cap * T / fabs(r);
    double lo = th_clamp(T / (1.0 + 4.0 * P.cap)), hi = th_clamp(T * (1.0 + 4.0 * P.cap));
    const double glo = lo - T - h * th_rate(lo, nh, ce, P, nullptr);
    const double ghi = hi - T - h * th_rate(hi, nh, ce, P, nullptr);
    double x;
    if (glo > 0.0 || ghi < 0.0) {
      *st |= TST_NO_BRACKET;
      x = th_clamp(T + h * r);
    } else {
      x = th_clamp(T + h * r);
      if (x < lo) x = lo;
      if (x > hi) x = hi;
      bool done = false;
      for (int it = 0; it < kMaxNewton; ++it) {
        double d;
        const double g = x - T - h * th_rate(x, nh, ce, P, &d);
        if (g == 0.0) {
          done = true;
          break;
        }
        if (g < 0.0) lo = x;
        else hi = x;
        const double gp = 1.0 - h * d;
        if (gp > 0.0) {
          const double xn = x - g / gp;
          if (fabs(xn - x) <= 1e-12 * x) {
            x = xn;
            done = true;
            break;
          }
          x = (xn > lo && xn < hi) ? xn : 0.5 * (lo + hi);
        } else {
          x = 0.5 * (lo + hi);
        }
      }
      if (!done) *st |= TST_NEWTON_CAP;
    }
    T = x;
    t += h;
    ++nsub;
  }
  *nsub_out = nsub;
  return T;
}

// Explicit estimate D of the change of log10 T over dt, in FP32 from the surrogate's inputs
// (log10 n_H, log10 T, log10 dt): the rate at T times dt, over T ln 10.  Since c_e is
// proportional to n_H, the rate is (Gamma - n_H Lambda(T, Z)) K with
// K = nh_per_rho t_per_pr (gamma - 1) / rate_unit; th_dlin_const folds K into the heating
// term and log10 of K times the metallicity factor into the cooling exponent.
// The surrogate predicts q = change / S with the saturated scale S = D / (1 + |D|): where the
// change is small S ~ D and q ~ 1, so the error is relative to the change (and S vanishes at
// equilibrium); for stiff cells |S| -> 1 and q is the change itself, so a large D never
// multiplies the network's error.
struct DlinConst {
  float gk;  // Gamma K
  float lk;  // log10(K (0.2 + 0.8 Z / 0.02))
};

static __constant__ float kLTf[kKnots] = {1.0f, 2.0f, 3.0f, 3.8f, 4.0f, 4.2f, 5.0f, 5.4f, 6.0f, 7.0f, 8.0f};
static __constant__ float kLLf[kKnots] = {-28.5f, -27.0f, -26.2f, -25.9f, -23.5f, -21.8f,
                                          -21.3f, -21.2f, -22.0f, -22.7f, -22.6f};

__device__ __forceinline__ DlinConst th_dlin_const(const ThermalDev& th, double gm1) {
  const double K = th.nh_per_rho * th.t_per_pr * gm1 / th.rate_unit;
  return {(float)(th.gamma_heat * K), (float)log10(K * (0.2 + 0.8 * th.z / 0.02))};
}

__device__ __forceinline__ float th_dlin(DlinConst c, float lnh, float lT, float ldt) {
  int k = 0;
#pragma unroll 1
  while (k < kKnots - 2 && lT >= kLTf[k + 1]) ++k;
  const float ll = kLLf[k] + (kLLf[k + 1] - kLLf[k]) / (kLTf[k + 1] - kLTf[k]) * (lT - kLTf[k]);
  const float rate = c.gk - exp10f(lnh + ll + c.lk);  // K per unit time
  return rate * exp10f(ldt - lT) * 0.4342944819f;      // 1 / ln 10
}

__device__ __forceinline__ float th_scale(float D) { return D / (1.0f + fabsf(D)); }

constexpr float kQClip = 8.0f;  // harvested targets are clipped to [-kQClip, kQClip]
constexpr int kHvCols = 6;      // harvested row: log10 n_H, log10 T, log10 dt, Z, q, change

// Temperature, n_H and c_e of interior cell (i, j, k) from the FP64 state.  The same
// arithmetic as the recovery of the step (no FP64 division, which costs the FP64 pipe about
// ten instructions here): 1/rho from the FP32 reciprocal and one FP64 Newton step (relative
// error ~1e-14), face sums with the factors (gamma-1)/2 and (gamma-1)/8 folded in;
// cef = 1 / (t_per_pr (gamma - 1)), computed once per launch by th_cef.
__device__ __forceinline__ double th_cef(const PatchDev& P, const ThermalDev& th) {
  return 1.0 / (th.t_per_pr * P.gm1);
}

// Pressure (FP64) of interior cell (i, j, k), with its density and 1/density.
__device__ __forceinline__ double th_pressure(const PatchDev& P, const double* __restrict__ U, int i, int j, int k,
                                              double& rho, double& irho) {
  const long long FS = P.FS, c = sidx(P, i, j, k);
  rho = U[c];
  irho = inv_density<float>(rho);
  const double mx = U[MX * FS + c], my = U[MY * FS + c], mz = U[MZ * FS + c];
  const double sbx = U[BXF * FS + c] + U[BXF * FS + sidx(P, fmap(P, 0, i + 1), j, k)];
  const double sby = U[BYF * FS + c] + U[BYF * FS + sidx(P, i, fmap(P, 1, j + 1), k)];
  const double sbz = U[BZF * FS + c] + U[BZF * FS + sidx(P, i, j, fmap(P, 2, k + 1))];
  return P.gm1 * U[EN * FS + c] - P.hgm1 * ((mx * mx + my * my + mz * mz) * irho) -
         P.egm1 * (sbx * sbx + sby * sby + sbz * sbz);
}

__device__ __forceinline__ void th_cell(const PatchDev& P, const ThermalDev& th, const double* __restrict__ U,
                                        int i, int j, int k, double cef, double& T, double& nh, double& ce) {
  double rho, irho;
  const double p = th_pressure(P, U, i, j, k, rho, irho);
  T = th.t_per_pr * p * irho;
  nh = th.nh_per_rho * rho;
  ce = rho * cef;
}

}  // namespace mhd
