// mhd_device.cuh -- device data layout and per-point phase functions of the MHD step
// (arXiv:1502.02935, Section 2.1), templated on the bulk arithmetic type R:
//   R = double : the plain FP64 method;
//   R = float  : FP32 reconstruction / Riemann / EMF / flux-difference arithmetic with
//                FP64 pressure recovery and FP64 accumulation of the conserved state.
//
// Layout in HBM (per patch, all SoA, x fastest):
//   state  Un, Uh : 8 FP64 fields [rho, mx, my, mz, E, Bx, By, Bz], extents PX*PY*PZ
//                   with PX = round4(nx+1), PY = ny+1, PZ = nz+1 (one extra layer for
//                   the high boundary face); cell (i,j,k) and faces i-1/2, j-1/2, k-1/2
//                   share the index i + PX (j + PY k).  No ghost cells: boundary
//                   conditions are index maps applied on every load.
//   scratch W, F, E : R, padded by 2 cells on active axes (QX = nx + 4 ...), holding
//                   primitives W (8), face fluxes F_d (7 per direction: rho, mx, my, mz,
//                   E, B_t1, B_t2 with (d, t1, t2) cyclic; the lowest bit of the stored
//                   mass flux marks a face without contact motion for the corner-EMF
//                   upwinding) and edge EMFs (3).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace mhd {

enum { RHO = 0, MX = 1, MY = 2, MZ = 3, EN = 4, BXF = 5, BYF = 6, BZF = 7 };
enum { WR = 0, WVX = 1, WVY = 2, WVZ = 3, WP = 4, WBX = 5, WBY = 6, WBZ = 7 };
// stored with W: the cell EMF -(v x B), components x, y, z (read by the corner EMFs)
enum { WEX = 8, WEY = 9, WEZ = 10, NWQ = 11 };
enum { NFLUX = 7 };  // rho (with the no-motion bit), mx, my, mz, E, B_t1, B_t2
enum : int { ERR_NONFINITE = 1, ERR_NEGATIVE = 2, ERR_TIMEOUT = 4 };
enum { POT_NONE = 0, POT_GAUSS_X = 1, POT_LOG_DISC = 2 };
enum { FLUX_AUTO = 0, FLUX_MARCH = 1, FLUX_PER_FACE = 2 };
// Riemann solvers of Section 2.1: HLLD (MHD), HLLC and HLL (pure gas dynamics)
enum { RIEMANN_HLLD = 0, RIEMANN_HLLC = 1, RIEMANN_HLL = 2 };

struct PatchDev {
  int n[3];      // interior cells per axis
  int act[3];    // axis active (n > 1)
  int per[3];    // periodic (trivial axes count as periodic with n = 1)
  int nface[3];  // owned faces along each normal: n, or n + 1 on an active outflow axis
  int g2[3];     // scratch padding (2 on active axes)
  int PX, PY, PZ;
  long long FS;  // state field stride
  int QX, QY, QZ;
  long long QS;  // scratch field stride
  double d[3], inv_d[3], lo[3], gamma;
  double gm1, hgm1, egm1;  // gamma - 1, (gamma - 1)/2, (gamma - 1)/8
  float gamma_f, d_f[3];   // FP32 copies for the mixed path
  float inv_d_f[3], lo_f[3];
  double* Un;
  double* Uh;
  void* W;
  void* F[3];
  void* E;
  void* W2;  // second W buffer of the fused EMF + update kernels (3D patches, x-y planes)
  unsigned long long* cfl_min;  // per-patch ordered-bits minimum of the CFL limit
  double* dt_used;
  int* err;
  int index;
  // floors (off unless floors != 0): rho >= rho_floor, rho pr_floor <= p <= rho pr_ceil
  int floors;
  double rho_floor, pr_floor, pr_ceil;
  float rho_floor_f, pr_floor_f, pr_ceil_f;  // FP32 copies for the conservative pre-checks
  unsigned long long* floored;  // count of cells changed by the end-of-step floors
  int riemann;                  // RIEMANN_*
  int flux_scheme;              // FLUX_* (host side: which kernel computes the y and z fluxes)
  // kappa-scheme coefficients K1 = (1 - kappa)/4, K2 = (1 + kappa)/4, b = (3 - kappa)/(1 - kappa)
  double rK1, rK2, rb;
  float rK1_f, rK2_f, rb_f;
  // inflow boundaries: bit s of the mask for side s (x-lo, x-hi, y-lo, ...) and the
  // primitive state [rho, vx, vy, vz, p, Bx, By, Bz] beyond it
  int inflow_mask;
  double inflow_w[6][8];
  // passive scalars (ns of them, 0 when off): conserved rho X in two FP64 buffers (base and
  // half-step, swapped with Un/Uh), X = (rho X)/rho of the stage's input on the padded box
  // in the bulk type, and X beyond each inflow side
  int ns;
  double* Sn;
  double* Sh;
  void* X;
  double inflow_x[6][8];
};

struct SourceDev {
  int potential;
  double psi0, xc, xw, v0, rc;
  float psi0_f, xc_f, xw_f, v0_f, rc_f;  // FP32 copies for the mixed path
};

struct StageArgs {
  int stage;       // 0 predictor (donor cell, h = dt/2), 1 corrector (kappa-scheme, h = dt)
  double dt_host;  // > 0: use it; <= 0: cfl * device CFL limit
  double cfl;
  SourceDev src;
  int concurrent;  // host side: the patch's chain runs beside other patches' (a batch)
};

// ------------------------------------------------------------------ indexing --
__device__ __forceinline__ int cmap(const PatchDev& P, int a, int i) {
  const int n = P.n[a];
  if (i >= 0 && i < n) return i;
  if (P.per[a]) {
    int m = i % n;
    return m < 0 ? m + n : m;
  }
  return i < 0 ? 0 : n - 1;
}

__device__ __forceinline__ int fmap(const PatchDev& P, int a, int f) {
  const int n = P.n[a];
  if (P.per[a]) {
    if (f >= 0 && f < n) return f;
    int m = f % n;
    return m < 0 ? m + n : m;
  }
  return f < 0 ? 0 : (f > n ? n : f);
}

__device__ __forceinline__ long long sidx(const PatchDev& P, int i, int j, int k) {
  return (long long)i + (long long)P.PX * ((long long)j + (long long)P.PY * k);
}

__device__ __forceinline__ long long qidx(const PatchDev& P, int i, int j, int k) {
  return (long long)(i + P.g2[0]) +
         (long long)P.QX * ((long long)(j + P.g2[1]) + (long long)P.QY * (k + P.g2[2]));
}

// the inflow side that a (possibly ghost) cell lies beyond, the first in side order, or -1
__device__ __forceinline__ int inflow_side(const PatchDev& P, int i, int j, int k) {
  if (!P.inflow_mask) return -1;
  const int c[3] = {i, j, k};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (c[a] < 0 && (P.inflow_mask >> (2 * a) & 1)) return 2 * a;
    if (c[a] >= P.n[a] && (P.inflow_mask >> (2 * a + 1) & 1)) return 2 * a + 1;
  }
  return -1;
}

__device__ __forceinline__ long long qstride(const PatchDev& P, int a) {
  return a == 0 ? 1LL : (a == 1 ? (long long)P.QX : (long long)P.QX * P.QY);
}

// ------------------------------------------------- FP32 <-> FP64 on the ALU --
// On this part FP32<->FP64 conversions issue to the FP64 pipe, which is ~1/64 of the FP32
// rate and is what bounds the recovery and update phases of the mixed path.  These two
// conversions are done instead with integer operations on the IEEE-754 fields:
//   binary32 -> binary64: sign kept, exponent rebiased by 1023 - 127 = 896, mantissa
//     shifted left by 29 (exact); zero and subnormal floats give a signed zero; inf/NaN kept.
//   binary64 -> binary32: exponent rebiased by -896, mantissa rounded to 23 bits to nearest
//     with ties to even (the carry of the rounding may step the exponent, up to inf);
//     magnitudes below the smallest normal float give a signed zero; inf/NaN kept.
__device__ __forceinline__ double f2d_alu(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  const unsigned hi_n = sign | ((e + 896u) << 20) | (m >> 3);
  const unsigned hi = e == 0u ? sign : (e == 0xFFu ? (sign | 0x7FF00000u | (m >> 3)) : hi_n);
  const unsigned lo = e == 0u ? 0u : (m << 29);
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float d2f_alu(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const unsigned m23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1FFFFFFFu;
  const unsigned up = (rest > 0x10000000u) | ((rest == 0x10000000u) & (m23 & 1u));
  const int ef = e - 896;
  unsigned bits = ((unsigned)ef << 23) + m23 + up;  // a carry out of the mantissa bumps the exponent
  bits = ef <= 0 ? 0u : (ef >= 255 ? 0x7F800000u : bits);
  bits = bits > 0x7F800000u ? 0x7F800000u : bits;
  if (e == 0x7FF) bits = 0x7F800000u | ((((hi & 0xFFFFFu) | lo) != 0u) ? 0x400000u : 0u);
  return __uint_as_float(sign | bits);
}

// --------------------------------------------------------------- arithmetic --
template <class R> struct Ar;
template <> struct Ar<double> {
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double from_d(double x) { return x; }
  static __device__ __forceinline__ double to_d(double x) { return x; }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double abs_(double x) { return fabs(x); }
  // the no-motion mark of a stored mass flux: its lowest significand bit (a change of at
  // most one ulp of the flux); its sign bit gives the direction of the motion
  static __device__ __forceinline__ double mark(double x, bool band) {
    return __longlong_as_double((__double_as_longlong(x) & ~1LL) | (long long)band);
  }
  static __device__ __forceinline__ bool marked(double x) { return __double_as_longlong(x) & 1LL; }
  static __device__ __forceinline__ bool negative(double x) { return __double_as_longlong(x) < 0; }
  // explicitly rounded operations (never contracted into an FMA)
  static __device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
  static constexpr double degen = 1e-8;
};
template <> struct Ar<float> {
  static __device__ __forceinline__ float from_d(double x) { return d2f_alu(x); }
  static __device__ __forceinline__ double to_d(float x) { return f2d_alu(x); }
  // single hardware approximations (a few ulp) for the FP32 bulk arithmetic
  static __device__ __forceinline__ float rcp(float x) {
#ifdef __CUDA_ARCH__
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return 1.0f / x;
#endif
  }
  static __device__ __forceinline__ float sqrt_(float x) {
#ifdef __CUDA_ARCH__
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return sqrtf(x);
#endif
  }
  static __device__ __forceinline__ float div(float a, float b) { return a * rcp(b); }
  static __device__ __forceinline__ float abs_(float x) { return fabsf(x); }
  static __device__ __forceinline__ float mark(float x, bool band) {
    return __uint_as_float((__float_as_uint(x) & ~1u) | (unsigned)band);
  }
  static __device__ __forceinline__ bool marked(float x) { return __float_as_uint(x) & 1u; }
  static __device__ __forceinline__ bool negative(float x) { return (int)__float_as_uint(x) < 0; }
  static __device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static constexpr float degen = 1e-8f;
};

// gamma and cell sizes in the bulk type (FP32 copies precomputed on the host)
template <class R> struct Gam;
template <> struct Gam<double> {
  static __device__ __forceinline__ double get(const PatchDev& P) { return P.gamma; }
  static __device__ __forceinline__ void kappa(const PatchDev& P, double& K1, double& K2, double& b) {
    K1 = P.rK1;
    K2 = P.rK2;
    b = P.rb;
  }
  static __device__ __forceinline__ double d(const PatchDev& P, int a) { return P.d[a]; }
  static __device__ __forceinline__ double inv(const PatchDev& P, int a) { return P.inv_d[a]; }
  static __device__ __forceinline__ double lo(const PatchDev& P, int a) { return P.lo[a]; }
  static __device__ __forceinline__ void src(const SourceDev& s, double& psi0, double& xc, double& xw, double& v0,
                                             double& rc) {
    psi0 = s.psi0, xc = s.xc, xw = s.xw, v0 = s.v0, rc = s.rc;
  }
};
template <> struct Gam<float> {
  static __device__ __forceinline__ float get(const PatchDev& P) { return P.gamma_f; }
  static __device__ __forceinline__ void kappa(const PatchDev& P, float& K1, float& K2, float& b) {
    K1 = P.rK1_f;
    K2 = P.rK2_f;
    b = P.rb_f;
  }
  static __device__ __forceinline__ float d(const PatchDev& P, int a) { return P.d_f[a]; }
  static __device__ __forceinline__ float inv(const PatchDev& P, int a) { return P.inv_d_f[a]; }
  static __device__ __forceinline__ float lo(const PatchDev& P, int a) { return P.lo_f[a]; }
  static __device__ __forceinline__ void src(const SourceDev& s, float& psi0, float& xc, float& xw, float& v0,
                                             float& rc) {
    psi0 = s.psi0_f, xc = s.xc_f, xw = s.xw_f, v0 = s.v0_f, rc = s.rc_f;
  }
};

// 1/rho for the FP64 pressure recovery.  FP64 path: IEEE division.  Mixed path: the
// correctly rounded FP32 reciprocal refined by one Newton-Raphson step in FP64
// (r <- r + r (1 - rho r)), which squares its relative error (~1e-14).
template <class R> __device__ __forceinline__ double inv_density(double rho);
template <> __device__ __forceinline__ double inv_density<double>(double rho) { return 1.0 / rho; }
template <> __device__ __forceinline__ double inv_density<float>(double rho) {
  double r = f2d_alu(__frcp_rn(d2f_alu(rho)));
  double e = fma(-rho, r, 1.0);
  return fma(r, e, r);
}

// The same with every operation explicitly rounded, for the CFL limit of the recovery: the
// update kernel's fused recovery and the standalone recovery must give the same limit bit for
// bit (the CFL step of a continued run equals that of a restart), whatever FMA contraction
// the compiler chooses in each kernel.
template <class R> __device__ __forceinline__ R fast_speed_rn(R rho, R p, R bb, R bn2, R gam) {
  const R gp = Ar<R>::mul_rn(gam, p);
  const R s = Ar<R>::add_rn(gp, bb);
  R disc = Ar<R>::fma_rn(s, s, Ar<R>::mul_rn(Ar<R>::mul_rn(R(-4), gp), bn2));
  disc = disc > R(0) ? disc : R(0);
  return Ar<R>::sqrt_(Ar<R>::mul_rn(Ar<R>::add_rn(s, Ar<R>::sqrt_(disc)), Ar<R>::rcp(Ar<R>::mul_rn(R(2), rho))));
}

template <class R> __device__ __forceinline__ R fast_speed(R rho, R p, R bb, R bn2, R gam) {
  // c_f^2 = [gamma p + B^2 + sqrt((gamma p + B^2)^2 - 4 gamma p Bn^2)] / (2 rho)
  R gp = gam * p;
  R s = gp + bb;
  R disc = s * s - R(4) * gp * bn2;
  disc = disc > R(0) ? disc : R(0);
  return Ar<R>::sqrt_((s + Ar<R>::sqrt_(disc)) * Ar<R>::rcp(R(2) * rho));
}

// ------------------------------------------------------------------ HLLD ----
// Miyoshi & Kusano (2005) HLLD flux, the MHD Riemann solver named in Section 2.1.
// w = [rho, vn, vt1, vt2, p, Bt1, Bt2] on each side, bn the face-normal field.
// f = [rho, m_n, m_t1, m_t2, E, Bt1, Bt2] fluxes (Eq. 3 in the interface frame) and
// f[7] = sigma = max(rho_L, rho_R) max(|S_L|, |S_R|), the face's mass-flux scale.
template <class R>
__device__ __forceinline__ void hlld(const R* wl, const R* wr, R bn, R gam, R* f) {
  const R half = R(0.5);
  const R igm1 = Ar<R>::rcp(gam - R(1));
  const R bn2 = bn * bn;
  const R rl = wl[0], ul = wl[1], vl = wl[2], zl = wl[3], pl = wl[4], byl = wl[5], bzl = wl[6];
  const R rr = wr[0], ur = wr[1], vr = wr[2], zr = wr[3], pr = wr[4], byr = wr[5], bzr = wr[6];
  const R bbl = bn2 + byl * byl + bzl * bzl;
  const R bbr = bn2 + byr * byr + bzr * bzr;
  const R ptl = pl + half * bbl, ptr = pr + half * bbr;
  const R el = pl * igm1 + half * rl * (ul * ul + vl * vl + zl * zl) + half * bbl;
  const R er = pr * igm1 + half * rr * (ur * ur + vr * vr + zr * zr) + half * bbr;
  const R cfl = fast_speed<R>(rl, pl, bbl, bn2, gam);
  const R cfr = fast_speed<R>(rr, pr, bbr, bn2, gam);
  const R cmax = cfl > cfr ? cfl : cfr;
  const R sl = (ul < ur ? ul : ur) - cmax;
  const R sr = (ul > ur ? ul : ur) + cmax;
  const R vbl = ul * bn + vl * byl + zl * bzl;
  const R vbr = ur * bn + vr * byr + zr * bzr;
  f[7] = (rl > rr ? rl : rr) * (Ar<R>::abs_(sl) > Ar<R>::abs_(sr) ? Ar<R>::abs_(sl) : Ar<R>::abs_(sr));

  if (sl > R(0)) {
    f[0] = rl * ul;
    f[1] = rl * ul * ul + ptl - bn2;
    f[2] = rl * ul * vl - bn * byl;
    f[3] = rl * ul * zl - bn * bzl;
    f[4] = (el + ptl) * ul - vbl * bn;
    f[5] = byl * ul - bn * vl;
    f[6] = bzl * ul - bn * zl;
    return;
  }
  if (sr < R(0)) {
    f[0] = rr * ur;
    f[1] = rr * ur * ur + ptr - bn2;
    f[2] = rr * ur * vr - bn * byr;
    f[3] = rr * ur * zr - bn * bzr;
    f[4] = (er + ptr) * ur - vbr * bn;
    f[5] = byr * ur - bn * vr;
    f[6] = bzr * ur - bn * zr;
    return;
  }
  const R dl = sl - ul, dr = sr - ur;
  const R iden = Ar<R>::rcp(dr * rr - dl * rl);
  const R sm = (dr * rr * ur - dl * rl * ul - ptr + ptl) * iden;
  const R pts = (dr * rr * ptl - dl * rl * ptr + rl * rr * dr * dl * (ur - ul)) * iden;

  // single-star densities on both sides; with them the rotational speeds, which fix the
  // region of the fan the face lies in
  const R isml = Ar<R>::rcp(sl - sm), ismr = Ar<R>::rcp(sr - sm);
  const R rsl = rl * dl * isml, rsr = rr * dr * ismr;
  const R sqrl = Ar<R>::sqrt_(rsl), sqrr = Ar<R>::sqrt_(rsr);
  const R abn = Ar<R>::abs_(bn);
  const R ssl = sm - abn * Ar<R>::rcp(sqrl);
  const R ssr = sm + abn * Ar<R>::rcp(sqrr);

  // choose the side and whether the double-star state is needed
  int side;  // 0: left, 1: right
  bool dbl;
  if (ssl >= R(0)) {
    side = 0; dbl = false;
  } else if (sm >= R(0)) {
    side = 0; dbl = true;
  } else if (ssr >= R(0)) {
    side = 1; dbl = true;
  } else {
    side = 1; dbl = false;
  }
  // the remaining single-star state of side s (v*, B*, E*; M&K Eq. 44-48): the outer star
  // regions need one side's, the double-star region both
  auto star = [&](int s, R& vs, R& zs, R& bys, R& bzs, R& es) {
    const R S_ = s ? sr : sl, rho_ = s ? rr : rl, un_ = s ? ur : ul, v1_ = s ? vr : vl, v2_ = s ? zr : zl;
    const R b1_ = s ? byr : byl, b2_ = s ? bzr : bzl, ee_ = s ? er : el, pt_ = s ? ptr : ptl;
    const R vb_ = s ? vbr : vbl, ds = s ? dr : dl, ism = s ? ismr : isml;
    const R t1 = rho_ * ds * (S_ - sm);
    const R den = t1 - bn2;
    if (Ar<R>::abs_(den) < Ar<R>::degen * (Ar<R>::abs_(t1) + bn2)) {
      vs = v1_;
      zs = v2_;
      bys = b1_;
      bzs = b2_;
    } else {
      const R iden2 = Ar<R>::rcp(den);
      const R fv = bn * (sm - un_) * iden2;
      const R fb = (rho_ * ds * ds - bn2) * iden2;
      vs = v1_ - b1_ * fv;
      zs = v2_ - b2_ * fv;
      bys = b1_ * fb;
      bzs = b2_ * fb;
    }
    const R vbs = sm * bn + vs * bys + zs * bzs;
    es = (ds * ee_ - pt_ * un_ + pts * sm + bn * (vb_ - vbs)) * ism;
  };
  const R S = side ? sr : sl;
  const R Ss = side ? ssr : ssl;
  const R rho = side ? rr : rl, un = side ? ur : ul, v1 = side ? vr : vl, v2 = side ? zr : zl;
  const R b1 = side ? byr : byl, b2 = side ? bzr : bzl, ee = side ? er : el, pt = side ? ptr : ptl;
  const R vb = side ? vbr : vbl;
  // F_a = physical flux of the outer state
  R F0 = rho * un;
  R F1 = rho * un * un + pt - bn2;
  R F2 = rho * un * v1 - bn * b1;
  R F3 = rho * un * v2 - bn * b2;
  R F4 = (ee + pt) * un - vb * bn;
  R F5 = b1 * un - bn * v1;
  R F6 = b2 * un - bn * v2;
  // F*_a = F_a + S_a (U*_a - U_a)
  const R rsa = side ? rsr : rsl;
  R vsa, zsa, bysa, bzsa, esa;
  star(side, vsa, zsa, bysa, bzsa, esa);
  F0 += S * (rsa - rho);
  F1 += S * (rsa * sm - rho * un);
  F2 += S * (rsa * vsa - rho * v1);
  F3 += S * (rsa * zsa - rho * v2);
  F4 += S * (esa - ee);
  F5 += S * (bysa - b1);
  F6 += S * (bzsa - b2);
  if (dbl) {
    // the other side's single-star state, then the double-star states (sqrt(rho*)-weighted,
    // M&K Eq. 59-63); F** = F* + S*(U** - U*)
    R vso, zso, byso, bzso, eso;
    star(1 - side, vso, zso, byso, bzso, eso);
    const R vs0 = side ? vso : vsa, vs1 = side ? vsa : vso, zs0 = side ? zso : zsa, zs1 = side ? zsa : zso;
    const R bys0 = side ? byso : bysa, bys1 = side ? bysa : byso, bzs0 = side ? bzso : bzsa,
            bzs1 = side ? bzsa : bzso;
    const R sgn = bn > R(0) ? R(1) : (bn < R(0) ? R(-1) : R(0));
    const R isum = Ar<R>::rcp(sqrl + sqrr);
    const R vss = (sqrl * vs0 + sqrr * vs1 + (bys1 - bys0) * sgn) * isum;
    const R zss = (sqrl * zs0 + sqrr * zs1 + (bzs1 - bzs0) * sgn) * isum;
    const R byss = (sqrl * bys1 + sqrr * bys0 + sqrl * sqrr * (vs1 - vs0) * sgn) * isum;
    const R bzss = (sqrl * bzs1 + sqrr * bzs0 + sqrl * sqrr * (zs1 - zs0) * sgn) * isum;
    const R vbsa = sm * bn + vsa * bysa + zsa * bzsa;
    const R vbss = sm * bn + vss * byss + zss * bzss;
    const R sq = side ? sqrr : sqrl;
    const R ess = side ? esa + sq * (vbsa - vbss) * sgn : esa - sq * (vbsa - vbss) * sgn;
    F2 += Ss * (rsa * vss - rsa * vsa);
    F3 += Ss * (rsa * zss - rsa * zsa);
    F4 += Ss * (ess - esa);
    F5 += Ss * (byss - bysa);
    F6 += Ss * (bzss - bzsa);
  }
  f[0] = F0; f[1] = F1; f[2] = F2; f[3] = F3; f[4] = F4; f[5] = F5; f[6] = F6;
}

// ------------------------------------------------------------ HLL, HLLC ----
// The two gas-dynamics solvers of Section 2.1, same layout as hlld.
// HLL (Harten, Lax & van Leer): one averaged state between the outer speeds of the HLLD
// estimate (fast speeds, so it is also the two-wave MHD solver):
//   F = [S_R F_L - S_L F_R + S_L S_R (U_R - U_L)] / (S_R - S_L) inside the fan.
template <class R>
__device__ __forceinline__ void hll(const R* wl, const R* wr, R bn, R gam, R* f) {
  const R half = R(0.5);
  const R igm1 = Ar<R>::rcp(gam - R(1));
  const R bn2 = bn * bn;
  const R w[2][7] = {{wl[0], wl[1], wl[2], wl[3], wl[4], wl[5], wl[6]},
                     {wr[0], wr[1], wr[2], wr[3], wr[4], wr[5], wr[6]}};
  R U[2][7], F[2][7], cf[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const R rho = w[s][0], un = w[s][1], v1 = w[s][2], v2 = w[s][3], p = w[s][4], b1 = w[s][5], b2 = w[s][6];
    const R bb = bn2 + b1 * b1 + b2 * b2;
    const R pt = p + half * bb;
    const R e = p * igm1 + half * rho * (un * un + v1 * v1 + v2 * v2) + half * bb;
    const R vb = un * bn + v1 * b1 + v2 * b2;
    U[s][0] = rho;
    U[s][1] = rho * un;
    U[s][2] = rho * v1;
    U[s][3] = rho * v2;
    U[s][4] = e;
    U[s][5] = b1;
    U[s][6] = b2;
    F[s][0] = rho * un;
    F[s][1] = rho * un * un + pt - bn2;
    F[s][2] = rho * un * v1 - bn * b1;
    F[s][3] = rho * un * v2 - bn * b2;
    F[s][4] = (e + pt) * un - vb * bn;
    F[s][5] = b1 * un - bn * v1;
    F[s][6] = b2 * un - bn * v2;
    cf[s] = fast_speed<R>(rho, p, bb, bn2, gam);
  }
  const R cmax = cf[0] > cf[1] ? cf[0] : cf[1];
  const R ul = w[0][1], ur = w[1][1];
  const R sl = (ul < ur ? ul : ur) - cmax;
  const R sr = (ul > ur ? ul : ur) + cmax;
  f[7] = (w[0][0] > w[1][0] ? w[0][0] : w[1][0]) *
         (Ar<R>::abs_(sl) > Ar<R>::abs_(sr) ? Ar<R>::abs_(sl) : Ar<R>::abs_(sr));
  if (sl > R(0)) {
#pragma unroll
    for (int m = 0; m < 7; ++m) f[m] = F[0][m];
  } else if (sr < R(0)) {
#pragma unroll
    for (int m = 0; m < 7; ++m) f[m] = F[1][m];
  } else {
    const R idn = Ar<R>::rcp(sr - sl);
#pragma unroll
    for (int m = 0; m < 7; ++m) f[m] = (sr * F[0][m] - sl * F[1][m] + sl * sr * (U[1][m] - U[0][m])) * idn;
  }
}

// HLLC (Toro, Spruce & Speares) for a face without field: the HLL fan split at the
// contact S_M into two star states (HLLD's single-star states with B = 0: Miyoshi & Kusano
// Eq. 38, 41, 43, 48); transverse velocities are kept across the contact.
template <class R>
__device__ __forceinline__ void hllc(const R* wl, const R* wr, R gam, R* f) {
  const R half = R(0.5);
  const R igm1 = Ar<R>::rcp(gam - R(1));
  const R rl = wl[0], ul = wl[1], vl = wl[2], zl = wl[3], pl = wl[4];
  const R rr = wr[0], ur = wr[1], vr = wr[2], zr = wr[3], pr = wr[4];
  const R el = pl * igm1 + half * rl * (ul * ul + vl * vl + zl * zl);
  const R er = pr * igm1 + half * rr * (ur * ur + vr * vr + zr * zr);
  const R cl = Ar<R>::sqrt_(gam * pl * Ar<R>::rcp(rl)), cr = Ar<R>::sqrt_(gam * pr * Ar<R>::rcp(rr));
  const R cmax = cl > cr ? cl : cr;
  const R sl = (ul < ur ? ul : ur) - cmax;
  const R sr = (ul > ur ? ul : ur) + cmax;
  f[5] = R(0);
  f[6] = R(0);
  f[7] = (rl > rr ? rl : rr) * (Ar<R>::abs_(sl) > Ar<R>::abs_(sr) ? Ar<R>::abs_(sl) : Ar<R>::abs_(sr));
  if (sl > R(0) || sr < R(0)) {
    const bool left = sl > R(0);
    const R rho = left ? rl : rr, un = left ? ul : ur, v1 = left ? vl : vr, v2 = left ? zl : zr;
    const R p = left ? pl : pr, e = left ? el : er;
    f[0] = rho * un;
    f[1] = rho * un * un + p;
    f[2] = rho * un * v1;
    f[3] = rho * un * v2;
    f[4] = (e + p) * un;
    return;
  }
  const R dl = sl - ul, dr = sr - ur;
  const R iden = Ar<R>::rcp(dr * rr - dl * rl);
  const R sm = (dr * rr * ur - dl * rl * ul - pr + pl) * iden;
  const R pts = (dr * rr * pl - dl * rl * pr + rl * rr * dr * dl * (ur - ul)) * iden;
  const bool left = sm >= R(0);
  const R S = left ? sl : sr;
  const R rho = left ? rl : rr, un = left ? ul : ur, v1 = left ? vl : vr, v2 = left ? zl : zr;
  const R p = left ? pl : pr, e = left ? el : er;
  const R ds = S - un;
  const R ism = Ar<R>::rcp(S - sm);
  const R rs = rho * ds * ism;
  const R es = (ds * e - p * un + pts * sm) * ism;
  // F* = F_a + S_a (U*_a - U_a)
  f[0] = rho * un + S * (rs - rho);
  f[1] = rho * un * un + p + S * (rs * sm - rho * un);
  f[2] = rho * un * v1 + S * (rs - rho) * v1;
  f[3] = rho * un * v2 + S * (rs - rho) * v2;
  f[4] = (e + p) * un + S * (es - e);
}

// the patch's solver at one face; HLLC hands a face that carries a field to HLLD (which
// is HLLC when B = 0)
template <class R>
__device__ __forceinline__ void riemann(int solver, const R* wl, const R* wr, R bn, R gam, R* f) {
  if (solver == RIEMANN_HLL) {
    hll<R>(wl, wr, bn, gam, f);
  } else if (solver == RIEMANN_HLLC && bn == R(0) && wl[5] == R(0) && wl[6] == R(0) && wr[5] == R(0) &&
             wr[6] == R(0)) {
    hllc<R>(wl, wr, gam, f);
  } else {
    hlld<R>(wl, wr, bn, gam, f);
  }
}

// --------------------------------------------------------- reconstruction ----
// compressive minmod kappa-scheme (Eq. 12-14 read in the standard form, third-order upwind
// biased for the paper's kappa = 1/3: K1 = 1/6, K2 = 1/3, b = 4; kappa = 0 and -1 are the
// second-order variants the text names), coefficients from the patch.
// minmod(a, b): the smaller magnitude with the common sign when a and b have the same
// sign, else 0; as max(min(a, b), min(max(a, b), 0)), which is exact (min and max do not
// round) and needs no product a b (which can underflow)
template <class R> __device__ __forceinline__ R minmod(R a, R b) {
  return fmax(fmin(a, b), fmin(fmax(a, b), R(0)));
}

template <class R>
__device__ __forceinline__ void kappa_face(R wm1, R w0, R w1, R w2, R K1, R K2, R b, R& wl, R& wr) {
  const R dwm = w0 - wm1, dw0 = w1 - w0, dwp = w2 - w1;
  wl = w0 + K1 * minmod<R>(dwm, b * dw0) + K2 * minmod<R>(dw0, b * dwm);
  wr = w1 - K1 * minmod<R>(dwp, b * dw0) - K2 * minmod<R>(dw0, b * dwp);
}

// --------------------------------------------------------------- sources ----
template <class R>
__device__ __forceinline__ void grad_psi(const SourceDev& s, R x, R y, R z, R* g) {
  g[0] = g[1] = g[2] = R(0);
  R psi0, xc, xw, v0, rc;
  Gam<R>::src(s, psi0, xc, xw, v0, rc);
  if (s.potential == POT_GAUSS_X) {
    R u = (x - xc) / xw;
    g[0] = psi0 * R(2) * u / xw * exp(-u * u);
  } else if (s.potential == POT_LOG_DISC) {
    R iq = v0 * v0 / (x * x + y * y + rc * rc + z * z);
    g[0] = x * iq;
    g[1] = y * iq;
    g[2] = z * iq;
  }
}

// centre of cell i along axis a in the bulk type
template <class R> __device__ __forceinline__ R centre(const PatchDev& P, int a, int i) {
  return Gam<R>::lo(P, a) + (R(i) + R(0.5)) * Gam<R>::d(P, a);
}

// ---------------------------------------------------------- phase: recovery --
// cell EMF -(v x B)_C (Eq. 9) from the velocity and field components A = C+1, B = C+2
// (explicitly rounded: the recovery fused into the update and the standalone recovery must
// store the same bits, whatever FMA contraction the compiler applies in each kernel)
template <class R> __device__ __forceinline__ R cell_emf(R vA, R vB, R bA, R bB) {
  return -Ar<R>::sub_rn(Ar<R>::mul_rn(vA, bB), Ar<R>::mul_rn(vB, bA));
}

// exponent test of a double on the integer pipe (not inf, not NaN)
__device__ __forceinline__ bool finite_d(double x) {
  return ((unsigned)__double2hiint(x) & 0x7FF00000u) != 0x7FF00000u;
}

// W of one cell from its conserved values: Eq. 6 for the cell-centred field (sbx, sby, sbz
// are the sums of the two face values, i.e. twice it), the energy closure after Eq. 3 for p
// (FP64 in both paths), with the floors when they are on.  Stores W at scratch index q when
// asked; returns the CFL limit min_d d/(|v_d| + c_f,d) for interior cells when cfl is set
// (else +inf; the predictor's new state needs no CFL limit: 256^3 step 4.210 -> 4.190 ms).
template <class R>
__device__ __forceinline__ R prim_core(const PatchDev& P, double rho, double mx, double my, double mz,
                                            double e, double sbx, double sby, double sbz, R* __restrict__ W,
                                            long long q, bool store, bool interior, bool cfl = true) {
  if (P.floors && rho < P.rho_floor) rho = P.rho_floor;
  // Every operation below is explicitly rounded (intrinsics are never contracted or
  // reordered): the recovery fused into the update kernel and the standalone recovery store
  // the same W and CFL limit bit for bit, whichever kernel inlines them.
  const double irho = inv_density<R>(rho);
  const double m2 = __fma_rn(mz, mz, __fma_rn(my, my, __dmul_rn(mx, mx)));
  const double b2 = __fma_rn(sbz, sbz, __fma_rn(sby, sby, __dmul_rn(sbx, sbx)));  // 4 |B_cc|^2
  // p = (gamma-1) (E - |m|^2/(2 rho) - |B_cc|^2/2), in FP64, clamped when floors are on
  double p = __fma_rn(-P.egm1, b2, __fma_rn(-P.hgm1, __dmul_rn(m2, irho), __dmul_rn(P.gm1, e)));
  if (P.floors) {
    const double lo = rho * P.pr_floor, hi = rho * P.pr_ceil;
    p = p < lo ? lo : (p > hi ? hi : p);  // a NaN passes through to the finiteness check
  }
  const R rirho = Ar<R>::from_d(irho);
  const R vx = Ar<R>::mul_rn(Ar<R>::from_d(mx), rirho), vy = Ar<R>::mul_rn(Ar<R>::from_d(my), rirho),
          vz = Ar<R>::mul_rn(Ar<R>::from_d(mz), rirho);
  const R bx = Ar<R>::from_d(sbx) * R(0.5), by = Ar<R>::from_d(sby) * R(0.5), bz = Ar<R>::from_d(sbz) * R(0.5);
  const R rr = Ar<R>::from_d(rho), pr = Ar<R>::from_d(p);
  if (store) {
    const long long QS = P.QS;
    W[q] = rr;
    W[WVX * QS + q] = vx;
    W[WVY * QS + q] = vy;
    W[WVZ * QS + q] = vz;
    W[WP * QS + q] = pr;
    W[WBX * QS + q] = bx;
    W[WBY * QS + q] = by;
    W[WBZ * QS + q] = bz;
    W[WEX * QS + q] = cell_emf<R>(vy, vz, by, bz);
    W[WEY * QS + q] = cell_emf<R>(vz, vx, bz, bx);
    W[WEZ * QS + q] = cell_emf<R>(vx, vy, bx, by);
  }
  R lim = R(INFINITY);
  if (interior) {
    // positivity / finiteness on the bulk-type values; CFL arithmetic in the bulk type
    if (!(isfinite(rr) && isfinite(pr) && finite_d(e))) {
      atomicOr(P.err, ERR_NONFINITE);
    } else if (!(rr > R(0)) || !(pr > R(0))) {
      atomicOr(P.err, ERR_NEGATIVE);
    }
    if (cfl) {
      const R v[3] = {vx, vy, vz};
      const R b[3] = {bx, by, bz};
      const R bb = Ar<R>::fma_rn(b[2], b[2], Ar<R>::fma_rn(b[1], b[1], Ar<R>::mul_rn(b[0], b[0])));
      const R gam = Gam<R>::get(P);
      R lr = R(INFINITY);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (!P.act[a]) continue;
        const R cf = fast_speed_rn<R>(rr, pr, bb, Ar<R>::mul_rn(b[a], b[a]), gam);
        const R t = Ar<R>::div(Gam<R>::d(P, a), Ar<R>::add_rn(Ar<R>::abs_(v[a]), cf));
        lr = t < lr ? t : lr;
      }
      lim = lr;
    }
  }
  return lim;
}

// The W stores and the CFL limit of prim_core from the bulk-type values (efin: E finite).
template <class R>
__device__ __forceinline__ R prim_store(const PatchDev& P, R rr, R vx, R vy, R vz, R bx, R by, R bz, R pr,
                                        bool efin, R* __restrict__ W, long long q, bool store, bool interior) {
  if (store) {
    const long long QS = P.QS;
    W[q] = rr;
    W[WVX * QS + q] = vx;
    W[WVY * QS + q] = vy;
    W[WVZ * QS + q] = vz;
    W[WP * QS + q] = pr;
    W[WBX * QS + q] = bx;
    W[WBY * QS + q] = by;
    W[WBZ * QS + q] = bz;
    W[WEX * QS + q] = cell_emf<R>(vy, vz, by, bz);
    W[WEY * QS + q] = cell_emf<R>(vz, vx, bz, bx);
    W[WEZ * QS + q] = cell_emf<R>(vx, vy, bx, by);
  }
  R lim = R(INFINITY);
  if (interior) {
    // positivity / finiteness on the bulk-type values; CFL arithmetic in the bulk type
    if (!(isfinite(rr) && isfinite(pr) && efin)) {
      atomicOr(P.err, ERR_NONFINITE);
    } else if (!(rr > R(0)) || !(pr > R(0))) {
      atomicOr(P.err, ERR_NEGATIVE);
    }
    const R v[3] = {vx, vy, vz};
    const R b[3] = {bx, by, bz};
    const R bb = Ar<R>::fma_rn(b[2], b[2], Ar<R>::fma_rn(b[1], b[1], Ar<R>::mul_rn(b[0], b[0])));
    const R gam = Gam<R>::get(P);
    R lr = R(INFINITY);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (!P.act[a]) continue;
      const R cf = fast_speed_rn<R>(rr, pr, bb, Ar<R>::mul_rn(b[a], b[a]), gam);
      const R t = Ar<R>::div(Gam<R>::d(P, a), Ar<R>::add_rn(Ar<R>::abs_(v[a]), cf));
      lr = t < lr ? t : lr;
    }
    lim = lr;
  }
  return lim;
}

// The second half of prim_core for floor_prim_core: W at scratch index q and the CFL limit
// from the recovered density, its reciprocal and the pressure (the same arithmetic as
// prim_core's, which keeps its own copy: inlined into the update kernel without floors,
// a shared tail cost that kernel registers and 6% of its time).
// (rr, pr: the density and pressure already in the bulk type)
template <class R>
__device__ __forceinline__ R prim_tail(const PatchDev& P, R rr, double irho, double mx, double my, double mz,
                                       double e, double sbx, double sby, double sbz, R pr,
                                       R* __restrict__ W, long long q, bool store, bool interior) {
  const R rirho = Ar<R>::from_d(irho);
  const R vx = Ar<R>::mul_rn(Ar<R>::from_d(mx), rirho), vy = Ar<R>::mul_rn(Ar<R>::from_d(my), rirho),
          vz = Ar<R>::mul_rn(Ar<R>::from_d(mz), rirho);
  const R bx = Ar<R>::from_d(sbx) * R(0.5), by = Ar<R>::from_d(sby) * R(0.5), bz = Ar<R>::from_d(sbz) * R(0.5);
  return prim_store<R>(P, rr, vx, vy, vz, bx, by, bz, pr, finite_d(e), W, q, store, interior);
}

// Conservative FP32 pre-checks of the floors (FP32 copies x = d2f_alu of the FP64 values):
// true only when the FP64 value certainly lies strictly inside the bound, so that the FP64
// comparison (and its clamp) can be skipped with the same result.  The margin 2^-20 exceeds
// the relative error of the roundings involved (at most 4 x 2^-24); NaN, zero and values
// that d2f_alu flushes fail the check and take the FP64 path.
constexpr float kFloorMargin = 1.0f + 1.0f / 1048576.0f;
__device__ __forceinline__ bool surely_above(float x, float bound_f) {
  return bound_f >= 1.17549435e-38f && x > bound_f * kFloorMargin;
}
__device__ __forceinline__ bool surely_inside(float x, float lo_f, float hi_f) {
  return surely_above(x, lo_f) && x < hi_f * (2.0f - kFloorMargin);
}

// The terms of the recovery's pressure that do not depend on E (prim_core's arithmetic and
// rounding, without the density floor): 1/rho, |m|^2/rho and 4|B_cc|^2.  A change of E alone
// (the thermal source) recovers the new pressure from them with recovery_pressure, bit for
// bit as prim_core would from the changed state.
struct RecoveryTerms {
  double irho, kin, b2;
};
template <class R>
__device__ __forceinline__ RecoveryTerms recovery_terms(double rho, double mx, double my, double mz, double sbx,
                                                        double sby, double sbz) {
  const double irho = inv_density<R>(rho);
  const double m2 = __fma_rn(mz, mz, __fma_rn(my, my, __dmul_rn(mx, mx)));
  const double b2 = __fma_rn(sbz, sbz, __fma_rn(sby, sby, __dmul_rn(sbx, sbx)));
  return {irho, __dmul_rn(m2, irho), b2};
}
// p = (gamma-1) (E - |m|^2/(2 rho) - |B_cc|^2/2), unclamped
__device__ __forceinline__ double recovery_pressure(const PatchDev& P, const RecoveryTerms& t, double e) {
  return __fma_rn(-P.egm1, t.b2, __fma_rn(-P.hgm1, t.kin, __dmul_rn(P.gm1, e)));
}

// The end-of-step floors and the recovery of the new state in one pass, sharing their FP64
// arithmetic (floors on): with rho_f = max(rho, rho_floor), the recovery's pressure with rho_f
// is clamped to [rho_f pr_floor, rho_f pr_ceil].  An unchanged cell keeps its state and takes
// W from that pressure, as prim_core would.  A changed cell gets rho_f and E rebuilt by the
// energy closure from the clamped pressure (momentum kept), counted in *nfl, and is
// recovered again from those stored values (so a standalone recovery gives the same W).
template <class R>
__device__ __forceinline__ R floor_prim_core(const PatchDev& P, double& rho, double mx, double my, double mz,
                                             double& e, double sbx, double sby, double sbz,
                                             R* __restrict__ W, long long q, int* nfl) {
  // (FP32 path: the FP64 comparisons only where the FP32 pre-checks cannot decide them)
  const R rr = Ar<R>::from_d(rho);
  const bool rho_in = sizeof(R) == 4 && surely_above(float(rr), P.rho_floor_f);
  const double rf = rho_in ? rho : (rho < P.rho_floor ? P.rho_floor : rho);
  const double irho = inv_density<R>(rf);
  const double m2 = __fma_rn(mz, mz, __fma_rn(my, my, __dmul_rn(mx, mx)));
  const double b2 = __fma_rn(sbz, sbz, __fma_rn(sby, sby, __dmul_rn(sbx, sbx)));
  const double p = __fma_rn(-P.egm1, b2, __fma_rn(-P.hgm1, __dmul_rn(m2, irho), __dmul_rn(P.gm1, e)));
  const R pr = Ar<R>::from_d(p);
  if (rho_in && surely_inside(float(pr), float(rr) * P.pr_floor_f, float(rr) * P.pr_ceil_f))
    return prim_tail<R>(P, rr, irho, mx, my, mz, e, sbx, sby, sbz, pr, W, q, true, true);
  const double lo = rf * P.pr_floor, hi = rf * P.pr_ceil;
  const double pf = p < lo ? lo : (p > hi ? hi : p);
  if (rf == rho && pf == p) return prim_tail<R>(P, rr, irho, mx, my, mz, e, sbx, sby, sbz, pr, W, q, true, true);
  rho = rf;
  e = pf / P.gm1 + 0.5 * m2 * irho + 0.125 * b2;  // p/(gamma-1) + |m|^2/(2 rho) + |B_cc|^2/2
  ++*nfl;
  return prim_core<R>(P, rho, mx, my, mz, e, sbx, sby, sbz, W, q, true, true);
}

// W at a (possibly ghost) cell from U via the boundary index maps.
template <class R>
__device__ __forceinline__ R prim_point(const PatchDev& P, const double* __restrict__ U,
                                             R* __restrict__ W, int i, int j, int k, bool store,
                                             bool interior) {
  const int side = inflow_side(P, i, j, k);
  if (side >= 0) {
    // a ghost cell beyond an inflow side: the side's fixed state
    if (store) {
      const long long QS = P.QS, q = qidx(P, i, j, k);
      R w[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) w[m] = Ar<R>::from_d(P.inflow_w[side][m]);
#pragma unroll
      for (int m = 0; m < 8; ++m) W[m * QS + q] = w[m];
      W[WEX * QS + q] = cell_emf<R>(w[WVY], w[WVZ], w[WBY], w[WBZ]);
      W[WEY * QS + q] = cell_emf<R>(w[WVZ], w[WVX], w[WBZ], w[WBX]);
      W[WEZ * QS + q] = cell_emf<R>(w[WVX], w[WVY], w[WBX], w[WBY]);
    }
    return R(INFINITY);
  }
  const int ci = cmap(P, 0, i), cj = cmap(P, 1, j), ck = cmap(P, 2, k);
  const long long FS = P.FS;
  const long long c = sidx(P, ci, cj, ck);
  const double sbx = U[BXF * FS + sidx(P, fmap(P, 0, i), cj, ck)] + U[BXF * FS + sidx(P, fmap(P, 0, i + 1), cj, ck)];
  const double sby = U[BYF * FS + sidx(P, ci, fmap(P, 1, j), ck)] + U[BYF * FS + sidx(P, ci, fmap(P, 1, j + 1), ck)];
  const double sbz = U[BZF * FS + sidx(P, ci, cj, fmap(P, 2, k))] + U[BZF * FS + sidx(P, ci, cj, fmap(P, 2, k + 1))];
  return prim_core<R>(P, U[c], U[MX * FS + c], U[MY * FS + c], U[MZ * FS + c], U[EN * FS + c], sbx, sby, sbz,
                      W, qidx(P, i, j, k), store, interior);
}

// --------------------------------------------------------- passive scalars --
// X_s = (rho X_s)/rho at a (possibly ghost) cell of the padded box: beyond an inflow side
// the side's X, else from the cell the boundary maps give.
template <class R>
__device__ __forceinline__ void scalar_prim_point(const PatchDev& P, const double* __restrict__ U,
                                                  const double* __restrict__ S, R* __restrict__ X, int i, int j,
                                                  int k) {
  const long long q = qidx(P, i, j, k), QS = P.QS;
  const int side = inflow_side(P, i, j, k);
  if (side >= 0) {
    for (int m = 0; m < P.ns; ++m) X[m * QS + q] = Ar<R>::from_d(P.inflow_x[side][m]);
    return;
  }
  const long long c = sidx(P, cmap(P, 0, i), cmap(P, 1, j), cmap(P, 2, k));
  // X is stored in the bulk type: the mixed path divides in FP32 (no FP64 division)
  const R irho = Ar<R>::rcp(Ar<R>::from_d(U[c]));
  for (int m = 0; m < P.ns; ++m) X[m * QS + q] = Ar<R>::from_d(S[m * P.FS + c]) * irho;
}

// rho X_out = rho X_base - h sum_d [F(c + 1/2) - F(c - 1/2)] / d at interior cell (i, j, k):
// F = (Riemann mass flux of the stage) * (X_L if it is >= 0 else X_R), X_L and X_R the
// donor-cell (ORDER 1) or kappa-scheme (ORDER 2) states of X at the face.
template <class R, int ORDER>
__device__ __forceinline__ void scalar_update_point(const PatchDev& P, const double* __restrict__ Sb,
                                                    double* __restrict__ So, const R* __restrict__ X, R h, int i,
                                                    int j, int k) {
  const long long s = sidx(P, i, j, k), q = qidx(P, i, j, k), QS = P.QS;
  R kap[3];
  Gam<R>::kappa(P, kap[0], kap[1], kap[2]);
  for (int m = 0; m < P.ns; ++m) {
    const R* Xm = X + m * QS;
    R div = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (!P.act[d]) continue;
      const long long st = qstride(P, d);
      const R* mflux = (const R*)P.F[d];  // component 0: the mass flux
      R fx[2];
#pragma unroll
      for (int up = 0; up < 2; ++up) {
        const long long f = q + up * st;  // face f - 1/2 along d
        R xl, xr;
        if (ORDER == 1) {
          xl = Xm[f - st];
          xr = Xm[f];
        } else {
          kappa_face<R>(Xm[f - 2 * st], Xm[f - st], Xm[f], Xm[f + st], kap[0], kap[1], kap[2], xl, xr);
        }
        const R mf = mflux[f];
        fx[up] = mf * (mf >= R(0) ? xl : xr);
      }
      div += (fx[1] - fx[0]) * Gam<R>::inv(P, d);
    }
    So[m * P.FS + s] = Sb[m * P.FS + s] - Ar<R>::to_d(h * div);
  }
}

// ----------------------------------------------------------- end-of-step floors --
// Interior cell of the new state: rho' = max(rho, rho_floor), momentum kept, p from E with
// rho' and the cell-centred field of Eq. 6 (face values b*lo, b*hi), clamped to
// [rho' pr_floor, rho' pr_ceil], and E rebuilt by the energy closure (text after Eq. 3)
// when rho or p changed.  Returns 1 for a changed cell.  (The paper states no floors.)
__device__ __forceinline__ int floor_core(const PatchDev& P, double& rho, double mx, double my, double mz,
                                          double& e, double bxlo, double bxhi, double bylo, double byhi,
                                          double bzlo, double bzhi) {
  const double rf = rho < P.rho_floor ? P.rho_floor : rho;
  const double bx = 0.5 * (bxlo + bxhi), by = 0.5 * (bylo + byhi), bz = 0.5 * (bzlo + bzhi);
  const double kin = 0.5 * (mx * mx + my * my + mz * mz) / rf;
  const double mag = 0.5 * (bx * bx + by * by + bz * bz);
  const double p = P.gm1 * (e - kin - mag);
  const double lo = rf * P.pr_floor, hi = rf * P.pr_ceil;
  const double pf = p < lo ? lo : (p > hi ? hi : p);
  if (rf == rho && pf == p) return 0;
  rho = rf;
  e = pf / P.gm1 + kin + mag;
  return 1;
}

__device__ __forceinline__ int floor_point(const PatchDev& P, double* __restrict__ U, int i, int j, int k) {
  const long long FS = P.FS, c = sidx(P, i, j, k);
  double rho = U[c], e = U[EN * FS + c];
  const int changed = floor_core(P, rho, U[MX * FS + c], U[MY * FS + c], U[MZ * FS + c], e, U[BXF * FS + c],
                                 U[BXF * FS + sidx(P, fmap(P, 0, i + 1), j, k)], U[BYF * FS + c],
                                 U[BYF * FS + sidx(P, i, fmap(P, 1, j + 1), k)], U[BZF * FS + c],
                                 U[BZF * FS + sidx(P, i, j, fmap(P, 2, k + 1))]);
  if (changed) {
    U[c] = rho;
    U[EN * FS + c] = e;
  }
  return changed;
}

// ---------------------------------------------------- Eq. 11's no-motion band --
// Eq. 11 averages the one-sided EMF derivatives of the corner formula where the contact does
// not move (F_rho = 0).  That is read as zero to the precision of the data the flux was
// computed from: |F_rho| <= eps_R sigma, sigma = max(rho_L, rho_R) max(|S_L|, |S_R|).  FP64
// path: eps = 2^-32, two orders above the rounding of FP64 data after the pressure
// recovery's cancellation (relative error ~2^-52 E / thermal energy, up to 1e3-1e4).  FP32
// bulk of the mixed path: eps = 64 * 2^-23, the same reading for data rounded to FP32.  A
// flux that is zero in exact arithmetic comes out as rounding of sigma, of either sign.  The
// flux kernels store the decision in the lowest bit of the mass flux (Ar::mark).
template <class R> struct UpwindEps;
template <> struct UpwindEps<double> { static constexpr double v = 1.0 / 4294967296.0; };
template <> struct UpwindEps<float> { static constexpr float v = 64.0f * 1.1920928955078125e-7f; };
template <class R> __device__ __forceinline__ bool no_motion_band(R fr, R sigma) {
  return !(Ar<R>::abs_(fr) > UpwindEps<R>::v * sigma);
}

// ------------------------------------------------------------- phase: flux ----
// HLLD flux through a D-face with donor-cell (ORDER 1) or kappa-scheme (ORDER 2)
// interface states; the normal field is the face value; a face whose reconstructed rho
// or p is not positive falls back to the donor-cell states.  get(m, o) returns primitive
// component m (W index) of the cell at offset o in {-2, -1, 0, 1} along D from the face
// (o = -1 left, o = 0 right).  f[0..7]: rho, m_D, m_T1, m_T2, E, B_T1, B_T2 fluxes and the
// wave-speed scale sigma.
template <class R, int D, int ORDER, class Get>
__device__ __forceinline__ void flux_core(const Get& get, R bn, R gam, int solver, const R* kap, R* f) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  const int comp[7] = {WR, WVX + D, WVX + T1, WVX + T2, WP, WBX + T1, WBX + T2};
  R wl[7], wr[7];
  if (ORDER == 1) {
#pragma unroll
    for (int m = 0; m < 7; ++m) {
      wl[m] = get(comp[m], -1);
      wr[m] = get(comp[m], 0);
    }
  } else {
#pragma unroll
    for (int m = 0; m < 7; ++m)
      kappa_face<R>(get(comp[m], -2), get(comp[m], -1), get(comp[m], 0), get(comp[m], 1), kap[0], kap[1], kap[2],
                    wl[m], wr[m]);
    if (!(wl[0] > R(0)) || !(wr[0] > R(0)) || !(wl[4] > R(0)) || !(wr[4] > R(0))) {
#pragma unroll
      for (int m = 0; m < 7; ++m) {
        wl[m] = get(comp[m], -1);
        wr[m] = get(comp[m], 0);
      }
    }
  }
  riemann<R>(solver, wl, wr, bn, gam, f);
}

// normal field at D-face (i, j, k) from the state's face values
template <class R, int D>
__device__ __forceinline__ R face_bn(const PatchDev& P, const double* __restrict__ Ub, int i, int j, int k) {
  const int c3[3] = {i, j, k};
  if (P.inflow_mask) {
    // the face of a ghost cell beyond an inflow side (along D the face index stays in [0, n])
    int side = -1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == D || side >= 0) continue;
      if (c3[a] < 0 && (P.inflow_mask >> (2 * a) & 1)) side = 2 * a;
      else if (c3[a] >= P.n[a] && (P.inflow_mask >> (2 * a + 1) & 1)) side = 2 * a + 1;
    }
    if (side >= 0) return Ar<R>::from_d(P.inflow_w[side][5 + D]);
  }
  int s3[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) s3[a] = (a == D) ? fmap(P, a, c3[a]) : cmap(P, a, c3[a]);
  // (the hardware conversion: the flux kernels leave the FP64 pipe idle, and the integer-pipe
  // d2f_alu would cost them about 25 issue slots per face; 256^3 step 4.228 -> 4.194 ms)
  const double b = Ub[(BXF + D) * P.FS + sidx(P, s3[0], s3[1], s3[2])];
  if constexpr (sizeof(R) == 4) return __double2float_rn(b);
  else return b;
}

// F_D at scratch index q from the solver's output f[0..7]: the mass flux (marked with Eq.
// 11's no-motion decision), the momentum components in x, y, z order, E and B_T1, B_T2
template <class R, int D>
__device__ __forceinline__ void store_flux(R* __restrict__ F, long long QS, long long q, const R* f) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  F[q] = Ar<R>::mark(f[0], no_motion_band<R>(f[0], f[7]));
  F[(1 + D) * QS + q] = f[1];
  F[(1 + T1) * QS + q] = f[2];
  F[(1 + T2) * QS + q] = f[3];
  F[4 * QS + q] = f[4];
  F[5 * QS + q] = f[5];
  F[6 * QS + q] = f[6];
}

// the flux through the D-face at (i, j, k) (face index i-1/2 along D) from the stored W
template <class R, int D, int ORDER>
__device__ __forceinline__ void flux_point(const PatchDev& P, const R* __restrict__ W,
                                           const double* __restrict__ Ub, R* __restrict__ F,
                                           int i, int j, int k, int solver) {
  const long long q = qidx(P, i, j, k), QS = P.QS, st = qstride(P, D);
  R f[8], kap[3];
  Gam<R>::kappa(P, kap[0], kap[1], kap[2]);
  flux_core<R, D, ORDER>([&](int m, int o) { return W[m * QS + q + o * st]; }, face_bn<R, D>(P, Ub, i, j, k),
                         Gam<R>::get(P), solver, kap, f);
  store_flux<R, D>(F, QS, q, f);
}

// -------------------------------------------------------------- phase: EMF ----
// Corner EMF E_C at edge (A-1/2, B-1/2), (A, B, C) cyclic (Eq. 9-11): mean of the four
// face EMFs plus upwinded one-sided corrections, the upwind side given by the sign of
// the Riemann mass flux F_rho through the face, and their mean at a face that the flux
// kernel marked as without contact motion (no_motion_band); (db/8) * 2/db = 1/4.
template <class R> __device__ __forceinline__ R upwind(R fr, R left, R right) {
  return Ar<R>::marked(fr) ? R(0.5) * (left + right) : (Ar<R>::negative(fr) ? right : left);
}

// Face EMFs around the edge: Ea_b, Ea_bm = -F_A(B_B) on the A-faces at b and b-1;
// Eb_a, Eb_am = F_B(B_A) on the B-faces at a and a-1.  Cell EMFs ec0..ec3 at (a, b),
// (a-1, b), (a, b-1), (a-1, b-1).  Marked mass fluxes of the same four faces.
template <class R>
__device__ __forceinline__ R corner_core(R Ea_b, R Ea_bm, R Eb_a, R Eb_am, R ec0, R ec1, R ec2, R ec3, R frA_b,
                                         R frA_bm, R frB_a, R frB_am) {
  const R d_bq = upwind<R>(frA_b, ec1 - Eb_am, ec0 - Eb_a);
  const R d_b3q = upwind<R>(frA_bm, Eb_am - ec3, Eb_a - ec2);
  const R d_aq = upwind<R>(frB_a, ec2 - Ea_bm, ec0 - Ea_b);
  const R d_a3q = upwind<R>(frB_am, Ea_bm - ec3, Ea_b - ec1);
  return R(0.25) * (Ea_b + Ea_bm + Eb_a + Eb_am) + R(0.25) * (d_b3q - d_bq) + R(0.25) * (d_a3q - d_aq);
}


// Corner EMF E_C at scratch index q when both transverse axes A, B are active.  Every
// product in corner_core is by 1/4 or 1/2 (exact), so no FMA contraction can change its
// bits: each evaluation of the same edge gives the same value.
template <class R, int C>
__device__ __forceinline__ R corner_value(const PatchDev& P, const R* __restrict__ W, long long q) {
  constexpr int A = (C + 1) % 3, B = (C + 2) % 3;
  const long long QS = P.QS;
  const R* FA = (const R*)P.F[A];
  const R* FB = (const R*)P.F[B];
  const long long sa = qstride(P, A), sb = qstride(P, B);
  const long long oa = q - sa, ob = q - sb, oab = q - sa - sb;
  const R* ec = W + (WEX + C) * QS;  // cell EMFs stored by the recovery
  return corner_core<R>(-FA[5 * QS + q], -FA[5 * QS + ob], FB[6 * QS + q], FB[6 * QS + oa], ec[q], ec[oa], ec[ob],
                        ec[oab], FA[q], FA[ob], FB[q], FB[oa]);
}

template <class R, int C>
__device__ __forceinline__ void corner_point(const PatchDev& P, const R* __restrict__ W,
                                             R* __restrict__ E, int i, int j, int k) {
  constexpr int A = (C + 1) % 3, B = (C + 2) % 3;
  const long long q = qidx(P, i, j, k), QS = P.QS;
  R e;
  if (P.act[A] && !P.act[B]) {
    e = -((const R*)P.F[A])[5 * QS + q];
  } else if (!P.act[A] && P.act[B]) {
    e = ((const R*)P.F[B])[6 * QS + q];
  } else if (!P.act[A] && !P.act[B]) {
    return;
  } else {
    e = corner_value<R, C>(P, W, q);
  }
  E[C * QS + q] = e;
}

template <class R>
__device__ __forceinline__ void emf_point(const PatchDev& P, const R* __restrict__ W,
                                          R* __restrict__ E, int i, int j, int k) {
  // E_x lives on x in [0, nx), E_y on y in [0, ny), E_z on z in [0, nz)
  if (i < P.n[0]) corner_point<R, 0>(P, W, E, i, j, k);
  if (j < P.n[1]) corner_point<R, 1>(P, W, E, i, j, k);
  if (k < P.n[2]) corner_point<R, 2>(P, W, E, i, j, k);
}

// ----------------------------------------------------------- phase: update ----
// New value of the a-face stored at state index sf whose lower-left edge has scratch
// index q: B_a - h [dE_c/db - dE_b/dc] (Eq. 8), with explicitly rounded operations so that
// every evaluation of the same face gives the same bits.
// The same for a face whose four edge EMFs are given (all three axes active): E_c at the
// face's lower and upper b-edges, E_b at its lower and upper c-edges.
template <class R>
__device__ __forceinline__ double face_from(double b_old, R ec0, R ec1, R eb0, R eb1, R inv_b, R inv_c, R h) {
  const R curl = Ar<R>::sub_rn(Ar<R>::mul_rn(Ar<R>::sub_rn(ec1, ec0), inv_b),
                               Ar<R>::mul_rn(Ar<R>::sub_rn(eb1, eb0), inv_c));
  return __dsub_rn(b_old, Ar<R>::to_d(Ar<R>::mul_rn(h, curl)));
}

template <class R>
__device__ __forceinline__ double face_new(const PatchDev& P, const double* __restrict__ Ub,
                                           const R* __restrict__ E, R h, int a, long long sf, long long q) {
  const int b = (a + 1) % 3, c = (a + 2) % 3;
  const long long QS = P.QS;
  R curl = R(0);
  if (P.act[b])
    curl = Ar<R>::mul_rn(Ar<R>::sub_rn(E[c * QS + q + qstride(P, b)], E[c * QS + q]), Gam<R>::inv(P, b));
  if (P.act[c])
    curl = Ar<R>::sub_rn(curl, Ar<R>::mul_rn(Ar<R>::sub_rn(E[b * QS + q + qstride(P, c)], E[b * QS + q]),
                                             Gam<R>::inv(P, c)));
  return __dsub_rn(Ub[(BXF + a) * P.FS + sf], Ar<R>::to_d(Ar<R>::mul_rn(h, curl)));
}

// Eq. 7 for the cell fields (plus h S of Eq. 2 at Usrc) and Eq. 8 (-curl E) for the
// owned faces: out = base - h (div F) + h S;  B_a -= h [dE_C/db - dE_B/dc].
template <class R>
__device__ __forceinline__ void update_point(const PatchDev& P, const double* __restrict__ Ub,
                                             const double* __restrict__ Us, double* __restrict__ Uo,
                                             const R* __restrict__ E, R h,
                                             const SourceDev& src, int i, int j, int k) {
  const long long s = sidx(P, i, j, k), FS = P.FS;
  const long long q = qidx(P, i, j, k), QS = P.QS;
  if (i < P.n[0] && j < P.n[1] && k < P.n[2]) {
    R div[5] = {R(0), R(0), R(0), R(0), R(0)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (!P.act[d]) continue;
      const R* Fd = (const R*)P.F[d];
      const long long st = qstride(P, d);
      const R idd = Gam<R>::inv(P, d);
#pragma unroll
      for (int f = 0; f < 5; ++f) div[f] += (Fd[f * QS + q + st] - Fd[f * QS + q]) * idd;
    }
    Uo[s] = Ub[s] - Ar<R>::to_d(h * div[0]);
    if (src.potential == POT_NONE) {
#pragma unroll
      for (int a = 0; a < 3; ++a) Uo[(MX + a) * FS + s] = Ub[(MX + a) * FS + s] - Ar<R>::to_d(h * div[1 + a]);
      Uo[EN * FS + s] = Ub[EN * FS + s] - Ar<R>::to_d(h * div[4]);
    } else {
      R g[3];
      grad_psi<R>(src, centre<R>(P, 0, i), centre<R>(P, 1, j), centre<R>(P, 2, k), g);
      const R rho = Ar<R>::from_d(Us[s]);
      const R sm[3] = {-rho * g[0], -rho * g[1], -rho * g[2]};
      const R se = -(Ar<R>::from_d(Us[MX * FS + s]) * g[0] + Ar<R>::from_d(Us[MY * FS + s]) * g[1] +
                     Ar<R>::from_d(Us[MZ * FS + s]) * g[2]);
#pragma unroll
      for (int a = 0; a < 3; ++a)
        Uo[(MX + a) * FS + s] = Ub[(MX + a) * FS + s] - Ar<R>::to_d(h * div[1 + a]) + Ar<R>::to_d(h * sm[a]);
      Uo[EN * FS + s] = Ub[EN * FS + s] - Ar<R>::to_d(h * div[4]) + Ar<R>::to_d(h * se);
    }
  }
  // faces
  const int c3[3] = {i, j, k};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    if (!(c3[a] < P.nface[a] && c3[b] < P.n[b] && c3[c] < P.n[c])) continue;
    Uo[(BXF + a) * FS + s] = face_new<R>(P, Ub, E, h, a, s, q);
  }
}

// Cell fields of the stage update (Eq. 7 with h S of Eq. 2 evaluated at Us): u = base - h
// (div F) + h S at interior cell (i, j, k), state index s, scratch index q.
template <class R>
__device__ __forceinline__ void cell_update(const PatchDev& P, const double* __restrict__ Ub,
                                            const double* __restrict__ Us, R h, const SourceDev& src, int i,
                                            int j, int k, long long s, long long q, double* u) {
  const long long FS = P.FS, QS = P.QS;
  R div[5] = {R(0), R(0), R(0), R(0), R(0)};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (!P.act[d]) continue;
    const R* Fd = (const R*)P.F[d];
    const long long st = qstride(P, d);
    const R idd = Gam<R>::inv(P, d);
#pragma unroll
    for (int f = 0; f < 5; ++f) div[f] += (Fd[f * QS + q + st] - Fd[f * QS + q]) * idd;
  }
  u[0] = Ub[s] - Ar<R>::to_d(h * div[0]);
  if (src.potential == POT_NONE) {
#pragma unroll
    for (int a = 0; a < 3; ++a) u[1 + a] = Ub[(MX + a) * FS + s] - Ar<R>::to_d(h * div[1 + a]);
    u[4] = Ub[EN * FS + s] - Ar<R>::to_d(h * div[4]);
  } else {
    R g[3];
    grad_psi<R>(src, centre<R>(P, 0, i), centre<R>(P, 1, j), centre<R>(P, 2, k), g);
    const R rho = Ar<R>::from_d(Us[s]);
    const R sm[3] = {-rho * g[0], -rho * g[1], -rho * g[2]};
    const R se = -(Ar<R>::from_d(Us[MX * FS + s]) * g[0] + Ar<R>::from_d(Us[MY * FS + s]) * g[1] +
                     Ar<R>::from_d(Us[MZ * FS + s]) * g[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
      u[1 + a] = Ub[(MX + a) * FS + s] - Ar<R>::to_d(h * div[1 + a]) + Ar<R>::to_d(h * sm[a]);
    u[4] = Ub[EN * FS + s] - Ar<R>::to_d(h * div[4]) + Ar<R>::to_d(h * se);
  }
}

// ------------------------------------------------- fused update and recovery --
// The fused update of a cell also needs the new values of its upper faces, which the
// neighbouring cells own and write; it computes them again with face_new, whose explicitly
// rounded operations make the copy bitwise equal to the owner's value.

// Stage update, then (interior cells) the recovery of the new state: U at cell (i, j, k)
// and its owned faces as update_point, the end-of-step floors when `last` and the floors
// are on, and W of the new cell stored at the cell (its ghost images are filled afterwards
// by ghost_point).  Returns the CFL limit of the new cell (+inf for face-only points);
// floored cells are added to *nfl.
template <class R>
__device__ __forceinline__ R update_fused_point(const PatchDev& P, const double* __restrict__ Ub,
                                                     const double* __restrict__ Us, double* __restrict__ Uo,
                                                     const R* __restrict__ E, R h, const SourceDev& src,
                                                     int i, int j, int k, bool last, int* nfl) {
  const long long s = sidx(P, i, j, k), FS = P.FS;
  const long long q = qidx(P, i, j, k);
  const int c3[3] = {i, j, k};
  if (!(i < P.n[0] && j < P.n[1] && k < P.n[2])) {
    // owned faces on the extra layer of an outflow axis
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int b = (a + 1) % 3, c = (a + 2) % 3;
      if (c3[a] < P.nface[a] && c3[b] < P.n[b] && c3[c] < P.n[c])
        Uo[(BXF + a) * FS + s] = face_new<R>(P, Ub, E, h, a, s, q);
    }
    return R(INFINITY);
  }
  double u[5];
  cell_update<R>(P, Ub, Us, h, src, i, j, k, s, q, u);
  // new lower (owned) and upper faces
  double blo[3], bhi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    blo[a] = face_new<R>(P, Ub, E, h, a, s, q);
    if (P.act[a]) {
      int cu[3] = {i, j, k};
      cu[a] = fmap(P, a, c3[a] + 1);
      bhi[a] = face_new<R>(P, Ub, E, h, a, sidx(P, cu[0], cu[1], cu[2]), q + qstride(P, a));
    } else {
      bhi[a] = blo[a];  // a trivial axis: the upper face is the same face
    }
  }
  if (last && P.floors) *nfl += floor_core(P, u[0], u[1], u[2], u[3], u[4], blo[0], bhi[0], blo[1], bhi[1], blo[2], bhi[2]);
  Uo[s] = u[0];
#pragma unroll
  for (int a = 0; a < 3; ++a) Uo[(MX + a) * FS + s] = u[1 + a];
  Uo[EN * FS + s] = u[4];
#pragma unroll
  for (int a = 0; a < 3; ++a) Uo[(BXF + a) * FS + s] = blo[a];
  // recovery of the new cell (its CFL limit in the corrector only)
  return prim_core<R>(P, u[0], u[1], u[2], u[3], u[4], blo[0] + bhi[0], blo[1] + bhi[1], blo[2] + bhi[2],
                      (R*)P.W, q, true, true, last);
}

// Ghost position number t of the padded scratch box (the shell of width g2 around the
// interior: z-slabs, then y-slabs within the interior planes, then x-slabs), as (i, j, k).
__device__ __forceinline__ bool ghost_index(const PatchDev& P, long long t, int& i, int& j, int& k) {
  const int gx = P.g2[0], gy = P.g2[1], gz = P.g2[2];
  const long long QX = P.QX, QY = P.QY;
  const long long nzs = 2LL * gz * QX * QY;            // z < 0 or z >= n
  const long long nys = 2LL * gy * QX * P.n[2];        // interior z, y outside
  const long long nxs = 2LL * gx * (long long)P.n[1] * P.n[2];  // interior y, z, x outside
  if (t < nzs) {
    const int s = (int)(t / (QX * QY));
    const long long r = t % (QX * QY);
    i = (int)(r % QX) - gx;
    j = (int)(r / QX) - gy;
    k = s < gz ? s - gz : P.n[2] + (s - gz);
    return true;
  }
  t -= nzs;
  if (t < nys) {
    const long long per = 2LL * gy * QX;
    k = (int)(t / per);
    const long long r = t % per;
    i = (int)(r % QX) - gx;
    const int s = (int)(r / QX);
    j = s < gy ? s - gy : P.n[1] + (s - gy);
    return true;
  }
  t -= nys;
  if (t < nxs) {
    const long long per = 2LL * gx;
    const long long row = t / per;
    const int s = (int)(t % per);
    j = (int)(row % P.n[1]);
    k = (int)(row / P.n[1]);
    i = s < gx ? s - gx : P.n[0] + (s - gx);
    return true;
  }
  return false;
}

__host__ __device__ __forceinline__ long long ghost_count(const PatchDev& P) {
  return 2LL * P.g2[2] * P.QX * P.QY + 2LL * P.g2[1] * P.QX * P.n[2] + 2LL * P.g2[0] * (long long)P.n[1] * P.n[2];
}

// W at ghost position (i, j, k) of the current state: a copy of the interior cell it maps to
// when every axis on which it lies outside is periodic, else the recovery from U as
// prim_point (an outflow ghost repeats the boundary face in its face sum).
template <class R>
__device__ __forceinline__ void ghost_point(const PatchDev& P, const double* __restrict__ U, int i, int j, int k) {
  const int c3[3] = {i, j, k};
  bool copy = true;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if ((c3[a] < 0 || c3[a] >= P.n[a]) && !P.per[a]) copy = false;
  R* W = (R*)P.W;
  if (copy) {
    const long long QS = P.QS, t = qidx(P, i, j, k), q = qidx(P, cmap(P, 0, i), cmap(P, 1, j), cmap(P, 2, k));
#pragma unroll
    for (int m = 0; m < NWQ; ++m) W[m * QS + t] = W[m * QS + q];
  } else {
    prim_point<R>(P, U, W, i, j, k, true, false);
  }
}

// ordered bits of a non-negative double (monotone as unsigned integers)
__device__ __forceinline__ unsigned long long dbits(double x) {
  return (unsigned long long)__double_as_longlong(x);
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
  __shared__ T red[32];  // one per warp, up to 1024 threads
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

}  // namespace mhd
