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

// (32-bit unsigned division when the plane of the box has fewer than 2^31 points, which
// is every practical size; 64-bit division is a long software sequence)
__device__ __forceinline__ bool range_point(const Range& rg, int& i, int& j, int& k) {
  const long long plane = (long long)rg.ext[0] * rg.ext[1];
  int ii, jj;
  if (plane < (1LL << 31)) {
    const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (unsigned)plane) return false;
    const unsigned e0 = (unsigned)rg.ext[0];
    const unsigned q = r / e0;
    jj = (int)q;
    ii = (int)(r - q * e0);
  } else {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= plane) return false;
    jj = (int)(r / rg.ext[0]);
    ii = (int)(r - (long long)jj * rg.ext[0]);
  }
  i = rg.lo[0] + ii;
  j = rg.lo[1] + jj;
  k = rg.lo[2] + (int)blockIdx.y;
  return true;
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

// one direction's fluxes with the Riemann solver S (RIEMANN_*) fixed at compile time.  The
// FP32 kernels are held to five resident CTAs per SM (48 registers, a few bytes spilled):
// the y and z donor-cell kernels then run 7-9% faster than at 56-58 registers and four CTAs
// (measured); the FP64 kernels would spill hundreds of bytes under that cap.
template <class R, int D, int ORDER, int S>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 5 : 1) k_flux(PatchDev P, const double* __restrict__ Ub,
                                                                      Range rg) {
  int i, j, k;
  if (!range_point(rg, i, j, k)) return;
  flux_point<R, D, ORDER>(P, (const R*)P.W, Ub, (R*)P.F[D], i, j, k, S);
}


// Fluxes through the D-faces (D = y or z) marching along D: each thread takes one position
// (x, the other transverse axis) of the flux range and a segment of kMarch consecutive faces,
// and loads one new cell of W per face (coalesced along x).  The kappa-scheme reconstructs
// each cell once: from its two one-sided differences dl, dr, the two limited slopes
// m1 = minmod(dl, b dr), m2 = minmod(dr, b dl) give its value at the upper face,
// w + K1 m1 + K2 m2 (w_L there), and at the lower face, w - K1 m2 - K2 m1 (w_R there) -- the
// expressions of kappa_face, where the per-face kernel evaluates both neighbours of every face.
// The donor-cell stage carries the previous cell.  The arithmetic is flux_point's (the
// compiler may contract its multiply-adds differently, so the bits can differ in the last
// place).
// Segments of seg faces (16 where the box gives enough columns, fewer on thinner boxes, see
// launch_flux); FP32 kernels at four (donor cell) and three (kappa-scheme) resident CTAs per
// SM: the fastest of 8, 16, 32, 64 faces and three or four CTAs at 256^3 (the kappa kernels
// spill at four).
constexpr int kMarch = 16;

// Block size of the marching kernels: 128 threads for the FP32 kappa-scheme, seven blocks per
// SM (72 registers, 28 warps; at 256^3 the y and z launches took 0.333 and 0.315 ms against
// 0.356 and 0.347 with three blocks of 256 threads at 78 registers, 24 warps; eight blocks
// spill), kBlock otherwise.
template <class R, int ORDER> constexpr int march_block() { return sizeof(R) == 4 && ORDER == 2 ? 128 : kBlock; }

template <class R, int D, int ORDER, int S>
__global__ void __launch_bounds__(march_block<R, ORDER>(), sizeof(R) == 4 ? (ORDER == 1 ? 4 : 7) : 1) k_flux_march(PatchDev P,
                                                                             const double* __restrict__ Ub,
                                                                             Range rg, int seg) {
  static_assert(D == 1 || D == 2, "marching along y or z");
  constexpr int T = D == 1 ? 2 : 1;  // the transverse axis other than x
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  const unsigned e0 = (unsigned)rg.ext[0];
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= e0 * (unsigned)rg.ext[T]) return;
  const unsigned qt = r / e0;
  int c3[3];
  c3[0] = rg.lo[0] + (int)(r - qt * e0);
  c3[T] = rg.lo[T] + (int)qt;
  const int f0 = rg.lo[D] + (int)blockIdx.y * seg;
  const int f1 = min(f0 + seg, rg.lo[D] + rg.ext[D]);
  const R* __restrict__ W = (const R*)P.W;
  R* __restrict__ F = (R*)P.F[D];
  const long long QS = P.QS, st = qstride(P, D);
  c3[D] = f0;
  long long q = qidx(P, c3[0], c3[1], c3[2]);  // cell of face f0 (its lower face)
  const R gam = Gam<R>::get(P);
  const int comp[7] = {WR, WVX + D, WVX + T1, WVX + T2, WP, WBX + T1, WBX + T2};
  R out[8];
  if (ORDER == 1) {
    R wm[7], w0[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) wm[m] = W[comp[m] * QS + q - st];
#pragma unroll 1
    for (int f = f0; f < f1; ++f, q += st) {
#pragma unroll
      for (int m = 0; m < 7; ++m) w0[m] = W[comp[m] * QS + q];
      c3[D] = f;
      riemann<R>(S, wm, w0, face_bn<R, D>(P, Ub, c3[0], c3[1], c3[2]), gam, out);
      store_flux<R, D>(F, QS, q, out);
#pragma unroll
      for (int m = 0; m < 7; ++m) wm[m] = w0[m];
    }
  } else {
    R K1, K2, kb;
    Gam<R>::kappa(P, K1, K2, kb);
    R b[7], c[7], up[7];  // W of cells f-1 and f; value of cell f-1 at face f (w_L there)
#pragma unroll
    for (int m = 0; m < 7; ++m) {
      const R a = W[comp[m] * QS + q - 2 * st];
      b[m] = W[comp[m] * QS + q - st];
      c[m] = W[comp[m] * QS + q];
      const R dl = b[m] - a, dr = c[m] - b[m];
      up[m] = b[m] + K1 * minmod<R>(dl, kb * dr) + K2 * minmod<R>(dr, kb * dl);
    }
#pragma unroll 1
    for (int f = f0; f < f1; ++f, q += st) {
      R wl[7], wr[7];
#pragma unroll
      for (int m = 0; m < 7; ++m) {
        const R d = W[comp[m] * QS + q + st];
        const R dl = c[m] - b[m], dr = d - c[m];
        const R m1 = minmod<R>(dl, kb * dr), m2 = minmod<R>(dr, kb * dl);
        wl[m] = up[m];
        wr[m] = c[m] - K1 * m2 - K2 * m1;
        up[m] = c[m] + K1 * m1 + K2 * m2;
        b[m] = c[m];
        c[m] = d;
      }
      // a face whose reconstructed rho or p is not positive takes the donor-cell states:
      // cells f - 1 (loaded again) and f (now in b)
      if (!(wl[0] > R(0)) || !(wr[0] > R(0)) || !(wl[4] > R(0)) || !(wr[4] > R(0))) {
#pragma unroll
        for (int m = 0; m < 7; ++m) {
          wl[m] = W[comp[m] * QS + q - st];
          wr[m] = b[m];
        }
      }
      c3[D] = f;
      riemann<R>(S, wl, wr, face_bn<R, D>(P, Ub, c3[0], c3[1], c3[2]), gam, out);
      store_flux<R, D>(F, QS, q, out);
    }
  }
}

// kappa-scheme fluxes through the x faces with each cell reconstructed once: a warp takes 32
// consecutive cells of the scratch rows of one plane of the flux range (rows run on through
// their padding, so a warp may span two rows).  Each lane reconstructs its cell's values at
// its lower and upper faces (w - K1 m2 - K2 m1 and w + K1 m1 + K2 m2, the expressions of
// kappa_face), and the face below lane l takes lane l - 1's upper value by a shuffle.  Windows
// overlap by one cell (lane 0 only passes its value on), so a warp computes 31 faces; faces in
// the x padding are computed and not stored.  Loads are clamped into the arrays (lanes past
// the last row read stored values and store nothing).  Measured at 256^3: 0.345 ms per launch
// against 0.362 for the per-face kernel (512 x 512 x 128: 0.566 against 0.609); the same
// scheme for the donor-cell stage, which has no reconstruction to share, was slower than its
// per-face kernel (0.302 against 0.284 ms), as was this kernel at four CTAs per SM (0.375 ms).
template <class R, int S>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 5 : 1) k_flux_xs(PatchDev P,
                                                                          const double* __restrict__ Ub,
                                                                          Range rg, unsigned nwin) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned win = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
  if (win >= nwin) return;  // whole warps
  const int k = rg.lo[2] + (int)blockIdx.y;
  const long long QS = P.QS;
  const long long q0 = qidx(P, -2, rg.lo[1], k);    // first cell of the plane's rows
  const long long len = (long long)rg.ext[1] * P.QX;  // cells of those rows
  const long long off = 31LL * win - 1 + lane;        // this lane's cell, from q0
  const long long q = q0 + off;
  const long long ql = q < 1 ? 1 : (q > QS - 2 ? QS - 2 : q);
  const R* __restrict__ W = (const R*)P.W;
  constexpr int comp[7] = {WR, WVX, WVY, WVZ, WP, WBY, WBZ};
  R K1, K2, kb;
  Gam<R>::kappa(P, K1, K2, kb);
  R wl[7], wr[7];
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    const R* Wm = W + comp[m] * QS;
    const R a = Wm[ql - 1], c = Wm[ql], e = Wm[ql + 1];
    const R dl = c - a, dr = e - c;
    const R m1 = minmod<R>(dl, kb * dr), m2 = minmod<R>(dr, kb * dl);
    const R up = c + K1 * m1 + K2 * m2;
    wr[m] = c - K1 * m2 - K2 * m1;
    wl[m] = __shfl_up_sync(0xffffffffu, up, 1);
  }
  // the face below this lane's cell: stored when its cell is a flux-range face
  if (lane == 0 || off < 0 || off >= len) return;
  const unsigned row = (unsigned)off / (unsigned)P.QX;
  const int i = (int)((unsigned)off - row * (unsigned)P.QX) - 2;
  if (i < 0 || i > P.n[0]) return;
  if (!(wl[0] > R(0)) || !(wr[0] > R(0)) || !(wl[4] > R(0)) || !(wr[4] > R(0))) {
    // a face whose reconstructed rho or p is not positive takes the donor-cell states
#pragma unroll
    for (int m = 0; m < 7; ++m) {
      wl[m] = W[comp[m] * QS + q - 1];
      wr[m] = W[comp[m] * QS + q];
    }
  }
  R out[8];
  riemann<R>(S, wl, wr, face_bn<R, 0>(P, Ub, i, rg.lo[1] + (int)row, k), Gam<R>::get(P), out);
  store_flux<R, 0>((R*)P.F[0], QS, q, out);
}

// Donor-cell fluxes of the predictor through the faces of all three directions in one
// kernel, for patches with three active axes: a thread takes one (x, y) column of
// [-1, n0] x [-1, n1] and a segment of seg planes of [-1, n2], marching up in z.  At each cell c
// it loads W(c) once and computes the x face between c - x and c, the y face between c - y and
// c, and the z face between c - z (carried from the previous plane) and c: 22 loads per cell
// for three faces, where the three separate kernels take 28 (the per-face x kernel loads both
// of its cells).  Each (i, j, k) computes exactly the faces the three flux ranges hold there.
// Measured at 256^3: step 4.266 -> 4.210 ms (disc 512 x 512 x 128: 9.24 -> 9.10 ms).
template <class R, int S>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 4 : 1) k_flux_d3(PatchDev P, const double* __restrict__ Ub,
                                                                          int seg) {
  const unsigned ex = (unsigned)P.n[0] + 2u, ey = (unsigned)P.n[1] + 2u;
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ex * ey) return;
  const unsigned qy = r / ex;
  const int i = -1 + (int)(r - qy * ex), j = -1 + (int)qy;
  const int k0 = -1 + (int)blockIdx.y * seg;
  const int k1 = min(k0 + seg, P.n[2] + 1);
  const R* __restrict__ W = (const R*)P.W;
  const long long QS = P.QS, QX = P.QX, QP = (long long)P.QX * P.QY;
  const R gam = Gam<R>::get(P);
  long long q = qidx(P, i, j, k0);
  R wz[8];  // W of the cell below
#pragma unroll
  for (int m = 0; m < 8; ++m) wz[m] = W[m * QS + q - QP];
  R out[8];
#pragma unroll 1
  for (int k = k0; k < k1; ++k, q += QP) {
    R w[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) w[m] = W[m * QS + q];
    if (i >= 0) {  // x face: [rho, vx, vy, vz, p, By, Bz]
      R wl[7], wr[7];
      const int cp[7] = {WR, WVX, WVY, WVZ, WP, WBY, WBZ};
#pragma unroll
      for (int m = 0; m < 7; ++m) {
        wl[m] = W[cp[m] * QS + q - 1];
        wr[m] = w[cp[m]];
      }
      riemann<R>(S, wl, wr, face_bn<R, 0>(P, Ub, i, j, k), gam, out);
      store_flux<R, 0>((R*)P.F[0], QS, q, out);
    }
    if (j >= 0) {  // y face: [rho, vy, vz, vx, p, Bz, Bx]
      R wl[7], wr[7];
      const int cp[7] = {WR, WVY, WVZ, WVX, WP, WBZ, WBX};
#pragma unroll
      for (int m = 0; m < 7; ++m) {
        wl[m] = W[cp[m] * QS + q - QX];
        wr[m] = w[cp[m]];
      }
      riemann<R>(S, wl, wr, face_bn<R, 1>(P, Ub, i, j, k), gam, out);
      store_flux<R, 1>((R*)P.F[1], QS, q, out);
    }
    if (k >= 0) {  // z face: [rho, vz, vx, vy, p, Bx, By]
      R wl[7], wr[7];
      const int cp[7] = {WR, WVZ, WVX, WVY, WP, WBX, WBY};
#pragma unroll
      for (int m = 0; m < 7; ++m) {
        wl[m] = wz[cp[m]];
        wr[m] = w[cp[m]];
      }
      riemann<R>(S, wl, wr, face_bn<R, 2>(P, Ub, i, j, k), gam, out);
      store_flux<R, 2>((R*)P.F[2], QS, q, out);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) wz[m] = w[m];
  }
}

// The same for patches whose active axes are x and y (a 2D plane): a thread per cell of
// [-1, n0] x [-1, n1] computes its lower x and y faces from W(c), W(c - x) and W(c - y).
template <class R, int S>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 4 : 1) k_flux_d2(PatchDev P, const double* __restrict__ Ub) {
  const unsigned ex = (unsigned)P.n[0] + 2u, ey = (unsigned)P.n[1] + 2u;
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ex * ey) return;
  const unsigned qy = r / ex;
  const int i = -1 + (int)(r - qy * ex), j = -1 + (int)qy;
  const R* __restrict__ W = (const R*)P.W;
  const long long QS = P.QS, QX = P.QX;
  const R gam = Gam<R>::get(P);
  const long long q = qidx(P, i, j, 0);
  R w[8], out[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) w[m] = W[m * QS + q];
  if (i >= 0) {  // x face: [rho, vx, vy, vz, p, By, Bz]
    R wl[7], wr[7];
    const int cp[7] = {WR, WVX, WVY, WVZ, WP, WBY, WBZ};
#pragma unroll
    for (int m = 0; m < 7; ++m) {
      wl[m] = W[cp[m] * QS + q - 1];
      wr[m] = w[cp[m]];
    }
    riemann<R>(S, wl, wr, face_bn<R, 0>(P, Ub, i, j, 0), gam, out);
    store_flux<R, 0>((R*)P.F[0], QS, q, out);
  }
  if (j >= 0) {  // y face: [rho, vy, vz, vx, p, Bz, Bx]
    R wl[7], wr[7];
    const int cp[7] = {WR, WVY, WVZ, WVX, WP, WBZ, WBX};
#pragma unroll
    for (int m = 0; m < 7; ++m) {
      wl[m] = W[cp[m] * QS + q - QX];
      wr[m] = w[cp[m]];
    }
    riemann<R>(S, wl, wr, face_bn<R, 1>(P, Ub, i, j, 0), gam, out);
    store_flux<R, 1>((R*)P.F[1], QS, q, out);
  }
}

// corner EMFs: memory-latency bound; eight resident blocks per SM (measured)
template <class R>
__global__ void __launch_bounds__(kBlock, 8) k_emf(PatchDev P, Range rg) {
  int i, j, k;
  if (!range_point(rg, i, j, k)) return;
  emf_point<R>(P, (const R*)P.W, (R*)P.E, i, j, k);
}

// Periodic images of the W of interior cell (i, j, k) for a patch with fewer than three active
// axes: the shifts by 0 or +-n that land in [-2, n + 1] along the active axes only (a trivial
// axis has no ghost shell).
template <class R>
__device__ __forceinline__ void periodic_images_act(const PatchDev& P, R* __restrict__ W, int i, int j, int k,
                                                    long long q) {
  const int c[3] = {i, j, k};
  bool near = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) near |= P.act[a] && (c[a] < 2 || c[a] >= P.n[a] - 2);
  if (!near) return;
  const long long QS = P.QS;
  R v[NWQ];
#pragma unroll
  for (int m = 0; m < NWQ; ++m) v[m] = W[m * QS + q];
  const int z0 = P.act[2] ? -1 : 0, y0 = P.act[1] ? -1 : 0, x0 = P.act[0] ? -1 : 0;
  for (int sz = z0; sz <= -z0; ++sz) {
    const int kk = k + sz * P.n[2];
    if (kk < -2 || kk > P.n[2] + 1) continue;
    for (int sy = y0; sy <= -y0; ++sy) {
      const int jj = j + sy * P.n[1];
      if (jj < -2 || jj > P.n[1] + 1) continue;
      for (int sx = x0; sx <= -x0; ++sx) {
        const int ii = i + sx * P.n[0];
        if (ii < -2 || ii > P.n[0] + 1 || (sx == 0 && sy == 0 && sz == 0)) continue;
        const long long t = qidx(P, ii, jj, kk);
#pragma unroll
        for (int m = 0; m < NWQ; ++m) W[m * QS + t] = v[m];
      }
    }
  }
}

// Stage update fused with the recovery of the new state (see update_fused_point).  Its FP64
// arithmetic is the bound; six resident blocks per SM (40 registers, a few spills to L1)
// hide the memory latency better than fewer blocks without spills (measured).  The
// predictor takes dt from the host or the CFL slot and records it; the corrector reuses the
// recorded dt and accumulates the CFL limit of the new state into the (reset) slot.
template <class R>
__global__ void __launch_bounds__(kBlock, 6) k_update_fused(PatchDev P, const double* __restrict__ Ub,
                                                         const double* __restrict__ Us,
                                                         double* __restrict__ Uo, Range rg, StageArgs a,
                                                         int images) {
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
  if (range_point(rg, i, j, k)) {
    lim = update_fused_point<R>(P, Ub, Us, Uo, (const R*)P.E, h, a.src, i, j, k, a.stage == 1, &nfl);
    // (every axis periodic: the new cell's W also at its images in the ghost shell)
    if (images && i < P.n[0] && j < P.n[1] && k < P.n[2]) periodic_images_act<R>(P, (R*)P.W, i, j, k, qidx(P, i, j, k));
  }
  if (a.stage == 1) {
    if (P.floors) {
      const unsigned tot = __reduce_add_sync(0xffffffffu, (unsigned)nfl);
      if ((threadIdx.x & 31) == 0 && tot) atomicAdd(P.floored, (unsigned long long)tot);
    }
    block_min_atomic(lim, P.cfl_min);
  }
}

constexpr int kTX = 32, kTY = 8;
constexpr int kEB = kTX * kTY;  // one thread per cell of a tile plane

template <class R>
__device__ __forceinline__ R emf_at(const PatchDev& P, const R* __restrict__ W, int c, int i, int j, int k) {
  const long long q = qidx(P, i, j, k);
  return c == 0 ? corner_value<R, 0>(P, W, q) : (c == 1 ? corner_value<R, 1>(P, W, q) : corner_value<R, 2>(P, W, q));
}

// asynchronous global -> shared copy of one 4- or 8-byte value (completion: cp_async_wait)
template <class R> __device__ __forceinline__ void cp_async(R* smem, const R* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(sizeof(R)) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The twelve values per cell that the edge EMFs of a plane read (the mass flux and the two
// transverse-field fluxes of each direction, and the three cell EMFs), staged in shared
// memory over the tile and a halo of one cell below and above it in x and y:
// (kTY + 2) x (kTX + 2) per array, point (ii, jj) of the tile at (jj + 1) * kSW + ii + 1.
// Rolling pairs [2] hold planes k and k + 1 of the march, the others plane k (the x and y
// faces) or the z faces at k + 1/2.
// Used by the FP32 update with the end-of-step floors (24.5 KB per CTA): there it is 3%
// faster per launch on the disc than reading the inputs from global memory (2.96 against
// 3.06 ms at 512 x 512 x 128), while without the floors it is 3% slower (1.30 against 1.26 ms
// at 256^3).  The FP64 arrays would take a CTA past 48 KB of static shared memory.
constexpr int kSW = kTX + 2, kSH = kTY + 2, kSP = kSW * kSH;
template <class R, bool ON> struct EdgeStage {
  static constexpr int N = ON ? kSP : 1;
  R x0[2][N], x6[2][N], x5[N];  // F_x: mass (marked), B_z flux, B_y flux
  R y0[2][N], y5[2][N], y6[N];  // F_y: mass (marked), B_z flux, B_x flux
  R z0[N], z5[N], z6[N];        // F_z at k + 1/2: mass (marked), B_x flux, B_y flux
  R ecx[2][N], ecy[2][N], ecz[N];
};

// Corner EMFs and the stage update in one kernel, for patches with three active axes.
// Five resident CTAs per SM (48 registers): five is the fastest of four, five and six on
// 128^3 and 256^3, and 32 x 8 tiles are faster than 32 x 16 at two or three CTAs per SM
// (measured at 256^3: 1.26 ms against 1.37 at four CTAs, 1.39 and 1.69 with 32 x 16).
// A CTA owns a kTX x kTY column of cells over lz consecutive z-planes and marches up in z.
// For plane k:
//  (S) with the floors (FP32, see EdgeStage): the edge EMFs' inputs of plane k + 1 are
//      copied to shared memory asynchronously while (B) and (C) run; plane k's arrived
//      during the previous plane;
//  (A) the edge EMFs the plane's faces need -- E_z at plane k, E_x and E_y at plane k + 1
//      (at the first plane also at k, from global memory) -- over the tile and its upper
//      halo row and column, into shared memory;
//  (B) from them, the new face values -- x and y faces at plane k, z faces at k + 1 (at the
//      first plane also at k) -- over the tile and its upper halo, into shared memory;
//      faces of the extra layer of an outflow axis, which no cell owns, are stored here;
//  (C) each cell: flux divergence and source, its owned (lower) faces stored, the floors
//      when asked, the recovery of the new state (W, cell EMFs) and its CFL limit.
// E_x, E_y and the z faces roll between two plane buffers.  Each face is
// computed about once (about 3.3 FP64 face updates per cell against 6 when every cell
// recomputes its upper faces), the edge EMFs do not go through HBM, and when staged the
// twelve edge inputs of a cell are read from global memory once instead of three times
// (without staging the second and third reads hit L1 or L2).  Edges and faces
// of the halo are computed by both CTAs that need them; both get the same bits
// (corner_core and face_from are insensitive to FMA contraction).  The cell EMFs are
// read from Win, the W of the stage's input, while CTAs of neighbouring tiles write the W
// of the new state: that goes to the other buffer, Wout.
constexpr int kEMinBlocks = 5;

// Periodic images of the W of interior cell (i, j, k) (scratch index q) in the ghost shell
// of width 2: every combination of shifts by 0 or +-n per axis that lands in [-2, n + 1],
// other than no shift.  Used when all three axes are periodic; it replaces the ghost-fill
// kernel, whose copies it makes.
template <class R>
__device__ __forceinline__ void periodic_images(const PatchDev& P, R* __restrict__ W, int i, int j, int k,
                                                long long q) {
  const int c[3] = {i, j, k};
  bool near = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) near |= c[a] < 2 || c[a] >= P.n[a] - 2;
  if (!near) return;
  const long long QS = P.QS;
  R v[NWQ];
#pragma unroll
  for (int m = 0; m < NWQ; ++m) v[m] = W[m * QS + q];
  for (int sz = -1; sz <= 1; ++sz) {
    const int kk = k + sz * P.n[2];
    if (kk < -2 || kk > P.n[2] + 1) continue;
    for (int sy = -1; sy <= 1; ++sy) {
      const int jj = j + sy * P.n[1];
      if (jj < -2 || jj > P.n[1] + 1) continue;
      for (int sx = -1; sx <= 1; ++sx) {
        const int ii = i + sx * P.n[0];
        if (ii < -2 || ii > P.n[0] + 1 || (sx == 0 && sy == 0 && sz == 0)) continue;
        const long long t = qidx(P, ii, jj, kk);
#pragma unroll
        for (int m = 0; m < NWQ; ++m) W[m * QS + t] = v[m];
      }
    }
  }
}

template <class R, bool FLOORS>
__global__ void __launch_bounds__(kEB, kEMinBlocks) k_emf_update(PatchDev P, const R* __restrict__ Win,
                                                       R* __restrict__ Wout, const double* __restrict__ Ub,
                                                       const double* __restrict__ Us, double* __restrict__ Uo,
                                                       StageArgs a, int lz, int images, int cells_out) {
  constexpr int SX = kTX + 1;  // row pitch of the arrays with an x halo
  __shared__ R sEz[(kTY + 1) * SX];
  __shared__ R sEx[2][(kTY + 1) * kTX];
  __shared__ R sEy[2][kTY * SX];
  __shared__ double sBx[kTY * SX];
  __shared__ double sBy[(kTY + 1) * kTX];
  __shared__ double sBz[2][kTY * kTX];
  constexpr bool STAGED = sizeof(R) == 4 && FLOORS;
  __shared__ EdgeStage<R, STAGED> G;
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
  // (staged: this barrier comes after the first plane's copies)
  if constexpr (!STAGED) __syncthreads();
  const int ntx = (P.n[0] + kTX - 1) / kTX;
  const int i0 = (int)(blockIdx.x % ntx) * kTX, j0 = (int)(blockIdx.x / ntx) * kTY;
  const int kz0 = (int)blockIdx.y * lz;
  const int kz1 = min(kz0 + lz, P.n[2]);
  const int ni = min(kTX, P.n[0] - i0), nj = min(kTY, P.n[1] - j0);
  const int ti = (int)threadIdx.x % kTX, tj = (int)threadIdx.x / kTX;  // warp tj holds row tj
  const bool own = ti < ni && tj < nj;
  const R ix = Gam<R>::inv(P, 0), iy = Gam<R>::inv(P, 1), iz = Gam<R>::inv(P, 2);
  const long long FS = P.FS, QX = P.QX, PX = P.PX;
  const long long QS = P.QS, QP = (long long)P.QX * P.QY;
  const R* __restrict__ Fx = (const R*)P.F[0];
  const R* __restrict__ Fy = (const R*)P.F[1];
  const R* __restrict__ Fz = (const R*)P.F[2];
  // (S) for plane kk: the x and y faces and cell E_z at kk, the rolling arrays at kk + 1
  // into buffer nb (and at kk into the other buffer when first), the z faces at kk + 1/2.
  // The points of the (ni + 2) x (nj + 2) box lie in the scratch arrays' padding of 2.
  auto stage = [&](int kk, int nb, bool first) {
    const int w = ni + 2, npts = w * (nj + 2);
    for (int t = (int)threadIdx.x; t < npts; t += kEB) {
      const int jj = t / w - 1, ii = t - (jj + 1) * w - 1;
      const int o = (jj + 1) * kSW + ii + 1;
      const long long q0 = qidx(P, i0 + ii, j0 + jj, kk), q1 = q0 + QP;
      cp_async(&G.x5[o], Fx + 5 * QS + q0);
      cp_async(&G.y6[o], Fy + 6 * QS + q0);
      cp_async(&G.ecz[o], Win + WEZ * QS + q0);
      cp_async(&G.x0[nb][o], Fx + q1);
      cp_async(&G.x6[nb][o], Fx + 6 * QS + q1);
      cp_async(&G.y0[nb][o], Fy + q1);
      cp_async(&G.y5[nb][o], Fy + 5 * QS + q1);
      cp_async(&G.ecx[nb][o], Win + WEX * QS + q1);
      cp_async(&G.ecy[nb][o], Win + WEY * QS + q1);
      cp_async(&G.z0[o], Fz + q1);
      cp_async(&G.z5[o], Fz + 5 * QS + q1);
      cp_async(&G.z6[o], Fz + 6 * QS + q1);
      if (first) {
        const int ob = nb ^ 1;
        cp_async(&G.x0[ob][o], Fx + q0);
        cp_async(&G.x6[ob][o], Fx + 6 * QS + q0);
        cp_async(&G.y0[ob][o], Fy + q0);
        cp_async(&G.y5[ob][o], Fy + 5 * QS + q0);
        cp_async(&G.ecx[ob][o], Win + WEX * QS + q0);
        cp_async(&G.ecy[ob][o], Win + WEY * QS + q0);
      }
    }
  };
  if constexpr (STAGED) {
    stage(kz0, 1, true);
    cp_async_wait();
    __syncthreads();
  }
  const R h = sh;
  const bool last = a.stage == 1;
  R lim = R(INFINITY);
  int nfl = 0;
  // edge EMFs at tile offset (ii, jj) from the staged inputs (corner_core's arguments as
  // corner_value takes them from global memory): E_z at plane k, E_x and E_y at k + 1/2
  auto ez_at = [&](int ii, int jj, int cur) {
    const int o = (jj + 1) * kSW + ii + 1;
    return corner_core<R>(-G.x5[o], -G.x5[o - kSW], G.y6[o], G.y6[o - 1], G.ecz[o], G.ecz[o - 1], G.ecz[o - kSW],
                          G.ecz[o - kSW - 1], G.x0[cur][o], G.x0[cur][o - kSW], G.y0[cur][o], G.y0[cur][o - 1]);
  };
  auto ex_at = [&](int ii, int jj, int cur) {
    const int o = (jj + 1) * kSW + ii + 1, nx = cur ^ 1;
    return corner_core<R>(-G.y5[nx][o], -G.y5[cur][o], G.z6[o], G.z6[o - kSW], G.ecx[nx][o], G.ecx[nx][o - kSW],
                          G.ecx[cur][o], G.ecx[cur][o - kSW], G.y0[nx][o], G.y0[cur][o], G.z0[o], G.z0[o - kSW]);
  };
  auto ey_at = [&](int ii, int jj, int cur) {
    const int o = (jj + 1) * kSW + ii + 1, nx = cur ^ 1;
    return corner_core<R>(-G.z5[o], -G.z5[o - 1], G.x6[nx][o], G.x6[cur][o], G.ecy[nx][o], G.ecy[cur][o],
                          G.ecy[nx][o - 1], G.ecy[cur][o - 1], G.z0[o], G.z0[o - 1], G.x0[nx][o], G.x0[cur][o]);
  };
  // unstaged: edge EMF c at tile offset (ii, jj) of plane kk into its shared array
  auto put_e = [&](int c, int ii, int jj, int kk, int buf) {
    const R e = emf_at<R>(P, Win, c, i0 + ii, j0 + jj, kk);
    if (c == 2) sEz[jj * SX + ii] = e;
    else if (c == 0) sEx[buf][jj * kTX + ii] = e;
    else sEy[buf][jj * SX + ii] = e;
  };
  for (int k = kz0; k < kz1; ++k) {
    const int cur = (k - kz0) & 1, nxt = cur ^ 1;
    const bool first = k == kz0;
    // (A) edge EMFs.  Each thread: E_z(k), E_x(k+1), E_y(k+1) at its own (ti, tj) (and
    // E_x(k), E_y(k) at the first plane); warps 0-2 (3-4 at the first plane) add the
    // upper halo row (jj = nj) and column (ii = ni).
    if constexpr (STAGED) {
      if (own) {
        sEz[tj * SX + ti] = ez_at(ti, tj, cur);
        sEx[nxt][tj * kTX + ti] = ex_at(ti, tj, cur);
        sEy[nxt][tj * SX + ti] = ey_at(ti, tj, cur);
        if (first) {
          sEx[cur][tj * kTX + ti] = emf_at<R>(P, Win, 0, i0 + ti, j0 + tj, k);
          sEy[cur][tj * SX + ti] = emf_at<R>(P, Win, 1, i0 + ti, j0 + tj, k);
        }
      }
      const int w = tj, l = ti;
      if (w == 0 && l < ni) sEz[nj * SX + l] = ez_at(l, nj, cur);
      if (w == 1 && l < ni) sEx[nxt][nj * kTX + l] = ex_at(l, nj, cur);
      if (w == 2) {
        if (l <= nj) sEz[l * SX + ni] = ez_at(ni, l, cur);
        else if (l >= 16 && l - 16 < nj) sEy[nxt][(l - 16) * SX + ni] = ey_at(ni, l - 16, cur);
      }
      if (first) {
        if (w == 3 && l < ni) sEx[cur][nj * kTX + l] = emf_at<R>(P, Win, 0, i0 + l, j0 + nj, k);
        if (w == 4 && l < nj) sEy[cur][l * SX + ni] = emf_at<R>(P, Win, 1, i0 + ni, j0 + l, k);
      }
    } else {
      // the same edges from global memory (corner_value)
      if (own) {
        put_e(2, ti, tj, k, 0);
        put_e(0, ti, tj, k + 1, nxt);
        put_e(1, ti, tj, k + 1, nxt);
        if (first) {
          put_e(0, ti, tj, k, cur);
          put_e(1, ti, tj, k, cur);
        }
      }
      const int w = tj, l = ti;
      if (w == 0 && l < ni) put_e(2, l, nj, k, 0);
      if (w == 1 && l < ni) put_e(0, l, nj, k + 1, nxt);
      if (w == 2) {
        if (l <= nj) put_e(2, ni, l, k, 0);
        else if (l >= 16 && l - 16 < nj) put_e(1, ni, l - 16, k + 1, nxt);
      }
      if (first) {
        if (w == 3 && l < ni) put_e(0, l, nj, k, cur);
        if (w == 4 && l < nj) put_e(1, ni, l, k, cur);
      }
    }
    __syncthreads();
    // (S) the next plane's edge inputs, in flight during (B) and (C): its rolling arrays go
    // to buffer cur, whose plane k (A) has just read
    if constexpr (STAGED)
      if (k + 1 < kz1) stage(k + 1, cur, false);
    // (B) new faces.  Each thread: the x and y faces of its cell at plane k and the z face
    // above it (and the z face below it at the first plane); warps 0-1 add the halo x-face
    // column (ii = ni) and y-face row (jj = nj).
    const long long sk = sidx(P, i0, j0, k);
    if (own) {
      const long long so = sk + ti + (long long)tj * PX;
      sBx[tj * SX + ti] = face_from<R>(Ub[BXF * FS + so], sEz[tj * SX + ti], sEz[(tj + 1) * SX + ti],
                                       sEy[cur][tj * SX + ti], sEy[nxt][tj * SX + ti], iy, iz, h);
      sBy[tj * kTX + ti] = face_from<R>(Ub[BYF * FS + so], sEx[cur][tj * kTX + ti], sEx[nxt][tj * kTX + ti],
                                        sEz[tj * SX + ti], sEz[tj * SX + ti + 1], iz, ix, h);
      const int ku = k + 1;
      const long long su = sidx(P, i0 + ti, j0 + tj, fmap(P, 2, ku));
      const double bz = face_from<R>(Ub[BZF * FS + su], sEy[nxt][tj * SX + ti], sEy[nxt][tj * SX + ti + 1],
                                     sEx[nxt][tj * kTX + ti], sEx[nxt][(tj + 1) * kTX + ti], ix, iy, h);
      sBz[nxt][tj * kTX + ti] = bz;
      if (ku == P.n[2] && P.nface[2] > P.n[2]) Uo[BZF * FS + sidx(P, i0 + ti, j0 + tj, ku)] = bz;
      if (first)
        sBz[cur][tj * kTX + ti] = face_from<R>(Ub[BZF * FS + so], sEy[cur][tj * SX + ti], sEy[cur][tj * SX + ti + 1],
                                               sEx[cur][tj * kTX + ti], sEx[cur][(tj + 1) * kTX + ti], ix, iy, h);
    }
    if (tj == 0 && ti < nj) {  // x face at the halo column
      const int jj = ti, i = i0 + ni, j = j0 + jj;
      const double b = face_from<R>(Ub[BXF * FS + sidx(P, fmap(P, 0, i), j, k)], sEz[jj * SX + ni],
                                    sEz[(jj + 1) * SX + ni], sEy[cur][jj * SX + ni], sEy[nxt][jj * SX + ni], iy, iz, h);
      sBx[jj * SX + ni] = b;
      if (i == P.n[0] && P.nface[0] > P.n[0]) Uo[BXF * FS + sidx(P, i, j, k)] = b;
    }
    if (tj == 1 && ti < ni) {  // y face at the halo row
      const int ii = ti, i = i0 + ii, j = j0 + nj;
      const double b = face_from<R>(Ub[BYF * FS + sidx(P, i, fmap(P, 1, j), k)], sEx[cur][nj * kTX + ii],
                                    sEx[nxt][nj * kTX + ii], sEz[nj * SX + ii], sEz[nj * SX + ii + 1], iz, ix, h);
      sBy[nj * kTX + ii] = b;
      if (j == P.n[1] && P.nface[1] > P.n[1]) Uo[BYF * FS + sidx(P, i, j, k)] = b;
    }
    __syncthreads();
    // (C) the cell
    if (own) {
      const long long s = sk + ti + (long long)tj * PX;
      const long long q = qidx(P, i0, j0, k) + ti + (long long)tj * QX;
      double u[5];
      cell_update<R>(P, Ub, Us, h, a.src, i0 + ti, j0 + tj, k, s, q, u);
      const double blo[3] = {sBx[tj * SX + ti], sBy[tj * kTX + ti], sBz[cur][tj * kTX + ti]};
      const double bhi[3] = {sBx[tj * SX + ti + 1], sBy[(tj + 1) * kTX + ti], sBz[nxt][tj * kTX + ti]};
      // the end-of-step floors (corrector) share the recovery's arithmetic and may change
      // rho and E before they are stored
      R l;
      if constexpr (!FLOORS) {
        // never taken in this instantiation (P.floors is off); with the call compiled in, the
        // kernel measured 1% faster at 256^3 (1.263 against 1.274 ms per launch) than
        // without it, through the compiler's scheduling of the rest
        if (last && P.floors)
          nfl += floor_core(P, u[0], u[1], u[2], u[3], u[4], blo[0], bhi[0], blo[1], bhi[1], blo[2], bhi[2]);
      }
      if constexpr (FLOORS) {
        l = last ? floor_prim_core<R>(P, u[0], u[1], u[2], u[3], u[4], blo[0] + bhi[0], blo[1] + bhi[1],
                                      blo[2] + bhi[2], Wout, q, &nfl)
                 : prim_core<R>(P, u[0], u[1], u[2], u[3], u[4], blo[0] + bhi[0], blo[1] + bhi[1],
                                blo[2] + bhi[2], Wout, q, true, true, false);
      }
      if (cells_out) {
        Uo[s] = u[0];
#pragma unroll
        for (int c = 0; c < 3; ++c) Uo[(MX + c) * FS + s] = u[1 + c];
        Uo[EN * FS + s] = u[4];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) Uo[(BXF + c) * FS + s] = blo[c];
      if constexpr (!FLOORS)
        l = prim_core<R>(P, u[0], u[1], u[2], u[3], u[4], blo[0] + bhi[0], blo[1] + bhi[1], blo[2] + bhi[2],
                         Wout, q, true, true, last);
      lim = l < lim ? l : lim;
      if (images) periodic_images<R>(P, Wout, i0 + ti, j0 + tj, k, q);
    }
    if constexpr (STAGED) {
      // the next plane's edge inputs have landed (each thread waits for its own copies; the
      // barrier makes all of them visible)
      cp_async_wait();
      __syncthreads();
    }
    // (unstaged: C(k) and A(k + 1) touch different shared arrays and share one barrier
    // interval)
  }
  if (a.stage == 1) {
    if (P.floors) {
      const unsigned tot = __reduce_add_sync(0xffffffffu, (unsigned)nfl);
      if ((threadIdx.x & 31) == 0 && tot) atomicAdd(P.floored, (unsigned long long)tot);
    }
    block_min_atomic(lim, P.cfl_min);
  }
}

// Corner EMFs and the stage update in one kernel for a 2D plane (x and y active, z trivial):
// the single-plane form of k_emf_update.  A CTA owns a kTX x kTY tile of cells:
//  (A) E_z at the tile's edges and its upper halo row and column (corner_value), into shared
//      memory;
//  (B) the new x and y faces of the tile and its upper halo (-curl E with E_z from shared
//      memory), and each cell's z face, whose edge EMFs along x and y are the fluxes of B_z
//      through the y and x faces (-F_y(B_z) and F_x(B_z), as corner_point takes them on a
//      trivial axis); faces of the extra layer of an outflow axis are stored here;
//  (C) each cell: flux divergence and source, its owned faces stored, the floors when asked,
//      the recovery of the new state and its CFL limit, and its periodic images.
// Every face takes face_from's operations in the order face_new gives them on a plane, so
// the state is bit for bit that of the corner-EMF kernel followed by k_update_fused.  The
// cell EMFs come from Win while neighbouring tiles write the new W to Wout.
template <class R>
__global__ void __launch_bounds__(kEB, kEMinBlocks) k_emf_update2(PatchDev P, const R* __restrict__ Win,
                                                        R* __restrict__ Wout, const double* __restrict__ Ub,
                                                        const double* __restrict__ Us, double* __restrict__ Uo,
                                                        StageArgs a, int images, int cells_out) {
  constexpr int SX = kTX + 1;  // row pitch of the arrays with an x halo
  __shared__ R sEz[(kTY + 1) * SX];
  __shared__ double sBx[kTY * SX];
  __shared__ double sBy[(kTY + 1) * kTX];
  __shared__ R sh;
  if (threadIdx.x == 0) {
    double dt;
    if (a.stage == 0) {
      dt = a.dt_host > 0.0 ? a.dt_host : a.cfl * __longlong_as_double((long long)*P.cfl_min);
      if (blockIdx.x == 0) *P.dt_used = dt;
    } else {
      dt = *P.dt_used;
    }
    sh = Ar<R>::from_d(a.stage == 0 ? 0.5 * dt : dt);
  }
  __syncthreads();
  const R h = sh;
  const int ntx = (P.n[0] + kTX - 1) / kTX;
  const int i0 = (int)(blockIdx.x % ntx) * kTX, j0 = (int)(blockIdx.x / ntx) * kTY;
  const int ni = min(kTX, P.n[0] - i0), nj = min(kTY, P.n[1] - j0);
  const int ti = (int)threadIdx.x % kTX, tj = (int)threadIdx.x / kTX;
  const bool own = ti < ni && tj < nj;
  const R ix = Gam<R>::inv(P, 0), iy = Gam<R>::inv(P, 1), iz = Gam<R>::inv(P, 2);
  const long long FS = P.FS, QS = P.QS, QX = P.QX;
  const R zero = R(0);
  // (A) E_z
  auto put_ez = [&](int ii, int jj) { sEz[jj * SX + ii] = emf_at<R>(P, Win, 2, i0 + ii, j0 + jj, 0); };
  if (own) put_ez(ti, tj);
  if (tj == 0 && ti < ni) put_ez(ti, nj);
  if (tj == 2 && ti <= nj) put_ez(ni, ti);
  __syncthreads();
  // (B) x and y faces (face_new on a plane: the x face has only the dE_z/dy term, the y face
  // only -dE_z/dx)
  if (own) {
    const long long so = sidx(P, i0 + ti, j0 + tj, 0);
    sBx[tj * SX + ti] = face_from<R>(Ub[BXF * FS + so], sEz[tj * SX + ti], sEz[(tj + 1) * SX + ti], zero, zero, iy,
                                     iz, h);
    sBy[tj * kTX + ti] = face_from<R>(Ub[BYF * FS + so], zero, zero, sEz[tj * SX + ti], sEz[tj * SX + ti + 1], iz,
                                      ix, h);
  }
  if (tj == 0 && ti < nj) {  // x face at the halo column
    const int jj = ti, i = i0 + ni, j = j0 + jj;
    const double b = face_from<R>(Ub[BXF * FS + sidx(P, fmap(P, 0, i), j, 0)], sEz[jj * SX + ni],
                                  sEz[(jj + 1) * SX + ni], zero, zero, iy, iz, h);
    sBx[jj * SX + ni] = b;
    if (i == P.n[0] && P.nface[0] > P.n[0]) Uo[BXF * FS + sidx(P, i, j, 0)] = b;
  }
  if (tj == 1 && ti < ni) {  // y face at the halo row
    const int ii = ti, i = i0 + ii, j = j0 + nj;
    const double b = face_from<R>(Ub[BYF * FS + sidx(P, i, fmap(P, 1, j), 0)], zero, zero, sEz[nj * SX + ii],
                                  sEz[nj * SX + ii + 1], iz, ix, h);
    sBy[nj * kTX + ii] = b;
    if (j == P.n[1] && P.nface[1] > P.n[1]) Uo[BYF * FS + sidx(P, i, j, 0)] = b;
  }
  __syncthreads();
  // (C) the cell
  R lim = R(INFINITY);
  int nfl = 0;
  if (own) {
    const int i = i0 + ti, j = j0 + tj;
    const long long s = sidx(P, i, j, 0);
    const long long q = qidx(P, i, j, 0);
    // its z face: E_y = F_x(B_z) at the x faces, E_x = -F_y(B_z) at the y faces
    const R* Fx = (const R*)P.F[0];
    const R* Fy = (const R*)P.F[1];
    const double bz = face_from<R>(Ub[BZF * FS + s], Fx[6 * QS + q], Fx[6 * QS + q + 1], -Fy[5 * QS + q],
                                   -Fy[5 * QS + q + QX], ix, iy, h);
    double u[5];
    cell_update<R>(P, Ub, Us, h, a.src, i, j, 0, s, q, u);
    const double blo[3] = {sBx[tj * SX + ti], sBy[tj * kTX + ti], bz};
    const double bhi[3] = {sBx[tj * SX + ti + 1], sBy[(tj + 1) * kTX + ti], bz};
    if (a.stage == 1 && P.floors)
      nfl += floor_core(P, u[0], u[1], u[2], u[3], u[4], blo[0], bhi[0], blo[1], bhi[1], blo[2], bhi[2]);
    if (cells_out) {
      Uo[s] = u[0];
#pragma unroll
      for (int c = 0; c < 3; ++c) Uo[(MX + c) * FS + s] = u[1 + c];
      Uo[EN * FS + s] = u[4];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) Uo[(BXF + c) * FS + s] = blo[c];
    lim = prim_core<R>(P, u[0], u[1], u[2], u[3], u[4], blo[0] + bhi[0], blo[1] + bhi[1], blo[2] + bhi[2], Wout, q,
                       true, true, a.stage == 1);
    if (images) periodic_images_act<R>(P, Wout, i, j, 0, q);
  }
  if (a.stage == 1) {
    if (P.floors) {
      const unsigned tot = __reduce_add_sync(0xffffffffu, (unsigned)nfl);
      if ((threadIdx.x & 31) == 0 && tot) atomicAdd(P.floored, (unsigned long long)tot);
    }
    block_min_atomic(lim, P.cfl_min);
  }
}

// X of the passive scalars over the padded box, from the stage's input state
template <class R>
__global__ void __launch_bounds__(kBlock) k_scalar_prim(PatchDev P, const double* __restrict__ U,
                                                        const double* __restrict__ S, Range rg) {
  int i, j, k;
  if (!range_point(rg, i, j, k)) return;
  scalar_prim_point<R>(P, U, S, (R*)P.X, i, j, k);
}

// the stage's scalar update over the interior cells; dt as the stage's update kernel takes it
template <class R, int ORDER>
__global__ void __launch_bounds__(kBlock) k_scalar_update(PatchDev P, const double* __restrict__ Sb,
                                                          double* __restrict__ So, Range rg, StageArgs a) {
  __shared__ R sh;
  if (threadIdx.x == 0) {
    const double dt = a.stage == 0 ? (a.dt_host > 0.0 ? a.dt_host : a.cfl * __longlong_as_double((long long)*P.cfl_min))
                                   : *P.dt_used;
    sh = Ar<R>::from_d(a.stage == 0 ? 0.5 * dt : dt);
  }
  __syncthreads();
  int i, j, k;
  if (!range_point(rg, i, j, k)) return;
  scalar_update_point<R, ORDER>(P, Sb, So, (const R*)P.X, sh, i, j, k);
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
__global__ void k_riemann(int solver, int n, const double* __restrict__ wl, const double* __restrict__ wr,
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
  riemann<R>(solver, a, b, (R)bn[q], (R)gam, f);
#pragma unroll
  for (int m = 0; m < 7; ++m) flux[8 * q + src[m]] = (double)f[m];
  flux[8 * q + 5] = 0.0;
}

// ------------------------------------------------------------- host side ----

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else
      n = 1;
  }
  return n;
}

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

// one direction's flux kernel for the patch's Riemann solver
template <class R, int D, int ORDER>
static void launch_flux(const PatchDev& P, const double* Ub, const Range& fr, cudaStream_t s) {
  if constexpr (D > 0) {
    // y and z faces: the marching kernel, one thread per (x, other transverse) position and
    // segment of seg faces.  seg = 16, 8, 4 or 2, the longest that still gives two waves of
    // 3 kBlock (768) resident threads per SM; a box too thin even for seg = 2 (a 2D plane, a
    // small patch) takes the per-face kernel, which has one thread per face
    constexpr int T = D == 1 ? 2 : 1;
    const long long plane = (long long)fr.ext[0] * fr.ext[T];
    const long long want = 2LL * 3 * kBlock * sm_count();
    int seg = kMarch;
    while (P.flux_scheme == FLUX_AUTO && seg > 2 && plane * ((fr.ext[D] + seg - 1) / seg) < want) seg >>= 1;
    if (P.flux_scheme == FLUX_MARCH ||
        (P.flux_scheme == FLUX_AUTO && plane * ((fr.ext[D] + seg - 1) / seg) >= want)) {
      constexpr int B = march_block<R, ORDER>();
      const dim3 g((unsigned)((plane + B - 1) / B), (unsigned)((fr.ext[D] + seg - 1) / seg), 1);
      if (P.riemann == RIEMANN_HLLC) k_flux_march<R, D, ORDER, RIEMANN_HLLC><<<g, B, 0, s>>>(P, Ub, fr, seg);
      else if (P.riemann == RIEMANN_HLL) k_flux_march<R, D, ORDER, RIEMANN_HLL><<<g, B, 0, s>>>(P, Ub, fr, seg);
      else k_flux_march<R, D, ORDER, RIEMANN_HLLD><<<g, B, 0, s>>>(P, Ub, fr, seg);
      return;
    }
  }
  if constexpr (D == 0 && ORDER == 2) {
    // kappa-scheme x faces: the shuffle kernel (each cell reconstructed once), unless the
    // per-face kernel is asked for
    if (P.flux_scheme != FLUX_PER_FACE) {
      const long long len = (long long)fr.ext[1] * P.QX;
      const unsigned nwin = (unsigned)((len + 30) / 31);  // window w: the faces below cells 31w .. 31w + 30
      const dim3 g((nwin + kBlock / 32 - 1) / (kBlock / 32), (unsigned)fr.ext[2], 1);
      if (P.riemann == RIEMANN_HLLC) k_flux_xs<R, RIEMANN_HLLC><<<g, kBlock, 0, s>>>(P, Ub, fr, nwin);
      else if (P.riemann == RIEMANN_HLL) k_flux_xs<R, RIEMANN_HLL><<<g, kBlock, 0, s>>>(P, Ub, fr, nwin);
      else k_flux_xs<R, RIEMANN_HLLD><<<g, kBlock, 0, s>>>(P, Ub, fr, nwin);
      return;
    }
  }
  const dim3 g = grid_of(fr);
  if (P.riemann == RIEMANN_HLLC) k_flux<R, D, ORDER, RIEMANN_HLLC><<<g, kBlock, 0, s>>>(P, Ub, fr);
  else if (P.riemann == RIEMANN_HLL) k_flux<R, D, ORDER, RIEMANN_HLL><<<g, kBlock, 0, s>>>(P, Ub, fr);
  else k_flux<R, D, ORDER, RIEMANN_HLLD><<<g, kBlock, 0, s>>>(P, Ub, fr);
}

// per-direction flux kernels of one stage, and the corner-EMF kernel when asked.  With a
// fork set (and no per-class profiling, whose events time one stream) the directions after
// the first active one run on the side streams, in parallel with it: each kernel fills the
// GPU, and the overlap fills the others' last partial waves (256^3: 4.299 -> 4.267 ms per
// step on the same box).
template <class R>
static int issue_fluxes(const PatchDev& P, const StageArgs& a, const double* Usrc, cudaStream_t s0, ProfRec* prof,
                        bool emf, const ForkSet* fk) {
  if (a.stage == 0 && P.act[0] && P.act[1] && P.act[2] && P.flux_scheme == FLUX_AUTO) {
    // the predictor's three directions in one marching kernel: segments of 8 planes (at 256^3
    // 0.651 ms per launch against 0.661 with 16, 0.664 with 24, 0.694 with 32), 4 or 2 while
    // the box gives fewer than two waves of four resident CTAs per SM; thinner boxes keep the
    // per-direction kernels, unless the patch's chain runs beside other patches' (the 64-patch
    // batch: 11.01 -> 10.92 ms per step with every 3D patch fused)
    const long long cols = (long long)(P.n[0] + 2) * (P.n[1] + 2), planes = P.n[2] + 2;
    const long long want = 2LL * 4 * kBlock * sm_count();
    int seg = 8;
    while (seg > 2 && cols * ((planes + seg - 1) / seg) < want) seg >>= 1;
    if (a.concurrent || cols * ((planes + seg - 1) / seg) >= want) {
      {
        ProfScope ps(prof, KC_FLUX1_XYZ, s0);
        const dim3 g((unsigned)((cols + kBlock - 1) / kBlock), (unsigned)((planes + seg - 1) / seg), 1);
        if (P.riemann == RIEMANN_HLLC) k_flux_d3<R, RIEMANN_HLLC><<<g, kBlock, 0, s0>>>(P, Usrc, seg);
        else if (P.riemann == RIEMANN_HLL) k_flux_d3<R, RIEMANN_HLL><<<g, kBlock, 0, s0>>>(P, Usrc, seg);
        else k_flux_d3<R, RIEMANN_HLLD><<<g, kBlock, 0, s0>>>(P, Usrc, seg);
      }
      if (!emf) return 1;
      const Range er = edge_range(P);
      ProfScope ps(prof, KC_EMF, s0);
      k_emf<R><<<grid_of(er), kBlock, 0, s0>>>(P, er);
      return 2;
    }
  }
  if (a.stage == 0 && P.act[0] && P.act[1] && !P.act[2] && P.flux_scheme == FLUX_AUTO) {
    // a 2D plane: the predictor's x and y faces in one kernel, a thread per cell; then the
    // corner EMFs as below
    {
      ProfScope ps(prof, KC_FLUX1_XYZ, s0);
      const long long cols = (long long)(P.n[0] + 2) * (P.n[1] + 2);
      const dim3 g((unsigned)((cols + kBlock - 1) / kBlock), 1, 1);
      if (P.riemann == RIEMANN_HLLC) k_flux_d2<R, RIEMANN_HLLC><<<g, kBlock, 0, s0>>>(P, Usrc);
      else if (P.riemann == RIEMANN_HLL) k_flux_d2<R, RIEMANN_HLL><<<g, kBlock, 0, s0>>>(P, Usrc);
      else k_flux_d2<R, RIEMANN_HLLD><<<g, kBlock, 0, s0>>>(P, Usrc);
    }
    if (!emf) return 1;
    const Range er = edge_range(P);
    ProfScope ps(prof, KC_EMF, s0);
    k_emf<R><<<grid_of(er), kBlock, 0, s0>>>(P, er);
    return 2;
  }
  int nl = 0;
  const bool par = fk && !prof && P.act[0] + P.act[1] + P.act[2] >= 2;
  if (par) {
    if (cudaEventRecord(fk->fork, s0) != cudaSuccess) return -1;
    for (int q = 0; q < 2; ++q)
      if (cudaStreamWaitEvent(fk->side[q], fk->fork, 0) != cudaSuccess) return -1;
  }
  int side = 0;
  bool first = true;
  for (int d = 0; d < 3; ++d) {
    if (!P.act[d]) continue;
    const cudaStream_t s = (par && !first) ? fk->side[side++] : s0;
    first = false;
    const Range fr = flux_range(P, d);
    ProfScope ps(prof, (a.stage == 0 ? KC_FLUX1 : KC_FLUX2) + d, s);
    if (a.stage == 0) {
      if (d == 0) launch_flux<R, 0, 1>(P, Usrc, fr, s);
      if (d == 1) launch_flux<R, 1, 1>(P, Usrc, fr, s);
      if (d == 2) launch_flux<R, 2, 1>(P, Usrc, fr, s);
    } else {
      if (d == 0) launch_flux<R, 0, 2>(P, Usrc, fr, s);
      if (d == 1) launch_flux<R, 1, 2>(P, Usrc, fr, s);
      if (d == 2) launch_flux<R, 2, 2>(P, Usrc, fr, s);
    }
    ++nl;
  }
  if (par) {
    for (int q = 0; q < side; ++q)
      if (cudaEventRecord(fk->join[q], fk->side[q]) != cudaSuccess ||
          cudaStreamWaitEvent(s0, fk->join[q], 0) != cudaSuccess)
        return -1;
  }
  if (!emf) return nl;
  const Range er = edge_range(P);
  ProfScope ps(prof, KC_EMF, s0);
  k_emf<R><<<grid_of(er), kBlock, 0, s0>>>(P, er);
  return nl + 1;
}

// One stage of the step for one patch: per-direction fluxes and the corner EMFs from the
// stored W, then the fused update + recovery and the ghost shell of W.  The predictor writes U^{n+1/2} into Uh; the corrector, whose base is U^n and whose
// source term is evaluated at U^{n+1/2}, writes U^{n+1} into Uh as well (each cell's
// U^{n+1/2} is read by the thread that overwrites it, and no kernel of the stage reads the
// faces of Uh after the fluxes), so the caller swaps Un and Uh after the corrector.
//
// Patches with three active axes use the fused EMF + update kernel, which reads the
// stage's W and writes the new W to the other buffer: the predictor reads W and writes
// W2, the corrector reads W2 and writes W, so W holds the new state's primitives after
// every step.  Other patches use the corner-EMF kernel and the fused update, in place.
template <class R>
static int issue_stage(const PatchDev& P, const StageArgs& a, cudaStream_t s, long long* launches,
                       ProfRec* prof, const ForkSet* fk) {
  const double* Usrc = a.stage == 0 ? P.Un : P.Uh;  // state the fluxes and S are built from
  const bool fused = P.act[0] && P.act[1] && P.act[2] && P.W2;
  // a 2D plane in x and y: the single-plane fused kernel
  const bool fused2 = P.act[0] && P.act[1] && !P.act[2] && P.W2;
  // all axes periodic (a trivial axis counts as periodic): the update kernel writes W's ghost
  // images itself
  const int images = P.per[0] && P.per[1] && P.per[2];
  PatchDev Q = P;  // Q.W: the W the stage reads
  PatchDev G = P;  // G.W: the W the stage writes
  if (fused || fused2) {
    Q.W = a.stage == 0 ? P.W : P.W2;
    G.W = a.stage == 0 ? P.W2 : P.W;
  }
  int nl = issue_fluxes<R>(Q, a, Usrc, s, prof, !(fused || fused2), fk);
  if (nl < 0) return -1;
  if (P.ns > 0) {
    // passive scalars, before the update overwrites the corrector's input state in Uh
    ProfScope ps(prof, KC_SCALARS, s);
    const Range pr = prim_range(P), ir = interior_range(P);
    k_scalar_prim<R><<<grid_of(pr), kBlock, 0, s>>>(P, Usrc, a.stage == 0 ? P.Sn : P.Sh, pr);
    if (a.stage == 0) k_scalar_update<R, 1><<<grid_of(ir), kBlock, 0, s>>>(P, P.Sn, P.Sh, ir, a);
    else k_scalar_update<R, 2><<<grid_of(ir), kBlock, 0, s>>>(P, P.Sn, P.Sh, ir, a);
    nl += 2;
  }
  if (fused) {
    ProfScope ps(prof, KC_EMF_UPDATE, s);
    // planes per CTA: 10, halved (down to 2) while the grid would be under two waves of
    // resident CTAs (10 against 8, 9, 12, 16 at 256^3: 1.238 ms per launch against 1.253,
    // 1.242, 1.267, 1.29; also faster on the disc and the batch: each CTA's first plane
    // recomputes its lower edges, and the grid's last partial wave idles)
    const int ntx = (P.n[0] + kTX - 1) / kTX, nty = (P.n[1] + kTY - 1) / kTY;
    int lz = 10;
    while (lz > 2 && (long long)ntx * nty * ((P.n[2] + lz - 1) / lz) < 2LL * kEMinBlocks * sm_count()) lz >>= 1;
    const dim3 grid((unsigned)(ntx * nty), (unsigned)((P.n[2] + lz - 1) / lz), 1);
    // the predictor's cell fields of U^n+1/2 are read by nobody when the corrector's source
    // term, the ghost fill and the passive scalars do not need them: only its faces are stored
    const int cells_out = !(a.stage == 0 && images && a.src.potential == POT_NONE && P.ns == 0);
    if (P.floors)
      k_emf_update<R, true><<<grid, kEB, 0, s>>>(Q, (const R*)Q.W, (R*)G.W, P.Un, Usrc, P.Uh, a, lz, images, cells_out);
    else
      k_emf_update<R, false><<<grid, kEB, 0, s>>>(Q, (const R*)Q.W, (R*)G.W, P.Un, Usrc, P.Uh, a, lz, images,
                                                  cells_out);
    ++nl;
  } else if (fused2) {
    ProfScope ps(prof, KC_EMF_UPDATE, s);
    const int ntx = (P.n[0] + kTX - 1) / kTX, nty = (P.n[1] + kTY - 1) / kTY;
    const int cells_out = !(a.stage == 0 && images && a.src.potential == POT_NONE && P.ns == 0);
    k_emf_update2<R><<<(unsigned)(ntx * nty), kEB, 0, s>>>(Q, (const R*)Q.W, (R*)G.W, P.Un, Usrc, P.Uh, a, images,
                                                          cells_out);
    ++nl;
  } else {
    const Range er = edge_range(P);
    ProfScope ps(prof, KC_UPDATE, s);
    k_update_fused<R><<<grid_of(er), kBlock, 0, s>>>(P, P.Un, Usrc, P.Uh, er, a, images);
    ++nl;
  }
  if (!images) {
    ProfScope ps(prof, KC_GHOST, s);
    const long long ng = ghost_count(P);
    if (ng > 0) {
      long long blocks = (ng + kBlock - 1) / kBlock;
      if (blocks > 65535) blocks = 65535;
      k_ghost<R><<<(unsigned)blocks, kBlock, 0, s>>>(G, P.Uh);
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
static int issue_ghost_w(const PatchDev& P, cudaStream_t s, long long* launches) {
  const long long ng = ghost_count(P);
  if (ng <= 0) return 0;
  long long blocks = (ng + kBlock - 1) / kBlock;
  if (blocks > 65535) blocks = 65535;
  k_ghost<R><<<(unsigned)blocks, kBlock, 0, s>>>(P, P.Un);
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
static int issue_riemann(int solver, int n, const double* wl, const double* wr, const double* bn, double gam,
                         double* flux, cudaStream_t s) {
  if (n <= 0) return 0;
  k_riemann<R><<<(unsigned)(((long long)n + 127) / 128), 128, 0, s>>>(solver, n, wl, wr, bn, gam, flux);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class R> Backend make_backend() {
  Backend b;
  b.scratch_elem = sizeof(R);
  b.stage = &issue_stage<R>;
  b.prim = &issue_prim<R>;
  b.cfl = &issue_cfl<R>;
  b.ghost_w = &issue_ghost_w<R>;
  b.riemann = &issue_riemann<R>;
  b.persistent = &issue_persistent<R>;
  b.occupancy = &persistent_occupancy<R>;
  return b;
}

}  // namespace mhd
