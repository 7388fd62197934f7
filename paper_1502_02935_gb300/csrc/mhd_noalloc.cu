// mhd_noalloc.cu -- CFL time step of a caller-held state, computed without any device
// allocation.
//
// This is a variant of the library's CFL reduction for callers that cannot allocate
// device memory.  Examples are applications that reserve the whole device through
// their own memory pool and do not let third-party code call cudaMalloc, and tight
// loops that cannot afford the device-wide synchronisation cudaMalloc/cudaFree imply.
// The regular reduction writes into memory that mhd_init_grid allocated.  Here the
// scratch (one partial minimum per thread block) is a fixed file-scope __device__
// array.  Every GPU that loads the library holds that array (32 KiB) until the
// process exits.
//
// The state is read in the library's host format (see mhd.h), from device pointers
// the caller owns.  The result goes to a device pointer the caller owns.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "mhd.h"
#include "mhd_device.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int kCellsPerThread = 8;
constexpr long long kCellsPerBlock = (long long)kBlock * kCellsPerThread;  // 2048
constexpr int kMaxBlocks = 4096;
static_assert(kMaxBlocks * kCellsPerBlock == MHD_NOALLOC_MAX_CELLS, "limit mismatch");

// One partial minimum per block of the first pass.  Shared by every call in the
// process: calls whose kernels overlap on the GPU race on it.  Each call writes every
// slot it later reads, so no slot has to be cleared between calls.
static __device__ __align__(256) double g_partials[kMaxBlocks];

// Host code may not use g_partials' name as a device address; the address is looked up
// once per device (with that device current) and kept here.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_partials_dev[kMaxDevices] = {nullptr};

struct DenseDesc {
  int n[3];
  int act[3];
  double d[3];
  double gamma;
};

// Minimum that keeps a NaN: a cell whose state cannot give a limit poisons the result.
__device__ __forceinline__ double nan_min(double a, double b) { return (a < b || a != a) ? a : b; }

// CFL limit min over active axes of d / (|v_d| + c_fast,d) at cell (i, j, k), in FP64,
// from the dense host-format arrays: the same formula as the step's recovery phase,
// without density or pressure floors.  A cell with rho <= 0, p <= 0 or a non-finite
// value has no limit: it returns NaN.
__device__ double cell_limit(const DenseDesc& D, const double* __restrict__ U,
                             const double* __restrict__ Bx, const double* __restrict__ By,
                             const double* __restrict__ Bz, int i, int j, int k) {
  const long long nx = D.n[0], ny = D.n[1], nz = D.n[2];
  const long long nc = nx * ny * nz;
  const long long c = i + nx * (j + ny * k);
  const double rho = U[c], mx = U[nc + c], my = U[2 * nc + c], mz = U[3 * nc + c], e = U[4 * nc + c];
  const double sbx = Bx[i + (nx + 1) * (j + ny * k)] + Bx[(i + 1) + (nx + 1) * (j + ny * k)];
  const double sby = By[i + nx * (j + (ny + 1) * k)] + By[i + nx * ((j + 1) + (ny + 1) * k)];
  const double sbz = Bz[i + nx * (j + ny * k)] + Bz[i + nx * (j + ny * (k + 1))];
  const double irho = 1.0 / rho;
  const double m2 = mx * mx + my * my + mz * mz;
  const double b2 = sbx * sbx + sby * sby + sbz * sbz;
  const double gm1 = D.gamma - 1.0;
  const double p = gm1 * e - (0.5 * gm1) * (m2 * irho) - (0.125 * gm1) * b2;
  const double v[3] = {mx * irho, my * irho, mz * irho};
  const double b[3] = {sbx * 0.5, sby * 0.5, sbz * 0.5};
  const double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  if (!(rho > 0.0) || !(p > 0.0) || !(fabs(e) < INFINITY) || !(bb < INFINITY) || !(m2 < INFINITY)) return NAN;
  double lim = INFINITY;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!D.act[a]) continue;
    const double cf = mhd::fast_speed<double>(rho, p, bb, b[a] * b[a], D.gamma);
    const double t = D.d[a] / (fabs(v[a]) + cf);
    lim = t < lim ? t : lim;
  }
  return lim;
}

__device__ double block_min(double v) {
  __shared__ double red[kBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v = nan_min(__shfl_xor_sync(0xffffffffu, v, o), v);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = (threadIdx.x < kBlock / 32) ? red[threadIdx.x] : INFINITY;
  if (warp == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v = nan_min(__shfl_xor_sync(0xffffffffu, v, o), v);
    }
  }
  return v;
}

// first pass: block b covers cells [b*2048, (b+1)*2048) and writes its minimum
__global__ void __launch_bounds__(kBlock) k_cfl_partials(DenseDesc D, const double* __restrict__ U,
                                                         const double* __restrict__ Bx,
                                                         const double* __restrict__ By,
                                                         const double* __restrict__ Bz,
                                                         double* __restrict__ partials) {
  const long long nc = (long long)D.n[0] * D.n[1] * D.n[2];
  double lim = INFINITY;
  for (int r = 0; r < kCellsPerThread; ++r) {
    const long long c = (long long)blockIdx.x * kCellsPerBlock + (long long)r * kBlock + threadIdx.x;
    if (c >= nc) break;
    const int i = (int)(c % D.n[0]);
    const long long q = c / D.n[0];
    const int j = (int)(q % D.n[1]);
    const int k = (int)(q / D.n[1]);
    lim = nan_min(cell_limit(D, U, Bx, By, Bz, i, j, k), lim);
  }
  lim = block_min(lim);
  if (threadIdx.x == 0) partials[blockIdx.x] = lim;
}

// second pass: one block folds the partials in a fixed order
__global__ void __launch_bounds__(kBlock) k_cfl_final(const double* __restrict__ partials, int nblocks,
                                                      double cfl, double* __restrict__ dt_out) {
  double lim = INFINITY;
  for (int b = threadIdx.x; b < nblocks; b += kBlock) lim = nan_min(partials[b], lim);
  lim = block_min(lim);
  if (threadIdx.x == 0) *dt_out = cfl * lim;
}

}  // namespace

extern "C" int mhd_cfl_dt_noalloc(const mhd_patch_desc* p, double cfl, const double* U,
                                  const double* Bface, double* dt_out, void* stream) {
  if (!p || !U || !Bface || !dt_out || !(cfl > 0.0) || !std::isfinite(cfl)) return MHD_ERR_ARG;
  const int n[3] = {p->nx, p->ny, p->nz};
  const double d[3] = {p->dx, p->dy, p->dz};
  DenseDesc D;
  long long nc = 1;
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 1 || !(d[a] > 0.0)) return MHD_ERR_ARG;
    D.n[a] = n[a];
    D.act[a] = n[a] > 1;
    D.d[a] = d[a];
    nc *= n[a];
  }
  if (!(p->gamma > 1.0)) return MHD_ERR_ARG;
  if (nc > MHD_NOALLOC_MAX_CELLS) return MHD_ERR_ARG;  // beyond the fixed scratch
  D.gamma = p->gamma;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MHD_ERR_CUDA;
  double* partials = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_partials_dev[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_partials) != cudaSuccess || !ptr) return MHD_ERR_CUDA;
      g_partials_dev[dev] = (double*)ptr;
    }
    partials = g_partials_dev[dev];
  }

  const long long nb = (nc + kCellsPerBlock - 1) / kCellsPerBlock;
  const double* Bx = Bface;
  const double* By = Bx + (long long)(n[0] + 1) * n[1] * n[2];
  const double* Bz = By + (long long)n[0] * (n[1] + 1) * n[2];
  cudaStream_t s = (cudaStream_t)stream;
  k_cfl_partials<<<(unsigned)nb, kBlock, 0, s>>>(D, U, Bx, By, Bz, partials);
  k_cfl_final<<<1, kBlock, 0, s>>>(partials, (int)nb, cfl, dt_out);
  return cudaGetLastError() == cudaSuccess ? MHD_OK : MHD_ERR_CUDA;
}
