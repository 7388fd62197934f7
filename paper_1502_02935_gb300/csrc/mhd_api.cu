// mhd_api.cu -- host runtime behind the C ABI of include/mhd.h: patch descriptors,
// device allocations, host<->device state exchange, the per-step launch sequence
// (optionally captured once into a CUDA graph and replayed), CFL queries and the
// sticky device error word.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mhd.h"
#include "mhd_backend.h"
#include "mhd_device.cuh"

using namespace mhd;

namespace {

struct PatchHost {
  PatchDev dev;
  mhd_patch_desc desc;
  long long ncell = 0, dense = 0;
  void* state = nullptr;
  void* scratch = nullptr;
};

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

__global__ void k_pack(PatchDev P, const double* __restrict__ U, double* __restrict__ out, long long total) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    pack_point(P, U, out, t);
}

__global__ void k_unpack(PatchDev P, const double* __restrict__ in, double* __restrict__ U, long long total) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    unpack_point(P, in, U, t);
}

unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 65535LL * 32 ? 65535LL * 32 : b));
}

}  // namespace

struct mhd_ctx {
  int np = 0, precision = 0, flags = 0;
  double cfl = 0.4;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<PatchHost> P;
  Backend be{};
  SourceDev src{};
  unsigned long long* cfl_min = nullptr;
  double* dt_used = nullptr;
  int* err = nullptr;
  double* staging = nullptr;
  cudaGraphExec_t gexec = nullptr;
  long long graph_launches = 0;
  long long launches = 0;
  bool profiling = false;
  ProfRec prof{};
  double prof_ms[KC_COUNT] = {0};
  long long prof_n[KC_COUNT] = {0};
  std::string last_error;
};

static int fail(mhd_ctx* c, int code, const std::string& msg) {
  if (c) c->last_error = msg;
  return code;
}

static int cuda_fail(mhd_ctx* c, cudaError_t e, const char* where) {
  return fail(c, MHD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                            \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

static void free_ctx(mhd_ctx* ctx) {
  if (!ctx) return;
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->profiling)
    for (int q = 0; q < ProfRec::kMax; ++q) {
      cudaEventDestroy(ctx->prof.a[q]);
      cudaEventDestroy(ctx->prof.b[q]);
    }
  for (auto& p : ctx->P) {
    if (p.state) cudaFree(p.state);
    if (p.scratch) cudaFree(p.scratch);
  }
  if (ctx->cfl_min) cudaFree(ctx->cfl_min);
  if (ctx->dt_used) cudaFree(ctx->dt_used);
  if (ctx->err) cudaFree(ctx->err);
  if (ctx->staging) cudaFree(ctx->staging);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

static int validate_patch(const mhd_patch_desc& d, std::string& why) {
  const int n[3] = {d.nx, d.ny, d.nz};
  const double dd[3] = {d.dx, d.dy, d.dz};
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 1 || n[a] > (1 << 20)) { why = "cell count out of range"; return -1; }
    if (!(dd[a] > 0.0) || !std::isfinite(dd[a])) { why = "cell size must be positive"; return -1; }
    if (n[a] > 1) {
      const int lo = d.bc[2 * a], hi = d.bc[2 * a + 1];
      if ((lo != MHD_BC_PERIODIC && lo != MHD_BC_OUTFLOW) || (hi != MHD_BC_PERIODIC && hi != MHD_BC_OUTFLOW)) {
        why = "unknown boundary condition"; return -1;
      }
      if ((lo == MHD_BC_PERIODIC) != (hi == MHD_BC_PERIODIC)) {
        why = "a periodic axis must be periodic on both sides"; return -1;
      }
      if (n[a] < 2) { why = "active axis needs at least 2 cells"; return -1; }
    }
  }
  if (!(d.gamma > 1.0) || !std::isfinite(d.gamma)) { why = "gamma must be > 1"; return -1; }
  return 0;
}

static int read_error_word(mhd_ctx* ctx) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h & ERR_TIMEOUT) return fail(ctx, MHD_ERR_TIMEOUT, "a bounded device wait ran out");
  if (h & ERR_NONFINITE) return fail(ctx, MHD_ERR_NONFINITE, "non-finite value in the state");
  if (h & ERR_NEGATIVE) return fail(ctx, MHD_ERR_NEGATIVE, "density or pressure <= 0");
  return MHD_OK;
}

// wait for the recorded launches and fold their event times into the per-class totals
static int flush_profile(mhd_ctx* ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  for (int q = 0; q < ctx->prof.n; ++q) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->prof.a[q], ctx->prof.b[q]));
    ctx->prof_ms[ctx->prof.cls[q]] += ms;
    ctx->prof_n[ctx->prof.cls[q]] += 1;
  }
  ctx->prof.n = 0;
  return MHD_OK;
}

static int issue_step(mhd_ctx* ctx, double dt) {
  CK(cudaMemsetAsync(ctx->cfl_min, 0xFF, sizeof(unsigned long long) * ctx->np, ctx->stream));
  StageArgs a{};
  a.dt_host = dt;
  a.cfl = ctx->cfl;
  a.src = ctx->src;
  for (int stage = 0; stage < 2; ++stage) {
    a.stage = stage;
    for (auto& p : ctx->P) {
      if (ctx->profiling && ctx->prof.n > ProfRec::kMax - 16) {
        int rc = flush_profile(ctx);
        if (rc) return rc;
      }
      if (ctx->be.stage(p.dev, a, ctx->stream, &ctx->launches, ctx->profiling ? &ctx->prof : nullptr))
        return cuda_fail(ctx, cudaGetLastError(), "stage launch");
    }
  }
  if (ctx->profiling) return flush_profile(ctx);
  return MHD_OK;
}

extern "C" {

int mhd_init_grid(mhd_ctx** out, const mhd_grid_desc* g, const double* const* U0,
                  const double* const* B0, int on_device) {
  if (!out) return MHD_ERR_ARG;
  *out = nullptr;
  if (!g || g->n_patches < 1 || !g->patches || !U0 || !B0) return MHD_ERR_ARG;
  if (g->precision != MHD_PREC_FP64 && g->precision != MHD_PREC_MIXED) return MHD_ERR_ARG;
  if (!(g->cfl > 0.0)) return MHD_ERR_ARG;
  mhd_ctx* ctx = new mhd_ctx();
  ctx->np = g->n_patches;
  ctx->precision = g->precision;
  ctx->flags = g->flags;
  ctx->cfl = g->cfl;
  ctx->be = g->precision == MHD_PREC_FP64 ? backend_fp64() : backend_mixed();
  auto bail = [&](int code) {
    free_ctx(ctx);
    return code;
  };
  if (g->cuda_stream) {
    ctx->stream = (cudaStream_t)g->cuda_stream;
  } else {
    if (cudaStreamCreate(&ctx->stream) != cudaSuccess) return bail(MHD_ERR_CUDA);
    ctx->own_stream = true;
  }
  if (cudaMalloc(&ctx->cfl_min, sizeof(unsigned long long) * ctx->np) != cudaSuccess ||
      cudaMalloc(&ctx->dt_used, sizeof(double) * ctx->np) != cudaSuccess ||
      cudaMalloc(&ctx->err, sizeof(int)) != cudaSuccess)
    return bail(MHD_ERR_NOMEM);
  cudaMemset(ctx->err, 0, sizeof(int));
  cudaMemset(ctx->dt_used, 0, sizeof(double) * ctx->np);
  long long max_dense = 0;
  ctx->P.resize(ctx->np);
  for (int p = 0; p < ctx->np; ++p) {
    const mhd_patch_desc& d = g->patches[p];
    std::string why;
    if (validate_patch(d, why) || !U0[p] || !B0[p]) return bail(MHD_ERR_ARG);
    PatchHost& H = ctx->P[p];
    H.desc = d;
    PatchDev& D = H.dev;
    memset(&D, 0, sizeof(D));
    const int n[3] = {d.nx, d.ny, d.nz};
    const double dd[3] = {d.dx, d.dy, d.dz}, lo[3] = {d.x0, d.y0, d.z0};
    for (int a = 0; a < 3; ++a) {
      D.n[a] = n[a];
      D.act[a] = n[a] > 1;
      D.per[a] = !D.act[a] || d.bc[2 * a] == MHD_BC_PERIODIC;
      D.nface[a] = (D.act[a] && !D.per[a]) ? n[a] + 1 : n[a];
      D.g2[a] = D.act[a] ? 2 : 0;
      D.d[a] = dd[a];
      D.inv_d[a] = 1.0 / dd[a];
      D.lo[a] = lo[a];
    }
    D.gamma = d.gamma;
    D.PX = (int)round_up(n[0] + 1, 4);
    D.PY = n[1] + 1;
    D.PZ = n[2] + 1;
    D.FS = round_up((long long)D.PX * D.PY * D.PZ, 32);
    D.QX = n[0] + 2 * D.g2[0];
    D.QY = n[1] + 2 * D.g2[1];
    D.QZ = n[2] + 2 * D.g2[2];
    D.QS = round_up((long long)D.QX * D.QY * D.QZ, 64);
    H.ncell = (long long)n[0] * n[1] * n[2];
    H.dense = 5 * H.ncell + (long long)(n[0] + 1) * n[1] * n[2] + (long long)n[0] * (n[1] + 1) * n[2] +
              (long long)n[0] * n[1] * (n[2] + 1);
    if (H.dense > max_dense) max_dense = H.dense;
    const size_t sbytes = sizeof(double) * 16 * (size_t)D.FS;
    const size_t qbytes = ctx->be.scratch_elem * (size_t)(8 + 3 * NFLUX + 3) * (size_t)D.QS;
    if (cudaMalloc(&H.state, sbytes) != cudaSuccess) return bail(MHD_ERR_NOMEM);
    if (cudaMalloc(&H.scratch, qbytes) != cudaSuccess) return bail(MHD_ERR_NOMEM);
    cudaMemset(H.state, 0, sbytes);
    cudaMemset(H.scratch, 0, qbytes);
    D.Un = (double*)H.state;
    D.Uh = D.Un + 8 * D.FS;
    char* q = (char*)H.scratch;
    const size_t fs = ctx->be.scratch_elem * (size_t)D.QS;
    D.W = q;
    q += 8 * fs;
    for (int a = 0; a < 3; ++a) {
      D.F[a] = q;
      q += NFLUX * fs;
    }
    D.E = q;
    D.cfl_min = ctx->cfl_min + p;
    D.dt_used = ctx->dt_used + p;
    D.err = ctx->err;
    D.index = p;
  }
  if (cudaMalloc(&ctx->staging, sizeof(double) * (size_t)max_dense) != cudaSuccess)
    return bail(MHD_ERR_NOMEM);
  for (int p = 0; p < ctx->np; ++p) {
    int rc = mhd_set_state(ctx, p, U0[p], B0[p], on_device);
    if (rc) return bail(rc);
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return bail(MHD_ERR_CUDA);
  *out = ctx;
  return MHD_OK;
}

int mhd_set_sources(mhd_ctx* ctx, const mhd_source_desc* s) {
  if (!ctx || !s) return MHD_ERR_ARG;
  if (s->potential != MHD_POT_NONE && s->potential != MHD_POT_GAUSS_X && s->potential != MHD_POT_LOG_DISC)
    return fail(ctx, MHD_ERR_ARG, "unknown potential");
  if (s->potential == MHD_POT_GAUSS_X && !(s->xw > 0.0)) return fail(ctx, MHD_ERR_ARG, "xw must be > 0");
  ctx->src.potential = s->potential;
  ctx->src.psi0 = s->psi0;
  ctx->src.xc = s->xc;
  ctx->src.xw = s->xw;
  ctx->src.v0 = s->v0;
  ctx->src.rc = s->rc;
  if (ctx->gexec) {  // sources are baked into captured launches
    cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
  }
  return MHD_OK;
}

int mhd_step(mhd_ctx* ctx, double dt) {
  if (!ctx) return MHD_ERR_ARG;
  if (!std::isfinite(dt)) return fail(ctx, MHD_ERR_ARG, "dt must be finite");
  if ((ctx->flags & MHD_FLAG_GRAPH) && dt <= 0.0 && !ctx->profiling) {
    if (!ctx->gexec) {
      cudaGraph_t graph;
      long long before = ctx->launches;
      CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      int rc = issue_step(ctx, -1.0);
      cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
      if (rc) return rc;
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
      ctx->graph_launches = ctx->launches - before;
      ctx->launches = before;
      e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
    ctx->launches += ctx->graph_launches;
    return MHD_OK;
  }
  return issue_step(ctx, dt);
}

int mhd_cfl_dt_patches(mhd_ctx* ctx, double* out) {
  if (!ctx || !out) return MHD_ERR_ARG;
  CK(cudaMemsetAsync(ctx->cfl_min, 0xFF, sizeof(unsigned long long) * ctx->np, ctx->stream));
  for (auto& p : ctx->P) {
    ProfScope ps(ctx->profiling && ctx->prof.n < ProfRec::kMax ? &ctx->prof : nullptr, KC_CFL, ctx->stream);
    if (ctx->be.cfl(p.dev, ctx->stream, &ctx->launches)) return cuda_fail(ctx, cudaGetLastError(), "cfl launch");
  }
  std::vector<unsigned long long> bits(ctx->np);
  CK(cudaMemcpyAsync(bits.data(), ctx->cfl_min, sizeof(unsigned long long) * ctx->np,
                     cudaMemcpyDeviceToHost, ctx->stream));
  int rc = read_error_word(ctx);
  if (rc) return rc;
  for (int p = 0; p < ctx->np; ++p) {
    double v;
    memcpy(&v, &bits[p], sizeof v);
    out[p] = ctx->cfl * v;
  }
  return MHD_OK;
}

int mhd_cfl_dt(mhd_ctx* ctx, double* out) {
  if (!ctx || !out) return MHD_ERR_ARG;
  std::vector<double> v(ctx->np);
  int rc = mhd_cfl_dt_patches(ctx, v.data());
  if (rc) return rc;
  double m = v[0];
  for (double x : v) m = x < m ? x : m;
  *out = m;
  return MHD_OK;
}

int mhd_get_state(mhd_ctx* ctx, int patch, double* U_out, double* B_out, int on_device) {
  if (!ctx || patch < 0 || patch >= ctx->np || !U_out || !B_out) return MHD_ERR_ARG;
  PatchHost& H = ctx->P[patch];
  k_pack<<<grid_for(H.dense), 256, 0, ctx->stream>>>(H.dev, H.dev.Un, ctx->staging, H.dense);
  ctx->launches += 1;
  CK(cudaGetLastError());
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(U_out, ctx->staging, sizeof(double) * 5 * H.ncell, kind, ctx->stream));
  CK(cudaMemcpyAsync(B_out, ctx->staging + 5 * H.ncell, sizeof(double) * (H.dense - 5 * H.ncell), kind,
                     ctx->stream));
  return read_error_word(ctx);
}

int mhd_set_state(mhd_ctx* ctx, int patch, const double* U, const double* B, int on_device) {
  if (!ctx || patch < 0 || patch >= ctx->np || !U || !B) return MHD_ERR_ARG;
  PatchHost& H = ctx->P[patch];
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(ctx->staging, U, sizeof(double) * 5 * H.ncell, kind, ctx->stream));
  CK(cudaMemcpyAsync(ctx->staging + 5 * H.ncell, B, sizeof(double) * (H.dense - 5 * H.ncell), kind,
                     ctx->stream));
  k_unpack<<<grid_for(H.dense), 256, 0, ctx->stream>>>(H.dev, ctx->staging, H.dev.Un, H.dense);
  ctx->launches += 1;
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream));
  return MHD_OK;
}

int mhd_sync(mhd_ctx* ctx) {
  if (!ctx) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  return read_error_word(ctx);
}

int mhd_get_metrics(mhd_ctx* ctx, mhd_metrics* m) {
  if (!ctx || !m) return MHD_ERR_ARG;
  memset(m, 0, sizeof(*m));
  CK(cudaMemcpyAsync(&m->dt_last, ctx->dt_used, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&m->error_word, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int p = 0; p < ctx->np; ++p) {
    PatchHost& H = ctx->P[p];
    std::vector<double> buf(H.dense);
    k_pack<<<grid_for(H.dense), 256, 0, ctx->stream>>>(H.dev, H.dev.Un, ctx->staging, H.dense);
    ctx->launches += 1;
    CK(cudaMemcpyAsync(buf.data(), ctx->staging, sizeof(double) * H.dense, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int nx = H.desc.nx, ny = H.desc.ny, nz = H.desc.nz;
    for (int f = 0; f < 5; ++f) {
      double s = 0.0;
      for (long long q = 0; q < H.ncell; ++q) s += buf[f * H.ncell + q];
      m->sums[f] += s;
    }
    const double* Bx = buf.data() + 5 * H.ncell;
    const double* By = Bx + (long long)(nx + 1) * ny * nz;
    const double* Bz = By + (long long)nx * (ny + 1) * nz;
    const double d[3] = {H.desc.dx, H.desc.dy, H.desc.dz};
    const int n[3] = {nx, ny, nz};
    double dmin = INFINITY;
    for (int a = 0; a < 3; ++a)
      if (n[a] > 1 && d[a] < dmin) dmin = d[a];
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          double div = 0.0;
          if (nx > 1) div += (Bx[(i + 1) + (long long)(nx + 1) * (j + (long long)ny * k)] -
                              Bx[i + (long long)(nx + 1) * (j + (long long)ny * k)]) / d[0];
          if (ny > 1) div += (By[i + (long long)nx * ((j + 1) + (long long)(ny + 1) * k)] -
                              By[i + (long long)nx * (j + (long long)(ny + 1) * k)]) / d[1];
          if (nz > 1) div += (Bz[i + (long long)nx * (j + (long long)ny * (k + 1))] -
                              Bz[i + (long long)nx * (j + (long long)ny * k)]) / d[2];
          double v = std::fabs(div) * dmin;
          if (v > m->max_divb) m->max_divb = v;
        }
  }
  return MHD_OK;
}

long long mhd_launch_count(const mhd_ctx* ctx) { return ctx ? ctx->launches : 0; }

int mhd_set_profiling(mhd_ctx* ctx, int on) {
  if (!ctx) return MHD_ERR_ARG;
  if (on && !ctx->profiling) {
    for (int q = 0; q < ProfRec::kMax; ++q) {
      CK(cudaEventCreate(&ctx->prof.a[q]));
      CK(cudaEventCreate(&ctx->prof.b[q]));
    }
    ctx->profiling = true;
  } else if (!on && ctx->profiling) {
    int rc = flush_profile(ctx);
    for (int q = 0; q < ProfRec::kMax; ++q) {
      cudaEventDestroy(ctx->prof.a[q]);
      cudaEventDestroy(ctx->prof.b[q]);
    }
    ctx->profiling = false;
    if (rc) return rc;
  }
  for (int c = 0; c < KC_COUNT; ++c) {
    ctx->prof_ms[c] = 0.0;
    ctx->prof_n[c] = 0;
  }
  return MHD_OK;
}

int mhd_get_profile(mhd_ctx* ctx, double* ms, long long* launches, int n) {
  if (!ctx || !ms || !launches || n < KC_COUNT) return MHD_ERR_ARG;
  if (ctx->profiling) {
    int rc = flush_profile(ctx);
    if (rc) return rc;
  }
  for (int c = 0; c < KC_COUNT; ++c) {
    ms[c] = ctx->prof_ms[c];
    launches[c] = ctx->prof_n[c];
  }
  return MHD_OK;
}

const char* mhd_last_error(const mhd_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

void mhd_destroy(mhd_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_ctx(ctx);
}

int mhd_riemann_hlld(int n, const double* wl, const double* wr, const double* bn, double gamma,
                     int precision, double* flux, void* stream) {
  if (n < 0 || (n > 0 && (!wl || !wr || !bn || !flux)) || !(gamma > 1.0)) return MHD_ERR_ARG;
  if (precision != MHD_PREC_FP64 && precision != MHD_PREC_MIXED) return MHD_ERR_ARG;
  Backend be = precision == MHD_PREC_FP64 ? backend_fp64() : backend_mixed();
  cudaStream_t s = (cudaStream_t)stream;
  if (be.hlld(n, wl, wr, bn, gamma, flux, s)) return MHD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ERR_CUDA;
  return MHD_OK;
}

}  // extern "C"
