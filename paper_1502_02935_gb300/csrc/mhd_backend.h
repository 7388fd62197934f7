// mhd_backend.h -- per-precision launch table shared by the host runtime.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace mhd {
struct PatchDev;
struct StageArgs;
struct PersistentArgs;

// Optional per-launch CUDA-event pairs recorded on the launching stream.
enum { KC_PRIM = 0, KC_FLUX1 = 1, KC_FLUX2 = 4, KC_EMF = 7, KC_UPDATE = 8, KC_CFL = 9, KC_PERSISTENT = 10,
       KC_THERMAL = 11, KC_FLOOR = 12, KC_GHOST = 13, KC_EMF_UPDATE = 14, KC_SCALARS = 15, KC_FLUX1_XYZ = 16,
       KC_COUNT = 17 };
struct ProfRec {
  static constexpr int kMax = 64;
  cudaEvent_t a[kMax], b[kMax];
  int cls[kMax];
  int n = 0;
};

struct ProfScope {
  ProfRec* p;
  int slot;
  cudaStream_t s;
  ProfScope(ProfRec* p_, int cls, cudaStream_t s_) : p(p_), slot(-1), s(s_) {
    if (p && p->n < ProfRec::kMax) {
      slot = p->n++;
      p->cls[slot] = cls;
      cudaEventRecord(p->a[slot], s);
    }
  }
  ~ProfScope() {
    if (slot >= 0) cudaEventRecord(p->b[slot], s);
  }
};

// Two side streams and their events for one issuing stream: a stage issues the y and z flux
// kernels on the side streams, beside the x kernel on its own stream, and joins them before
// the update (in a captured graph: three parallel branches).
struct ForkSet {
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[2] = {nullptr, nullptr};
};

struct Backend {
  size_t scratch_elem;  // bytes per scratch value (8 for FP64, 4 for the mixed path)
  // one stage (0 predictor, 1 corrector) of a van Leer step of one patch; both write Uh
  // (fk: side streams for the flux kernels, or null to issue everything on the stream)
  int (*stage)(const PatchDev&, const StageArgs&, cudaStream_t, long long* launches, ProfRec* prof,
               const ForkSet* fk);
  // W and CFL limit of the current state Un (the recovery that starts a step)
  int (*prim)(const PatchDev&, cudaStream_t, long long* launches, ProfRec* prof);
  // CFL limit of the current state into the patch's cfl_min slot
  int (*cfl)(const PatchDev&, cudaStream_t, long long* launches);
  // W of the ghost shell from the interior W and the current state Un
  int (*ghost_w)(const PatchDev&, cudaStream_t, long long* launches);
  // unit-level Riemann fluxes (solver: 0 HLLD, 1 HLLC, 2 HLL)
  int (*riemann)(int solver, int n, const double* wl, const double* wr, const double* bn, double gamma,
                 double* flux, cudaStream_t s);
  // one whole step of every patch in one cooperative launch of `blocks` CTAs
  int (*persistent)(const PersistentArgs&, int blocks, cudaStream_t, long long* launches);
  int (*occupancy)(int block, int* blocks_per_sm);
};

Backend backend_fp64();
Backend backend_mixed();
}  // namespace mhd
