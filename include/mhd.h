/*
 * mhd.h -- C ABI of the GB300 magneto-gas-dynamics step library (libmhd.so).
 *
 * The library advances the ideal-MHD system of Khoperskov, Vasiliev, Khoperskov &
 * Lubimov, "Numerical code for multi-component galaxies" (arXiv:1502.02935),
 * Section 2.1: conserved U = [rho, rho v, E, B] (Eq. 1), dU/dt + div(F, G, H) = S
 * (Eq. 2, fluxes Eq. 3, P* = P + B^2/2), finite-volume update with n+1/2 fluxes
 * (Eq. 7), constrained-transport induction on face-centred B (Eq. 4-6, Eq. 8)
 * with corner EMFs (Eq. 9-11), HLLD Riemann fluxes and kappa = 1/3 minmod MUSCL
 * reconstruction of primitives (Eq. 12-14), two-stage van Leer time stepping.
 * Every step runs in the library's CUDA kernels on one GPU.
 *
 * Conventions
 *  - Status: every call returns an int; MHD_OK (0) or a negative MHD_ERR_* code.
 *    Nothing throws or aborts across this boundary.  mhd_last_error() gives text.
 *  - Ownership: the caller owns every array it passes; the library copies from
 *    and into them and keeps no pointer after the call returns.  The library owns
 *    all device memory it allocates (freed by mhd_destroy).
 *  - Host state format per patch (FP64, x fastest):
 *      U     : 5 cell fields [rho, rho vx, rho vy, rho vz, E], each nz*ny*nx.
 *      Bface : Bx (nz, ny, nx+1), then By (nz, ny+1, nx), then Bz (nz+1, ny, nx),
 *              concatenated; index i of Bx is the face x_{i-1/2}.  On periodic
 *              axes and on trivial axes (n = 1) the last layer repeats the first.
 *  - on_device = 1: the U / Bface pointers are device pointers (for example a
 *    torch CUDA tensor's data_ptr()) with the same layout; 0: host pointers.
 *  - Streams: all work is issued on the cudaStream_t given in mhd_grid_desc
 *    (NULL = the legacy default stream).  A context is not thread-safe.
 *  - Device-side errors (non-finite or non-positive density/pressure, a bounded
 *    wait that ran out) set a sticky device error word; it is read, and returned
 *    as a status, by mhd_sync, mhd_cfl_dt and mhd_get_state.
 */
#ifndef MHD_H
#define MHD_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MHD_OK = 0,
  MHD_ERR_ARG = -1,       /* invalid argument (sizes, pointers, combination) */
  MHD_ERR_CUDA = -2,      /* a CUDA runtime call failed */
  MHD_ERR_NONFINITE = -3, /* a non-finite value appeared in the state */
  MHD_ERR_NEGATIVE = -4,  /* density or pressure <= 0 after recovery */
  MHD_ERR_TIMEOUT = -5,   /* a bounded device wait ran out (persistent mode) */
  MHD_ERR_STATE = -6,     /* call not valid in the context's current state */
  MHD_ERR_NOMEM = -7      /* device allocation failed */
};

enum { MHD_BC_PERIODIC = 0, MHD_BC_OUTFLOW = 1 };

enum {
  MHD_PREC_FP64 = 0, /* every stage in FP64 */
  MHD_PREC_MIXED = 1 /* FP32 reconstruction/Riemann/EMF arithmetic; FP64 pressure
                        recovery p = (gamma-1)(E - kinetic - magnetic) and FP64
                        accumulation of the conserved state */
};

enum {
  MHD_FLAG_GRAPH = 1,      /* replay each step from a captured CUDA graph */
  MHD_FLAG_PERSISTENT = 2  /* all patches, all phases of a step in one persistent launch */
};

enum { MHD_POT_NONE = 0, MHD_POT_GAUSS_X = 1, MHD_POT_LOG_DISC = 2 };

/* One rectangular patch.  Axes with n = 1 are trivial (no fluxes along them). */
typedef struct {
  int nx, ny, nz;
  double x0, y0, z0; /* coordinate of the low face of cell 0 */
  double dx, dy, dz;
  int bc[6];         /* x-lo, x-hi, y-lo, y-hi, z-lo, z-hi: MHD_BC_*; a periodic axis
                        must be periodic on both sides */
  double gamma;      /* ratio of specific heats, > 1 */
} mhd_patch_desc;

typedef struct {
  int n_patches;                 /* >= 1; patches are independent */
  const mhd_patch_desc* patches; /* n_patches descriptors */
  int precision;                 /* MHD_PREC_* */
  double cfl;                    /* Courant number used when dt <= 0 */
  int flags;                     /* MHD_FLAG_* */
  void* cuda_stream;             /* cudaStream_t or NULL */
} mhd_grid_desc;

/* External potential entering the source vector S of Eq. 2:
 * S = [0, -rho grad Psi, -rho v . grad Psi, 0, 0, 0].
 *   MHD_POT_GAUSS_X : Psi = -psi0 exp(-((x - xc)/xw)^2)
 *   MHD_POT_LOG_DISC: Psi = v0^2/2 ln(x^2 + y^2 + rc^2 + z^2) */
typedef struct {
  int potential;
  double psi0, xc, xw;
  double v0, rc;
} mhd_source_desc;

typedef struct {
  double dt_last;        /* dt used by the last step of patch 0 */
  double sums[5];        /* interior totals of rho, rho v, E over all patches */
  double max_divb;       /* max over cells of |div B| * min(dx) */
  int error_word;        /* sticky device error bits */
} mhd_metrics;

typedef struct mhd_ctx mhd_ctx; /* opaque, library-owned */

/* Create a context, allocate the device state of every patch and copy the
 * initial state in.  U0[p] / Bface0[p] follow the host state format above.
 * On failure *out is NULL and nothing stays allocated. */
int mhd_init_grid(mhd_ctx** out, const mhd_grid_desc* grid, const double* const* U0,
                  const double* const* Bface0, int on_device);

/* Set the external potential (Eq. 2 source vector).  Default: none. */
int mhd_set_sources(mhd_ctx* ctx, const mhd_source_desc* src);

/* Advance every patch by one van Leer step (Eq. 7, Eq. 8).  dt > 0: that dt for
 * every patch.  dt <= 0: each patch uses cfl * its own CFL limit of its current
 * state, computed on the device (no host synchronisation).  Asynchronous. */
int mhd_step(mhd_ctx* ctx, double dt);

/* cfl * min over all patches, cells and active axes of d/(|v_d| + c_fast,d) for the
 * current state.  Synchronises the stream. */
int mhd_cfl_dt(mhd_ctx* ctx, double* dt_out);

/* Per-patch CFL time steps, n_patches values.  Synchronises. */
int mhd_cfl_dt_patches(mhd_ctx* ctx, double* dt_out);

/* Copy the state of one patch out (host format above; on_device as in init). */
int mhd_get_state(mhd_ctx* ctx, int patch, double* U_out, double* Bface_out, int on_device);

/* Replace the state of one patch (same format).  Used for resume and for
 * end-to-end runs that stream each step's input from the host. */
int mhd_set_state(mhd_ctx* ctx, int patch, const double* U, const double* Bface, int on_device);

/* Wait for all issued work and return the device error status. */
int mhd_sync(mhd_ctx* ctx);

int mhd_get_metrics(mhd_ctx* ctx, mhd_metrics* out);

/* Number of kernel launches the library issued since the context was created
 * (graph replays count the kernels inside the graph). */
long long mhd_launch_count(const mhd_ctx* ctx);

/* Per-kernel timing.  While on, every launch is bracketed by a CUDA event pair on the
 * context's stream (steps are not replayed from a graph) and the elapsed times are summed
 * per kernel class: 0 recovery+CFL, 1-3 donor-cell HLLD fluxes x/y/z, 4-6 kappa-scheme
 * HLLD fluxes x/y/z, 7 corner EMFs, 8 update, 9 standalone CFL.  Switching on or off
 * clears the totals. */
int mhd_set_profiling(mhd_ctx* ctx, int on);

/* Totals since profiling was switched on: ms[c] milliseconds and launches[c] launches of
 * class c, for c < n (n >= 10).  Synchronises. */
int mhd_get_profile(mhd_ctx* ctx, double* ms, long long* launches, int n);

const char* mhd_last_error(const mhd_ctx* ctx);

void mhd_destroy(mhd_ctx* ctx);

/* Unit-level entry for parity tests: HLLD fluxes (Miyoshi & Kusano 2005, the solver
 * named in Section 2.1) of n interfaces in the interface frame, computed by the
 * same device function the step uses.  wl, wr: n*8 values [rho, vn, vt1, vt2, p,
 * unused, Bt1, Bt2]; bn: n normal fields; flux: n*8 outputs [rho, mn, mt1, mt2, E,
 * 0, Bt1, Bt2].  All four are device pointers; precision MHD_PREC_FP64 computes in
 * FP64, MHD_PREC_MIXED in FP32 (inputs/outputs stay FP64).  stream may be NULL. */
int mhd_riemann_hlld(int n, const double* wl, const double* wr, const double* bn, double gamma,
                     int precision, double* flux, void* stream);

/* Largest patch (nx*ny*nz cells) that mhd_cfl_dt_noalloc accepts. */
#define MHD_NOALLOC_MAX_CELLS 8388608

/* CFL time step of a state held by the caller, computed without allocating device
 * memory.  The paper has no counterpart: this exists for callers that cannot allocate
 * (an application that reserves the whole device through its own memory pool, or a
 * loop that cannot afford the synchronisation cudaMalloc/cudaFree imply).
 *   p        : one patch descriptor (boundary conditions are not used).
 *   cfl      : Courant number, > 0.
 *   U, Bface : device pointers to the state in the host format above (FP64).
 *   dt_out   : device pointer; receives cfl * min over cells and active axes of
 *              d / (|v_d| + c_fast,d), computed in FP64 as mhd_cfl_dt of an FP64 context.
 *   stream   : cudaStream_t or NULL; the call is asynchronous on it.
 * Scratch is a fixed 32 KiB __device__ array inside the library, held by every GPU
 * that loads it until the process exits; the call allocates and frees nothing.
 * Returns MHD_ERR_ARG for bad arguments or nx*ny*nz > MHD_NOALLOC_MAX_CELLS, and
 * MHD_ERR_CUDA if a launch fails.  The first call on each device looks up the
 * scratch array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture.  All calls share the one array:
 * calls whose work overlaps on the GPU (e.g. on two streams) race and must be
 * serialised by the caller. */
int mhd_cfl_dt_noalloc(const mhd_patch_desc* p, double cfl, const double* U, const double* Bface,
                       double* dt_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
