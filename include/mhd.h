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
  MHD_ERR_NEGATIVE = -4,  /* density or pressure <= 0 after recovery (reported before
                             MHD_ERR_NONFINITE when both occurred) */
  MHD_ERR_TIMEOUT = -5,   /* a bounded device wait ran out (persistent mode) */
  MHD_ERR_STATE = -6,     /* call not valid in the context's current state */
  MHD_ERR_NOMEM = -7      /* device allocation failed */
};

/* Boundaries (Section 3 names free and inflow boundaries): periodic; outflow = zero-gradient
 * copy of the cell fields and transverse faces; inflow = a fixed state beyond the boundary
 * (mhd_set_inflow).  Normal faces on the boundary itself are CT-updated for outflow and
 * inflow alike. */
enum { MHD_BC_PERIODIC = 0, MHD_BC_OUTFLOW = 1, MHD_BC_INFLOW = 2 };

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
/* Riemann solvers (Section 2.1): HLLD for magneto-gas dynamics (the default); HLLC and
 * HLL for pure gas dynamics (B = 0). */
enum { MHD_RIEMANN_HLLD = 0, MHD_RIEMANN_HLLC = 1, MHD_RIEMANN_HLL = 2 };
/* Reconstruction of the corrector (Eq. 12-14): kappa = 1/3, third-order upwind biased (the
 * paper's choice, default); kappa = 0, second-order upwind biased; kappa = -1, second-order
 * fully upwind. */
enum { MHD_RECON_KAPPA_THIRD = 0, MHD_RECON_KAPPA_ZERO = 1, MHD_RECON_KAPPA_UPWIND = 2 };

enum { MHD_THERMAL_OFF = 0, MHD_THERMAL_PLAIN = 1, MHD_THERMAL_SURROGATE = 2 };

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
 *   MHD_POT_LOG_DISC: Psi = v0^2/2 ln(x^2 + y^2 + rc^2 + z^2)
 * Floors (the paper states none; rho_floor > 0 turns them on, 0 leaves the step bitwise
 * unchanged): the primitive recovery uses rho_f = max(rho, rho_floor) and clamps p to
 * [rho_f pr_floor, rho_f pr_ceil]; after each full step, before the thermal term, every
 * interior cell gets rho' = max(rho, rho_floor), its momentum kept, p recomputed with rho'
 * and clamped the same way, and E rebuilt from them; changed cells are counted
 * (mhd_metrics.floored).  pr_floor <= 0: no pressure floor; pr_ceil <= 0: no ceiling. */
typedef struct {
  int potential;
  double psi0, xc, xw;
  double v0, rc;
  double rho_floor, pr_floor, pr_ceil;
} mhd_source_desc;

/* Thermal source term (heating and cooling in S of Eq. 2; the thermal module of
 * Section 3.10), applied operator-split after each step: per interior cell, isochoric
 *   e = c_e T,   de/dt = (n_H gamma_heat - n_H^2 Lambda(T, z)) / rate_unit,
 * T = t_per_pr p/rho, n_H = nh_per_rho rho, c_e = rho/(t_per_pr (gamma-1)).  Lambda is a
 * built-in piecewise power law over 10 K..1e8 K standing in for the paper's tables.
 * MHD_THERMAL_PLAIN integrates it in FP64 by sub-stepped backward Euler (sub-step change
 * capped at cap*T, Newton with bisection safeguard); MHD_THERMAL_SURROGATE evaluates the
 * trained MLP (mhd_surrogate_train) and falls back to the plain integrator per cell. */
typedef struct {
  int mode;          /* MHD_THERMAL_* */
  double gamma_heat; /* heating per hydrogen atom, erg/s */
  double z;          /* metallicity */
  double rate_unit;  /* erg cm^-3 s^-1 per code energy density per code time */
  double cap;        /* largest relative temperature change per sub-step, (0, 1] */
  double nh_per_rho; /* hydrogen number density [cm^-3] per code density */
  double t_per_pr;   /* temperature [K] per code p/rho */
} mhd_thermal_desc;

typedef struct {
  double dt_last;        /* dt used by the last step of patch 0 */
  double sums[5];        /* interior totals of rho, rho v, E over all patches */
  double max_divb;       /* max over cells of |div B| * min(dx) */
  int error_word;        /* sticky device error bits */
  unsigned long long floored; /* cells changed by the end-of-step floors since init */
} mhd_metrics;

typedef struct mhd_ctx mhd_ctx; /* opaque, library-owned */

/* Create a context, allocate the device state of every patch and copy the
 * initial state in.  U0[p] / Bface0[p] follow the host state format above.
 * On failure *out is NULL and nothing stays allocated.  MHD_ERR_ARG for a bad
 * descriptor: a cell count outside [1, 2^20] per axis or above 2^40 per patch, an
 * active axis (more than one cell) without a boundary condition on each side or
 * with periodicity on one side only, a non-positive spacing, gamma <= 1, a null
 * state pointer, an unknown precision, a Courant number that is not finite and > 0.  MHD_ERR_NOMEM when the device cannot hold the buffers; the
 * runtime's error state is left clear, so other contexts are unaffected. */
int mhd_init_grid(mhd_ctx** out, const mhd_grid_desc* grid, const double* const* U0,
                  const double* const* Bface0, int on_device);

/* Set the external potential (Eq. 2 source vector) and the floors.  Default: none. */
int mhd_set_sources(mhd_ctx* ctx, const mhd_source_desc* src);

/* Interface flux solver of every patch for the following steps (Section 2.1 names HLL and
 * HLLC for pure gas dynamics and HLLD for magneto-gas dynamics):
 *   MHD_RIEMANN_HLLD: Miyoshi & Kusano's five-wave solver (default);
 *   MHD_RIEMANN_HLLC: the three-wave gas-dynamics solver at faces where every field
 *                     component is zero on both sides, HLLD at the others (HLLD is HLLC
 *                     when B = 0, so a field-free run only gets cheaper);
 *   MHD_RIEMANN_HLL:  the two-wave solver with the same outer speeds, at every face.
 * The outer speed estimate and the mass-flux scale of the corner EMFs are the same for
 * all three.  MHD_ERR_ARG for another value. */
int mhd_set_riemann(mhd_ctx* ctx, int solver);

/* Which kernels compute the fluxes (the same fluxes, Eq. 3 with the interface states of
 * Eq. 12-14; a choice of schedule).  MHD_FLUX_MARCH: through y and z faces, threads marching
 * along the flux direction over segments of 16 faces (8, 4 or 2 on thinner boxes), each cell
 * loaded and reconstructed once; through x faces of the kappa-scheme stage, warps of 32
 * consecutive cells that pass each cell's upper-face value to the next lane by a shuffle;
 * the donor-cell stage's x faces one thread per face.  MHD_FLUX_PER_FACE: one thread per face
 * in every direction.  MHD_FLUX_AUTO (the default): as MARCH, except that y and z go per face
 * where the box gives fewer than two waves of marching threads (2D planes, small patches),
 * and that on patches with three active axes and enough columns the donor-cell stage
 * computes all three directions in one kernel marching in z.  Drops captured graphs. */
enum { MHD_FLUX_AUTO = 0, MHD_FLUX_MARCH = 1, MHD_FLUX_PER_FACE = 2 };
int mhd_set_flux_scheme(mhd_ctx* ctx, int scheme);

/* Reconstruction of every patch for the following steps, MHD_RECON_* (the minmod
 * kappa-scheme with K1 = (1 - kappa)/4, K2 = (1 + kappa)/4, b = (3 - kappa)/(1 - kappa)).
 * MHD_ERR_ARG for another value. */
int mhd_set_reconstruction(mhd_ctx* ctx, int recon);

/* State beyond side `side` (0 x-lo, 1 x-hi, 2 y-lo, 3 y-hi, 4 z-lo, 5 z-hi) of patch
 * `patch`, whose bc must be MHD_BC_INFLOW: w = [rho, vx, vy, vz, p, Bx, By, Bz] (host
 * array, copied).  Ghost cells beyond the side hold it, with their faces; a ghost cell
 * beyond several inflow sides takes the first in the order above.  Until it is set, an
 * inflow side holds rho = 1, p = 1 at rest without field.  MHD_ERR_ARG if the side is not
 * an inflow side or rho, p are not positive and finite. */
int mhd_set_inflow(mhd_ctx* ctx, int patch, int side, const double* w);

/* Passive scalars: several gas components carried by the flow.  Each is a conserved
 * rho X advected with the Riemann mass flux of the step and the upwind X at each face
 * (X_L where the mass flux is >= 0, else X_R), X = (rho X)/rho reconstructed like the
 * primitives (donor cell in the predictor, the patch's kappa-scheme in the corrector,
 * without the positivity fallback), accumulated in FP64; they do not act on the flow. */
#define MHD_MAX_SCALARS 8

/* n scalars (0 <= n <= MHD_MAX_SCALARS; 0 removes them) on every patch, all rho X = 0.
 * MHD_ERR_STATE on a context made with MHD_FLAG_PERSISTENT (that step carries none). */
int mhd_set_scalars(mhd_ctx* ctx, int n);

/* rho X of one patch, dense [n][nz][ny][nx] (access as mhd_set_state / mhd_get_state).
 * MHD_ERR_STATE without scalars.  The get synchronises. */
int mhd_set_scalar_state(mhd_ctx* ctx, int patch, const double* S, int on_device);
int mhd_get_scalar_state(mhd_ctx* ctx, int patch, double* S_out, int on_device);

/* X (n values, host array) beyond an inflow side of a patch (default 0). */
int mhd_set_inflow_scalars(mhd_ctx* ctx, int patch, int side, const double* X);

/* Advance every patch by one van Leer step (Eq. 7, Eq. 8).  dt > 0: that dt for
 * every patch.  dt <= 0: each patch uses cfl * its own CFL limit of its current
 * state, computed on the device (no host synchronisation).  Asynchronous.
 * Runs are bitwise reproducible: a state read out with mhd_get_state and set back
 * with mhd_set_state continues exactly as the uninterrupted run. */
int mhd_step(mhd_ctx* ctx, double dt);

/* cfl * min over all patches, cells and active axes of d/(|v_d| + c_fast,d) for the
 * current state: bit for bit the dt that mhd_step(ctx, -1) takes next (for one patch;
 * with several, each patch takes its own, mhd_cfl_dt_patches).  Synchronises the
 * stream. */
int mhd_cfl_dt(mhd_ctx* ctx, double* dt_out);

/* Per-patch CFL time steps, n_patches values.  Synchronises. */
int mhd_cfl_dt_patches(mhd_ctx* ctx, double* dt_out);

/* Copy the state of one patch out (host format above; on_device as in init).  A kernel
 * writes the caller's arrays directly when the device can address them: device memory,
 * or page-locked host memory mapped into the device's address space (cudaHostAlloc;
 * pinned PyTorch tensors are), in which case the data cross the host link from the
 * kernel's stores.  Other host memory is filled from a device staging buffer by one copy
 * per array.  Synchronises; the arrays are complete on return. */
int mhd_get_state(mhd_ctx* ctx, int patch, double* U_out, double* Bface_out, int on_device);

/* Replace the state of one patch (same format; same direct or staged access as
 * mhd_get_state).  Used for resume and for end-to-end runs that stream each step's input
 * from the host.  Asynchronous: the caller keeps the arrays unchanged until the stream
 * has passed this call (mhd_sync, or any synchronising call). */
int mhd_set_state(mhd_ctx* ctx, int patch, const double* U, const double* Bface, int on_device);

/* Wait for all issued work and return the device error status. */
int mhd_sync(mhd_ctx* ctx);

int mhd_get_metrics(mhd_ctx* ctx, mhd_metrics* out);

/* Number of kernel launches the library issued since the context was created
 * (graph replays count the kernels inside the graph). */
long long mhd_launch_count(const mhd_ctx* ctx);

/* Set the thermal source term (default off).  Thermal cells are applied after each step
 * with that step's dt of the patch. */
int mhd_set_thermal(mhd_ctx* ctx, const mhd_thermal_desc* th);

/* Thermal counters since the thermal term was first set: out4[0] cells integrated,
 * [1] backward-Euler sub-steps, [2] cells that hit a sub-step or Newton cap,
 * [3] surrogate cells that fell back to the plain integrator.  Synchronises. */
int mhd_thermal_stats(mhd_ctx* ctx, unsigned long long* out4);

/* Surrogate of the thermal source (a 4 -> 64 -> 64 -> 1 tanh network on x = (log10 n_H,
 * log10 T, log10 dt, Z) mapped to [-1, 1] by the training range; the 64x64 layer on BF16
 * tensor cores with FP32 accumulation).  The network predicts q, the change of log10 T
 * over dt in units of S = D / (1 + |D|), where D = rate(T) dt / (T ln 10) is the explicit
 * estimate of the change, rate = (n_H Gamma - n_H^2 Lambda(T, Z)) / (rate_unit c_e), both
 * evaluated in FP32 at x; the change applied is q S.  (Small changes: S ~ D and the error is
 * relative to the change; stiff cells: |S| -> 1 and q is the change itself.)  A cell falls
 * back to the plain integrator when a standardised input leaves [-1, 1], when |q| > qmax,
 * or when |q S| > dmax or is not finite.  Harvested rows are 6 floats (log10 n_H, log10 T,
 * log10 dt, Z, q, change) with q clipped to [-8, 8] (q = 1 where S is 0).
 *
 * mhd_surrogate_harvest: while the thermal mode is MHD_THERMAL_PLAIN, record training pairs
 * from the plain integrator into a device ring of `capacity` rows, from about one cell in
 * `stride` per step (a hash of the cell index salted by the step's dt).  Each sampled cell
 * gives four rows: its own (n_H, T, dt) pair and three pairs integrated again at n_H, T and dt
 * each shifted by an independent hashed offset uniform in [-0.5, 0.5] decades (c_e scaled with
 * n_H), so that the training set covers a neighbourhood of the visited states.  capacity 0
 * stops.
 *
 * mhd_surrogate_train: train on the harvested pairs on the GPU: MSE loss, Adam (beta1 0.9,
 * beta2 0.999) on FP32 master weights with the learning rate decayed from lr to lr/20 on a
 * cosine, minibatches of `batch` rows drawn with a hash of (seed, step, row), `epochs`
 * passes of rows/batch steps, weights initialised from seed.
 * qmax > 0 is the fallback bound on the predicted |q|; qmax <= 0 takes 1.25 times the
 * largest |q| in the training set.  dmax is 1.25 times the largest |change| there.  loss_out receives the mean squared error of the
 * last epoch, rows_out the number of training rows (either may be NULL).  Harvesting stops.
 *
 * mhd_surrogate_params: copy the FP32 parameters out (4545 floats: W1[64][4], b1[64],
 * W2[64][64], b2[64], w3[64], b3) and, if range_out is not NULL, 10 floats: the input
 * offsets lo[4], scales s[4] (x_s = (x - lo) s - 1), qmax and dmax.
 *
 * mhd_surrogate_rows: copy up to max_rows harvested rows (6 floats each, in ring order) to
 * the host buffer rows_out; count_out (may be NULL) receives the number of rows held.
 * MHD_ERR_STATE if harvesting was never set up.  Synchronises the context's stream.
 *
 * mhd_surrogate_fallback_cells: the cells that the last surrogate thermal phase (of the
 * context's last patch) handed to the plain integrator, as interior cell indices
 * i + nx (j + ny k) in no particular order: up to max_cells of them into the host buffer
 * cells_out; count_out (may be NULL) receives how many there were.  MHD_ERR_STATE before the
 * first surrogate phase.  Synchronises the context's stream.  A diagnostic of the fallback
 * rule (Section 3.10 stand-in; the paper has no surrogate). */
int mhd_surrogate_harvest(mhd_ctx* ctx, long long capacity, int stride);
int mhd_surrogate_train(mhd_ctx* ctx, int epochs, int batch, double lr, unsigned long long seed, double qmax,
                        double* loss_out, long long* rows_out);
int mhd_surrogate_params(mhd_ctx* ctx, float* params_out, float* range_out);
int mhd_surrogate_rows(mhd_ctx* ctx, float* rows_out, long long max_rows, long long* count_out);
int mhd_surrogate_fallback_cells(mhd_ctx* ctx, int* cells_out, long long max_cells, long long* count_out);

/* Per-kernel timing.  While on, every launch is bracketed by a CUDA event pair on the
 * context's stream (steps are not replayed from a graph) and the elapsed times are summed
 * per kernel class: 0 recovery+CFL, 1-3 donor-cell HLLD fluxes x/y/z, 4-6 kappa-scheme
 * HLLD fluxes x/y/z, 7 corner EMFs, 8 update, 9 standalone CFL, 10 persistent step,
 * 11 thermal source, 12 end-of-step floors, 13 ghost W fill, 14 corner EMFs fused with the
 * update (patches with three active axes; they launch no class 7 or 8 kernel), 15 passive
 * scalars.  Switching on or off clears the totals. */
int mhd_set_profiling(mhd_ctx* ctx, int on);

/* Totals since profiling was switched on: ms[c] milliseconds and launches[c] launches of
 * class c, for c < n (n >= 17).  Synchronises. */
int mhd_get_profile(mhd_ctx* ctx, double* ms, long long* launches, int n);

/* Autotuner of the batched step (context made with MHD_FLAG_PERSISTENT; a schedule, not part
 * of the paper's method).  It times the
 * persistent step for each candidate tile shape (TX x TY points of one z-plane per CTA) and
 * CTA count per SM and keeps the fastest; then it times that persistent step against the
 * per-phase scheme (each patch's kernels as one chain on one of up to eight streams) over
 * three whole steps from the same state, and the context runs its steps with the faster
 * scheme from then on (mhd_step_scheme tells which; passive scalars only run per phase).
 * The result is recorded in a JSON cache file at cache_path, keyed by GPU name, precision
 * and patch sizes (NULL: no cache); force = 0 uses a cached entry without timing.  The state
 * is restored after the timing runs and captured graphs are dropped.  tile_out (may be NULL)
 * receives TX, TY.  MHD_ERR_STATE without MHD_FLAG_PERSISTENT. */
int mhd_autotune(mhd_ctx* ctx, const char* cache_path, int force, int* tile_out);

/* The scheme the context's steps run with (the schedule of the same step, Eq. 7-8, over a
 * batch of independent patches; the paper runs one grid per MPI rank and has no
 * counterpart): *persistent_out = 1 for one persistent launch per step
 * (MHD_FLAG_PERSISTENT, until mhd_autotune picks the per-phase scheme), 0 for per-phase
 * launches.  mhd_set_step_scheme chooses it: 1 needs MHD_FLAG_PERSISTENT and no passive
 * scalars (MHD_ERR_STATE otherwise); switching drops the captured graphs and the next step
 * starts with the recovery.  Both schemes advance the same state. */
int mhd_step_scheme(mhd_ctx* ctx, int* persistent_out);
int mhd_set_step_scheme(mhd_ctx* ctx, int persistent);

/* Bounded waits of the persistent step.  limit_ms: the longest a CTA waits at a grid
 * barrier before it sets the device error word to MHD_ERR_TIMEOUT and the launch ends
 * (default 2000).  phantom_blocks: CTAs that never arrive but that the barrier also waits
 * for (default 0; a positive value makes every wait run out, which exercises the timeout
 * path without faulting or hanging the GPU). */
int mhd_set_wait_limit(mhd_ctx* ctx, double limit_ms, int phantom_blocks);

const char* mhd_last_error(const mhd_ctx* ctx);

void mhd_destroy(mhd_ctx* ctx);

/* The unit-level entries below (mhd_riemann_hlld, mhd_riemann_flux, mhd_thermal_cells,
 * mhd_mlp_forward[_tc], mhd_convert_fp) accept n = 0, launch nothing and then allow NULL
 * array pointers; n < 0 is MHD_ERR_ARG.  mhd_mlp_grad[_tc] need 1 <= n <= 2^20. */

/* Unit-level entry for parity tests: HLLD fluxes (Miyoshi & Kusano 2005, the solver
 * named in Section 2.1) of n interfaces in the interface frame, computed by the
 * same device function the step uses.  wl, wr: n*8 values [rho, vn, vt1, vt2, p,
 * unused, Bt1, Bt2]; bn: n normal fields; flux: n*8 outputs [rho, mn, mt1, mt2, E,
 * 0, Bt1, Bt2].  All four are device pointers; precision MHD_PREC_FP64 computes in
 * FP64, MHD_PREC_MIXED in FP32 (inputs/outputs stay FP64).  stream may be NULL. */
int mhd_riemann_hlld(int n, const double* wl, const double* wr, const double* bn, double gamma,
                     int precision, double* flux, void* stream);

/* The same for the solver MHD_RIEMANN_* (MHD_RIEMANN_HLLC: HLLD at faces with a field). */
int mhd_riemann_flux(int solver, int n, const double* wl, const double* wr, const double* bn, double gamma,
                     int precision, double* flux, void* stream);

/* Unit-level entry for parity tests: the plain FP64 thermal integrator of
 * MHD_THERMAL_PLAIN on n independent cells (device pointers): temperature T0 [K],
 * n_H [cm^-3], c_e (code energy density per K), dt (code time) -> T_out, and per-cell
 * status bits (1 sub-step cap, 2 Newton cap, 4 no bracket; status may be NULL).
 * d->mode is ignored.  Synchronises stream (NULL allowed). */
int mhd_thermal_cells(long long n, const double* T0, const double* nh, const double* ce, const double* dt,
                      const mhd_thermal_desc* d, double* T_out, int* status, void* stream);

/* Unit-level entries for parity tests of the surrogate kernels (device pointers; params
 * in the layout of mhd_surrogate_params; inputs already in [-1, 1]):
 * mhd_mlp_forward: y[n] for xs[n][4].
 * mhd_mlp_grad: gradient (4545 floats) of the mean squared error over rows[n][6] in the
 * harvested-row layout (x0..x3, target, one column the gradient ignores) and the sum of
 * squared errors in *loss_sum.  Synchronise stream. */
int mhd_mlp_forward(long long n, const float* xs, const float* params, float* y, void* stream);
/* The same forward pass with the 64x64 layer on tcgen05 tensor cores (TMEM accumulator);
 * MHD_ERR_TIMEOUT if the bounded wait for the MMA ran out. */
int mhd_mlp_forward_tc(long long n, const float* xs, const float* params, float* y, void* stream);
int mhd_mlp_grad(long long n, const float* rows, const float* params, float* grad, float* loss_sum, void* stream);
/* The same gradient with the three 64-wide products of the backward pass (Z2 = H1 W2^T,
 * dH1 = dZ2 W2, dW2 = dZ2^T H1) on tcgen05 tensor cores, 128 rows per CTA; the kernel
 * mhd_surrogate_train uses.  MHD_ERR_TIMEOUT if a bounded wait for the MMAs ran out. */
int mhd_mlp_grad_tc(long long n, const float* rows, const float* params, float* grad, float* loss_sum,
                    void* stream);

/* Unit-level entry for a parity test of the mixed path's FP64 <-> FP32 conversions (the
 * precision split's plumbing; the paper has none), which run on the integer pipe: for n
 * elements of device arrays, d2f_out = d_in rounded to FP32 (nearest, ties to even; a
 * result below the smallest normal float becomes a signed zero; overflow gives inf; NaN a
 * quiet NaN) and f2d_out = f_in widened exactly (subnormal floats become a signed zero).
 * Synchronises stream. */
int mhd_convert_fp(long long n, const double* d_in, const float* f_in, float* d2f_out, double* f2d_out,
                   void* stream);

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
 *              d / (|v_d| + c_fast,d), computed in FP64 as mhd_cfl_dt of an FP64 context
 *              without floors (density and pressure floors set by mhd_set_sources are
 *              not applied here).  If any cell has rho <= 0, p <= 0 or a non-finite
 *              value, *dt_out is NaN: the call is asynchronous, so the failure that
 *              mhd_cfl_dt returns as a status arrives here in the result.
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
