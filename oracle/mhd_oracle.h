/*
 * mhd_oracle.h -- plain, slow FP64 CPU oracle of the magneto-gas-dynamics step of
 * Khoperskov, Vasiliev, Khoperskov & Lubimov (arXiv:1502.02935), Section 2.1.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call
 * this file; only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * --impl reference legs use it.  It shares no code with the CUDA library.
 *
 * State format (identical to the library's host format, so both can be fed the
 * same arrays):
 *   U     : 5 cell fields [rho, rho*vx, rho*vy, rho*vz, E], each nz*ny*nx, x fastest.
 *   Bx    : (nz, ny, nx+1) x-face values, Bx[k][j][i] sits on face x_{i-1/2}.
 *   By    : (nz, ny+1, nx) y-face values on y_{j-1/2}.
 *   Bz    : (nz+1, ny, nx) z-face values on z_{k-1/2}.
 * For periodic axes and for trivial axes (n == 1) the last face layer repeats
 * the first one.
 */
#ifndef MHD_ORACLE_H
#define MHD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Boundary conditions (Section 3 prose names free and inflow boundaries): periodic;
 * outflow = zero-gradient copy; inflow = a fixed state beyond the boundary. */
enum { ORC_BC_PERIODIC = 0, ORC_BC_OUTFLOW = 1, ORC_BC_INFLOW = 2 };
/* Riemann solver (Section 2.1: HLL or HLLC for pure gas dynamics, HLLD for MHD).
 * HLLC is the gas-dynamics solver: a face that carries a field (B_n or a transverse
 * component non-zero on either side) takes HLLD, which is HLLC when B = 0. */
enum { ORC_RIEMANN_HLLD = 0, ORC_RIEMANN_HLLC = 1, ORC_RIEMANN_HLL = 2 };
/* Reconstruction of Eq. 12-14: kappa = 1/3 (third-order upwind biased, the paper's
 * choice), 0 (second-order upwind biased), -1 (second-order fully upwind), in the
 * standard compressive kappa-scheme arrangement; and kappa = 1/3 in the arrangement of
 * K1, K2 and b exactly as printed (a cross-check of that reading; second order only). */
enum { ORC_RECON_KAPPA_THIRD = 0, ORC_RECON_KAPPA_ZERO = 1, ORC_RECON_KAPPA_UPWIND = 2,
       ORC_RECON_PRINTED = 3 };
enum { ORC_POT_NONE = 0, ORC_POT_GAUSS_X = 1, ORC_POT_LOG_DISC = 2 };

typedef struct {
  int nx, ny, nz;
  double x0, y0, z0;   /* coordinate of the low face of cell 0 along each axis */
  double dx, dy, dz;
  int bc[6];           /* x-lo, x-hi, y-lo, y-hi, z-lo, z-hi */
  double gamma;
  int riemann;         /* ORC_RIEMANN_* (0: HLLD) */
  int recon;           /* ORC_RECON_* (0: kappa = 1/3) */
  /* primitive state [rho, vx, vy, vz, p, Bx, By, Bz] beyond each side whose bc is
   * ORC_BC_INFLOW (same side order as bc) */
  double inflow[6][8];
  /* Eq. 11 takes the mean of the two one-sided EMF derivatives where the face's mass flux
   * is zero; here: where |F_rho| <= upwind_eps * rho_max * max|S|.  0 takes 2^-32, zero to
   * the precision of FP64 data after the pressure recovery's cancellation; 64 * 2^-23 is
   * the same reading for data rounded to FP32. */
  double upwind_eps;
} orc_patch;

typedef struct {
  int potential;
  double psi0, xc, xw; /* Gaussian well Psi = -psi0 exp(-((x-xc)/xw)^2) (bow-shock test) */
  double v0, rc;       /* logarithmic potential Psi = v0^2/2 ln(x^2+y^2+rc^2+z^2) */
  /* Floors (the paper states none; reading for the disc run).  rho_floor > 0 turns them
   * on: the primitive recovery uses rho_f = max(rho, rho_floor) and clamps p to
   * [rho_f pr_floor, rho_f pr_ceil]; after each full step every interior cell gets
   * rho' = max(rho, rho_floor), momentum kept, p recomputed with rho' and clamped the
   * same way, E rebuilt from them.  pr_ceil <= 0: no ceiling. */
  double rho_floor, pr_floor, pr_ceil;
} orc_source;

/* One van Leer predictor-corrector step of size dt (Eq. 7, Eq. 8).  Arrays are
 * updated in place.  Returns the number of interior cells the end-of-step floors
 * changed (0 with floors off), or -1 on bad arguments. */
int orc_step(const orc_patch* p, const orc_source* s, double* U, double* Bx,
             double* By, double* Bz, double dt);

/* One step of orc_step that also advects ns passive scalars (multi-species gas carried by
 * the flow): S holds the conserved rho X_s, [ns][nz][ny][nx], updated in place.  Their
 * face flux is the Riemann mass flux times the upwind X (X_L where the mass flux is >= 0,
 * else X_R), X = (rho X)/rho reconstructed like the primitives (donor cell in the
 * predictor, the patch's kappa-scheme in the corrector, without the positivity fallback).
 * inflow_x[side * ns + s] is X beyond an inflow side (may be NULL: 0).  Returns as
 * orc_step. */
int orc_step_scalars(const orc_patch* p, const orc_source* s, double* U, double* Bx, double* By,
                     double* Bz, int ns, double* S, const double* inflow_x, double dt);

/* The corner EMFs E_x, E_y, E_z of one stage (Eq. 9-11) for the state given: order 1 is
 * the predictor's donor-cell stage, order 2 the corrector's reconstruction.  E holds
 * [3][nz][ny][nx]; E[c] at cell (i, j, k) is the edge along c at the cell's low corner
 * (E_z at (i-1/2, j-1/2, k)).  The state is not changed.  Returns 0, or -1 on bad arguments. */
int orc_stage_emf(const orc_patch* p, const double* U, const double* Bx, const double* By,
                  const double* Bz, int order, double* E);

/* cfl * min over interior cells and active axes of d/(|v_d| + c_f,d), from the
 * recovered primitives (with the floors of s when s is not NULL). */
double orc_cfl_dt(const orc_patch* p, const orc_source* s, const double* U, const double* Bx,
                  const double* By, const double* Bz, double cfl);

/* Advance to t_end with CFL steps (the last one clipped so t_end is hit).
 * Returns the number of steps taken (max_steps caps it), -1 on bad arguments. */
int orc_run(const orc_patch* p, const orc_source* s, double* U, double* Bx,
            double* By, double* Bz, double cfl, double t_end, int max_steps);

/* HLLD flux (Miyoshi & Kusano 2005) for a batch of n interfaces, in the frame of
 * the interface normal: w = [rho, vn, vt1, vt2, p, (unused), Bt1, Bt2], bn = normal
 * field.  flux = [rho, mn, mt1, mt2, E, 0, Bt1, Bt2] fluxes, 8 per interface. */
void orc_hlld_batch(int n, const double* wl, const double* wr, const double* bn,
                    double gamma, double* flux);

/* The same for the solver ORC_RIEMANN_* (HLLC: HLLD at faces with a field). */
void orc_riemann_batch(int solver, int n, const double* wl, const double* wr, const double* bn,
                       double gamma, double* flux);

/* kappa = 1/3 compressive minmod reconstruction on a 1D array of n values:
 * for interfaces m = 2..n-2 (between w[m-1] and w[m]) writes wl[m], wr[m]. */
void orc_reconstruct_1d(int n, const double* w, double* wl, double* wr);

/* The same for the reconstruction ORC_RECON_*. */
void orc_reconstruct_1d_ex(int recon, int n, const double* w, double* wl, double* wr);

/* Total over the interior of the 5 cell fields (fixed order) and the maximum of
 * |div B| * min(d) over interior cells. */
void orc_diagnostics(const orc_patch* p, const double* U, const double* Bx,
                     const double* By, const double* Bz, double sums[5],
                     double* max_divb);

/* Number of OpenMP threads used by the step (1 when built without OpenMP). */
int orc_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
