/*
 * mhd_oracle.c -- plain FP64 CPU oracle of the TVD-MUSCL magneto-gas-dynamics step
 * of arXiv:1502.02935, Section 2.1.  TEST INFRASTRUCTURE ONLY (see mhd_oracle.h).
 *
 * Written for a reader who checks it against the paper by eye: ghost-padded arrays,
 * one loop nest per operation, no fusion, no blocking, FP64 throughout, built with
 * -ffp-contract=off.  Each function cites the passage it follows.  Where the paper
 * is garbled or silent the reading taken is stated at the function.
 *
 *   conserved vector U ........................ Eq. 1
 *   conservation law with sources S ............ Eq. 2
 *   fluxes F, G, H, P* = P + B^2/2, E closure .. Eq. 3 and the text after it
 *   face-centred B, cell-centred gas ........... Eq. 4, Eq. 5
 *   cell-centred B as face average ............. Eq. 6
 *   finite-volume update with n+1/2 fluxes ..... Eq. 7
 *   constrained-transport induction ............ Eq. 8 (second bracket read as E_y)
 *   E = -v x B ................................. Eq. 9
 *   corner EMF with upwinded derivatives ....... Eq. 10, Eq. 11
 *   HLLD Riemann solver ........................ Section 2.1 (Miyoshi & Kusano 2005)
 *   kappa = 1/3 minmod MUSCL of primitives ..... Eq. 12-14
 * Time integration: the "time- and area-averaged fluxes at n+1/2" of Eq. 7 are
 * obtained with the two-stage van Leer predictor-corrector (donor-cell half step,
 * then MUSCL full step), the unsplit CT scheme of the Athena code that the paper
 * compares against in Section 3.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "mhd_oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

enum { RHO = 0, MX = 1, MY = 2, MZ = 3, EN = 4, BXF = 5, BYF = 6, BZF = 7, NF = 8 };
/* primitive vector W: rho, vx, vy, vz, p, Bx, By, Bz (cell-centred B) */
enum { WR = 0, WVX = 1, WVY = 2, WVZ = 3, WP = 4, WBX = 5, WBY = 6, WBZ = 7 };

#define GHOST 3

/* Default width of Eq. 11's "no contact motion" band, relative to the face's mass-flux
 * scale (see the corner EMFs below). */
#define UPWIND_EPS_FP64 (1.0 / 4294967296.0)

typedef struct {
  int n[3];     /* interior cells */
  int g[3];     /* ghost layers (GHOST on active axes, 0 on trivial ones) */
  int N[3];     /* padded extent n + 2g + 1 (the +1 holds the high face) */
  int act[3];   /* axis active (n > 1) */
  int per[3];   /* periodic (trivial axes count as periodic with n = 1) */
  double d[3], lo[3], gamma;
  int riemann; /* ORC_RIEMANN_* */
  int recon;   /* ORC_RECON_* */
  double upwind_eps; /* width of Eq. 11's "no contact motion" band, relative to sigma */
  int inflow[6];           /* side has an inflow boundary */
  double in_u[6][NF];      /* its state: conserved cell fields and the three field components */
  double in_w[6][NF];      /* and its primitives rho, vx, vy, vz, p, Bx, By, Bz */
  long tot;
  int floors;                         /* floors on (rho_floor > 0) */
  double rho_floor, pr_floor, pr_ceil; /* pr_ceil = +inf when no ceiling is set */
} grid;

static long ix(const grid* G, int i, int j, int k) {
  return (long)(i + G->g[0]) +
         (long)G->N[0] * ((long)(j + G->g[1]) + (long)G->N[1] * (long)(k + G->g[2]));
}

static long ixv(const grid* G, const int c[3]) { return ix(G, c[0], c[1], c[2]); }

static int make_grid(const orc_patch* p, grid* G) {
  int n[3] = {p->nx, p->ny, p->nz};
  double d[3] = {p->dx, p->dy, p->dz}, lo[3] = {p->x0, p->y0, p->z0};
  G->tot = 1;
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 1 || !(d[a] > 0)) return -1;
    G->n[a] = n[a];
    G->act[a] = n[a] > 1;
    G->g[a] = G->act[a] ? GHOST : 0;
    G->N[a] = n[a] + 2 * G->g[a] + 1;
    int blo = p->bc[2 * a], bhi = p->bc[2 * a + 1];
    G->inflow[2 * a] = G->inflow[2 * a + 1] = 0;
    if (!G->act[a]) {
      G->per[a] = 1;
    } else {
      if ((blo == ORC_BC_PERIODIC) != (bhi == ORC_BC_PERIODIC)) return -1;
      if (blo < ORC_BC_PERIODIC || blo > ORC_BC_INFLOW || bhi < ORC_BC_PERIODIC || bhi > ORC_BC_INFLOW) return -1;
      G->per[a] = blo == ORC_BC_PERIODIC;
      G->inflow[2 * a] = blo == ORC_BC_INFLOW;
      G->inflow[2 * a + 1] = bhi == ORC_BC_INFLOW;
    }
    G->d[a] = d[a];
    G->lo[a] = lo[a];
    G->tot *= G->N[a];
  }
  if (!(p->gamma > 1.0)) return -1;
  G->gamma = p->gamma;
  if (p->riemann < ORC_RIEMANN_HLLD || p->riemann > ORC_RIEMANN_HLL) return -1;
  G->riemann = p->riemann;
  if (p->recon < ORC_RECON_KAPPA_THIRD || p->recon > ORC_RECON_PRINTED) return -1;
  G->recon = p->recon;
  if (!(p->upwind_eps >= 0.0) || !(p->upwind_eps < 1.0)) return -1;
  G->upwind_eps = p->upwind_eps > 0.0 ? p->upwind_eps : UPWIND_EPS_FP64;
  for (int side = 0; side < 6; ++side) {
    if (!G->inflow[side]) continue;
    const double* w = p->inflow[side];
    if (!(w[0] > 0.0) || !(w[4] > 0.0)) return -1;
    G->in_u[side][RHO] = w[0];
    G->in_u[side][MX] = w[0] * w[1];
    G->in_u[side][MY] = w[0] * w[2];
    G->in_u[side][MZ] = w[0] * w[3];
    G->in_u[side][EN] = w[4] / (G->gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) +
                        0.5 * (w[5] * w[5] + w[6] * w[6] + w[7] * w[7]);
    for (int m = 0; m < NF; ++m) G->in_w[side][m] = w[m];
    G->in_u[side][BXF] = w[5];
    G->in_u[side][BYF] = w[6];
    G->in_u[side][BZF] = w[7];
  }
  G->floors = 0;
  G->rho_floor = G->pr_floor = 0.0;
  G->pr_ceil = INFINITY;
  return 0;
}

/* Floors from the source description (reading: the paper states none). */
static void set_floors(grid* G, const orc_source* s) {
  if (!s || !(s->rho_floor > 0.0)) return;
  G->floors = 1;
  G->rho_floor = s->rho_floor;
  G->pr_floor = s->pr_floor > 0.0 ? s->pr_floor : 0.0;
  G->pr_ceil = s->pr_ceil > 0.0 ? s->pr_ceil : INFINITY;
}

static double clamp_p(const grid* G, double p, double rho) {
  double lo = rho * G->pr_floor, hi = rho * G->pr_ceil;
  return p < lo ? lo : (p > hi ? hi : p);
}

/* ---------------------------------------------------------------- boundaries --
 * The paper names boundary conditions only in prose (free outflow, inflow, Section
 * 3.3).  Reading: periodic wrap, or outflow = zero-gradient copy of the nearest
 * interior cell value (cell fields and transverse faces) and of the boundary face
 * (normal faces).  Boundary normal faces themselves are interior and CT-updated. */
static int src_index(const grid* G, int a, int v, int is_face_axis) {
  int n = G->n[a];
  if (G->per[a]) {
    int m = v % n;
    return m < 0 ? m + n : m;
  }
  if (v < 0) return 0;
  if (is_face_axis) return v > n ? n : v;
  return v > n - 1 ? n - 1 : v;
}

/* Inflow: a cell beyond an inflow side (the first such side in axis order) holds that
 * side's state, cell fields and the faces it owns alike; the boundary face itself (index
 * 0 or n along the axis) is a face of the domain and is CT-updated. */
static int inflow_side(const grid* G, const int c[3], int fa) {
  for (int a = 0; a < 3; ++a) {
    int hi = G->n[a] - 1 + (a == fa ? 1 : 0); /* last index inside along a */
    if (c[a] < 0 && G->inflow[2 * a]) return 2 * a;
    if (c[a] > hi && G->inflow[2 * a + 1]) return 2 * a + 1;
  }
  return -1;
}

static void fill_ghosts(const grid* G, double* const F[NF]) {
  for (int f = 0; f < NF; ++f) {
    int fa = f >= BXF ? f - BXF : -1; /* face axis of this field */
    double* q = F[f];
#pragma omp parallel for schedule(static)
    for (int kk = 0; kk < G->N[2]; ++kk)
      for (int jj = 0; jj < G->N[1]; ++jj)
        for (int ii = 0; ii < G->N[0]; ++ii) {
          int c[3] = {ii - G->g[0], jj - G->g[1], kk - G->g[2]};
          int side = inflow_side(G, c, fa);
          if (side >= 0) {
            q[ixv(G, c)] = G->in_u[side][f];
            continue;
          }
          int s[3];
          for (int a = 0; a < 3; ++a) s[a] = src_index(G, a, c[a], a == fa);
          if (s[0] == c[0] && s[1] == c[1] && s[2] == c[2]) continue;
          q[ixv(G, c)] = q[ixv(G, s)];
        }
  }
}

/* ------------------------------------------------------ primitive recovery --
 * Eq. 6: cell-centred B is the mean of the two face values.
 * Text after Eq. 3: E = P/(gamma-1) + rho v^2/2 + B^2/2, so
 * P = (gamma-1) (E - rho v^2/2 - B^2/2).
 * With floors on, rho is raised to rho_floor before v = m/rho, and P is clamped to
 * [rho pr_floor, rho pr_ceil]. */
static void cons_to_prim(const grid* G, double* const U[NF], double* const W[NF]) {
  double gm1 = G->gamma - 1.0;
#pragma omp parallel for schedule(static)
  for (int k = -G->g[2]; k < G->n[2] + G->g[2]; ++k)
    for (int j = -G->g[1]; j < G->n[1] + G->g[1]; ++j)
      for (int i = -G->g[0]; i < G->n[0] + G->g[0]; ++i) {
        {
          /* a cell beyond an inflow side holds the side's primitive state */
          int cc[3] = {i, j, k};
          int side = inflow_side(G, cc, -1);
          if (side >= 0) {
            long c0 = ix(G, i, j, k);
            for (int m = 0; m < NF; ++m) W[m][c0] = G->in_w[side][m];
            continue;
          }
        }
        long c = ix(G, i, j, k);
        double rho = U[RHO][c];
        if (G->floors && rho < G->rho_floor) rho = G->rho_floor;
        double vx = U[MX][c] / rho, vy = U[MY][c] / rho, vz = U[MZ][c] / rho;
        double bx = 0.5 * (U[BXF][c] + U[BXF][ix(G, i + 1, j, k)]);
        double by = 0.5 * (U[BYF][c] + U[BYF][ix(G, i, j + 1, k)]);
        double bz = 0.5 * (U[BZF][c] + U[BZF][ix(G, i, j, k + 1)]);
        double kin = 0.5 * rho * (vx * vx + vy * vy + vz * vz);
        double mag = 0.5 * (bx * bx + by * by + bz * bz);
        W[WR][c] = rho;
        W[WVX][c] = vx;
        W[WVY][c] = vy;
        W[WVZ][c] = vz;
        double p = gm1 * (U[EN][c] - kin - mag);
        W[WP][c] = G->floors ? clamp_p(G, p, rho) : p;
        W[WBX][c] = bx;
        W[WBY][c] = by;
        W[WBZ][c] = bz;
      }
}

/* ------------------------------------------------------------------ HLLD ----
 * Section 2.1 names HLLD for magneto-gas dynamics and refers to Miyoshi & Kusano
 * (2005, JCP 208, 315) for it.  The steps below follow that paper:
 *   fast speed c_f^2 = [gp + B^2 + sqrt((gp + B^2)^2 - 4 gp Bn^2)] / (2 rho);
 *   outer speeds S_L = min(uL,uR) - max(cfL,cfR), S_R = max(uL,uR) + max(cfL,cfR);
 *   contact speed S_M and star total pressure from the HLL jump conditions;
 *   single-star states across S_L, S_R; Alfven speeds S*_{L,R} = S_M -/+ |Bn|/sqrt(rho*);
 *   double-star states as sqrt(rho*)-weighted averages;
 *   flux picked by the sign of S_L, S*_L, S_M, S*_R, S_R (ties: S_L > 0 -> F_L,
 *   S*_L >= 0 -> F*_L, S_M >= 0 -> F**_L, S*_R >= 0 -> F**_R, S_R >= 0 -> F*_R, else F_R).
 * Reading of the degenerate case (Bn^2 = rho (S-u)(S-S_M)): when that denominator is
 * below 1e-8 of the sum of the magnitudes of its two terms, the transverse velocity
 * and field keep their outer values.
 * w = [rho, un, ut1, ut2, p, -, Bt1, Bt2] in the interface frame. */
#define HLLD_DEGEN 1e-8

static double fast_speed(double rho, double p, double bn, double bt1, double bt2, double gam) {
  double gp = gam * p;
  double b2 = bn * bn + bt1 * bt1 + bt2 * bt2;
  double disc = (gp + b2) * (gp + b2) - 4.0 * gp * bn * bn;
  if (disc < 0.0) disc = 0.0;
  return sqrt((gp + b2 + sqrt(disc)) / (2.0 * rho));
}

/* conserved state in the interface frame */
static void frame_cons(const double* w, double bn, double gam, double* u) {
  double rho = w[0], un = w[1], v1 = w[2], v2 = w[3], p = w[4], b1 = w[6], b2 = w[7];
  u[0] = rho;
  u[1] = rho * un;
  u[2] = rho * v1;
  u[3] = rho * v2;
  u[4] = p / (gam - 1.0) + 0.5 * rho * (un * un + v1 * v1 + v2 * v2) +
         0.5 * (bn * bn + b1 * b1 + b2 * b2);
  u[5] = bn;
  u[6] = b1;
  u[7] = b2;
}

/* Eq. 3 (F column) in the interface frame */
static void frame_flux(const double* w, double bn, double gam, double* f) {
  double rho = w[0], un = w[1], v1 = w[2], v2 = w[3], p = w[4], b1 = w[6], b2 = w[7];
  double pstar = p + 0.5 * (bn * bn + b1 * b1 + b2 * b2);
  double e = p / (gam - 1.0) + 0.5 * rho * (un * un + v1 * v1 + v2 * v2) +
             0.5 * (bn * bn + b1 * b1 + b2 * b2);
  double vb = un * bn + v1 * b1 + v2 * b2;
  f[0] = rho * un;
  f[1] = rho * un * un + pstar - bn * bn;
  f[2] = rho * un * v1 - bn * b1;
  f[3] = rho * un * v2 - bn * b2;
  f[4] = (e + pstar) * un - vb * bn;
  f[5] = 0.0;
  f[6] = b1 * un - bn * v1;
  f[7] = b2 * un - bn * v2;
}

/* flux[5] (the normal-field flux, identically zero) returns the face's mass-flux
 * scale max(rho_L, rho_R) * max(|S_L|, |S_R|), used by the corner-EMF upwinding. */
static void hlld(const double* wl, const double* wr, double bn, double gam, double* flux) {
  double UL[8], UR[8], FL[8], FR[8];
  frame_cons(wl, bn, gam, UL);
  frame_cons(wr, bn, gam, UR);
  frame_flux(wl, bn, gam, FL);
  frame_flux(wr, bn, gam, FR);

  double rl = wl[0], ul = wl[1], pl = wl[4];
  double rr = wr[0], ur = wr[1], pr = wr[4];
  double ptl = pl + 0.5 * (bn * bn + wl[6] * wl[6] + wl[7] * wl[7]);
  double ptr = pr + 0.5 * (bn * bn + wr[6] * wr[6] + wr[7] * wr[7]);
  double cfl = fast_speed(rl, pl, bn, wl[6], wl[7], gam);
  double cfr = fast_speed(rr, pr, bn, wr[6], wr[7], gam);
  double cmax = cfl > cfr ? cfl : cfr;
  double sl = (ul < ur ? ul : ur) - cmax;
  double sr = (ul > ur ? ul : ur) + cmax;

  double sigma = (rl > rr ? rl : rr) * (fabs(sl) > fabs(sr) ? fabs(sl) : fabs(sr));
  if (sl > 0.0) {
    memcpy(flux, FL, sizeof FL);
    flux[5] = sigma;
    return;
  }
  if (sr < 0.0) {
    memcpy(flux, FR, sizeof FR);
    flux[5] = sigma;
    return;
  }

  /* contact speed and star total pressure (M&K Eq. 38 and Eq. 41) */
  double dl = sl - ul, dr = sr - ur;
  double den = dr * rr - dl * rl;
  double sm = (dr * rr * ur - dl * rl * ul - ptr + ptl) / den;
  double pts = (dr * rr * ptl - dl * rl * ptr + rl * rr * dr * dl * (ur - ul)) / den;

  /* single-star states (M&K Eq. 43-48) */
  double US[2][8];
  double rs[2], vs1[2], vs2[2], bs1[2], bs2[2];
  const double* w[2] = {wl, wr};
  const double* Uo[2] = {UL, UR};
  double S[2] = {sl, sr};
  for (int s = 0; s < 2; ++s) {
    double rho = w[s][0], un = w[s][1], v1 = w[s][2], v2 = w[s][3];
    double b1 = w[s][6], b2 = w[s][7];
    double ds = S[s] - un;
    rs[s] = rho * ds / (S[s] - sm);
    double t1 = rho * ds * (S[s] - sm);
    double denom = t1 - bn * bn;
    if (fabs(denom) < HLLD_DEGEN * (fabs(t1) + bn * bn)) {
      vs1[s] = v1;
      vs2[s] = v2;
      bs1[s] = b1;
      bs2[s] = b2;
    } else {
      vs1[s] = v1 - bn * b1 * (sm - un) / denom;
      vs2[s] = v2 - bn * b2 * (sm - un) / denom;
      bs1[s] = b1 * (rho * ds * ds - bn * bn) / denom;
      bs2[s] = b2 * (rho * ds * ds - bn * bn) / denom;
    }
    double vb = un * bn + v1 * b1 + v2 * b2;
    double vbs = sm * bn + vs1[s] * bs1[s] + vs2[s] * bs2[s];
    double es = (ds * Uo[s][4] - (s == 0 ? ptl : ptr) * un + pts * sm + bn * (vb - vbs)) /
                (S[s] - sm);
    US[s][0] = rs[s];
    US[s][1] = rs[s] * sm;
    US[s][2] = rs[s] * vs1[s];
    US[s][3] = rs[s] * vs2[s];
    US[s][4] = es;
    US[s][5] = bn;
    US[s][6] = bs1[s];
    US[s][7] = bs2[s];
  }

  /* Alfven (rotational) speeds (M&K Eq. 51) */
  double sqrl = sqrt(rs[0]), sqrr = sqrt(rs[1]);
  double ssl = sm - fabs(bn) / sqrl;
  double ssr = sm + fabs(bn) / sqrr;

  /* double-star states (M&K Eq. 59-63) */
  double sgn = bn > 0.0 ? 1.0 : (bn < 0.0 ? -1.0 : 0.0);
  double isum = 1.0 / (sqrl + sqrr);
  double vss1 = (sqrl * vs1[0] + sqrr * vs1[1] + (bs1[1] - bs1[0]) * sgn) * isum;
  double vss2 = (sqrl * vs2[0] + sqrr * vs2[1] + (bs2[1] - bs2[0]) * sgn) * isum;
  double bss1 = (sqrl * bs1[1] + sqrr * bs1[0] + sqrl * sqrr * (vs1[1] - vs1[0]) * sgn) * isum;
  double bss2 = (sqrl * bs2[1] + sqrr * bs2[0] + sqrl * sqrr * (vs2[1] - vs2[0]) * sgn) * isum;
  double vbss = sm * bn + vss1 * bss1 + vss2 * bss2;
  double USS[2][8];
  for (int s = 0; s < 2; ++s) {
    double vbs = sm * bn + vs1[s] * bs1[s] + vs2[s] * bs2[s];
    double sq = s == 0 ? sqrl : sqrr;
    double ess = s == 0 ? US[0][4] - sq * (vbs - vbss) * sgn : US[1][4] + sq * (vbs - vbss) * sgn;
    USS[s][0] = rs[s];
    USS[s][1] = rs[s] * sm;
    USS[s][2] = rs[s] * vss1;
    USS[s][3] = rs[s] * vss2;
    USS[s][4] = ess;
    USS[s][5] = bn;
    USS[s][6] = bss1;
    USS[s][7] = bss2;
  }

  /* F*_a = F_a + S_a (U*_a - U_a);  F**_a = F*_a + S*_a (U**_a - U*_a)  (M&K Eq. 64-65) */
  double fs[8];
  if (ssl >= 0.0) {
    for (int m = 0; m < 8; ++m) flux[m] = FL[m] + sl * (US[0][m] - UL[m]);
  } else if (sm >= 0.0) {
    for (int m = 0; m < 8; ++m) {
      fs[m] = FL[m] + sl * (US[0][m] - UL[m]);
      flux[m] = fs[m] + ssl * (USS[0][m] - US[0][m]);
    }
  } else if (ssr >= 0.0) {
    for (int m = 0; m < 8; ++m) {
      fs[m] = FR[m] + sr * (US[1][m] - UR[m]);
      flux[m] = fs[m] + ssr * (USS[1][m] - US[1][m]);
    }
  } else {
    for (int m = 0; m < 8; ++m) flux[m] = FR[m] + sr * (US[1][m] - UR[m]);
  }
  flux[5] = sigma;
}

/* HLL (Harten, Lax & van Leer), one of the two gas-dynamics solvers of Section 2.1: the
 * single averaged state between the outer waves S_L, S_R (the estimate above; with a field
 * the fast speeds make it the two-wave MHD solver), from the integral form of the
 * conservation law over the fan:
 *   F = F_L (S_L > 0),  F_R (S_R < 0),  else
 *   F = [S_R F_L - S_L F_R + S_L S_R (U_R - U_L)] / (S_R - S_L). */
static void hll(const double* wl, const double* wr, double bn, double gam, double* flux) {
  double UL[8], UR[8], FL[8], FR[8];
  frame_cons(wl, bn, gam, UL);
  frame_cons(wr, bn, gam, UR);
  frame_flux(wl, bn, gam, FL);
  frame_flux(wr, bn, gam, FR);
  double rl = wl[0], ul = wl[1], rr = wr[0], ur = wr[1];
  double cfl = fast_speed(rl, wl[4], bn, wl[6], wl[7], gam);
  double cfr = fast_speed(rr, wr[4], bn, wr[6], wr[7], gam);
  double cmax = cfl > cfr ? cfl : cfr;
  double sl = (ul < ur ? ul : ur) - cmax;
  double sr = (ul > ur ? ul : ur) + cmax;
  double sigma = (rl > rr ? rl : rr) * (fabs(sl) > fabs(sr) ? fabs(sl) : fabs(sr));
  if (sl > 0.0) {
    memcpy(flux, FL, sizeof FL);
  } else if (sr < 0.0) {
    memcpy(flux, FR, sizeof FR);
  } else {
    for (int m = 0; m < 8; ++m) flux[m] = (sr * FL[m] - sl * FR[m] + sl * sr * (UR[m] - UL[m])) / (sr - sl);
  }
  flux[5] = sigma;
}

/* HLLC (Toro, Spruce & Speares), the other gas-dynamics solver of Section 2.1, for B = 0:
 * the HLL fan split by the contact S_M into two star states.  In the notation of the HLLD
 * solver above with every field component zero (M&K Eq. 38, 41, 43, 48):
 *   S_M = [(S_R - u_R) rho_R u_R - (S_L - u_L) rho_L u_L - p_R + p_L]
 *         / [(S_R - u_R) rho_R - (S_L - u_L) rho_L],
 *   p*  = [(S_R - u_R) rho_R p_L - (S_L - u_L) rho_L p_R
 *          + rho_L rho_R (S_R - u_R)(S_L - u_L)(u_R - u_L)] / (same denominator),
 *   rho*_a = rho_a (S_a - u_a)/(S_a - S_M), transverse velocities kept,
 *   E*_a = [(S_a - u_a) E_a - p_a u_a + p* S_M] / (S_a - S_M),
 *   F = F_L (S_L > 0), F_L + S_L (U*_L - U_L) (S_M >= 0), F_R + S_R (U*_R - U_R)
 *   (S_R >= 0 > S_M), F_R (S_R < 0). */
static void hllc(const double* wl, const double* wr, double gam, double* flux) {
  double UL[8], UR[8], FL[8], FR[8];
  frame_cons(wl, 0.0, gam, UL);
  frame_cons(wr, 0.0, gam, UR);
  frame_flux(wl, 0.0, gam, FL);
  frame_flux(wr, 0.0, gam, FR);
  double rl = wl[0], ul = wl[1], pl = wl[4];
  double rr = wr[0], ur = wr[1], pr = wr[4];
  double cl = fast_speed(rl, pl, 0.0, 0.0, 0.0, gam);
  double cr = fast_speed(rr, pr, 0.0, 0.0, 0.0, gam);
  double cmax = cl > cr ? cl : cr;
  double sl = (ul < ur ? ul : ur) - cmax;
  double sr = (ul > ur ? ul : ur) + cmax;
  double sigma = (rl > rr ? rl : rr) * (fabs(sl) > fabs(sr) ? fabs(sl) : fabs(sr));
  if (sl > 0.0) {
    memcpy(flux, FL, sizeof FL);
    flux[5] = sigma;
    return;
  }
  if (sr < 0.0) {
    memcpy(flux, FR, sizeof FR);
    flux[5] = sigma;
    return;
  }
  double dl = sl - ul, dr = sr - ur;
  double den = dr * rr - dl * rl;
  double sm = (dr * rr * ur - dl * rl * ul - pr + pl) / den;
  double pts = (dr * rr * pl - dl * rl * pr + rl * rr * dr * dl * (ur - ul)) / den;
  const double* w = sm >= 0.0 ? wl : wr;
  const double* Ua = sm >= 0.0 ? UL : UR;
  const double* Fa = sm >= 0.0 ? FL : FR;
  double S = sm >= 0.0 ? sl : sr;
  double ds = S - w[1];
  double rs = w[0] * ds / (S - sm);
  double Us[8] = {rs, rs * sm, rs * w[2], rs * w[3], (ds * Ua[4] - w[4] * w[1] + pts * sm) / (S - sm),
                  0.0, 0.0, 0.0};
  for (int m = 0; m < 8; ++m) flux[m] = Fa[m] + S * (Us[m] - Ua[m]);
  flux[5] = sigma;
}

/* the solver of the grid at one face; flux[5] is the face's mass-flux scale */
static void riemann(int solver, const double* wl, const double* wr, double bn, double gam, double* flux) {
  if (solver == ORC_RIEMANN_HLL) {
    hll(wl, wr, bn, gam, flux);
  } else if (solver == ORC_RIEMANN_HLLC && bn == 0.0 && wl[6] == 0.0 && wl[7] == 0.0 && wr[6] == 0.0 &&
             wr[7] == 0.0) {
    hllc(wl, wr, gam, flux);
  } else {
    hlld(wl, wr, bn, gam, flux);
  }
}

void orc_hlld_batch(int n, const double* wl, const double* wr, const double* bn,
                    double gamma, double* flux) {
  for (int q = 0; q < n; ++q) {
    hlld(wl + 8 * q, wr + 8 * q, bn[q], gamma, flux + 8 * q);
    flux[8 * q + 5] = 0.0;
  }
}

void orc_riemann_batch(int solver, int n, const double* wl, const double* wr, const double* bn,
                       double gamma, double* flux) {
  for (int q = 0; q < n; ++q) {
    riemann(solver, wl + 8 * q, wr + 8 * q, bn[q], gamma, flux + 8 * q);
    flux[8 * q + 5] = 0.0;
  }
}

/* --------------------------------------------------------- reconstruction ----
 * Eq. 12-14 with kappa = 1/3 (K1 = (1-kappa)/4, K2 = (1+kappa)/4, b = (3-kappa)/(1-kappa)),
 * minmod(a, b) = sign(a) max(0, min(|a|, sign(a) b)).
 * Reading: the printed arrangement of K1, K2 and b is taken in the standard
 * compressive kappa-scheme form, the one that is third-order upwind biased for
 * kappa = 1/3 as the text states:
 *   w_L(i+1/2) = w_i     + K1 minmod(dw_{i-1}, b dw_i) + K2 minmod(dw_i, b dw_{i-1})
 *   w_R(i+1/2) = w_{i+1} - K1 minmod(dw_{i+1}, b dw_i) - K2 minmod(dw_i, b dw_{i+1})
 * with dw_i = w_{i+1} - w_i. */
static double minmod(double a, double b) {
  double s = a > 0.0 ? 1.0 : (a < 0.0 ? -1.0 : 0.0);
  double m = fabs(a) < s * b ? fabs(a) : s * b;
  return s * (m > 0.0 ? m : 0.0);
}

static double recon_kappa(int recon) {
  return recon == ORC_RECON_KAPPA_ZERO ? 0.0 : (recon == ORC_RECON_KAPPA_UPWIND ? -1.0 : 1.0 / 3.0);
}

/* values w_{i-1}, w_i, w_{i+1}, w_{i+2} -> states left and right of face i+1/2.
 * ORC_RECON_PRINTED: dW_i = K2 minmod(dw_{i-1}, dw_i) + K1 minmod(dw_i, b dw_{i-1}),
 * dW_{i+1} = K2 minmod(dw_{i+1}, dw_i) + K1 minmod(dw_i, b dw_{i+1}), w_L = w_i + dW_i,
 * w_R = w_{i+1} - dW_{i+1} (Eq. 13-14 as printed). */
static void kappa_face(int recon, const double* w4, double* wl, double* wr) {
  double kappa = recon_kappa(recon);
  double K1 = (1.0 - kappa) / 4.0, K2 = (1.0 + kappa) / 4.0, b = (3.0 - kappa) / (1.0 - kappa);
  double dwm = w4[1] - w4[0]; /* dw_{i-1} */
  double dw0 = w4[2] - w4[1]; /* dw_i     */
  double dwp = w4[3] - w4[2]; /* dw_{i+1} */
  if (recon == ORC_RECON_PRINTED) {
    *wl = w4[1] + K2 * minmod(dwm, dw0) + K1 * minmod(dw0, b * dwm);
    *wr = w4[2] - K2 * minmod(dwp, dw0) - K1 * minmod(dw0, b * dwp);
    return;
  }
  *wl = w4[1] + K1 * minmod(dwm, b * dw0) + K2 * minmod(dw0, b * dwm);
  *wr = w4[2] - K1 * minmod(dwp, b * dw0) - K2 * minmod(dw0, b * dwp);
}

void orc_reconstruct_1d(int n, const double* w, double* wl, double* wr) {
  for (int m = 2; m <= n - 2; ++m) kappa_face(ORC_RECON_KAPPA_THIRD, w + m - 2, wl + m, wr + m);
}

void orc_reconstruct_1d_ex(int recon, int n, const double* w, double* wl, double* wr) {
  for (int m = 2; m <= n - 2; ++m) kappa_face(recon, w + m - 2, wl + m, wr + m);
}

/* ------------------------------------------------------------ face fluxes ----
 * Interface states for face d-1/2 of cell c (left cell c-1, right cell c).
 * order 1: donor cell (predictor); order 2: kappa-scheme on w = {rho, P, v, B}
 * (Eq. 12-14).  The normal field is the face value on both sides.  If the
 * reconstructed density or pressure is not positive on either side, the face
 * falls back to the donor-cell states (reading; the paper is silent). */
static const int CYC[3][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}}; /* normal, t1, t2 */

static void compute_fluxes(const grid* G, int d, int order, double* const W[NF],
                           double* const U[NF], double* const Fl[NF]) {
  int t1 = CYC[d][1], t2 = CYC[d][2];
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    if (a == d) {
      lo[a] = 0;
      hi[a] = G->n[a];
    } else if (G->act[a]) {
      lo[a] = -1;
      hi[a] = G->n[a];
    } else {
      lo[a] = 0;
      hi[a] = 0;
    }
  }
  const int vmap[8] = {WR, WVX + d, WVX + t1, WVX + t2, WP, -1, WBX + t1, WBX + t2};
#pragma omp parallel for schedule(static)
  for (int k = lo[2]; k <= hi[2]; ++k)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int i = lo[0]; i <= hi[0]; ++i) {
        int c[3] = {i, j, k};
        long cell[4];
        for (int s = -2; s <= 1; ++s) {
          int e[3] = {i, j, k};
          e[d] += s;
          cell[s + 2] = ixv(G, e);
        }
        double wl[8], wr[8];
        for (int m = 0; m < 8; ++m) {
          if (vmap[m] < 0) {
            wl[m] = wr[m] = 0.0;
            continue;
          }
          const double* q = W[vmap[m]];
          if (order == 1) {
            wl[m] = q[cell[1]];
            wr[m] = q[cell[2]];
          } else {
            double w4[4] = {q[cell[0]], q[cell[1]], q[cell[2]], q[cell[3]]};
            kappa_face(G->recon, w4, &wl[m], &wr[m]);
          }
        }
        if (order != 1 && (wl[0] <= 0.0 || wr[0] <= 0.0 || wl[4] <= 0.0 || wr[4] <= 0.0)) {
          for (int m = 0; m < 8; ++m) {
            if (vmap[m] < 0) continue;
            wl[m] = W[vmap[m]][cell[1]];
            wr[m] = W[vmap[m]][cell[2]];
          }
        }
        double bn = U[BXF + d][ixv(G, c)];
        double f[8];
        riemann(G->riemann, wl, wr, bn, G->gamma, f);
        long o = ixv(G, c);
        Fl[RHO][o] = f[0];
        Fl[MX + d][o] = f[1];
        Fl[MX + t1][o] = f[2];
        Fl[MX + t2][o] = f[3];
        Fl[EN][o] = f[4];
        Fl[BXF + d][o] = f[5]; /* mass-flux scale (the normal-field flux itself is zero) */
        Fl[BXF + t1][o] = f[6];
        Fl[BXF + t2][o] = f[7];
      }
}

/* ------------------------------------------------------------ corner EMFs ----
 * Eq. 9: cell-centre EMF E = -v x B.  Face EMFs from the Godunov fluxes (Eq. 3):
 * at a-faces E_c = -F_a[B_b], at b-faces E_c = +F_b[B_a], (a, b, c) cyclic.
 * Eq. 10-11 for the edge E_c at (a-1/2, b-1/2):
 *   E = 1/4 [E_a(a-1/2, b) + E_a(a-1/2, b-1) + E_b(a, b-1/2) + E_b(a-1, b-1/2)]
 *     + db/8 [(dE/db)(a-1/2, b-3/4) - (dE/db)(a-1/2, b-1/4)]
 *     + da/8 [(dE/da)(a-3/4, b-1/2) - (dE/da)(a-1/4, b-1/2)].
 * Readings: the four face points are the ones that surround the edge; the sign of
 * the corrections is the one for which a flow that varies along one axis only
 * gives back the face EMF exactly; the upwind side in Eq. 11 is chosen by the sign
 * of the Riemann mass flux F_rho through that face.  Eq. 11's "otherwise" (no
 * contact motion, F_rho = 0) is taken as zero to the precision of the data: |F_rho| <=
 * eps * sigma, sigma = max(rho_L, rho_R) max(|S_L|, |S_R|) the face's mass-flux scale.
 * A mass flux that is zero in exact arithmetic comes out of the HLLD formulas as rounding
 * of sigma, of either sign, and that rounding includes the one of the recovered pressure:
 * p = (gamma-1)(E - kinetic - magnetic) keeps a relative error of about 2^-52 times
 * E / (thermal energy), which reaches 1e3-1e4 at Mach 30-100 or low beta.  The default
 * eps = 2^-32 (UPWIND_EPS_FP64) lies two orders above that rounding; any slower motion is
 * upwinded.  A patch may set another eps (orc_patch.upwind_eps): the same reading for
 * data rounded to FP32 takes 64 * 2^-23.
 * If only one of a, b is active the edge EMF is that axis' face EMF. */
static double upwind(double fr, double sigma, double eps, double left, double right) {
  if (fr > eps * sigma) return left;
  if (fr < -eps * sigma) return right;
  return 0.5 * (left + right);
}

static void compute_emf(const grid* G, double* const W[NF], double* const Fl[3][NF],
                        double* const Ed[3]) {
  for (int c = 0; c < 3; ++c) {
    int a = CYC[c][1], b = CYC[c][2]; /* (a, b, c) cyclic */
    int lo[3] = {0, 0, 0}, hi[3];
    for (int x = 0; x < 3; ++x) hi[x] = (x == c) ? G->n[x] - 1 : (G->act[x] ? G->n[x] : 0);
    double* E = Ed[c];
    if (!G->act[a] && !G->act[b]) {
      for (long q = 0; q < G->tot; ++q) E[q] = 0.0;
      continue;
    }
#pragma omp parallel for schedule(static)
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          int p[3] = {i, j, k};
          long o = ixv(G, p);
          if (G->act[a] && !G->act[b]) {
            E[o] = -Fl[a][BXF + b][o];
            continue;
          }
          if (!G->act[a] && G->act[b]) {
            E[o] = Fl[b][BXF + a][o];
            continue;
          }
          /* neighbours: s = shift by -1 along a, t = shift by -1 along b */
          int pa[3] = {i, j, k}, pb[3] = {i, j, k}, pab[3] = {i, j, k};
          pa[a] -= 1;
          pb[b] -= 1;
          pab[a] -= 1;
          pab[b] -= 1;
          long oa = ixv(G, pa), ob = ixv(G, pb), oab = ixv(G, pab);
          /* face EMFs */
          double Ea_b = -Fl[a][BXF + b][o];    /* a-face (a-1/2, b)   */
          double Ea_bm = -Fl[a][BXF + b][ob];  /* a-face (a-1/2, b-1) */
          double Eb_a = Fl[b][BXF + a][o];     /* b-face (a, b-1/2)   */
          double Eb_am = Fl[b][BXF + a][oa];   /* b-face (a-1, b-1/2) */
          /* cell EMFs E_c = -(v_a B_b - v_b B_a) */
          double ec[4];
          long cells[4] = {o, oa, ob, oab}; /* (a,b) (a-1,b) (a,b-1) (a-1,b-1) */
          for (int q = 0; q < 4; ++q) {
            long cc = cells[q];
            ec[q] = -(W[WVX + a][cc] * W[WBX + b][cc] - W[WVX + b][cc] * W[WBX + a][cc]);
          }
          double da = G->d[a], db = G->d[b];
          /* d/db on a-face (a-1/2, b): between face point b and corner b-1/2 -> (b-1/4) */
          double dEdb_q = upwind(Fl[a][RHO][o], Fl[a][BXF + a][o], G->upwind_eps, 2.0 * (ec[1] - Eb_am) / db,
                                 2.0 * (ec[0] - Eb_a) / db);
          /* d/db on a-face (a-1/2, b-1): between corner b-1/2 and face point b-1 -> (b-3/4) */
          double dEdb_3q = upwind(Fl[a][RHO][ob], Fl[a][BXF + a][ob], G->upwind_eps, 2.0 * (Eb_am - ec[3]) / db,
                                  2.0 * (Eb_a - ec[2]) / db);
          /* d/da on b-face (a, b-1/2) -> (a-1/4) */
          double dEda_q = upwind(Fl[b][RHO][o], Fl[b][BXF + b][o], G->upwind_eps, 2.0 * (ec[2] - Ea_bm) / da,
                                 2.0 * (ec[0] - Ea_b) / da);
          /* d/da on b-face (a-1, b-1/2) -> (a-3/4) */
          double dEda_3q = upwind(Fl[b][RHO][oa], Fl[b][BXF + b][oa], G->upwind_eps, 2.0 * (Ea_bm - ec[3]) / da,
                                  2.0 * (Ea_b - ec[1]) / da);
          E[o] = 0.25 * (Ea_b + Ea_bm + Eb_a + Eb_am) + db / 8.0 * (dEdb_3q - dEdb_q) +
                 da / 8.0 * (dEda_3q - dEda_q);
        }
  }
}

/* --------------------------------------------------------------- sources ----
 * Eq. 2 source vector for an external potential: S = [0, -rho grad Psi,
 * -rho v . grad Psi, 0, 0, 0], evaluated at cell centres. */
static void grad_psi(const orc_source* s, double x, double y, double z, double g[3]) {
  g[0] = g[1] = g[2] = 0.0;
  if (!s) return;
  if (s->potential == ORC_POT_GAUSS_X) {
    double u = (x - s->xc) / s->xw;
    g[0] = s->psi0 * 2.0 * u / s->xw * exp(-u * u);
  } else if (s->potential == ORC_POT_LOG_DISC) {
    double q = x * x + y * y + s->rc * s->rc + z * z;
    g[0] = s->v0 * s->v0 * x / q;
    g[1] = s->v0 * s->v0 * y / q;
    g[2] = s->v0 * s->v0 * z / q;
  }
}

/* --------------------------------------------------------------- update -----
 * Eq. 7 for the cell fields, Eq. 8 for the faces (the second bracket of the printed
 * Eq. 8 is read as E_y, the component that -curl E requires):
 *   B_a -= h [ (E_c(b+1/2) - E_c(b-1/2))/db - (E_b(c+1/2) - E_b(c-1/2))/dc ]
 * out = base - h * divergence + h * S(src). */
static void update(const grid* G, const orc_source* s, double h, double* const base[NF],
                   double* const srcU[NF], double* const Fl[3][NF], double* const Ed[3],
                   double* const out[NF]) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        long o = ix(G, i, j, k);
        for (int f = RHO; f <= EN; ++f) {
          double div = 0.0;
          for (int d = 0; d < 3; ++d) {
            if (!G->act[d]) continue;
            int p[3] = {i, j, k};
            p[d] += 1;
            div += (Fl[d][f][ixv(G, p)] - Fl[d][f][o]) / G->d[d];
          }
          out[f][o] = base[f][o] - h * div;
        }
        double x = G->lo[0] + (i + 0.5) * G->d[0];
        double y = G->lo[1] + (j + 0.5) * G->d[1];
        double z = G->lo[2] + (k + 0.5) * G->d[2];
        double g[3];
        grad_psi(s, x, y, z, g);
        double rho = srcU[RHO][o];
        out[MX][o] += h * (-rho * g[0]);
        out[MY][o] += h * (-rho * g[1]);
        out[MZ][o] += h * (-rho * g[2]);
        out[EN][o] += h * (-(srcU[MX][o] * g[0] + srcU[MY][o] * g[1] + srcU[MZ][o] * g[2]));
      }
  for (int fa = 0; fa < 3; ++fa) {
    int b = CYC[fa][1], c = CYC[fa][2];
    int hi[3];
    for (int x = 0; x < 3; ++x) hi[x] = G->n[x] - 1;
    if (G->act[fa] && !G->per[fa]) hi[fa] = G->n[fa]; /* outflow: high boundary face is owned */
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= hi[2]; ++k)
      for (int j = 0; j <= hi[1]; ++j)
        for (int i = 0; i <= hi[0]; ++i) {
          int p[3] = {i, j, k};
          long o = ixv(G, p);
          double curl = 0.0;
          if (G->act[b]) {
            int q[3] = {i, j, k};
            q[b] += 1;
            curl += (Ed[c][ixv(G, q)] - Ed[c][o]) / G->d[b];
          }
          if (G->act[c]) {
            int q[3] = {i, j, k};
            q[c] += 1;
            curl -= (Ed[b][ixv(G, q)] - Ed[b][o]) / G->d[c];
          }
          out[BXF + fa][o] = base[BXF + fa][o] - h * curl;
        }
  }
}

/* ----------------------------------------------------------- host layout ---- */
static long host_cell(const grid* G, int i, int j, int k) {
  return (long)i + (long)G->n[0] * ((long)j + (long)G->n[1] * k);
}

static long host_face(const grid* G, int fa, int i, int j, int k) {
  int e[3] = {G->n[0], G->n[1], G->n[2]};
  e[fa] += 1;
  return (long)i + (long)e[0] * ((long)j + (long)e[1] * k);
}

static void load_state(const grid* G, const double* U, const double* B[3], double* const S[NF]) {
  long nc = (long)G->n[0] * G->n[1] * G->n[2];
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i)
        for (int f = 0; f < 5; ++f) S[f][ix(G, i, j, k)] = U[f * nc + host_cell(G, i, j, k)];
  for (int fa = 0; fa < 3; ++fa) {
    int e[3] = {G->n[0], G->n[1], G->n[2]};
    e[fa] += 1;
    for (int k = 0; k < e[2]; ++k)
      for (int j = 0; j < e[1]; ++j)
        for (int i = 0; i < e[0]; ++i) S[BXF + fa][ix(G, i, j, k)] = B[fa][host_face(G, fa, i, j, k)];
  }
}

static void store_state(const grid* G, double* const S[NF], double* U, double* B[3]) {
  long nc = (long)G->n[0] * G->n[1] * G->n[2];
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i)
        for (int f = 0; f < 5; ++f) U[f * nc + host_cell(G, i, j, k)] = S[f][ix(G, i, j, k)];
  for (int fa = 0; fa < 3; ++fa) {
    int e[3] = {G->n[0], G->n[1], G->n[2]};
    e[fa] += 1;
    for (int k = 0; k < e[2]; ++k)
      for (int j = 0; j < e[1]; ++j)
        for (int i = 0; i < e[0]; ++i) B[fa][host_face(G, fa, i, j, k)] = S[BXF + fa][ix(G, i, j, k)];
  }
}

/* -------------------------------------------------------------- the step ---- */
typedef struct {
  double* Un[NF];
  double* Uh[NF];
  double* Uo[NF];
  double* W[NF];
  double* Fl[3][NF];
  double* Ed[3];
  double* block;
} work;

static int work_alloc(const grid* G, work* w) {
  int nbuf = 4 * NF + 3 * NF + 3;
  w->block = (double*)calloc((size_t)nbuf * (size_t)G->tot, sizeof(double));
  if (!w->block) return -1;
  double* q = w->block;
  for (int f = 0; f < NF; ++f, q += G->tot) w->Un[f] = q;
  for (int f = 0; f < NF; ++f, q += G->tot) w->Uh[f] = q;
  for (int f = 0; f < NF; ++f, q += G->tot) w->Uo[f] = q;
  for (int f = 0; f < NF; ++f, q += G->tot) w->W[f] = q;
  for (int d = 0; d < 3; ++d)
    for (int f = 0; f < NF; ++f, q += G->tot) w->Fl[d][f] = q;
  for (int d = 0; d < 3; ++d, q += G->tot) w->Ed[d] = q;
  return 0;
}

/* End-of-step floors on the conserved state (reading: the paper states none):
 * rho' = max(rho, rho_floor), momentum kept, P from E with rho' and the cell-centred
 * field of Eq. 6, clamped to [rho' pr_floor, rho' pr_ceil], and E rebuilt by the
 * closure after Eq. 3 when rho or P changed.  Returns the number of cells changed. */
static long floor_state(const grid* G, double* const U[NF]) {
  if (!G->floors) return 0;
  double gm1 = G->gamma - 1.0;
  long count = 0;
#pragma omp parallel for schedule(static) reduction(+ : count)
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        long c = ix(G, i, j, k);
        double rho = U[RHO][c];
        double rf = rho < G->rho_floor ? G->rho_floor : rho;
        double m2 = U[MX][c] * U[MX][c] + U[MY][c] * U[MY][c] + U[MZ][c] * U[MZ][c];
        double bx = 0.5 * (U[BXF][c] + U[BXF][ix(G, i + 1, j, k)]);
        double by = 0.5 * (U[BYF][c] + U[BYF][ix(G, i, j + 1, k)]);
        double bz = 0.5 * (U[BZF][c] + U[BZF][ix(G, i, j, k + 1)]);
        double kin = 0.5 * m2 / rf;
        double mag = 0.5 * (bx * bx + by * by + bz * bz);
        double p = gm1 * (U[EN][c] - kin - mag);
        double pf = clamp_p(G, p, rf);
        if (rf != rho || pf != p) {
          U[RHO][c] = rf;
          U[EN][c] = pf / gm1 + kin + mag;
          ++count;
        }
      }
  return count;
}

/* Two-stage van Leer step: donor-cell fluxes and EMFs from W^n give U^{n+1/2}
 * (h = dt/2, S at U^n); kappa-scheme fluxes and EMFs from W^{n+1/2} give U^{n+1}
 * (h = dt, S at U^{n+1/2}), both from the base U^n. */
static long vl2_step(const grid* G, const orc_source* s, work* w, double dt) {
  fill_ghosts(G, w->Un);
  cons_to_prim(G, w->Un, w->W);
  for (int d = 0; d < 3; ++d)
    if (G->act[d]) compute_fluxes(G, d, 1, w->W, w->Un, w->Fl[d]);
  compute_emf(G, w->W, w->Fl, w->Ed);
  update(G, s, 0.5 * dt, w->Un, w->Un, w->Fl, w->Ed, w->Uh);
  fill_ghosts(G, w->Uh);
  cons_to_prim(G, w->Uh, w->W);
  for (int d = 0; d < 3; ++d)
    if (G->act[d]) compute_fluxes(G, d, 2, w->W, w->Uh, w->Fl[d]);
  compute_emf(G, w->W, w->Fl, w->Ed);
  update(G, s, dt, w->Un, w->Uh, w->Fl, w->Ed, w->Uo);
  for (int f = 0; f < NF; ++f) {
    double* t = w->Un[f];
    w->Un[f] = w->Uo[f];
    w->Uo[f] = t;
  }
  fill_ghosts(G, w->Un); /* the floors read the high faces of the last interior cells */
  long floored = floor_state(G, w->Un);
  if (floored) fill_ghosts(G, w->Un);
  return floored;
}

/* ------------------------------------------------------- passive scalars ----
 * X_s = (rho X_s)/rho on the padded box: interior cells from the state, ghost cells
 * beyond an inflow side from inflow_x, other ghost cells from their mapped source cell. */
static void scalar_prim(const grid* G, double* const U[NF], int ns, double* const S[], const double* inflow_x,
                        double* const X[]) {
#pragma omp parallel for schedule(static)
  for (int kk = 0; kk < G->N[2]; ++kk)
    for (int jj = 0; jj < G->N[1]; ++jj)
      for (int ii = 0; ii < G->N[0]; ++ii) {
        int c[3] = {ii - G->g[0], jj - G->g[1], kk - G->g[2]};
        long o = ixv(G, c);
        int side = inflow_side(G, c, -1);
        if (side >= 0) {
          for (int q = 0; q < ns; ++q) X[q][o] = inflow_x ? inflow_x[side * ns + q] : 0.0;
          continue;
        }
        int m[3];
        for (int a = 0; a < 3; ++a) m[a] = src_index(G, a, c[a], 0);
        long src = ixv(G, m);
        for (int q = 0; q < ns; ++q) X[q][o] = S[q][src] / U[RHO][src];
      }
}

/* rho X_out = rho X_base - h sum_d [F_d(c + 1/2) - F_d(c - 1/2)] / dx_d over interior cells,
 * F_d = (mass flux) * (X_L if mass flux >= 0 else X_R) at each face */
static void scalar_update(const grid* G, int order, double h, double* const Fl[3][NF], int ns,
                          double* const X[], double* const Sb[], double* const So[]) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        int c[3] = {i, j, k};
        long o = ixv(G, c);
        for (int q = 0; q < ns; ++q) {
          double div = 0.0;
          for (int d = 0; d < 3; ++d) {
            if (!G->act[d]) continue;
            double fx[2];
            for (int up = 0; up < 2; ++up) {
              int f[3] = {i, j, k};
              f[d] += up; /* face f[d] - 1/2 */
              long cell[4];
              for (int t = -2; t <= 1; ++t) {
                int e[3] = {f[0], f[1], f[2]};
                e[d] += t;
                cell[t + 2] = ixv(G, e);
              }
              double xl, xr;
              if (order == 1) {
                xl = X[q][cell[1]];
                xr = X[q][cell[2]];
              } else {
                double w4[4] = {X[q][cell[0]], X[q][cell[1]], X[q][cell[2]], X[q][cell[3]]};
                kappa_face(G->recon, w4, &xl, &xr);
              }
              double mf = Fl[d][RHO][ixv(G, f)];
              fx[up] = mf * (mf >= 0.0 ? xl : xr);
            }
            div += (fx[1] - fx[0]) / G->d[d];
          }
          So[q][o] = Sb[q][o] - h * div;
        }
      }
}

int orc_step_scalars(const orc_patch* p, const orc_source* s, double* U, double* Bx, double* By,
                     double* Bz, int ns, double* S, const double* inflow_x, double dt) {
  grid G;
  work w;
  if (ns < 0 || (ns > 0 && !S)) return -1;
  if (make_grid(p, &G) || work_alloc(&G, &w)) return -1;
  set_floors(&G, s);
  const double* Bin[3] = {Bx, By, Bz};
  double* Bout[3] = {Bx, By, Bz};
  load_state(&G, U, Bin, w.Un);
  /* per scalar: base, half-step, new, X (padded) */
  double* blk = (double*)calloc((size_t)(4 * (ns > 0 ? ns : 1)) * (size_t)G.tot, sizeof(double));
  double** Sn = (double**)calloc((size_t)(4 * (ns > 0 ? ns : 1)), sizeof(double*));
  if (!blk || !Sn) {
    free(blk);
    free(Sn);
    free(w.block);
    return -1;
  }
  double** Sh = Sn + ns;
  double** So = Sh + ns;
  double** X = So + ns;
  for (int q = 0; q < 4 * ns; ++q) Sn[q] = blk + (size_t)q * G.tot;
  const long cells = (long)G.n[0] * G.n[1] * G.n[2];
  for (int q = 0; q < ns; ++q)
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i)
          Sn[q][ix(&G, i, j, k)] = S[q * cells + ((long)k * G.n[1] + j) * G.n[0] + i];
  /* the step of vl2_step, with the scalars carried on each stage's mass fluxes */
  fill_ghosts(&G, w.Un);
  cons_to_prim(&G, w.Un, w.W);
  for (int d = 0; d < 3; ++d)
    if (G.act[d]) compute_fluxes(&G, d, 1, w.W, w.Un, w.Fl[d]);
  scalar_prim(&G, w.Un, ns, Sn, inflow_x, X);
  scalar_update(&G, 1, 0.5 * dt, w.Fl, ns, X, Sn, Sh);
  compute_emf(&G, w.W, w.Fl, w.Ed);
  update(&G, s, 0.5 * dt, w.Un, w.Un, w.Fl, w.Ed, w.Uh);
  fill_ghosts(&G, w.Uh);
  cons_to_prim(&G, w.Uh, w.W);
  for (int d = 0; d < 3; ++d)
    if (G.act[d]) compute_fluxes(&G, d, 2, w.W, w.Uh, w.Fl[d]);
  scalar_prim(&G, w.Uh, ns, Sh, inflow_x, X);
  scalar_update(&G, 2, dt, w.Fl, ns, X, Sn, So);
  compute_emf(&G, w.W, w.Fl, w.Ed);
  update(&G, s, dt, w.Un, w.Uh, w.Fl, w.Ed, w.Uo);
  for (int f = 0; f < NF; ++f) {
    double* t = w.Un[f];
    w.Un[f] = w.Uo[f];
    w.Uo[f] = t;
  }
  fill_ghosts(&G, w.Un);
  long floored = floor_state(&G, w.Un);
  if (floored) fill_ghosts(&G, w.Un);
  store_state(&G, w.Un, U, Bout);
  for (int q = 0; q < ns; ++q)
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i)
          S[q * cells + ((long)k * G.n[1] + j) * G.n[0] + i] = So[q][ix(&G, i, j, k)];
  free(blk);
  free(Sn);
  free(w.block);
  return floored > 2147483647L ? 2147483647 : (int)floored;
}

/* Time step from the CFL condition (the paper does not state it; reading:
 * dt = C min over cells and active axes of d / (|v_d| + c_f,d), c_f the fast
 * magnetosonic speed along that axis). */
static double cfl_from(const grid* G, double* const U[NF], double* const W[NF], double cfl) {
  double best = INFINITY;
  cons_to_prim(G, U, W);
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        long c = ix(G, i, j, k);
        for (int d = 0; d < 3; ++d) {
          if (!G->act[d]) continue;
          int t1 = CYC[d][1], t2 = CYC[d][2];
          double cf = fast_speed(W[WR][c], W[WP][c], W[WBX + d][c], W[WBX + t1][c], W[WBX + t2][c],
                                 G->gamma);
          double dtd = G->d[d] / (fabs(W[WVX + d][c]) + cf);
          if (dtd < best) best = dtd;
        }
      }
  return cfl * best;
}

int orc_step(const orc_patch* p, const orc_source* s, double* U, double* Bx, double* By,
             double* Bz, double dt) {
  grid G;
  work w;
  if (make_grid(p, &G) || work_alloc(&G, &w)) return -1;
  set_floors(&G, s);
  const double* Bin[3] = {Bx, By, Bz};
  double* Bout[3] = {Bx, By, Bz};
  load_state(&G, U, Bin, w.Un);
  long floored = vl2_step(&G, s, &w, dt);
  store_state(&G, w.Un, U, Bout);
  free(w.block);
  return floored > 2147483647L ? 2147483647 : (int)floored;
}

/* The corner EMFs of one stage (Eq. 9-11) for the state given, without updating it:
 * order 1 is the predictor's donor-cell stage, order 2 the corrector's reconstruction.
 * E[c][k][j][i] receives E_c at the cell's low edge along c (for E_z: (i-1/2, j-1/2, k)). */
int orc_stage_emf(const orc_patch* p, const double* U, const double* Bx, const double* By,
                  const double* Bz, int order, double* E) {
  grid G;
  work w;
  if (order < 1 || order > 2 || make_grid(p, &G) || work_alloc(&G, &w)) return -1;
  set_floors(&G, NULL);
  const double* Bin[3] = {Bx, By, Bz};
  load_state(&G, U, Bin, w.Un);
  fill_ghosts(&G, w.Un);
  cons_to_prim(&G, w.Un, w.W);
  for (int d = 0; d < 3; ++d)
    if (G.act[d]) compute_fluxes(&G, d, order, w.W, w.Un, w.Fl[d]);
  compute_emf(&G, w.W, w.Fl, w.Ed);
  long nc = (long)G.n[0] * G.n[1] * G.n[2];
  for (int c = 0; c < 3; ++c)
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i)
          E[c * nc + host_cell(&G, i, j, k)] = w.Ed[c][ix(&G, i, j, k)];
  free(w.block);
  return 0;
}

double orc_cfl_dt(const orc_patch* p, const orc_source* s, const double* U, const double* Bx,
                  const double* By, const double* Bz, double cfl) {
  grid G;
  work w;
  if (make_grid(p, &G) || work_alloc(&G, &w)) return -1.0;
  set_floors(&G, s);
  const double* Bin[3] = {Bx, By, Bz};
  load_state(&G, U, Bin, w.Un);
  fill_ghosts(&G, w.Un);
  double dt = cfl_from(&G, w.Un, w.W, cfl);
  free(w.block);
  return dt;
}

int orc_run(const orc_patch* p, const orc_source* s, double* U, double* Bx, double* By,
            double* Bz, double cfl, double t_end, int max_steps) {
  grid G;
  work w;
  if (make_grid(p, &G) || work_alloc(&G, &w)) return -1;
  set_floors(&G, s);
  const double* Bin[3] = {Bx, By, Bz};
  double* Bout[3] = {Bx, By, Bz};
  load_state(&G, U, Bin, w.Un);
  fill_ghosts(&G, w.Un);
  double t = 0.0;
  int steps = 0;
  while (t < t_end && steps < max_steps) {
    double dt = cfl_from(&G, w.Un, w.W, cfl);
    if (t + dt > t_end) dt = t_end - t;
    vl2_step(&G, s, &w, dt);
    t += dt;
    ++steps;
  }
  store_state(&G, w.Un, U, Bout);
  free(w.block);
  return steps;
}

void orc_diagnostics(const orc_patch* p, const double* U, const double* Bx, const double* By,
                     const double* Bz, double sums[5], double* max_divb) {
  grid G;
  if (make_grid(p, &G)) return;
  long nc = (long)G.n[0] * G.n[1] * G.n[2];
  for (int f = 0; f < 5; ++f) {
    double acc = 0.0;
    for (long q = 0; q < nc; ++q) acc += U[f * nc + q];
    sums[f] = acc;
  }
  const double* B[3] = {Bx, By, Bz};
  double dmin = INFINITY;
  for (int a = 0; a < 3; ++a)
    if (G.act[a] && G.d[a] < dmin) dmin = G.d[a];
  double m = 0.0;
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        double div = 0.0;
        int c[3] = {i, j, k};
        for (int a = 0; a < 3; ++a) {
          if (!G.act[a]) continue;
          int h[3] = {i, j, k};
          h[a] += 1;
          div += (B[a][host_face(&G, a, h[0], h[1], h[2])] - B[a][host_face(&G, a, c[0], c[1], c[2])]) /
                 G.d[a];
        }
        if (fabs(div) * dmin > m) m = fabs(div) * dmin;
      }
  *max_divb = m;
}

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
