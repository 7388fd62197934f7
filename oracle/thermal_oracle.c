/*
 * thermal_oracle.c -- plain FP64 oracle of the thermal source term and of the MLP
 * surrogate that replaces it.  TEST INFRASTRUCTURE ONLY (see mhd_oracle.h).
 *
 * Thermal module (Section 3.10 of arXiv:1502.02935): per-cell heating and cooling enter
 * the energy equation through S (Eq. 2).  The paper's rate tables are not available, so
 * the cooling function here is a documented stand-in: Lambda(T, Z) is a piecewise power
 * law in T between knots (log10 T, log10 Lambda) spanning 10 K .. 1e8 K, with a steep rise
 * at 1e4 K, a metal peak near 2.5e5 K and a declining, thermally unstable segment above
 * it; it scales as (0.2 + 0.8 Z/0.02).  Heating is a constant Gamma per hydrogen atom.
 *
 * Isochoric update of one cell over dt (operator split after the MHD step):
 *   e = c_e T,   de/dt = (n_H Gamma - n_H^2 Lambda(T, Z)) / rate_unit,
 * integrated by backward Euler in T on sub-steps whose explicit change is capped at
 * |dT| <= cap * T, each solved by Newton's method with a bisection safeguard
 * (at most 30 iterations, relative tolerance 1e-12), T clamped to [10, 1e8] K.  Hitting
 * a cap is reported in the status word, never by looping on.
 */
#include <math.h>
#include <stddef.h>

#define NKNOT 11
static const double LT[NKNOT] = {1.0, 2.0, 3.0, 3.8, 4.0, 4.2, 5.0, 5.4, 6.0, 7.0, 8.0};
static const double LL[NKNOT] = {-28.5, -27.0, -26.2, -25.9, -23.5, -21.8, -21.3, -21.2, -22.0, -22.7, -22.6};
#define T_MIN 10.0
#define T_MAX 1e8
#define MAX_SUB 4096
#define MAX_NEWTON 30

enum { ST_SUBSTEP_CAP = 1, ST_NEWTON_CAP = 2, ST_NO_BRACKET = 4 };

typedef struct {
  double gamma_heat; /* Gamma, erg s^-1 per H */
  double z;          /* metallicity */
  double rate_unit;  /* erg cm^-3 s^-1 per code energy density per code time */
  double cap;        /* largest explicit relative change of T per sub-step */
} th_par;

/* Lambda(T, Z) [erg cm^3 s^-1] and its logarithmic slope d ln Lambda / d ln T */
static double cooling(double T, double z, double* slope) {
  double lt = log10(T);
  int k = 0;
  while (k < NKNOT - 2 && lt >= LT[k + 1]) ++k;
  double a = (LL[k + 1] - LL[k]) / (LT[k + 1] - LT[k]);
  double ll = LL[k] + a * (lt - LT[k]);
  if (slope) *slope = a;
  return pow(10.0, ll) * (0.2 + 0.8 * z / 0.02);
}

/* dT/dt and its derivative with respect to T */
static double rate(double T, double nh, double ce, const th_par* P, double* dfdT) {
  double a;
  double lam = cooling(T, P->z, &a);
  double f = (nh * P->gamma_heat - nh * nh * lam) / (P->rate_unit * ce);
  if (dfdT) *dfdT = -(nh * nh * lam * a / T) / (P->rate_unit * ce);
  return f;
}

static double clampT(double T) { return T < T_MIN ? T_MIN : (T > T_MAX ? T_MAX : T); }

/* one cell: returns T(dt), status bits in *st */
static double integrate(double T0, double nh, double ce, double dt, const th_par* P, int* st) {
  double T = clampT(T0), t = 0.0;
  int nsub = 0;
  *st = 0;
  while (t < dt) {
    if (nsub == MAX_SUB) {
      *st |= ST_SUBSTEP_CAP;
      break;
    }
    double r = rate(T, nh, ce, P, NULL);
    double h = dt - t;
    if (fabs(r) * h > P->cap * T) h = P->cap * T / fabs(r);
    /* bracket of the backward-Euler root g(x) = x - T - h f(x) */
    double lo = clampT(T / (1.0 + 4.0 * P->cap)), hi = clampT(T * (1.0 + 4.0 * P->cap));
    double glo = lo - T - h * rate(lo, nh, ce, P, NULL);
    double ghi = hi - T - h * rate(hi, nh, ce, P, NULL);
    double x;
    if (glo > 0.0 || ghi < 0.0) {
      /* no sign change inside the bracket: take the explicit estimate, clamped */
      *st |= ST_NO_BRACKET;
      x = clampT(T + h * r);
    } else {
      x = clampT(T + h * r);
      if (x < lo) x = lo;
      if (x > hi) x = hi;
      int it = 0, done = 0;
      for (; it < MAX_NEWTON; ++it) {
        double d;
        double g = x - T - h * rate(x, nh, ce, P, &d);
        if (g == 0.0) {
          done = 1;
          break;
        }
        if (g < 0.0) lo = x;
        else hi = x;
        double gp = 1.0 - h * d;
        if (gp > 0.0) {
          double xn = x - g / gp;
          if (fabs(xn - x) <= 1e-12 * x) { /* converged Newton step */
            x = xn;
            done = 1;
            break;
          }
          x = (xn > lo && xn < hi) ? xn : 0.5 * (lo + hi);
        } else {
          x = 0.5 * (lo + hi); /* bisection safeguard */
        }
      }
      if (!done) *st |= ST_NEWTON_CAP;
    }
    T = x;
    t += h;
    ++nsub;
  }
  return T;
}

typedef struct {
  double gamma_heat, z, rate_unit, cap;
  double nh_per_rho; /* n_H [cm^-3] per code density */
  double t_per_pr;   /* T [K] per code p/rho */
} orc_thermal;

static th_par par_of(const orc_thermal* q) {
  th_par P = {q->gamma_heat, q->z, q->rate_unit, q->cap};
  return P;
}

void orc_cooling(long n, const double* T, double z, double* lam, double* slope) {
  for (long q = 0; q < n; ++q) lam[q] = cooling(T[q], z, slope ? slope + q : NULL);
}

/* Cells given by (T0, n_H, c_e, dt): T_out after dt; status bits OR-ed per cell. */
int orc_thermal_cells(long n, const double* T0, const double* nh, const double* ce, const double* dt,
                      const orc_thermal* q, double* T_out, int* st_out) {
  th_par P = par_of(q);
  int any = 0;
  for (long i = 0; i < n; ++i) {
    int st;
    T_out[i] = integrate(T0[i], nh[i], ce[i], dt[i], &P, &st);
    if (st_out) st_out[i] = st;
    any |= st;
  }
  return any;
}

/* Operator-split thermal update of a state in the library's host format: per cell
 * p from the closure after Eq. 3 (cell-centred field of Eq. 6), T = t_per_pr p/rho,
 * n_H = nh_per_rho rho, c_e = rho/(t_per_pr (gamma-1)); E += c_e (T(dt) - T). */
int orc_thermal_apply(int nx, int ny, int nz, double gamma, const orc_thermal* q, double* U,
                      const double* Bx, const double* By, const double* Bz, double dt) {
  th_par P = par_of(q);
  long nc = (long)nx * ny * nz;
  int any = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : any)
  for (long c = 0; c < nc; ++c) {
    int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long)nx * ny));
    double rho = U[c], mx = U[nc + c], my = U[2 * nc + c], mz = U[3 * nc + c], e = U[4 * nc + c];
    double bx = 0.5 * (Bx[i + (long)(nx + 1) * (j + (long)ny * k)] + Bx[i + 1 + (long)(nx + 1) * (j + (long)ny * k)]);
    double by = 0.5 * (By[i + (long)nx * (j + (long)(ny + 1) * k)] + By[i + (long)nx * (j + 1 + (long)(ny + 1) * k)]);
    double bz = 0.5 * (Bz[i + (long)nx * (j + (long)ny * k)] + Bz[i + (long)nx * (j + (long)ny * (k + 1))]);
    double vx = mx / rho, vy = my / rho, vz = mz / rho;
    double p = (gamma - 1.0) * (e - 0.5 * rho * (vx * vx + vy * vy + vz * vz) - 0.5 * (bx * bx + by * by + bz * bz));
    double T = q->t_per_pr * p / rho;
    double nh = q->nh_per_rho * rho;
    double ce = rho / (q->t_per_pr * (gamma - 1.0));
    int st;
    double T1 = integrate(T, nh, ce, dt, &P, &st);
    any |= st;
    U[4 * nc + c] = e + ce * (T1 - T);
  }
  return any;
}

/* ------------------------------------------------------------- MLP oracle ----
 * Surrogate network 4 -> H -> H -> 1 with tanh hidden layers (H = 64):
 *   h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = w3 . h2 + b3,
 * W1 row-major H x 4, W2 row-major H x H.  Loss = mean over the batch of (y - t)^2.
 * Backward pass by the chain rule, plain loops, FP64. */
#define HID 64

static void fwd1(const double* x, const double* W1, const double* b1, const double* W2, const double* b2,
                 const double* w3, const double* b3, double* h1, double* h2, double* y) {
  for (int a = 0; a < HID; ++a) {
    double z = b1[a];
    for (int k = 0; k < 4; ++k) z += W1[a * 4 + k] * x[k];
    h1[a] = tanh(z);
  }
  for (int a = 0; a < HID; ++a) {
    double z = b2[a];
    for (int k = 0; k < HID; ++k) z += W2[a * HID + k] * h1[k];
    h2[a] = tanh(z);
  }
  double out = b3[0];
  for (int k = 0; k < HID; ++k) out += w3[k] * h2[k];
  *y = out;
}

void orc_mlp_forward(long n, const double* X, const double* W1, const double* b1, const double* W2,
                     const double* b2, const double* w3, const double* b3, double* Y) {
  double h1[HID], h2[HID];
  for (long q = 0; q < n; ++q) fwd1(X + 4 * q, W1, b1, W2, b2, w3, b3, h1, h2, Y + q);
}

double orc_mlp_backward(long n, const double* X, const double* Tg, const double* W1, const double* b1,
                        const double* W2, const double* b2, const double* w3, const double* b3, double* gW1,
                        double* gb1, double* gW2, double* gb2, double* gw3, double* gb3) {
  double h1[HID], h2[HID], d2[HID], d1[HID];
  for (int a = 0; a < HID * 4; ++a) gW1[a] = 0.0;
  for (int a = 0; a < HID * HID; ++a) gW2[a] = 0.0;
  for (int a = 0; a < HID; ++a) gb1[a] = gb2[a] = gw3[a] = 0.0;
  gb3[0] = 0.0;
  double loss = 0.0;
  for (long q = 0; q < n; ++q) {
    const double* x = X + 4 * q;
    double y;
    fwd1(x, W1, b1, W2, b2, w3, b3, h1, h2, &y);
    double r = y - Tg[q];
    loss += r * r;
    double dy = 2.0 * r / (double)n; /* d loss / d y */
    gb3[0] += dy;
    for (int a = 0; a < HID; ++a) {
      gw3[a] += dy * h2[a];
      d2[a] = dy * w3[a] * (1.0 - h2[a] * h2[a]);
    }
    for (int a = 0; a < HID; ++a) {
      gb2[a] += d2[a];
      for (int k = 0; k < HID; ++k) gW2[a * HID + k] += d2[a] * h1[k];
    }
    for (int k = 0; k < HID; ++k) {
      double s = 0.0;
      for (int a = 0; a < HID; ++a) s += W2[a * HID + k] * d2[a];
      d1[k] = s * (1.0 - h1[k] * h1[k]);
    }
    for (int a = 0; a < HID; ++a) {
      gb1[a] += d1[a];
      for (int k = 0; k < 4; ++k) gW1[a * 4 + k] += d1[a] * x[k];
    }
  }
  return loss / (double)n;
}

/* -------------------------------------------------- surrogate thermal step ----
 * The learned replacement of the integration above, as the step applies it per cell
 * (Section 3.10 via S of Eq. 2; the network is the project's stand-in for the tabulated
 * integration).  For each cell:
 *   T, n_H, c_e as in orc_thermal_apply; Tc = T clamped to [10, 1e8] K;
 *   features (log10 n_H, log10 Tc, log10 dt, Z), standardised x_s = (x - lo) s - 1;
 *   explicit estimate D = rate(Tc) dt / (Tc ln 10) and its saturated scale S = D / (1 + |D|);
 *   q = network(x_s), in FP64 with the hidden activations h1 and the weights W2 rounded to
 *   BF16 (the operands of the 64 x 64 layer), the change of log10 T is d = q S;
 *   fallback to the plain integrator when a standardised feature leaves [-1, 1], |q| > qmax,
 *   |d| > dmax, or d is not finite;
 *   otherwise T1 = Tc 10^d and dT = T1 - T, written Tc expm1(d ln 10) when no clamp acts
 *   (Tc = T and T1 inside [10, 1e8]) and clamp(T1) - T otherwise; E += c_e dT. */

/* round to the nearest BF16 value (8 significant bits), ties to even */
static double bf16_round(double v) {
  if (v == 0.0 || !isfinite(v)) return v;
  int e;
  double m = frexp(v, &e); /* v = m 2^e, 0.5 <= |m| < 1 */
  return ldexp(nearbyint(ldexp(m, 8)), e - 8);
}

void orc_bf16_round(long n, const double* v, double* out) {
  for (long q = 0; q < n; ++q) out[q] = bf16_round(v[q]);
}

static double net_forward_bf16(const double* x, const double* W1, const double* b1, const double* W2b,
                               const double* b2, const double* w3, double b3) {
  double h1[HID];
  for (int a = 0; a < HID; ++a) {
    double z = b1[a];
    for (int k = 0; k < 4; ++k) z += W1[a * 4 + k] * x[k];
    h1[a] = bf16_round(tanh(z));
  }
  double y = b3;
  for (int a = 0; a < HID; ++a) {
    double z = b2[a];
    for (int k = 0; k < HID; ++k) z += W2b[a * HID + k] * h1[k];
    y += w3[a] * tanh(z);
  }
  return y;
}

/* The surrogate's network on rows X[n][4] (already standardised), as the step evaluates it:
 * FP64 with h1 and W2 rounded to BF16.  params as below. */
void orc_mlp_forward_bf16(long n, const double* X, const double* params, double* Y) {
  const double *W1 = params, *b1 = W1 + HID * 4, *W2 = b1 + HID, *b2 = W2 + HID * HID, *w3 = b2 + HID;
  double W2b[HID * HID];
  for (int a = 0; a < HID * HID; ++a) W2b[a] = bf16_round(W2[a]);
  for (long q = 0; q < n; ++q) Y[q] = net_forward_bf16(X + 4 * q, W1, b1, W2b, b2, w3, w3[HID]);
}

/* params: W1[64][4], b1[64], W2[64][64], b2[64], w3[64], b3 (4545 values); range: lo[4],
 * s[4], qmax, dmax.  U is updated in place.  fallback[c] (may be NULL) receives 1 where the
 * cell took the integrator; feat[6 c + 0..5] (may be NULL) the standardised features, q and S.
 * Returns the integrator's status bits OR-ed over the fallback cells. */
int orc_surrogate_apply(int nx, int ny, int nz, double gamma, const orc_thermal* q, const double* params,
                        const double* range, double* U, const double* Bx, const double* By, const double* Bz,
                        double dt, int* fallback, double* feat) {
  th_par P = par_of(q);
  const double *W1 = params, *b1 = W1 + HID * 4, *W2 = b1 + HID, *b2 = W2 + HID * HID, *w3 = b2 + HID;
  const double b3 = w3[HID];
  double W2b[HID * HID];
  for (int a = 0; a < HID * HID; ++a) W2b[a] = bf16_round(W2[a]);
  long nc = (long)nx * ny * nz;
  int any = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : any)
  for (long c = 0; c < nc; ++c) {
    int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long)nx * ny));
    double rho = U[c], mx = U[nc + c], my = U[2 * nc + c], mz = U[3 * nc + c], e = U[4 * nc + c];
    double bx = 0.5 * (Bx[i + (long)(nx + 1) * (j + (long)ny * k)] + Bx[i + 1 + (long)(nx + 1) * (j + (long)ny * k)]);
    double by = 0.5 * (By[i + (long)nx * (j + (long)(ny + 1) * k)] + By[i + (long)nx * (j + 1 + (long)(ny + 1) * k)]);
    double bz = 0.5 * (Bz[i + (long)nx * (j + (long)ny * k)] + Bz[i + (long)nx * (j + (long)ny * (k + 1))]);
    double vx = mx / rho, vy = my / rho, vz = mz / rho;
    double p = (gamma - 1.0) * (e - 0.5 * rho * (vx * vx + vy * vy + vz * vz) - 0.5 * (bx * bx + by * by + bz * bz));
    double T = q->t_per_pr * p / rho;
    double nh = q->nh_per_rho * rho;
    double ce = rho / (q->t_per_pr * (gamma - 1.0));
    double Tc = clampT(T);
    double raw[4] = {log10(nh), log10(Tc), log10(dt), q->z};
    double xs[4];
    int inside = 1;
    for (int f = 0; f < 4; ++f) {
      xs[f] = (raw[f] - range[f]) * range[4 + f] - 1.0;
      inside = inside && xs[f] >= -1.0 && xs[f] <= 1.0;
    }
    double D = rate(Tc, nh, ce, &P, NULL) * dt / (Tc * log(10.0));
    double S = D / (1.0 + fabs(D));
    double y = net_forward_bf16(xs, W1, b1, W2b, b2, w3, b3);
    double d = y * S;
    int fb = !(inside && fabs(y) <= range[8] && fabs(d) <= range[9]);
    double dT;
    if (fb) {
      int st;
      dT = integrate(T, nh, ce, dt, &P, &st) - T;
      any |= st;
    } else {
      double T1 = Tc * pow(10.0, d);
      if (Tc != T || !(T1 >= T_MIN && T1 <= T_MAX)) dT = clampT(T1) - T;
      else dT = Tc * expm1(d * log(10.0));
    }
    U[4 * nc + c] = e + ce * dT;
    if (fallback) fallback[c] = fb;
    if (feat) {
      for (int f = 0; f < 4; ++f) feat[6 * c + f] = xs[f];
      feat[6 * c + 4] = y;
      feat[6 * c + 5] = S;
    }
  }
  return any;
}
