/*
 * oracle.c -- plain FP64 CPU reference of per-cell constant-volume adiabatic chemistry.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker of the GPU library: only the tests,
 * the smoke check and the benchmark's CPU-baseline leg load it.  It shares no code, header
 * or table with the CUDA path.
 *
 * What it computes (arxiv 2510.23993, Sec. 2.1):
 *   - each cell is a 0-D reactor at constant volume (rho fixed) and constant internal
 *     energy e (adiabatic), Eq. 5:  dY_k/dt = W_k * omega_k / rho;
 *   - the temperature follows from e by a Newton iteration at fixed rho and Y (Sec. 2.1,
 *     the sentence after Eq. 6); Eq. 6 itself is garbled in the paper, its corrected form
 *     dT/dt = -sum_k u_k W_k omega_k / (rho c_v) is only used as a cross-check;
 *   - cells with T < T_min are not integrated (Algorithm 2/3, "T_reaction_min").
 * The method under test is an approximation of the exact solution of that ODE at t = dt;
 * the oracle therefore integrates the ODE to a tolerance far below the 1e-4 parity bar,
 * with an integrator unrelated to the GPU's: 3-stage Radau IIA (order 5), step doubling for
 * the error estimate, finite-difference Jacobian, full Newton on the 3n stage system.
 *
 * Rates use direct products of concentrations (no logarithms), k_f = A T^b exp(-Ea/RT),
 * k_r = k_f / K_c with K_c = K_p (p0/RT)^(sum dnu), ln K_p = -sum dnu_k g_k/(RT) from NASA-7.
 * Thermo outside [T_lo, T_hi] holds cp constant at the boundary value (h, s continuous).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define R_GAS 8.314462618
#define P_REF 101325.0
#define T_BRACKET_LO 50.0
#define T_BRACKET_HI 20000.0
#define MAXN 64

/* diagnostics switch for debugging the oracle itself (0 = silent) */
int o_verbose = 0;

typedef struct {
  int ns, nr;
  const double *W;        /* [ns] */
  const double *thermo;   /* [ns][9] a1..a7, T_lo, T_hi */
  const int8_t *nu_f;     /* [nr][ns] */
  const int8_t *nu_r;     /* [nr][ns] */
  const double *A, *b, *Ea;
  const uint8_t *rev, *tb;
  const double *eff;      /* [nr][ns] */
} omech;

/* ---------------- thermodynamics ---------------- */

/* cp/R, h/(RT), s/R of species k at T (NASA-7, constant-cp extrapolation). */
void o_thermo(const omech *m, int k, double T, double *cpR, double *hRT, double *sR) {
  const double *a = m->thermo + 9 * k;
  double Te = T;
  if (Te < a[7]) Te = a[7];
  if (Te > a[8]) Te = a[8];
  double cp = a[0] + a[1] * Te + a[2] * Te * Te + a[3] * pow(Te, 3) + a[4] * pow(Te, 4);
  double h = a[0] * Te + a[1] * Te * Te / 2.0 + a[2] * pow(Te, 3) / 3.0 + a[3] * pow(Te, 4) / 4.0 +
             a[4] * pow(Te, 5) / 5.0 + a[5];
  double s = a[0] * log(Te) + a[1] * Te + a[2] * Te * Te / 2.0 + a[3] * pow(Te, 3) / 3.0 +
             a[4] * pow(Te, 4) / 4.0 + a[6];
  if (Te != T) {
    h += cp * (T - Te);
    s += cp * log(T / Te);
  }
  if (cpR) *cpR = cp;
  if (hRT) *hRT = h / T;
  if (sR) *sR = s;
}

/* mass-specific internal energy of species k, J/kg: u = (h - R T) / W */
double o_u_species(const omech *m, int k, double T) {
  double hRT;
  o_thermo(m, k, T, NULL, &hRT, NULL);
  return R_GAS * T * (hRT - 1.0) / m->W[k];
}

/* mixture e(T) = sum Y_k u_k(T) and c_v = sum Y_k cv_k (J/kg, J/kg/K) */
void o_mixture_energy(const omech *m, const double *Y, double T, double *e, double *cv) {
  double se = 0.0, sc = 0.0;
  for (int k = 0; k < m->ns; ++k) {
    double cpR, hRT;
    o_thermo(m, k, T, &cpR, &hRT, NULL);
    se += Y[k] * R_GAS * T * (hRT - 1.0) / m->W[k];
    sc += Y[k] * R_GAS * (cpR - 1.0) / m->W[k];
  }
  if (e) *e = se;
  if (cv) *cv = sc;
}

/* T such that e(T, Y) = e0: Newton, safeguarded by bisection on [50, 20000] K.
 * Returns T; *ok = 0 if the root is not bracketed. */
double o_T_from_e(const omech *m, const double *Y, double e0, double Tguess, int *ok) {
  double lo = T_BRACKET_LO, hi = T_BRACKET_HI, f_lo, f_hi;
  o_mixture_energy(m, Y, lo, &f_lo, NULL);
  o_mixture_energy(m, Y, hi, &f_hi, NULL);
  f_lo -= e0;
  f_hi -= e0;
  if (ok) *ok = 1;
  if (!(f_lo <= 0.0 && f_hi >= 0.0)) {
    if (ok) *ok = 0;
    return NAN;
  }
  double T = (Tguess > lo && Tguess < hi) ? Tguess : 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    double e, cv;
    o_mixture_energy(m, Y, T, &e, &cv);
    double f = e - e0;
    if (f > 0) hi = T; else lo = T;
    double Tn = (cv > 0) ? T - f / cv : 0.5 * (lo + hi);
    if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
    if (fabs(Tn - T) <= 1e-13 * T) return Tn;
    T = Tn;
  }
  return T;
}

/* ---------------- kinetics ---------------- */

/* Rates of progress q_f, q_r (third-body factor included) and species production rates
 * omega (mol/m^3/s), Eq. 5.  C_k = max(rho Y_k / W_k, 0). */
void o_rates(const omech *m, double rho, double T, const double *Y,
             double *qf_out, double *qr_out, double *omega) {
  int ns = m->ns, nr = m->nr;
  double C[MAXN], gRT[MAXN];
  for (int k = 0; k < ns; ++k) {
    /* the exact solution never has negative concentrations; round-off negatives count as 0 */
    C[k] = fmax(rho * Y[k] / m->W[k], 0.0);
    double hRT, sR;
    o_thermo(m, k, T, NULL, &hRT, &sR);
    gRT[k] = hRT - sR;
  }
  for (int k = 0; k < ns; ++k) omega[k] = 0.0;
  for (int r = 0; r < nr; ++r) {
    const int8_t *nf = m->nu_f + (size_t)r * ns, *nb = m->nu_r + (size_t)r * ns;
    double kf = m->A[r] * pow(T, m->b[r]) * exp(-m->Ea[r] / (R_GAS * T));
    double qf = kf, qr = 0.0;
    for (int k = 0; k < ns; ++k)
      for (int j = 0; j < nf[k]; ++j) qf *= C[k];
    if (m->rev[r]) {
      double dG = 0.0, dn = 0.0;
      for (int k = 0; k < ns; ++k) {
        dG += (nb[k] - nf[k]) * gRT[k];
        dn += (nb[k] - nf[k]);
      }
      double Kc = exp(-dG) * pow(P_REF / (R_GAS * T), dn);
      qr = kf / Kc;
      for (int k = 0; k < ns; ++k)
        for (int j = 0; j < nb[k]; ++j) qr *= C[k];
    }
    double M = 1.0;
    if (m->tb[r]) {
      M = 0.0;
      for (int k = 0; k < ns; ++k) M += m->eff[(size_t)r * ns + k] * C[k];
    }
    if (qf_out) qf_out[r] = qf * M;
    if (qr_out) qr_out[r] = qr * M;
    double q = M * (qf - qr);
    for (int k = 0; k < ns; ++k) omega[k] += (nb[k] - nf[k]) * q;
  }
}

/* Right-hand side of Eq. 5 with T from e.  *T is the guess on entry, the solution on exit. */
static int rhs(const omech *m, double rho, double e0, const double *Y, double *T, double *f) {
  int ok;
  double Tn = o_T_from_e(m, Y, e0, *T, &ok);
  if (!ok || !(Tn > 0)) return 0;
  *T = Tn;
  double omega[MAXN];
  o_rates(m, rho, Tn, Y, NULL, NULL, omega);
  for (int k = 0; k < m->ns; ++k) f[k] = m->W[k] * omega[k] / rho;
  return 1;
}

/* ---------------- dense linear algebra ---------------- */

static int lu_factor(double *a, int n, int *piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(a[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
    piv[k] = p;
    if (best == 0.0) return 0;
    if (p != k)
      for (int j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
    for (int i = k + 1; i < n; ++i) {
      double l = a[i * n + k] / a[k * n + k];
      a[i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
    }
  }
  return 1;
}

static void lu_solve(const double *a, int n, const int *piv, double *x) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) x[i] -= a[i * n + j] * x[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) x[i] -= a[i * n + j] * x[j];
    x[i] /= a[i * n + i];
  }
}

/* ---------------- Radau IIA (3 stages, order 5) ---------------- */

static double RA[3][3], RC[3];
static int radau_ready = 0;

static void radau_init(void) {
  double s6 = sqrt(6.0);
  RC[0] = (4.0 - s6) / 10.0;
  RC[1] = (4.0 + s6) / 10.0;
  RC[2] = 1.0;
  RA[0][0] = (88.0 - 7.0 * s6) / 360.0;
  RA[0][1] = (296.0 - 169.0 * s6) / 1800.0;
  RA[0][2] = (-2.0 + 3.0 * s6) / 225.0;
  RA[1][0] = (296.0 + 169.0 * s6) / 1800.0;
  RA[1][1] = (88.0 + 7.0 * s6) / 360.0;
  RA[1][2] = (-2.0 - 3.0 * s6) / 225.0;
  RA[2][0] = (16.0 - s6) / 36.0;
  RA[2][1] = (16.0 + s6) / 36.0;
  RA[2][2] = 1.0 / 9.0;
  radau_ready = 1;
}

/* exported so that a test can check the tableau against the order conditions */
void oracle_radau_tableau(double *A9, double *c3) {
  if (!radau_ready) radau_init();
  for (int i = 0; i < 3; ++i) {
    c3[i] = RC[i];
    for (int j = 0; j < 3; ++j) A9[i * 3 + j] = RA[i][j];
  }
}

typedef struct {
  const omech *m;
  double rho, e0, rtol, atol;
} oprob;

/* finite-difference Jacobian of f at y (forward differences, FP64) */
static int fd_jacobian(const oprob *P, const double *y, const double *f0, double T, double *J) {
  int n = P->m->ns;
  double yp[MAXN], fp[MAXN];
  memcpy(yp, y, sizeof(double) * n);
  for (int j = 0; j < n; ++j) {
    double d = 1.5e-8 * fmax(fabs(y[j]), 1e-6);
    yp[j] = y[j] + d;
    double Tp = T;
    if (!rhs(P->m, P->rho, P->e0, yp, &Tp, fp)) return 0;
    for (int i = 0; i < n; ++i) J[i * n + j] = (fp[i] - f0[i]) / d;
    yp[j] = y[j];
  }
  return 1;
}

/* one Radau IIA step of size h from y; writes y1, returns 1 on Newton convergence.
 * J is the Jacobian at y. */
static int radau_step(const oprob *P, const double *y, double h, const double *J, double *T,
                      double *y1, double *lu, int *piv) {
  int n = P->m->ns, N = 3 * n;
  for (int i = 0; i < 3; ++i)
    for (int p = 0; p < n; ++p)
      for (int j = 0; j < 3; ++j)
        for (int q = 0; q < n; ++q)
          lu[(i * n + p) * N + (j * n + q)] = ((i == j && p == q) ? 1.0 : 0.0) - h * RA[i][j] * J[p * n + q];
  if (!lu_factor(lu, N, piv)) return 0;
  double Z[3 * MAXN], F[3][MAXN], res[3 * MAXN], ys[MAXN];
  memset(Z, 0, sizeof(double) * N);
  double Ts[3] = {*T, *T, *T};
  double prev = 0.0;
  for (int it = 0; it < 15; ++it) {
    for (int i = 0; i < 3; ++i) {
      for (int p = 0; p < n; ++p) ys[p] = y[p] + Z[i * n + p];
      if (!rhs(P->m, P->rho, P->e0, ys, &Ts[i], F[i])) return 0;
    }
    for (int i = 0; i < 3; ++i)
      for (int p = 0; p < n; ++p) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j) s += RA[i][j] * F[j][p];
        res[i * n + p] = -(Z[i * n + p] - h * s);
      }
    lu_solve(lu, N, piv, res);
    double nrm = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int p = 0; p < n; ++p) {
        Z[i * n + p] += res[i * n + p];
        double w = P->atol + P->rtol * fabs(y[p]);
        double v = fabs(res[i * n + p]) / w;
        if (v > nrm) nrm = v;
      }
    if (!(nrm == nrm)) return 0;
    /* converged when the update, or the remaining error estimated from the contraction
     * rate theta, is far below the integration tolerance */
    double theta = (it > 0 && prev > 0) ? nrm / prev : 1.0;
    if (o_verbose > 1) fprintf(stderr, "      newton h=%.3e it=%d nrm=%.3e\n", h, it, nrm);
    int conv = nrm < 1e-2 || (it > 0 && theta < 0.9 && nrm * theta / (1.0 - theta) < 1e-2);
    if (conv) {
      for (int p = 0; p < n; ++p) y1[p] = y[p] + Z[2 * n + p];
      *T = Ts[2];
      return 1;
    }
    if (it > 0 && theta >= 1.0) return 0;   /* diverging */
    prev = nrm;
  }
  return 0;
}

/* Integrate one cell over [0, dt].  Y (in/out), T (in: guess; out: final).  Returns
 * the number of accepted steps, or -1 on failure. */
int o_integrate_cell(const omech *m, double rho, double e0, double *Y, double *T, double dt,
                     double rtol, double atol, int max_steps) {
  if (!radau_ready) radau_init();
  int n = m->ns;
  oprob P = {m, rho, e0, rtol, atol};
  double y[MAXN], f0[MAXN], J[MAXN * MAXN], yfull[MAXN], yhalf[MAXN], y2[MAXN];
  int N = 3 * n;
  double *lu = (double *)malloc(sizeof(double) * N * N);
  int *piv = (int *)malloc(sizeof(int) * N);
  memcpy(y, Y, sizeof(double) * n);
  double t = 0.0, Tc = *T;
  if (!rhs(m, rho, e0, y, &Tc, f0)) { free(lu); free(piv); return -1; }
  double h = fmin(dt, 1e-12);
  int steps = 0, fails = 0;
  while (t < dt) {
    if (steps + fails > max_steps) { free(lu); free(piv); return -1; }
    int last = 0;
    if (t + h >= dt) { h = dt - t; last = 1; }
    if (!fd_jacobian(&P, y, f0, Tc, J)) { free(lu); free(piv); return -1; }
    double T1 = Tc, T2 = Tc, Th = Tc;
    int ok = radau_step(&P, y, h, J, &T1, yfull, lu, piv);
    if (ok) ok = radau_step(&P, y, 0.5 * h, J, &Th, yhalf, lu, piv);
    double fh[MAXN];
    if (ok) {
      T2 = Th;
      double Jh[MAXN * MAXN];
      ok = rhs(m, rho, e0, yhalf, &T2, fh) && fd_jacobian(&P, yhalf, fh, T2, Jh) &&
           radau_step(&P, yhalf, 0.5 * h, Jh, &T2, y2, lu, piv);
    }
    if (o_verbose) fprintf(stderr, "t=%.6e h=%.3e ok=%d steps=%d fails=%d T=%.3f\n", t, h, ok, steps, fails, Tc);
    if (!ok) {
      h *= 0.25;
      fails++;
      if (h < 1e-30) { free(lu); free(piv); return -1; }
      continue;
    }
    /* step doubling: error of the two-half-step solution, order 5 => divide by 2^5 - 1 */
    double err = 0.0;
    int arg = -1;
    for (int p = 0; p < n; ++p) {
      double e = (y2[p] - yfull[p]) / 31.0;
      double w = atol + rtol * fmax(fabs(y[p]), fabs(y2[p]));
      double v = fabs(e) / w;
      if (v > err) { err = v; arg = p; }
    }
    if (o_verbose) fprintf(stderr, "   argmax species %d y=%.3e\n", arg, arg >= 0 ? y2[arg] : 0.0);
    if (err <= 1.0) {
      t = last ? dt : t + h;
      memcpy(y, y2, sizeof(double) * n);
      Tc = T2;
      steps++;
      if (!rhs(m, rho, e0, y, &Tc, f0)) { free(lu); free(piv); return -1; }
    } else {
      fails++;
    }
    double fac = (err > 0) ? 0.9 * pow(err, -1.0 / 6.0) : 4.0;
    if (fac > 4.0) fac = 4.0;
    if (fac < 0.2) fac = 0.2;
    h *= fac;
  }
  memcpy(Y, y, sizeof(double) * n);
  int okT;
  *T = o_T_from_e(m, y, e0, Tc, &okT);
  free(lu);
  free(piv);
  return okT ? steps : -1;
}

/* ---------------- batch entry points (SoA arrays, Y is [ns][ld]) ---------------- */

static omech make_mech(int ns, int nr, const double *W, const double *thermo, const int8_t *nu_f,
                       const int8_t *nu_r, const double *A, const double *b, const double *Ea,
                       const uint8_t *rev, const uint8_t *tb, const double *eff) {
  omech m = {ns, nr, W, thermo, nu_f, nu_r, A, b, Ea, rev, tb, eff};
  return m;
}

#define MECH_ARGS int ns, int nr, const double *W, const double *thermo, const int8_t *nu_f, \
  const int8_t *nu_r, const double *A, const double *b, const double *Ea, const uint8_t *rev, \
  const uint8_t *tb, const double *eff
#define MECH_PASS ns, nr, W, thermo, nu_f, nu_r, A, b, Ea, rev, tb, eff

/* rho = p / (R T sum Y/W), e = sum Y_k u_k(T) */
void oracle_state_from_TpY(MECH_ARGS, int64_t n, const double *T, const double *p,
                           const double *Y, int64_t ld, double *rho, double *e) {
  omech m = make_mech(MECH_PASS);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double y[MAXN], s = 0.0;
    for (int k = 0; k < ns; ++k) { y[k] = Y[k * ld + i]; s += y[k] / W[k]; }
    rho[i] = p[i] / (R_GAS * T[i] * s);
    o_mixture_energy(&m, y, T[i], &e[i], NULL);
  }
}

void oracle_T_from_e(MECH_ARGS, int64_t n, const double *Y, int64_t ld, const double *e,
                     const double *Tguess, double *T) {
  omech m = make_mech(MECH_PASS);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double y[MAXN];
    for (int k = 0; k < ns; ++k) y[k] = Y[k * ld + i];
    int ok;
    T[i] = o_T_from_e(&m, y, e[i], Tguess[i], &ok);
  }
}

/* dY/dt [ns][ld] at given (rho, T, Y); qf/qr [nr][n] optional (third-body factor included) */
void oracle_rates(MECH_ARGS, int64_t n, const double *rho, const double *T, const double *Y,
                  int64_t ld, double *dYdt, double *qf, double *qr) {
  omech m = make_mech(MECH_PASS);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double y[MAXN], om[MAXN], qfl[1024], qrl[1024];
    for (int k = 0; k < ns; ++k) y[k] = Y[k * ld + i];
    o_rates(&m, rho[i], T[i], y, nr <= 1024 ? qfl : NULL, nr <= 1024 ? qrl : NULL, om);
    for (int k = 0; k < ns; ++k) dYdt[k * ld + i] = W[k] * om[k] / rho[i];
    if (qf && nr <= 1024)
      for (int r = 0; r < nr; ++r) { qf[r * n + i] = qfl[r]; qr[r * n + i] = qrl[r]; }
  }
}

/* cp/R, h/RT, s/R of every species at each T [n] -> out [3][ns][n] */
void oracle_thermo(MECH_ARGS, int64_t n, const double *T, double *out) {
  omech m = make_mech(MECH_PASS);
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < ns; ++k)
      o_thermo(&m, k, T[i], &out[(0 * ns + k) * n + i], &out[(1 * ns + k) * n + i],
               &out[(2 * ns + k) * n + i]);
}

/* Advance n cells over dt (constant rho, e).  T, Y in/out; p out (p = rho R T sum Y/W).
 * Cells with T < T_min are left untouched (steps = 0).  steps[i] = accepted steps or -1. */
void oracle_advance(MECH_ARGS, int64_t n, const double *rho, const double *e, double *T,
                    double *p, double *Y, int64_t ld, double dt, double rtol, double atol,
                    double T_min, int max_steps, int32_t *steps) {
  omech m = make_mech(MECH_PASS);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i) {
    if (!(T[i] >= T_min)) { steps[i] = 0; continue; }
    double y[MAXN], Ti = T[i];
    for (int k = 0; k < ns; ++k) y[k] = Y[k * ld + i];
    int s = o_integrate_cell(&m, rho[i], e[i], y, &Ti, dt, rtol, atol, max_steps);
    steps[i] = s;
    if (s < 0) continue;
    double sw = 0.0;
    for (int k = 0; k < ns; ++k) { Y[k * ld + i] = y[k]; sw += y[k] / W[k]; }
    T[i] = Ti;
    if (p) p[i] = rho[i] * R_GAS * Ti * sw;
  }
}

/* Brute force: fixed-step backward Euler with nsteps uniform steps, full Newton with a fresh
 * FD Jacobian each iteration, converged to round-off.  Used for the step-halving pin. */
int oracle_backward_euler(MECH_ARGS, double rho, double e0, double *Y, double *T, double dt,
                          int64_t nsteps) {
  omech m = make_mech(MECH_PASS);
  oprob P = {&m, rho, e0, 1e-14, 1e-300};
  int n = ns;
  double h = dt / (double)nsteps, y[MAXN], yn[MAXN], f[MAXN], J[MAXN * MAXN], g[MAXN];
  int piv[MAXN];
  double Tc = *T;
  memcpy(y, Y, sizeof(double) * n);
  for (int64_t s = 0; s < nsteps; ++s) {
    memcpy(yn, y, sizeof(double) * n);
    int conv = 0;
    for (int it = 0; it < 30; ++it) {
      if (!rhs(&m, rho, e0, y, &Tc, f)) return 0;
      if (!fd_jacobian(&P, y, f, Tc, J)) return 0;
      for (int i = 0; i < n; ++i) {
        g[i] = -(y[i] - yn[i] - h * f[i]);
        for (int j = 0; j < n; ++j) J[i * n + j] = (i == j ? 1.0 : 0.0) - h * J[i * n + j];
      }
      if (!lu_factor(J, n, piv)) return 0;
      lu_solve(J, n, piv, g);
      double nrm = 0.0;
      for (int i = 0; i < n; ++i) {
        y[i] += g[i];
        double v = fabs(g[i]) / (1e-20 + 1e-13 * fabs(y[i]));
        if (v > nrm) nrm = v;
      }
      if (o_verbose > 1) fprintf(stderr, "      be step %lld it=%d nrm=%.3e\n", (long long)s, it, nrm);
      if (nrm < 1.0) { conv = 1; break; }
    }
    if (!conv) return 0;
  }
  memcpy(Y, y, sizeof(double) * n);
  int ok;
  *T = o_T_from_e(&m, y, e0, Tc, &ok);
  return ok;
}

/* Temperature ODE cross-check (corrected Eq. 6): integrate (Y, T) with
 * dT/dt = -sum_k u_k(T) W_k omega_k / (rho c_v), using classical RK4 with nsteps steps. */
int oracle_temperature_ode(MECH_ARGS, double rho, double *Y, double *T, double dt, int64_t nsteps) {
  omech m = make_mech(MECH_PASS);
  int n = ns;
  double h = dt / (double)nsteps;
  double y[MAXN + 1], k[4][MAXN + 1], tmp[MAXN + 1];
  memcpy(y, Y, sizeof(double) * n);
  y[n] = *T;
  for (int64_t s = 0; s < nsteps; ++s) {
    for (int st = 0; st < 4; ++st) {
      const double c = (st == 0) ? 0.0 : (st == 3 ? 1.0 : 0.5);
      for (int i = 0; i <= n; ++i) tmp[i] = y[i] + (st ? c * h * k[st - 1][i] : 0.0);
      double om[MAXN], cv, num = 0.0;
      o_rates(&m, rho, tmp[n], tmp, NULL, NULL, om);
      o_mixture_energy(&m, tmp, tmp[n], NULL, &cv);
      for (int i = 0; i < n; ++i) {
        k[st][i] = W[i] * om[i] / rho;
        num += o_u_species(&m, i, tmp[n]) * W[i] * om[i];
      }
      k[st][n] = -num / (rho * cv);
    }
    for (int i = 0; i <= n; ++i) y[i] += h * (k[0][i] + 2 * k[1][i] + 2 * k[2][i] + k[3][i]) / 6.0;
  }
  memcpy(Y, y, sizeof(double) * n);
  *T = y[n];
  return 1;
}

/* The paper's own explicit scheme (Sec. 2.1; the per-cell loop of Algorithm 2, which Algorithm 3
 * runs in pieces without changing any cell's sequence of substeps): forward Euler on Eq. 5 with
 * each substep as long as keeps every |dY_k| within frac * max(|Y_k|, y_floor) and never past dt,
 * T from e after every substep.  Cells with T < T_min are untouched (steps 0); steps = -1 when
 * k_max substeps do not reach dt or T(e) fails (the state reached is kept). */
void oracle_explicit(MECH_ARGS, int64_t n, const double *rho, const double *e, double *T, double *p,
                     double *Y, int64_t ld, double dt, double frac, double y_floor, double T_min,
                     int64_t k_max, int64_t *steps) {
  omech m = make_mech(MECH_PASS);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i) {
    if (!(T[i] >= T_min)) { steps[i] = 0; continue; }
    double y[MAXN], S[MAXN], om[MAXN];
    for (int k = 0; k < ns; ++k) y[k] = Y[k * ld + i];
    int ok;
    double Ti = o_T_from_e(&m, y, e[i], T[i], &ok);
    double t = 0.0;
    int64_t K = 0;
    while (ok && t < dt && K < k_max) {
      o_rates(&m, rho[i], Ti, y, NULL, NULL, om);
      const double rem = dt - t;
      double h = rem;
      for (int k = 0; k < ns; ++k) {
        S[k] = W[k] * om[k] / rho[i];
        if (S[k] != 0.0) h = fmin(h, frac * fmax(fabs(y[k]), y_floor) / fabs(S[k]));
      }
      double y1[MAXN];
      for (int k = 0; k < ns; ++k) y1[k] = y[k] + h * S[k];
      double T1 = o_T_from_e(&m, y1, e[i], Ti, &ok);
      if (!ok) break;
      memcpy(y, y1, sizeof(double) * ns);
      Ti = T1;
      t = h >= rem ? dt : t + h;
      ++K;
    }
    steps[i] = (ok && t >= dt) ? K : -1;
    double sw = 0.0;
    for (int k = 0; k < ns; ++k) { Y[k * ld + i] = y[k]; sw += y[k] / W[k]; }
    T[i] = Ti;
    if (p) p[i] = rho[i] * R_GAS * Ti * sw;
  }
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
