/*
 * qed_oracle.c -- plain, slow, FP64 CPU oracle of the QED Monte-Carlo particle step of
 * Ridgers et al., "Modelling Gamma-Ray Photon Emission & Pair Production in High-Intensity
 * Laser-Matter Interactions" (arXiv:1311.5551).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls this file:
 * only the test-suite, the smoke check and the CPU-baseline leg of the benchmark use it.
 * It shares no code, header, table or constant generator with the CUDA library.
 *
 * Every quantity is IEEE double.  Compile with -ffp-contract=off so that results do not
 * depend on whether the host compiler fuses multiply-adds.
 *
 * Units used throughout (the paper's normalisation, Sec. 2):
 *   momenta u = p/(m_e c); photon momentum k = (h nu/m_e c^2) * khat, eps = |k|;
 *   fields E and cB in units of the Schwinger field E_s;
 *   time in units of hbar/(m_e c^2) (so e E_s/(m_e c) = 1), length in hbar/(m_e c).
 * In these units du/dt = q (E + (u/gamma) x cB) and dx/dt = u/gamma.
 *
 * Parity unpinned: the inverse-CDF interpolation artefacts of P_chi and P_f (Sec. 3) between the
 * table nodes have no printed values; they are pinned only statistically (moments and KS against
 * quadrature).  At the nodes the inversion is pinned exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_ALPHA 7.2973525693e-3 /* fine-structure constant (CODATA 2018) */

/* =====================================================================================
 * 1. Modified Bessel functions of the second kind from their integral representations.
 *    K_nu(x)  = int_0^inf exp(-x cosh t) cosh(nu t) dt
 *    Ki_nu(y) = int_y^inf K_nu(s) ds = int_0^inf exp(-y cosh t) cosh(nu t) / cosh t dt
 *    The integrands are even and analytic in a strip about the real axis, so the
 *    trapezoid rule converges exponentially in 1/h.  For large x the integrand is a
 *    Gaussian of width 1/sqrt(x) about t = 0 and the step shrinks accordingly.
 * ===================================================================================== */
static double trap_h(double x) { double h = 0.25 / sqrt(x); return h < 0.1 ? h : 0.1; }

/* One trapezoid sum of exp(-x cosh t) * w(t), w(t) = cosh(nu t) [/cosh t if over_cosh]. */
static double bessel_trap(double nu, double x, int over_cosh) {
  if (!(x > 0.0)) return INFINITY;
  if (x > 745.0) return 0.0; /* exp(-x) underflows double */
  const double h = trap_h(x);
  const double t_peak = asinh(nu / x);
  double sum = 0.5 * exp(-x); /* t = 0 term, halved */
  for (int m = 1; m < 200000; ++m) {
    const double t = m * h, ch = cosh(t);
    const double arg = x * ch;
    if (arg > 745.0 + nu * t) break; /* remaining terms underflow */
    double term = cosh(nu * t) * exp(-arg);
    if (over_cosh) term /= ch;
    sum += term;
    if (t > t_peak && term < 1e-18 * sum) break;
  }
  return h * sum;
}

double orc_besselk(double nu, double x) { return bessel_trap(nu, x, 0); }
double orc_besselk_int(double nu, double y) { return bessel_trap(nu, y, 1); }

/* =====================================================================================
 * 2. Adaptive Gauss-Legendre quadrature.  Nodes and weights of the n-point rule are found
 *    by Newton iteration on the Legendre polynomial P_n (three-term recurrence).
 * ===================================================================================== */
#define GL_N 10
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

static void gl_init(void) {
  if (gl_ready) return;
  for (int i = 0; i < GL_N; ++i) {
    double x = cos(ORC_PI * (i + 0.75) / (GL_N + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= GL_N; ++k) { double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
      dp = GL_N * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-17) break;
    }
    gl_x[i] = x;
    gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  gl_ready = 1;
}

typedef double (*orc_fn)(double v, const void* ctx);

static double gl_fixed(orc_fn f, const void* ctx, double a, double b) {
  const double c = 0.5 * (a + b), r = 0.5 * (b - a);
  double s = 0.0;
  for (int i = 0; i < GL_N; ++i) s += gl_w[i] * f(c + r * gl_x[i], ctx);
  return r * s;
}

static double gl_adapt_rec(orc_fn f, const void* ctx, double a, double b, double whole, double abstol, int depth) {
  const double m = 0.5 * (a + b);
  const double left = gl_fixed(f, ctx, a, m), right = gl_fixed(f, ctx, m, b);
  const double both = left + right;
  /* accept when within the share of the tolerance, or when the difference is at the
   * level of the round-off of the integrand values themselves (about 1e-15 relative) */
  const double diff = fabs(both - whole);
  if (depth >= 40 || diff <= abstol || diff <= 2e-14 * fabs(both)) return both;
  return gl_adapt_rec(f, ctx, a, m, left, 0.5 * abstol, depth + 1) +
         gl_adapt_rec(f, ctx, m, b, right, 0.5 * abstol, depth + 1);
}

/* Integral of f over [a,b] to an absolute tolerance abstol. */
double orc_integrate(orc_fn f, const void* ctx, double a, double b, double abstol) {
  gl_init();
  if (!(b > a)) return 0.0;
  return gl_adapt_rec(f, ctx, a, b, gl_fixed(f, ctx, a, b), abstol, 0);
}

/* =====================================================================================
 * 3. Emissivities (Appendices A and B).
 * ===================================================================================== */

/* Quantum synchrotron function F(eta, chi), App. A: for chi < eta/2
 *   F = (4 chi^2/eta^2) y K_{2/3}(y) + (1 - 2 chi/eta) y Ki_{5/3}(y),
 *   y = 4 chi / [3 eta (eta - 2 chi)];   F = 0 for chi >= eta/2.
 * Written in xi = 2 chi/eta (so 4chi^2/eta^2 = xi^2 and y = 2 xi/[3 eta (1 - xi)]);
 * one_minus_xi is passed separately so that it keeps full precision near xi = 1. */
static double F_xi(double eta, double xi, double one_minus_xi) {
  if (!(xi > 0.0) || !(one_minus_xi > 0.0)) return 0.0;
  const double y = 2.0 * xi / (3.0 * eta * one_minus_xi);
  return xi * xi * y * orc_besselk(2.0 / 3.0, y) + one_minus_xi * y * orc_besselk_int(5.0 / 3.0, y);
}

double orc_F(double eta, double chi) {
  if (!(eta > 0.0) || !(chi > 0.0) || chi >= 0.5 * eta) return 0.0;
  return F_xi(eta, 2.0 * chi / eta, (eta - 2.0 * chi) / eta);
}

/* Classical synchrotron spectrum, App. A: F_c = y_c Ki_{5/3}(y_c), y_c = 4 chi/(3 eta^2). */
double orc_F_classical(double eta, double chi) {
  const double yc = 4.0 * chi / (3.0 * eta * eta);
  return yc * orc_besselk_int(5.0 / 3.0, yc);
}

typedef struct { double eta; } eta_ctx;

/* Integrands in s, xi = s^3 (removes the xi^{-2/3} endpoint behaviour of F/xi). */
static double ig_F_over_xi_s(double s, const void* c) { /* (F/xi) dxi = 3 F / s ds */
  const double eta = ((const eta_ctx*)c)->eta;
  if (!(s > 0.0)) return 0.0;
  const double xi = s * s * s, omx = (1.0 - s) * (1.0 + s + s * s);
  return 3.0 * F_xi(eta, xi, omx) / s;
}
static double ig_F_s(double s, const void* c) { /* F dxi = 3 s^2 F ds */
  const double eta = ((const eta_ctx*)c)->eta;
  if (!(s > 0.0)) return 0.0;
  const double xi = s * s * s, omx = (1.0 - s) * (1.0 + s + s * s);
  return 3.0 * s * s * F_xi(eta, xi, omx);
}
/* xi and 1 - xi from zeta = ln(xi/(1-xi)), each to full relative precision. */
static double xi_of_zeta(double z) { return 1.0 / (1.0 + exp(-z)); }
static double omxi_of_zeta(double z) { return 1.0 / (1.0 + exp(z)); }

/* Integrand in zeta: dxi = xi (1-xi) dzeta, so (F/xi) dxi = F (1-xi) dzeta. */
static double ig_F_zeta(double z, const void* c) {
  const double eta = ((const eta_ctx*)c)->eta;
  const double omx = omxi_of_zeta(z);
  return F_xi(eta, xi_of_zeta(z), omx) * omx;
}

/* Integral over xi in [0,1] of an s-integrand; a coarse pass sets the absolute tolerance. */
static double int01_s(orc_fn f, double eta, double rel) {
  eta_ctx c = {eta};
  const double rough = orc_integrate(f, &c, 0.0, 1.0, 1e-6 * 5.0);
  return orc_integrate(f, &c, 0.0, 1.0, rel * fabs(rough));
}

/* h(eta) = int_0^{eta/2} F/chi dchi = int_0^1 F/xi dxi   (App. A). */
double orc_h(double eta) { return int01_s(ig_F_over_xi_s, eta, 1e-15); }

/* g(eta) = 3 sqrt3/(2 pi eta^2) int_0^{eta/2} F dchi = 3 sqrt3/(4 pi eta) int_0^1 F dxi. */
double orc_g(double eta) { return 3.0 * sqrt(3.0) / (4.0 * ORC_PI * eta) * int01_s(ig_F_s, eta, 1e-15); }

/* Fit of g quoted in Sec. 2.1. */
double orc_g_fit(double eta) {
  return pow(1.0 + 4.8 * (1.0 + eta) * log(1.0 + 1.7 * eta) + 2.44 * eta * eta, -2.0 / 3.0);
}

/* Pair emissivity, App. B: T(chi) = 0.16 K_{1/3}^2[2/(3 chi)] / chi. */
double orc_T(double chi) {
  if (!(chi > 0.0)) return 0.0;
  const double k = orc_besselk(1.0 / 3.0, 2.0 / (3.0 * chi));
  return 0.16 * k * k / chi;
}

/* Unnormalised pair-split density, App. B: [2 + f(1-f)]/[f(1-f)] K_{2/3}[1/(3 chi f (1-f))].
 * Dividing by k(chi) = int_0^1 of it gives p_f. */
double orc_pf_unnorm(double f, double chi) {
  const double q = f * (1.0 - f);
  if (!(q > 0.0) || !(chi > 0.0)) return 0.0;
  return (2.0 + q) / q * orc_besselk(2.0 / 3.0, 1.0 / (3.0 * q * chi));
}

typedef struct { double chi; } chi_ctx;
static double ig_pf(double f, const void* c) { return orc_pf_unnorm(f, ((const chi_ctx*)c)->chi); }

/* k(chi) = int_0^1 [unnormalised p_f] df   (App. B normalisation). */
double orc_k(double chi) {
  chi_ctx c = {chi};
  const double rough = orc_integrate(ig_pf, &c, 0.0, 0.5, 1e-6 * orc_pf_unnorm(0.5, chi));
  return 2.0 * orc_integrate(ig_pf, &c, 0.0, 0.5, 1e-15 * rough);
}

/* =====================================================================================
 * 4. Look-up tables (Sec. 3).
 *    eta grid : ln eta_i = ln eta_min + i d_eta, i = 0..n_eta-1.
 *    ln_h[i]  : ln h(eta_i);   g[i] : g(eta_i).
 *    Photon-energy cumulative P_chi at eta_i, as a function of xi = 2chi/eta:
 *      xi_min(eta_i) is the cut-off of Sec. 3: the photons below it carry 1e-9 (energy_cut)
 *      of the spectrum's energy, int_0^{xi_min} F dxi = cut * int_0^1 F dxi.
 *      Nodes are uniform in zeta = ln(xi/(1-xi)) from zeta_lo = logit(xi_min) to
 *      zeta_hi = ln(90 eta), where y = 2xi/(3 eta (1-xi)) = 60 and the spectrum is below
 *      e^-60 of its peak, so both the low-energy end and the xi -> 1 tail are resolved:
 *      xi_ij = 1/(1 + exp(-zeta_ij)), zeta_ij = zeta_lo_i + j (zeta_hi_i - zeta_lo_i)/(n_xi-1).
 *      P[i][j] = int_0^{xi_ij} (F/xi) dxi / h(eta_i)  (includes the ignored photons), and
 *      Q[i][j] = int_{xi_ij}^1 (F/xi) dxi / h(eta_i)  (its complement, kept for precision).
 *    chi grid : ln chi_k = ln chi_min + k d_chi;   ln_T[k] = ln T(chi_k).
 *    Pair split, half-table by the symmetry p_f(f) = p_f(1-f) of App. B: f_j = j/(2(n_f-1)),
 *      Pf[k][j] = int_0^{f_j} p_f df / int_0^{1/2} p_f df.
 * ===================================================================================== */
typedef struct {
  int n_eta, n_xi, n_chi, n_f;
  double ln_eta_min, ln_eta_max, ln_chi_min, ln_chi_max, energy_cut;
  double* ln_h;      /* [n_eta] */
  double* g;         /* [n_eta] */
  double* zeta_lo;   /* [n_eta] logit(xi_min) */
  double* zeta_hi;   /* [n_eta] ln(90 eta) */
  double* P;         /* [n_eta * n_xi] */
  double* Q;         /* [n_eta * n_xi] */
  double* ln_T;      /* [n_chi] */
  double* Pf;        /* [n_chi * n_f] */
} orc_tables;

/* Energy fraction below xi: int_0^xi F dxi' / int_0^1 F dxi'. */
static double energy_below(double eta, double xi, double total_F, double rel) {
  eta_ctx c = {eta};
  return orc_integrate(ig_F_s, &c, 0.0, cbrt(xi), rel * total_F) / total_F;
}

/* Solve energy_below(xi) = cut for xi by Newton iteration in ln xi (d/dln xi = xi F / total). */
static double find_xi_min(double eta, double cut, double total_F) {
  /* classical small-xi behaviour F ~ c xi^{1/3} gives a starting guess; refine */
  double lx = log(1e-3 * eta < 1e-3 ? 1e-3 * eta : 1e-3);
  for (int it = 0; it < 200; ++it) {
    const double xi = exp(lx);
    const double e = energy_below(eta, xi, total_F, 1e-16);
    const double de = xi * F_xi(eta, xi, -expm1(lx)) / total_F;
    double step = (e - cut) / de;
    /* guard: e(xi) grows like xi^{4/3}; limit the step in ln xi */
    if (step > 2.0) step = 2.0;
    if (step < -2.0) step = -2.0;
    lx -= step;
    if (fabs(step) < 1e-14) break;
  }
  return lx;
}

static void build_eta_row(orc_tables* T, int i) {
  const double d_eta = (T->ln_eta_max - T->ln_eta_min) / (T->n_eta - 1);
  const double eta = exp(T->ln_eta_min + i * d_eta);
  eta_ctx c = {eta};
  const double h = orc_h(eta);
  const double totF = int01_s(ig_F_s, eta, 1e-15);
  T->ln_h[i] = log(h);
  T->g[i] = 3.0 * sqrt(3.0) / (4.0 * ORC_PI * eta) * totF;
  const double lxm = find_xi_min(eta, T->energy_cut, totF);
  const double zlo = lxm - log(-expm1(lxm)), zhi = log(90.0 * eta);
  T->zeta_lo[i] = zlo;
  T->zeta_hi[i] = zhi;
  const int n = T->n_xi;
  double* P = T->P + (size_t)i * n;
  double* Q = T->Q + (size_t)i * n;
  /* interval integrals in zeta between consecutive nodes */
  double* I = (double*)malloc(sizeof(double) * n);
  for (int j = 0; j + 1 < n; ++j) {
    const double z0 = zlo + j * (zhi - zlo) / (n - 1), z1 = zlo + (j + 1) * (zhi - zlo) / (n - 1);
    I[j] = orc_integrate(ig_F_zeta, &c, z0, z1, 1e-17 * h);
  }
  /* below the first node: int_0^{xi_min} F/xi dxi in s = xi^{1/3};
   * above the last node: the e^-60 tail, in zeta up to where F underflows */
  const double below = orc_integrate(ig_F_over_xi_s, &c, 0.0, exp(lxm / 3.0), 1e-17 * h);
  const double above = orc_integrate(ig_F_zeta, &c, zhi, zhi + 8.0, 1e-30 * h);
  double acc = below;
  P[0] = below / h;
  for (int j = 1; j < n; ++j) { acc += I[j - 1]; P[j] = acc / h; }
  acc = above;
  Q[n - 1] = above / h;
  for (int j = n - 2; j >= 0; --j) { acc += I[j]; Q[j] = acc / h; }
  free(I);
}

static void build_chi_row(orc_tables* T, int k) {
  const double d_chi = (T->ln_chi_max - T->ln_chi_min) / (T->n_chi - 1);
  const double chi = exp(T->ln_chi_min + k * d_chi);
  T->ln_T[k] = log(orc_T(chi));
  chi_ctx c = {chi};
  const int n = T->n_f;
  double* Pf = T->Pf + (size_t)k * n;
  const double half = orc_integrate(ig_pf, &c, 0.0, 0.5, 1e-6 * orc_pf_unnorm(0.5, chi));
  double acc = 0.0;
  Pf[0] = 0.0;
  double total = 0.0;
  double* J = (double*)malloc(sizeof(double) * n);
  for (int j = 0; j + 1 < n; ++j) {
    const double f0 = 0.5 * j / (n - 1), f1 = 0.5 * (j + 1) / (n - 1);
    J[j] = orc_integrate(ig_pf, &c, f0, f1, 1e-17 * half);
    total += J[j];
  }
  for (int j = 1; j < n; ++j) { acc += J[j - 1]; Pf[j] = acc / total; }
  Pf[n - 1] = 1.0;
  free(J);
}

/* Fill all tables; the caller owns the arrays.  Rows are independent (OpenMP over rows). */
int orc_tables_build(orc_tables* T) {
  gl_init();
  if (T->n_eta < 2 || T->n_xi < 2 || T->n_chi < 2 || T->n_f < 2) return 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < T->n_eta; ++i) build_eta_row(T, i);
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < T->n_chi; ++k) build_chi_row(T, k);
  return 0;
}

/* ---------- table look-ups: linear interpolation (Sec. 3) ----------
 * Reading: h and T are interpolated linearly in (ln eta, ln h) and (ln chi, ln T). */
static void grid_pos(double lnv, double lo, double hi, int n, int* idx, double* w, int* oor) {
  const double d = (hi - lo) / (n - 1);
  double s = (lnv - lo) / d;
  *oor = 0;
  if (!(s > 0.0)) { *idx = 0; *w = 0.0; if (s < 0.0) *oor = -1; return; }
  if (s >= n - 1) { *idx = n - 2; *w = 1.0; if (s > n - 1) *oor = 1; return; }
  int i = (int)floor(s);
  if (i > n - 2) i = n - 2;
  *idx = i;
  *w = s - i;
}

/* h(eta) by table; eta above the table is clamped (and flagged by *oor = 1). */
double orc_lookup_h(const orc_tables* T, double eta, int* oor) {
  int i, o; double w;
  grid_pos(log(eta), T->ln_eta_min, T->ln_eta_max, T->n_eta, &i, &w, &o);
  if (oor) *oor = o;
  return exp((1.0 - w) * T->ln_h[i] + w * T->ln_h[i + 1]);
}

/* T(chi) by table: 0 below the table; chi^{-1/3} continuation above it (App. B). */
double orc_lookup_T(const orc_tables* T, double chi, int* oor) {
  if (oor) *oor = 0;
  if (!(chi >= exp(T->ln_chi_min))) return 0.0;
  int i, o; double w;
  grid_pos(log(chi), T->ln_chi_min, T->ln_chi_max, T->n_chi, &i, &w, &o);
  if (o > 0) {
    if (oor) *oor = 1;
    return exp(T->ln_T[T->n_chi - 1]) * pow(chi / exp(T->ln_chi_max), -1.0 / 3.0);
  }
  return exp((1.0 - w) * T->ln_T[i] + w * T->ln_T[i + 1]);
}

/* Invert one P_chi row at U (with V = 1 - U): xi linearly interpolated in P between the
 * bracketing nodes.  The complement Q is used when U > 1/2 (same interpolation, kept
 * precise near P = 1).  U at or below the first node returns xi_min. */
static double invert_xi_row(const orc_tables* T, int r, double U, double V) {
  const int n = T->n_xi;
  const double* P = T->P + (size_t)r * n;
  const double* Q = T->Q + (size_t)r * n;
  const double zlo = T->zeta_lo[r], zhi = T->zeta_hi[r];
  if (U <= P[0]) return xi_of_zeta(zlo);
  if (V <= Q[n - 1]) return xi_of_zeta(zhi);
  int j;
  double frac;
  if (U <= 0.5) {
    int lo = 0, hi = n - 1; /* invariant P[lo] < U <= P[hi] */
    while (hi - lo > 1) { const int mid = (lo + hi) / 2; if (P[mid] < U) lo = mid; else hi = mid; }
    j = lo;
    frac = (U - P[j]) / (P[j + 1] - P[j]);
  } else {
    int lo = 0, hi = n - 1; /* invariant Q[lo] > V >= Q[hi] */
    while (hi - lo > 1) { const int mid = (lo + hi) / 2; if (Q[mid] > V) lo = mid; else hi = mid; }
    j = lo;
    frac = (Q[j] - V) / (Q[j] - Q[j + 1]);
  }
  const double x0 = xi_of_zeta(zlo + j * (zhi - zlo) / (n - 1));
  const double x1 = xi_of_zeta(zlo + (j + 1) * (zhi - zlo) / (n - 1));
  return x0 + frac * (x1 - x0);
}

/* Photon-energy sample, Sec. 3: returns 1 and *xi = 2chi/eta for the photon, or 0 when U
 * falls below the cut-off (the photon is ignored).  Between eta rows xi is interpolated
 * linearly in ln eta; below the table it keeps the classical scaling xi ~ eta. */
int orc_sample_xi(const orc_tables* T, double eta, double U, double* xi) {
  const double V = 1.0 - U;
  int i, o; double w;
  grid_pos(log(eta), T->ln_eta_min, T->ln_eta_max, T->n_eta, &i, &w, &o);
  const int n = T->n_xi;
  const double pcut = (1.0 - w) * T->P[(size_t)i * n] + w * T->P[(size_t)(i + 1) * n];
  if (U < pcut) return 0;
  double x = (1.0 - w) * invert_xi_row(T, i, U, V);
  if (w > 0.0) x += w * invert_xi_row(T, i + 1, U, V);
  if (o < 0) x *= eta / exp(T->ln_eta_min);
  if (x > 1.0) x = 1.0;
  *xi = x;
  return 1;
}

static double invert_f_row(const orc_tables* T, int r, double V) {
  const int n = T->n_f;
  const double* P = T->Pf + (size_t)r * n;
  int lo = 0, hi = n - 1; /* P[lo] < V <= P[hi] */
  while (hi - lo > 1) { const int mid = (lo + hi) / 2; if (P[mid] < V) lo = mid; else hi = mid; }
  const double frac = (V - P[lo]) / (P[lo + 1] - P[lo]);
  const double f0 = 0.5 * lo / (n - 1), f1 = 0.5 * (lo + 1) / (n - 1);
  return f0 + frac * (f1 - f0);
}

/* Pair-split sample, Sec. 3 / App. B: the positron's energy fraction f.  U < 1/2 maps to
 * the lower half (f <= 1/2) via V = 2U, U >= 1/2 to the upper half via V = 2(1-U). */
double orc_sample_f(const orc_tables* T, double chi, double U) {
  int i, o; double w;
  grid_pos(log(chi), T->ln_chi_min, T->ln_chi_max, T->n_chi, &i, &w, &o);
  const int lower = U < 0.5;
  const double V = lower ? 2.0 * U : 2.0 * (1.0 - U);
  double fh = (1.0 - w) * invert_f_row(T, i, V);
  if (w > 0.0) fh += w * invert_f_row(T, i + 1, V);
  return lower ? fh : 1.0 - fh;
}

/* =====================================================================================
 * 5. Philox4x64-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11).
 * ===================================================================================== */
void orc_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    const unsigned __int128 p0 = (unsigned __int128)M0 * c0, p1 = (unsigned __int128)M1 * c2;
    const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform double strictly inside (0,1) from the top 52 bits of a word: (m + 1/2) 2^-52 with
 * m < 2^52 is exact in double, so the largest value is 1 - 2^-53 and the smallest 2^-53. */
double orc_u01(uint64_t w) { return ((double)(w >> 12) + 0.5) * 0x1.0p-52; }

enum { ORC_ELECTRON = 0, ORC_POSITRON = 1, ORC_PHOTON = 2 };
enum { ORC_PURPOSE_EVENT = 0, ORC_PURPOSE_INIT = 1 };

/* Stream layout: key = (seed, scenario); counter = (particle id, step, species kind, purpose). */
static void draw4(uint64_t seed, uint64_t scenario, uint64_t id, uint64_t step, uint64_t kind, uint64_t purpose, double U[4]) {
  const uint64_t ctr[4] = {id, step, kind, purpose}, key[2] = {seed, scenario};
  uint64_t w[4];
  orc_philox4x64(ctr, key, w);
  for (int i = 0; i < 4; ++i) U[i] = orc_u01(w[i]);
}

/* =====================================================================================
 * 6. Fields (the analytic stand-ins for the PIC gather of Sec. 3.2).
 * ===================================================================================== */
enum { ORC_FIELD_UNIFORM = 0, ORC_FIELD_ROTATING_E = 1, ORC_FIELD_PLANE_LP = 2, ORC_FIELD_PLANE_CP = 3,
       ORC_FIELD_GRID = 4 };

typedef struct {
  int kind;
  double E[3], B[3];       /* uniform E and cB */
  double E0;               /* amplitude (rotating E, plane waves) */
  double omega;            /* angular frequency; for plane waves also the wavenumber (c = 1) */
  double phase0;           /* rotating E: E = E0 (cos(omega t + phase0), sin(omega t + phase0), 0) */
  double phi_start;        /* plane wave: phase phi = omega (t - x) - phi_start */
  double phi_len;          /* sin^2 field envelope over 0 <= phi <= phi_len; <= 0: no envelope */
  /* grid: components Ex, Ey, Ez, cBx, cBy, cBz, each n[0]*n[1]*n[2] values, x fastest */
  const double* grid;
  int n[3];
  int shape;               /* 1: cloud-in-cell, 2: triangular-shaped cloud */
  double origin[3], spacing[3];
} orc_field;

/* Weight of grid node i for a particle at continuous index s (node units) with the particle
 * shape of the PIC gather (Sec. 3.2; the paper does not fix the shape, the two usual ones are
 * offered): the overlap of a cell-wide top hat (cloud-in-cell) or of a triangle two cells wide
 * (triangular-shaped cloud) centred on the particle with the node's cell. */
static double orc_shape_weight(int shape, double s, int i) {
  const double d = fabs(s - (double)i);
  if (shape == 1) return d < 1.0 ? 1.0 - d : 0.0;
  if (d <= 0.5) return 0.75 - d * d;
  if (d < 1.5) return 0.5 * (1.5 - d) * (1.5 - d);
  return 0.0;
}

/* Component c (0..2: E_x..E_z, 3..5: cB_x..cB_z) at x, Yee-staggered: E_c sits half a cell along
 * axis c, cB_c half a cell along the two other axes.  Sum over every grid node of
 * weight_x * weight_y * weight_z * value (nodes outside the grid do not exist). */
static double orc_grid_component(const orc_field* F, int c, const double x[3]) {
  double s[3];
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    const int staggered = c < 3 ? (a == c) : (a != c - 3);
    s[a] = (x[a] - F->origin[a]) / F->spacing[a] - (staggered ? 0.5 : 0.0);
    /* the nodes whose weight can be non-zero */
    lo[a] = (int)floor(s[a]) - 2;
    hi[a] = (int)floor(s[a]) + 2;
    if (lo[a] < 0) lo[a] = 0;
    if (hi[a] > F->n[a] - 1) hi[a] = F->n[a] - 1;
  }
  const size_t N = (size_t)F->n[0] * F->n[1] * F->n[2];
  const double* G = F->grid + (size_t)c * N;
  double v = 0.0;
  for (int k = lo[2]; k <= hi[2]; ++k)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int i = lo[0]; i <= hi[0]; ++i) {
        const double w = orc_shape_weight(F->shape, s[0], i) * orc_shape_weight(F->shape, s[1], j) *
                         orc_shape_weight(F->shape, s[2], k);
        if (w != 0.0) v += w * G[((size_t)k * F->n[1] + j) * F->n[0] + i];
      }
  return v;
}

void orc_field_eval(const orc_field* F, double t, const double x[3], double E[3], double B[3]) {
  E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = 0.0;
  if (F->kind == ORC_FIELD_GRID) {
    /* far outside the grid nothing contributes (and floor() stays within int range) */
    for (int a = 0; a < 3; ++a) {
      const double s = (x[a] - F->origin[a]) / F->spacing[a];
      if (!(s > -3.0 && s < F->n[a] + 2.0)) return;
    }
    for (int c = 0; c < 3; ++c) {
      E[c] = orc_grid_component(F, c, x);
      B[c] = orc_grid_component(F, c + 3, x);
    }
    return;
  }
  if (F->kind == ORC_FIELD_UNIFORM) {
    for (int c = 0; c < 3; ++c) { E[c] = F->E[c]; B[c] = F->B[c]; }
  } else if (F->kind == ORC_FIELD_ROTATING_E) {
    const double ph = F->omega * t + F->phase0;
    E[0] = F->E0 * cos(ph);
    E[1] = F->E0 * sin(ph);
  } else { /* plane wave travelling along +x */
    const double phi = F->omega * (t - x[0]) - F->phi_start;
    double env = 1.0;
    if (F->phi_len > 0.0) {
      if (phi <= 0.0 || phi >= F->phi_len) return;
      const double s = sin(ORC_PI * phi / F->phi_len);
      env = s * s;
    }
    const double a = F->E0 * env;
    if (F->kind == ORC_FIELD_PLANE_LP) {
      E[1] = a * cos(phi);
      B[2] = a * cos(phi);
    } else {
      E[1] = a * cos(phi); E[2] = a * sin(phi);
      B[1] = -a * sin(phi); B[2] = a * cos(phi);
    }
  }
}

/* =====================================================================================
 * 7. Classical propagation between events: Boris push of e+- (Vlasov eq. LHS, Sec. 2.3).
 *    u^{n-1/2} -> u^{n+1/2} with the fields at (x^n, t^n):
 *    half electric kick, rotation about cB using gamma of the half-kicked momentum,
 *    second half electric kick.
 * ===================================================================================== */
void orc_boris(double q, double dt, const double E[3], const double B[3], double u[3]) {
  const double hq = 0.5 * q * dt;
  double um[3] = {u[0] + hq * E[0], u[1] + hq * E[1], u[2] + hq * E[2]};
  const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  const double tv[3] = {hq * B[0] / gm, hq * B[1] / gm, hq * B[2] / gm};
  const double t2 = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
  const double sv[3] = {2.0 * tv[0] / (1.0 + t2), 2.0 * tv[1] / (1.0 + t2), 2.0 * tv[2] / (1.0 + t2)};
  const double up[3] = {um[0] + (um[1] * tv[2] - um[2] * tv[1]),
                        um[1] + (um[2] * tv[0] - um[0] * tv[2]),
                        um[2] + (um[0] * tv[1] - um[1] * tv[0])};
  const double uq[3] = {um[0] + (up[1] * sv[2] - up[2] * sv[1]),
                        um[1] + (up[2] * sv[0] - up[0] * sv[2]),
                        um[2] + (up[0] * sv[1] - up[1] * sv[0])};
  for (int c = 0; c < 3; ++c) u[c] = uq[c] + hq * E[c];
}

/* eta = |F_{mu nu} p^nu| / (m c E_s) (Sec. 2):  eta^2 = (gamma E + u x cB)^2 - (u.E)^2,
 * evaluated as E^2 + |u x E|^2 + 2 gamma E.(u x cB) + |u x cB|^2 (same value, using
 * gamma^2 = 1 + u^2, without the cancellation of the first form when u is parallel to E). */
static void cross(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

double orc_eta(const double u[3], double gamma, const double E[3], const double B[3]) {
  double uxE[3], uxB[3];
  cross(u, E, uxE);
  cross(u, B, uxB);
  const double e2 = dot(E, E) + dot(uxE, uxE) + 2.0 * gamma * dot(E, uxB) + dot(uxB, uxB);
  return e2 > 0.0 ? sqrt(e2) : 0.0;
}

/* chi = (1/2)|F^{mu nu} k_nu| / (m c E_s) (Sec. 2, half the usual chi_gamma):
 * 4 chi^2 = (eps E + k x cB)^2 - (k.E)^2 = |k x E|^2 + 2 eps E.(k x cB) + |k x cB|^2. */
double orc_chi(const double k[3], double eps, const double E[3], const double B[3]) {
  double kxE[3], kxB[3];
  cross(k, E, kxE);
  cross(k, B, kxB);
  const double c2 = dot(kxE, kxE) + 2.0 * eps * dot(E, kxB) + dot(kxB, kxB);
  return c2 > 0.0 ? 0.5 * sqrt(c2) : 0.0;
}

/* Rates in units of m c^2/hbar:
 *   lambda_gamma = (sqrt3 alpha c/lambda_c)(eta/gamma) h(eta)  (eq. rate_photons), with
 *   lambda_c = h/(m c) so c/lambda_c = 1/(2 pi):  (sqrt3 alpha/(2 pi)) (eta/gamma) h(eta);
 *   lambda_pm = (2 pi alpha c/lambda_c)(m c^2/h nu) chi T(chi)  (eq. pair_prod_rate)
 *             = alpha (chi/eps) T(chi). */
double orc_rate_photon(const orc_tables* T, double eta, double gamma, int* oor) {
  if (!(eta > 0.0)) { if (oor) *oor = 0; return 0.0; }
  return sqrt(3.0) * ORC_ALPHA / (2.0 * ORC_PI) * (eta / gamma) * orc_lookup_h(T, eta, oor);
}
double orc_rate_pair(const orc_tables* T, double chi, double eps, int* oor) {
  if (!(chi > 0.0)) { if (oor) *oor = 0; return 0.0; }
  return ORC_ALPHA * (chi / eps) * orc_lookup_T(T, chi, oor);
}

/* =====================================================================================
 * 8. The Monte-Carlo step (Sec. 3), one scenario.
 * ===================================================================================== */
typedef struct {
  double *x, *y, *z, *ux, *uy, *uz, *tau;
  uint32_t* id;
  int64_t n, cap;
  uint32_t next_id;
  double* w;  /* macroparticle weight: the physical particles it stands for (children inherit it) */
} orc_species;

typedef struct {
  double dt, t0;
  uint64_t step, seed, scenario;
  int emit_photons, make_pairs, drain_photons;
  int recoil_energy; /* 0: momentum-conserving recoil of Sec. 3 (default); 1: energy-conserving */
  orc_field field;
} orc_step_params;

typedef struct {
  double n[3], energy[3];            /* live particles and their energy after the step */
  double emitted_n, emitted_energy;  /* photons created this step (kept or drained) */
  double dropped_n;                  /* emission events below the table cut-off */
  double emit_defect;                /* sum over emissions of (gamma_f + eps) - gamma_i */
  double pairs_n, pair_energy;       /* photons converted this step and their energy */
  double pair_defect;                /* sum over pairs of (gamma_- + gamma_+) - eps */
  double drained_n, drained_energy;
  double oor_eta, oor_chi;           /* look-ups outside the tables */
} orc_ledger;

typedef struct { double x[3], u[3], tau, w; uint32_t parent; } child_t;
typedef struct { child_t* v; int64_t n, cap; } child_list;

static void push_child(child_list* L, const child_t* c) {
  if (L->n == L->cap) { L->cap = L->cap ? 2 * L->cap : 1024; L->v = (child_t*)realloc(L->v, sizeof(child_t) * L->cap); }
  L->v[L->n++] = *c;
}

/* Kahan-compensated sum */
typedef struct { double s, c; } ksum;
static void kadd(ksum* k, double v) { const double y = v - k->c, t = k->s + y; k->c = (t - k->s) - y; k->s = t; }

static int append_children(orc_species* S, const child_list* L) {
  if (S->n + L->n > S->cap) return 2;
  for (int64_t r = 0; r < L->n; ++r) {
    const int64_t d = S->n + r;
    S->x[d] = L->v[r].x[0]; S->y[d] = L->v[r].x[1]; S->z[d] = L->v[r].x[2];
    S->ux[d] = L->v[r].u[0]; S->uy[d] = L->v[r].u[1]; S->uz[d] = L->v[r].u[2];
    S->tau[d] = L->v[r].tau;
    S->w[d] = L->v[r].w;
    S->id[d] = S->next_id + (uint32_t)r;
  }
  S->n += L->n;
  S->next_id += (uint32_t)L->n;
  return 0;
}

/* sp[0] electrons, sp[1] positrons, sp[2] photons; drained receives the emitted photons
 * when p->drain_photons (the paper deletes photons right after generation when pair
 * production is negligible, Sec. 3.1).  New particles join at the next step, ordered by
 * (parent species, parent index).  Returns 0, or 2 when a capacity would be exceeded. */
int orc_step(const orc_tables* T, const orc_step_params* p, orc_species* sp[3], orc_species* drained, orc_ledger* L) {
  const double dt = p->dt, t = p->t0 + (double)p->step * p->dt;
  const double c_gamma = sqrt(3.0) * ORC_ALPHA / (2.0 * ORC_PI);
  child_list ph_new = {0, 0, 0}, el_new = {0, 0, 0}, po_new = {0, 0, 0};
  memset(L, 0, sizeof(*L));
  ksum emitted_e = {0, 0}, defect_e = {0, 0}, pair_e = {0, 0}, defect_p = {0, 0};

  /* --- electrons and positrons --- */
  for (int kind = ORC_ELECTRON; kind <= ORC_POSITRON; ++kind) {
    orc_species* S = sp[kind];
    const double q = kind == ORC_ELECTRON ? -1.0 : 1.0;
    for (int64_t i = 0; i < S->n; ++i) {
      double x[3] = {S->x[i], S->y[i], S->z[i]}, u[3] = {S->ux[i], S->uy[i], S->uz[i]};
      double E[3], B[3];
      orc_field_eval(&p->field, t, x, E, B);
      orc_boris(q, dt, E, B, u);
      const double gamma = sqrt(1.0 + dot(u, u));
      for (int c = 0; c < 3; ++c) x[c] += dt * u[c] / gamma;
      const double eta = orc_eta(u, gamma, E, B);
      int oor = 0;
      const double lam = eta > 0.0 ? c_gamma * (eta / gamma) * orc_lookup_h(T, eta, &oor) : 0.0;
      if (oor > 0) L->oor_eta += 1.0;
      double tau = S->tau[i] - lam * dt;
      if (p->emit_photons && tau <= 0.0) {
        double U[4];
        draw4(p->seed, p->scenario, S->id[i], p->step, (uint64_t)kind, ORC_PURPOSE_EVENT, U);
        double xi;
        if (orc_sample_xi(T, eta, U[0], &xi)) {
          const double eps = xi * gamma;
          const double um = sqrt(dot(u, u));
          const double uh[3] = {u[0] / um, u[1] / um, u[2] / um};
          child_t c;
          for (int k = 0; k < 3; ++k) { c.x[k] = x[k]; c.u[k] = eps * uh[k]; }
          c.tau = -log(U[2]);
          c.parent = (uint32_t)i;
          c.w = S->w[i];
          /* recoil p_f = p_i - (h nu/c) phat_i (Sec. 3) */
          double umf;
          if (p->recoil_energy) {
            const double gf = gamma - eps;
            umf = gf > 1.0 ? sqrt(gf * gf - 1.0) : 0.0;
          } else {
            umf = um > eps ? um - eps : 0.0;
          }
          for (int k = 0; k < 3; ++k) u[k] = umf * uh[k];
          const double gf = sqrt(1.0 + umf * umf);
          kadd(&defect_e, (gf + eps) - gamma);
          kadd(&emitted_e, eps);
          L->emitted_n += 1.0;
          push_child(&ph_new, &c);
        } else {
          L->dropped_n += 1.0;
        }
        tau = -log(U[1]);
      }
      S->x[i] = x[0]; S->y[i] = x[1]; S->z[i] = x[2];
      S->ux[i] = u[0]; S->uy[i] = u[1]; S->uz[i] = u[2];
      S->tau[i] = tau;
    }
  }
  /* photon children of electrons come first, then those of positrons: ph_new already holds
   * them in that order because electrons were processed first; keep the parent kind
   * boundary for the caller's bookkeeping implicit. */

  /* --- photons --- */
  {
    orc_species* S = sp[ORC_PHOTON];
    int64_t keep = 0;
    for (int64_t i = 0; i < S->n; ++i) {
      double x[3] = {S->x[i], S->y[i], S->z[i]}, k[3] = {S->ux[i], S->uy[i], S->uz[i]};
      double E[3], B[3];
      orc_field_eval(&p->field, t, x, E, B);
      const double eps = sqrt(dot(k, k));
      const double chi = orc_chi(k, eps, E, B);
      int oor = 0;
      const double lam = chi > 0.0 ? ORC_ALPHA * (chi / eps) * orc_lookup_T(T, chi, &oor) : 0.0;
      if (oor > 0) L->oor_chi += 1.0;
      for (int c = 0; c < 3; ++c) x[c] += dt * k[c] / eps; /* null geodesic at c */
      double tau = S->tau[i] - lam * dt;
      if (p->make_pairs && tau <= 0.0) {
        double U[4];
        draw4(p->seed, p->scenario, S->id[i], p->step, ORC_PHOTON, ORC_PURPOSE_EVENT, U);
        const double f = orc_sample_f(T, chi, U[0]);
        child_t ce, cp;
        double fe = 1.0 - f, fp = f;
        double se = fe, sp_ = fp; /* momentum scale factors along k */
        if (p->recoil_energy && eps >= 2.0) {
          const double gp = 1.0 + f * (eps - 2.0), gm = 1.0 + (1.0 - f) * (eps - 2.0);
          sp_ = sqrt(gp * gp - 1.0) / eps;
          se = sqrt(gm * gm - 1.0) / eps;
        }
        for (int c = 0; c < 3; ++c) {
          ce.x[c] = x[c]; cp.x[c] = x[c];
          ce.u[c] = se * k[c]; cp.u[c] = sp_ * k[c];
        }
        ce.tau = -log(U[1]);
        cp.tau = -log(U[2]);
        ce.parent = cp.parent = (uint32_t)i;
        ce.w = cp.w = S->w[i];
        const double gm = sqrt(1.0 + dot(ce.u, ce.u)), gp = sqrt(1.0 + dot(cp.u, cp.u));
        kadd(&defect_p, (gm + gp) - eps);
        kadd(&pair_e, eps);
        L->pairs_n += 1.0;
        push_child(&el_new, &ce);
        push_child(&po_new, &cp);
        continue; /* the photon is annihilated */
      }
      S->x[keep] = x[0]; S->y[keep] = x[1]; S->z[keep] = x[2];
      S->ux[keep] = k[0]; S->uy[keep] = k[1]; S->uz[keep] = k[2];
      S->tau[keep] = tau; S->id[keep] = S->id[i]; S->w[keep] = S->w[i];
      ++keep;
    }
    S->n = keep;
  }

  /* --- new particles join --- */
  int rc = 0;
  rc |= append_children(sp[ORC_ELECTRON], &el_new);
  rc |= append_children(sp[ORC_POSITRON], &po_new);
  if (p->drain_photons) {
    ksum de = {0, 0};
    for (int64_t r = 0; r < ph_new.n; ++r) kadd(&de, sqrt(dot(ph_new.v[r].u, ph_new.v[r].u)));
    L->drained_n = (double)ph_new.n;
    L->drained_energy = de.s;
    if (drained) rc |= append_children(drained, &ph_new);
    else sp[ORC_PHOTON]->next_id += (uint32_t)ph_new.n;
  } else {
    rc |= append_children(sp[ORC_PHOTON], &ph_new);
  }
  free(ph_new.v); free(el_new.v); free(po_new.v);

  L->emitted_energy = emitted_e.s;
  L->emit_defect = defect_e.s;
  L->pair_energy = pair_e.s;
  L->pair_defect = defect_p.s;
  for (int kind = 0; kind < 3; ++kind) {
    const orc_species* S = sp[kind];
    ksum e = {0, 0};
    for (int64_t i = 0; i < S->n; ++i) {
      const double u2 = S->ux[i] * S->ux[i] + S->uy[i] * S->uy[i] + S->uz[i] * S->uz[i];
      kadd(&e, kind == ORC_PHOTON ? sqrt(u2) : sqrt(1.0 + u2));
    }
    L->n[kind] = (double)S->n;
    L->energy[kind] = e.s;
  }
  return rc;
}

/* Initial optical depths, Sec. 3: P = 1 - exp(-tau_em) drawn uniformly, i.e. tau = -ln U. */
/* =====================================================================================
 * 9. Macroparticle merging.  Sec. 3.1 names merging macroparticles as the way to keep a
 *    growing population (an e+e- cascade) bounded and leaves it unimplemented; this is one
 *    definition of it that conserves what the ledger tracks (stated for photons; electrons and
 *    positrons merge the same way with their energy gamma).  Photons are grouped by a cell of
 *    a position grid, a direction bin and an energy bin; every group of at least min_group
 *    photons is replaced by two photons of half the group's weight each, placed at the group's
 *    weighted mean position, that carry exactly the group's total weight W = sum w, momentum
 *    P = sum w k and energy E = sum w |k|: both have energy E/W, and momenta P/W + d and
 *    P/W - d with d perpendicular to P and |d|^2 = (E/W)^2 - |P/W|^2.  The two survivors are the
 *    group's two lowest-index photons (they keep their ids and optical depths); the others
 *    are removed and the remaining photons keep their order.
 *
 *    The bins use exact arithmetic only, so that any IEEE double implementation finds the same
 *    groups: the cell is floor((x - origin)/cell) per axis (photons outside the grid are not
 *    merged), the direction is the face of the cube [-1, 1]^3 that k points through (the axis
 *    of largest |k_a| and its sign) and an n_face x n_face bin of the other two components
 *    divided by |k_a| on that face, and the energy is the binary exponent of |k| and one of
 *    n_sub equal sub-bins of its mantissa.
 * ===================================================================================== */
typedef struct {
  double origin[3], cell[3];
  int n_cells[3];
  int n_face;     /* direction bins per cube-face axis */
  int n_sub;      /* energy sub-bins per octave */
  int min_group;  /* smallest group that is merged (>= 3) */
} orc_merge_params;

/* Group key of photon i, or UINT64_MAX when it is not merged (outside the grid, k = 0). */
static uint64_t merge_key(const orc_species* S, int64_t i, const orc_merge_params* M) {
  const double x[3] = {S->x[i], S->y[i], S->z[i]}, k[3] = {S->ux[i], S->uy[i], S->uz[i]};
  uint64_t cell = 0;
  for (int a = 2; a >= 0; --a) {
    const double c = floor((x[a] - M->origin[a]) / M->cell[a]);
    if (!(c >= 0.0 && c < (double)M->n_cells[a])) return UINT64_MAX;
    cell = cell * (uint64_t)M->n_cells[a] + (uint64_t)c;
  }
  int ax = 0;
  for (int a = 1; a < 3; ++a)
    if (fabs(k[a]) > fabs(k[ax])) ax = a;
  const double m = fabs(k[ax]);
  if (!(m > 0.0)) return UINT64_MAX;
  const int face = 2 * ax + (k[ax] < 0.0 ? 1 : 0);
  int fb[2], q = 0;
  for (int a = 0; a < 3; ++a) {
    if (a == ax) continue;
    int b = (int)floor((k[a] / m + 1.0) * 0.5 * M->n_face);
    if (b < 0) b = 0;
    if (b >= M->n_face) b = M->n_face - 1;
    fb[q++] = b;
  }
  const uint64_t dir = ((uint64_t)face * M->n_face + fb[0]) * M->n_face + fb[1];
  int e2 = 0;
  const double mant = frexp(sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]), &e2); /* [0.5, 1) */
  int sub = (int)floor((mant - 0.5) * 2.0 * M->n_sub);
  if (sub >= M->n_sub) sub = M->n_sub - 1;
  const uint64_t en = (uint64_t)(e2 + 1100) * (uint64_t)M->n_sub + (uint64_t)sub;
  return (cell << 32) | (dir << 16) | en;
}

typedef struct { uint64_t key; int64_t i; } key_index;
static int cmp_key_index(const void* a, const void* b) {
  const key_index *p = (const key_index*)a, *q = (const key_index*)b;
  if (p->key != q->key) return p->key < q->key ? -1 : 1;
  return p->i < q->i ? -1 : (p->i > q->i ? 1 : 0);
}

/* Merges the particles of S (photons when massless, else electrons or positrons: the merged pair
 * then has gamma = E/W each and |u| = sqrt(gamma^2 - 1), and |d|^2 = |u|^2 - |P/W|^2, which is
 * >= 0 because gamma(u) is convex); returns the number of groups merged. */
int64_t orc_merge(orc_species* S, const orc_merge_params* M, int massless) {
  key_index* v = (key_index*)malloc(sizeof(key_index) * (size_t)(S->n > 0 ? S->n : 1));
  unsigned char* gone = (unsigned char*)calloc((size_t)(S->n > 0 ? S->n : 1), 1);
  int64_t m = 0, groups = 0;
  for (int64_t i = 0; i < S->n; ++i) {
    const uint64_t key = merge_key(S, i, M);
    if (key != UINT64_MAX) { v[m].key = key; v[m].i = i; ++m; }
  }
  qsort(v, (size_t)m, sizeof(key_index), cmp_key_index);
  for (int64_t a = 0; a < m;) {
    int64_t b = a;
    while (b < m && v[b].key == v[a].key) ++b;
    if (b - a >= M->min_group) {
      /* totals in index order */
      double W = 0.0, P[3] = {0.0, 0.0, 0.0}, E = 0.0, X[3] = {0.0, 0.0, 0.0};
      for (int64_t r = a; r < b; ++r) {
        const int64_t i = v[r].i;
        const double w = S->w[i], k[3] = {S->ux[i], S->uy[i], S->uz[i]}, x[3] = {S->x[i], S->y[i], S->z[i]};
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        W += w;
        E += w * (massless ? sqrt(k2) : sqrt(1.0 + k2));
        for (int c = 0; c < 3; ++c) { P[c] += w * k[c]; X[c] += w * x[c]; }
      }
      const double et = E / W, mv[3] = {P[0] / W, P[1] / W, P[2] / W};
      const double m2 = mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2];
      const double d2 = (massless ? et * et : et * et - 1.0) - m2;
      const double dl = d2 > 0.0 ? sqrt(d2) : 0.0;
      /* d perpendicular to P: P x e, e the axis with the smallest |P_a| (the lowest on ties) */
      int ax = 0;
      for (int c = 1; c < 3; ++c)
        if (fabs(mv[c]) < fabs(mv[ax])) ax = c;
      double e[3] = {0.0, 0.0, 0.0};
      e[ax] = 1.0;
      double dv[3] = {mv[1] * e[2] - mv[2] * e[1], mv[2] * e[0] - mv[0] * e[2], mv[0] * e[1] - mv[1] * e[0]};
      const double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
      if (dn > 0.0) for (int c = 0; c < 3; ++c) dv[c] *= dl / dn;
      else { for (int c = 0; c < 3; ++c) dv[c] = 0.0; dv[ax] = dl; }
      const int64_t s0 = v[a].i, s1 = v[a + 1].i;  /* the two lowest indices (sorted by index) */
      const int64_t surv[2] = {s0, s1};
      for (int q = 0; q < 2; ++q) {
        const int64_t i = surv[q];
        const double sg = q == 0 ? 1.0 : -1.0;
        S->ux[i] = mv[0] + sg * dv[0]; S->uy[i] = mv[1] + sg * dv[1]; S->uz[i] = mv[2] + sg * dv[2];
        S->x[i] = X[0] / W; S->y[i] = X[1] / W; S->z[i] = X[2] / W;
        S->w[i] = 0.5 * W;
      }
      for (int64_t r = a + 2; r < b; ++r) gone[v[r].i] = 1;
      ++groups;
    }
    a = b;
  }
  int64_t keep = 0;
  for (int64_t i = 0; i < S->n; ++i) {
    if (gone[i]) continue;
    S->x[keep] = S->x[i]; S->y[keep] = S->y[i]; S->z[keep] = S->z[i];
    S->ux[keep] = S->ux[i]; S->uy[keep] = S->uy[i]; S->uz[keep] = S->uz[i];
    S->tau[keep] = S->tau[i]; S->id[keep] = S->id[i]; S->w[keep] = S->w[i];
    ++keep;
  }
  S->n = keep;
  free(v);
  free(gone);
  return groups;
}

int64_t orc_merge_photons(orc_species* S, const orc_merge_params* M) { return orc_merge(S, M, 1); }

/* Physical totals of a species: out[0] = sum w, out[1] = sum w * energy (|k| for photons,
 * gamma for e+-), out[2..4] = sum w * momentum. */
void orc_species_totals(const orc_species* S, int massless, double out[5]) {
  for (int c = 0; c < 5; ++c) out[c] = 0.0;
  for (int64_t i = 0; i < S->n; ++i) {
    const double u[3] = {S->ux[i], S->uy[i], S->uz[i]}, w = S->w[i];
    const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    out[0] += w;
    out[1] += w * (massless ? sqrt(u2) : sqrt(1.0 + u2));
    for (int c = 0; c < 3; ++c) out[2 + c] += w * u[c];
  }
}

void orc_init_tau(orc_species* S, int kind, uint64_t seed, uint64_t scenario) {
  for (int64_t i = 0; i < S->n; ++i) {
    double U[4];
    draw4(seed, scenario, S->id[i], 0, (uint64_t)kind, ORC_PURPOSE_INIT, U);
    S->tau[i] = -log(U[0]);
  }
}
