// qed_tables.cpp -- host construction of the look-up tables of Sec. 3 (h, T, P_chi, P_f)
// from the emissivities of Apps. A and B.
//
// Numerical route: modified Bessel functions from libstdc++ (std::cyl_bessel_k); the
// integral Ki_{5/3}(y) = int_y^inf K_{5/3} from the recurrence K'_{2/3} = -(K_{1/3}+K_{5/3})/2,
// i.e. Ki_{5/3} = 2 K_{2/3} - Ki_{1/3}, with Ki_{1/3} accumulated once on a geometric ladder
// of y and completed by an 8-point Gauss-Legendre panel; all table integrals by fixed
// Gauss-Legendre panels.  Rows are independent and are built on all host threads.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "qed_internal.h"

namespace qedlib {
namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- Gauss-Legendre rules
struct GaussRule {
  std::vector<double> node, weight;  // on [-1, 1]
  explicit GaussRule(int n) : node(n), weight(n) {
    // roots of P_n by Newton's method from the asymptotic guess cos(pi (k - 1/4)/(n + 1/2))
    for (int k = 0; k < n; ++k) {
      double r = std::cos(kPi * (k + 0.75) / (n + 0.5));
      double deriv = 1.0;
      for (int iter = 0; iter < 64; ++iter) {
        double pm1 = 1.0, p = r;  // P_0, P_1
        for (int m = 1; m < n; ++m) {
          const double pp1 = ((2 * m + 1) * r * p - m * pm1) / (m + 1);
          pm1 = p;
          p = pp1;
        }
        deriv = n * (pm1 - r * p) / (1.0 - r * r);
        const double delta = p / deriv;
        r -= delta;
        if (std::fabs(delta) <= 1e-16 * std::fabs(r) + 1e-300) break;
      }
      node[k] = r;
      weight[k] = 2.0 / ((1.0 - r * r) * deriv * deriv);
    }
  }
  template <class Fn>
  double integrate(Fn&& f, double a, double b) const {
    const double half = 0.5 * (b - a), mid = 0.5 * (a + b);
    double acc = 0.0;
    for (size_t k = 0; k < node.size(); ++k) acc += weight[k] * f(mid + half * node[k]);
    return acc * half;
  }
};

double bessel_k(double nu, double x) {
  if (!(x > 0.0)) return INFINITY;
  if (x > 700.0) return 0.0;
  return std::cyl_bessel_k(nu, x);
}

// ---------------------------------------------------------------- Ki_{1/3} ladder
class KiOneThird {
 public:
  KiOneThird() : gl_(8) {
    const double y0 = 1e-20, ratio = 1.02;
    double y = y0;
    while (y < 720.0) { y_.push_back(y); y *= ratio; }
    y_.push_back(y);
    ki_.assign(y_.size(), 0.0);
    // downward accumulation; K_{1/3}(720) ~ 1e-314 so the top value is zero
    for (size_t k = y_.size() - 1; k-- > 0;) ki_[k] = ki_[k + 1] + segment(y_[k], y_[k + 1]);
    log_y0_ = std::log(y0);
    inv_log_ratio_ = 1.0 / std::log(ratio);
  }
  // int_a^b K_{1/3}(t) dt in s = ln t (t K_{1/3}(t) is smooth in s)
  double segment(double a, double b) const {
    return gl_.integrate([](double s) { const double t = std::exp(s); return t * bessel_k(1.0 / 3.0, t); },
                         std::log(a), std::log(b));
  }
  double operator()(double y) const {
    if (!(y > y_.front())) return ki_.front();
    if (y >= y_.back()) return 0.0;
    size_t k = (size_t)((std::log(y) - log_y0_) * inv_log_ratio_);
    if (k + 1 >= y_.size()) k = y_.size() - 2;
    while (k > 0 && y_[k] > y) --k;
    while (k + 2 < y_.size() && y_[k + 1] <= y) ++k;
    return ki_[k + 1] + segment(y, y_[k + 1]);
  }

 private:
  GaussRule gl_;
  std::vector<double> y_, ki_;
  double log_y0_, inv_log_ratio_;
};

// ---------------------------------------------------------------- emissivities
struct Emissivity {
  KiOneThird ki13;
  // F(eta, chi) of App. A in xi = 2chi/eta, one_minus_xi passed separately for precision
  double F(double eta, double xi, double one_minus_xi) const {
    if (!(xi > 0.0) || !(one_minus_xi > 0.0)) return 0.0;
    const double y = 2.0 * xi / (3.0 * eta * one_minus_xi);
    if (y > 700.0) return 0.0;
    const double k23 = bessel_k(2.0 / 3.0, y);
    const double ki53 = 2.0 * k23 - ki13(y);
    return xi * xi * y * k23 + one_minus_xi * y * ki53;
  }
  // T(chi) of App. B
  static double T(double chi) {
    const double k = bessel_k(1.0 / 3.0, 2.0 / (3.0 * chi));
    return 0.16 * k * k / chi;
  }
  // unnormalised p_f of App. B
  static double pf(double f, double chi) {
    const double q = f * (1.0 - f);
    if (!(q > 0.0)) return 0.0;
    return (2.0 + q) / q * bessel_k(2.0 / 3.0, 1.0 / (3.0 * chi * q));
  }
};

inline double logistic(double z) { return 1.0 / (1.0 + std::exp(-z)); }
inline double logistic_c(double z) { return 1.0 / (1.0 + std::exp(z)); }  // 1 - logistic(z)

struct RowBuilder {
  const Emissivity& em;
  const qed_table_params& p;
  TableHost& out;
  GaussRule gl8{8}, gl16{16};

  // F dxi over [0, xi] in s = xi^{1/3}: 3 s^2 F(s^3) ds, one 16-point panel (xi small)
  double energy_below(double eta, double xi) const {
    return gl16.integrate([&](double s) { const double x = s * s * s; return 3.0 * s * s * em.F(eta, x, 1.0 - x); },
                          0.0, std::cbrt(xi));
  }
  // (F/xi) dxi over [0, xi] in s: 3 F(s^3)/s ds
  double number_below(double eta, double xi) const {
    return gl16.integrate([&](double s) { const double x = s * s * s; return 3.0 * em.F(eta, x, 1.0 - x) / s; },
                          0.0, std::cbrt(xi));
  }
  // in zeta: (F/xi) dxi = F (1 - xi) dzeta, F dxi = F xi (1 - xi) dzeta
  double number_zeta(double eta, double z0, double z1) const {
    return gl8.integrate([&](double z) { const double om = logistic_c(z); return em.F(eta, logistic(z), om) * om; }, z0, z1);
  }
  double energy_zeta(double eta, double z0, double z1) const {
    return gl8.integrate([&](double z) { const double om = logistic_c(z), x = logistic(z); return em.F(eta, x, om) * x * om; },
                         z0, z1);
  }

  void eta_row(int i) {
    const double lmin = std::log(p.eta_min), lmax = std::log(p.eta_max);
    const double eta = std::exp(lmin + (lmax - lmin) * i / (p.n_eta - 1));
    const double zhi = std::log(90.0 * eta);
    // total int_0^1 F dxi: below xi = 1e-13 in s, above in zeta panels of width 1/8
    const double za = std::log(1e-13);
    double total = energy_below(eta, 1e-13);
    const int npan = (int)std::ceil((zhi + 6.0 - za) * 8.0);
    for (int k = 0; k < npan; ++k) total += energy_zeta(eta, za + k * 0.125, za + (k + 1) * 0.125);
    // cut-off xi_min: energy fraction below it equals energy_cut (Sec. 3); Newton in ln xi on
    // ln(fraction), whose slope tends to 4/3
    double lx = std::log(1e-9);
    for (int it = 0; it < 100; ++it) {
      const double x = std::exp(lx);
      const double eb = energy_below(eta, x);
      const double slope = x * em.F(eta, x, 1.0 - x) / eb;
      const double step = (std::log(eb / total) - std::log(p.energy_cut)) / slope;
      lx -= std::max(-3.0, std::min(3.0, step));
      if (std::fabs(step) < 1e-15) break;
    }
    const double xmin = std::exp(lx);
    const double zlo = std::log(xmin / (1.0 - xmin));
    const int n = p.n_xi;
    std::vector<double> seg(n - 1);
    const double dz = (zhi - zlo) / (n - 1);
    for (int j = 0; j + 1 < n; ++j) seg[j] = number_zeta(eta, zlo + j * dz, zlo + (j + 1) * dz);
    const double below = number_below(eta, xmin);
    const double above = number_zeta(eta, zhi, zhi + 3.0) + number_zeta(eta, zhi + 3.0, zhi + 6.0);
    double h = below + above;
    for (double v : seg) h += v;
    double* P = &out.P[(size_t)i * n];
    double* Q = &out.Q[(size_t)i * n];
    double acc = below;
    P[0] = acc / h;
    for (int j = 1; j < n; ++j) { acc += seg[j - 1]; P[j] = acc / h; }
    acc = above;
    Q[n - 1] = acc / h;
    for (int j = n - 2; j >= 0; --j) { acc += seg[j]; Q[j] = acc / h; }
    out.ln_h[i] = std::log(h);
    out.g[i] = 3.0 * std::sqrt(3.0) / (4.0 * kPi * eta) * total;
    out.zeta_lo[i] = zlo;
    out.zeta_hi[i] = zhi;
  }

  void chi_row(int k) {
    const double lmin = std::log(p.chi_min), lmax = std::log(p.chi_max);
    const double chi = std::exp(lmin + (lmax - lmin) * k / (p.n_chi - 1));
    out.ln_T[k] = std::log(Emissivity::T(chi));
    const int n = p.n_f;
    std::vector<double> seg(n - 1);
    double tot = 0.0;
    // in s = f^{1/3}: for chi f >> 1 the density behaves as f^{-1/3} near f = 0, which the
    // substitution turns into the smooth 3 s^2 p_f(s^3); two 16-point panels per interval
    auto ig = [&](double s) { return 3.0 * s * s * Emissivity::pf(s * s * s, chi); };
    for (int j = 0; j + 1 < n; ++j) {
      const double s0 = std::cbrt(0.5 * j / (n - 1)), s1 = std::cbrt(0.5 * (j + 1) / (n - 1));
      const double sm = 0.5 * (s0 + s1);
      seg[j] = gl16.integrate(ig, s0, sm) + gl16.integrate(ig, sm, s1);
      tot += seg[j];
    }
    double* row = &out.Pf[(size_t)k * n];
    double acc = 0.0;
    row[0] = 0.0;
    for (int j = 1; j < n; ++j) { acc += seg[j - 1]; row[j] = acc / tot; }
    row[n - 1] = 1.0;
  }
};

}  // namespace

bool validate_table_params(const qed_table_params& p, std::string& err) {
  if (p.n_eta < 2 || p.n_xi < 2 || p.n_chi < 2 || p.n_f < 2) { err = "table sizes must be >= 2"; return false; }
  if (p.n_eta > 65536 || p.n_xi > 65536 || p.n_chi > 65536 || p.n_f > 65536) { err = "table sizes must be <= 65536"; return false; }
  if (!(p.eta_min > 0.0) || !(p.eta_max > p.eta_min)) { err = "need 0 < eta_min < eta_max"; return false; }
  if (!(p.chi_min > 0.0) || !(p.chi_max > p.chi_min)) { err = "need 0 < chi_min < chi_max"; return false; }
  if (!(p.energy_cut > 0.0) || !(p.energy_cut < 1e-3)) { err = "energy_cut must be in (0, 1e-3)"; return false; }
  return true;
}

void TableHost::resize(const qed_table_params& prm) {
  p = prm;
  ln_h.assign(p.n_eta, 0.0);
  g.assign(p.n_eta, 0.0);
  zeta_lo.assign(p.n_eta, 0.0);
  zeta_hi.assign(p.n_eta, 0.0);
  P.assign((size_t)p.n_eta * p.n_xi, 0.0);
  Q.assign((size_t)p.n_eta * p.n_xi, 0.0);
  ln_T.assign(p.n_chi, 0.0);
  Pf.assign((size_t)p.n_chi * p.n_f, 0.0);
}

bool build_tables_host(const qed_table_params& p, TableHost& out, std::string& err) {
  if (!validate_table_params(p, err)) return false;
  out.resize(p);
  static const Emissivity em;  // the Ki_{1/3} ladder is built once per process
  const int rows = p.n_eta + p.n_chi;
  std::atomic<int> next{0};
  auto worker = [&]() {
    RowBuilder rb{em, p, out};
    for (int r; (r = next.fetch_add(1)) < rows;) {
      if (r < p.n_eta) rb.eta_row(r);
      else rb.chi_row(r - p.n_eta);
    }
  };
  unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (unsigned t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& t : pool) t.join();
  for (size_t i = 0; i < out.ln_h.size(); ++i)
    if (!std::isfinite(out.ln_h[i])) { err = "non-finite h in table build"; return false; }
  return true;
}

}  // namespace qedlib
