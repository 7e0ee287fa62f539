// Relaxation-parameter fitting (Sec. 4.1): host FP64, no device needed.
//
// The multiple-relaxation model's attenuation and phase velocity follow from
// the dispersion relation (Eq. dispersion_relations with the sums gamma of
// Eq. gamma1); the fit minimises
//   J = w_alpha NMSE(alpha_model, alpha_target) + (1 - w_alpha) NMSE(c_model, c_target)
// (Eq. relaxation_parameter_optimization; NMSE = mean squared error over the
// variance of the target) for a power-law target alpha0 f^y and its
// Kramers-Kronig phase velocity.  The paper's search is a coarse-to-fine
// grid inside the bounds of Table 2 (kappa linear, d and alpha in log10),
// each finer search centred on the best point so far with every range 30 %
// narrower; a Nelder-Mead polish in the same coordinates may follow.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <thread>
#include <vector>

#include "fw2.h"

namespace fw2 {
void set_global_error(const char *msg);
}

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kNpPerDb = 2.302585092994045684 / 20.0;  // ln(10) / 20

struct Target {
  std::vector<double> w;       // angular frequencies
  std::vector<double> att, c;  // target attenuation [dB/cm] and phase velocity [m/s]
  double var_att = 0, var_c = 0, c0 = 0, w_alpha = 0.1;
  int N = 0;
};

double variance(const std::vector<double> &v) {
  double m = 0;
  for (double x : v) m += x;
  m /= (double)v.size();
  double s = 0;
  for (double x : v) s += (x - m) * (x - m);
  return s / (double)v.size();
}

// Point of the search space: kappa1, kappa2, log10 d1[N], log10 d2[N],
// log10 alpha1[N], log10 alpha2[N].
struct Params {
  double k1, k2, d1[FW2_FIT_MAX_RELAX], d2[FW2_FIT_MAX_RELAX], a1[FW2_FIT_MAX_RELAX], a2[FW2_FIT_MAX_RELAX];
};
Params unpack(const double *x, int N) {
  Params p{};
  p.k1 = x[0];
  p.k2 = x[1];
  for (int n = 0; n < N; ++n) {
    p.d1[n] = std::pow(10.0, x[2 + n]);
    p.d2[n] = std::pow(10.0, x[2 + N + n]);
    p.a1[n] = std::pow(10.0, x[2 + 2 * N + n]);
    p.a2[n] = std::pow(10.0, x[2 + 3 * N + n]);
  }
  return p;
}

// Principal square root of a complex number: the larger part from
// sqrt((|z| + |x|) / 2), the other as y / (2 that), free of cancellation.
std::complex<double> csqrt(std::complex<double> z) {
  const double x = z.real(), y = z.imag();
  if (x == 0.0 && y == 0.0) return {0.0, 0.0};
  const double t = std::sqrt(0.5 * (std::hypot(x, y) + std::fabs(x)));
  if (x >= 0.0) return {t, y / (2.0 * t)};
  return {std::fabs(y) / (2.0 * t), y < 0 ? -t : t};
}

// attenuation [dB/cm] and phase velocity from the sums gamma of both
// operators (Eq. dispersion_relations): k = (w / c0) (1/(kappa1 kappa2) -
// gamma1/kappa2 - gamma2/kappa1 + gamma1 gamma2)^(-1/2), waves exp(i(w t - k x))
inline void curves_of(std::complex<double> g1, std::complex<double> g2, double k1, double k2, double c0, double w,
                      double &att, double &c) {
  const std::complex<double> inner = 1.0 / (k1 * k2) - g1 / k2 - g2 / k1 + g1 * g2;
  const std::complex<double> k = (w / c0) / csqrt(inner);
  att = -k.imag() / kNpPerDb / 100.0;
  c = w / k.real();
}

// attenuation [dB/cm] and phase velocity of the model at angular frequency w
void model_at(const Params &p, int N, double c0, double w, double &att, double &c) {
  using cd = std::complex<double>;
  cd g1 = 0, g2 = 0;
  for (int n = 0; n < N; ++n) {
    g1 += (p.d1[n] / (p.k1 * p.k1)) / cd(p.d1[n] / p.k1 + p.a1[n], w);
    g2 += (p.d2[n] / (p.k2 * p.k2)) / cd(p.d2[n] / p.k2 + p.a2[n], w);
  }
  curves_of(g1, g2, p.k1, p.k2, c0, w, att, c);
}

double cost(const Target &T, const double *x) {
  const Params p = unpack(x, T.N);
  double ea = 0, ec = 0;
  const size_t F = T.w.size();
  for (size_t i = 0; i < F; ++i) {
    double a, c;
    model_at(p, T.N, T.c0, T.w[i], a, c);
    ea += (a - T.att[i]) * (a - T.att[i]);
    ec += (c - T.c[i]) * (c - T.c[i]);
  }
  const double J = T.w_alpha * (ea / F) / T.var_att + (1.0 - T.w_alpha) * (ec / F) / T.var_c;
  return std::isfinite(J) ? J : INFINITY;
}

// Best point of the grid: `pts` values per dimension over [centre - width/2,
// centre + width/2] clamped to the bounds, searched by `threads` threads.
// A term d/kappa^2 / (d/kappa + alpha + i w) of gamma depends on three axes
// only (kappa, d and alpha of one mechanism and operator), so every term of
// the grid is computed once into a table; each grid point then sums N table
// entries per operator and frequency.
double grid_level(const Target &T, int D, int pts, const double *centre, const double *width, const double *lo,
                  const double *hi, int threads, std::vector<double> &best, long long &evals) {
  using cd = std::complex<double>;
  const int N = T.N;
  const int F = (int)T.w.size();
  std::vector<std::vector<double>> axes(D, std::vector<double>(pts));
  for (int d = 0; d < D; ++d)
    for (int i = 0; i < pts; ++i) {
      const double v = pts > 1 ? centre[d] - width[d] / 2 + width[d] * i / (pts - 1) : centre[d];
      axes[d][i] = std::min(std::max(v, lo[d]), hi[d]);
    }
  // term tables [op][n][i_kappa][i_d][i_alpha][f]
  const size_t per = (size_t)pts * pts * pts * F;
  std::vector<cd> tab((size_t)2 * N * per);
  for (int op = 0; op < 2; ++op)
    for (int n = 0; n < N; ++n) {
      const int dk = op, dd = 2 + op * N + n, da = 2 + 2 * N + op * N + n;
      cd *t = tab.data() + ((size_t)op * N + n) * per;
      for (int ik = 0; ik < pts; ++ik)
        for (int id = 0; id < pts; ++id)
          for (int ia = 0; ia < pts; ++ia) {
            const double kap = axes[dk][ik], dv = std::pow(10.0, axes[dd][id]), av = std::pow(10.0, axes[da][ia]);
            cd *row = t + (((size_t)ik * pts + id) * pts + ia) * F;
            for (int f = 0; f < F; ++f) row[f] = (dv / (kap * kap)) / cd(dv / kap + av, T.w[f]);
          }
    }
  long long total = 1;
  for (int d = 0; d < D; ++d) total *= pts;
  std::vector<double> bj(threads, INFINITY);
  std::vector<long long> bi(threads, -1);
  auto work = [&](int t) {
    const long long a = total * t / threads, b = total * (t + 1) / threads;
    std::vector<int> ix(D);
    std::vector<const cd *> rows(2 * N);
    for (long long g = a; g < b; ++g) {
      long long r = g;
      for (int d = 0; d < D; ++d) {
        ix[d] = (int)(r % pts);
        r /= pts;
      }
      for (int op = 0; op < 2; ++op)
        for (int n = 0; n < N; ++n) {
          const int ik = ix[op], id = ix[2 + op * N + n], ia = ix[2 + 2 * N + op * N + n];
          rows[op * N + n] = tab.data() + ((size_t)op * N + n) * per + (((size_t)ik * pts + id) * pts + ia) * F;
        }
      const double k1 = axes[0][ix[0]], k2 = axes[1][ix[1]];
      double ea = 0, ec = 0;
      for (int f = 0; f < F; ++f) {
        cd g1 = 0, g2 = 0;
        for (int n = 0; n < N; ++n) {
          g1 += rows[n][f];
          g2 += rows[N + n][f];
        }
        double at, c;
        curves_of(g1, g2, k1, k2, T.c0, T.w[f], at, c);
        ea += (at - T.att[f]) * (at - T.att[f]);
        ec += (c - T.c[f]) * (c - T.c[f]);
      }
      double j = T.w_alpha * (ea / F) / T.var_att + (1.0 - T.w_alpha) * (ec / F) / T.var_c;
      if (!std::isfinite(j)) j = INFINITY;
      if (j < bj[t]) {
        bj[t] = j;
        bi[t] = g;
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
  work(0);
  for (auto &th : pool) th.join();
  evals += total;
  int tb = 0;
  for (int t = 1; t < threads; ++t)
    if (bj[t] < bj[tb] || (bj[t] == bj[tb] && bi[t] < bi[tb])) tb = t;
  if (bi[tb] < 0) return INFINITY;
  long long r = bi[tb];
  best.assign(D, 0.0);
  for (int d = 0; d < D; ++d) {
    best[d] = axes[d][r % pts];
    r /= pts;
  }
  return bj[tb];
}

// Nelder-Mead in the search coordinates, points clamped to the bounds.
double polish(const Target &T, int D, const double *lo, const double *hi, std::vector<double> &x, long long &evals,
              int max_iter) {
  auto clampv = [&](std::vector<double> &v) {
    for (int d = 0; d < D; ++d) v[d] = std::min(std::max(v[d], lo[d]), hi[d]);
  };
  std::vector<std::vector<double>> s(D + 1, x);
  std::vector<double> f(D + 1);
  for (int d = 0; d < D; ++d) {
    const double step = 0.05 * (hi[d] - lo[d]);
    s[d + 1][d] += (s[d + 1][d] + step <= hi[d]) ? step : -step;
  }
  for (int i = 0; i <= D; ++i) {
    clampv(s[i]);
    f[i] = cost(T, s[i].data());
    ++evals;
  }
  std::vector<double> c(D), xr(D), xe(D), xc(D);
  for (int it = 0; it < max_iter; ++it) {
    std::vector<int> ord(D + 1);
    for (int i = 0; i <= D; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return f[a] < f[b]; });
    const int ib = ord[0], iw = ord[D], is = ord[D - 1];
    if (std::fabs(f[iw] - f[ib]) <= 1e-15 * std::max(1.0, std::fabs(f[ib]))) break;
    std::fill(c.begin(), c.end(), 0.0);
    for (int i = 0; i <= D; ++i)
      if (i != iw)
        for (int d = 0; d < D; ++d) c[d] += s[i][d] / D;
    for (int d = 0; d < D; ++d) xr[d] = c[d] + (c[d] - s[iw][d]);
    clampv(xr);
    const double fr = cost(T, xr.data());
    ++evals;
    if (fr < f[ib]) {
      for (int d = 0; d < D; ++d) xe[d] = c[d] + 2.0 * (c[d] - s[iw][d]);
      clampv(xe);
      const double fe = cost(T, xe.data());
      ++evals;
      if (fe < fr) { s[iw] = xe; f[iw] = fe; }
      else { s[iw] = xr; f[iw] = fr; }
    } else if (fr < f[is]) {
      s[iw] = xr;
      f[iw] = fr;
    } else {
      const bool outside = fr < f[iw];
      for (int d = 0; d < D; ++d) xc[d] = outside ? c[d] + 0.5 * (xr[d] - c[d]) : c[d] + 0.5 * (s[iw][d] - c[d]);
      const double fc = cost(T, xc.data());
      ++evals;
      if (fc < std::min(fr, f[iw])) {
        s[iw] = xc;
        f[iw] = fc;
      } else {  // shrink toward the best point
        for (int i = 0; i <= D; ++i) {
          if (i == ib) continue;
          for (int d = 0; d < D; ++d) s[i][d] = s[ib][d] + 0.5 * (s[i][d] - s[ib][d]);
          f[i] = cost(T, s[i].data());
          ++evals;
        }
      }
    }
  }
  int ib = 0;
  for (int i = 1; i <= D; ++i)
    if (f[i] < f[ib]) ib = i;
  x = s[ib];
  return f[ib];
}

}  // namespace

extern "C" {

fw2_status fw2_fit_request_init(fw2_fit_request *r) {
  if (!r) return FW2_EINVAL;
  std::memset(r, 0, sizeof *r);
  r->alpha0 = 0.5;
  r->y = 1.0;
  r->n_relax = 2;
  r->c0 = 1540.0;
  r->f_ref = 0.0;
  r->f_lo = 1e6;
  r->f_hi = 20e6;
  r->n_freq = 77;
  r->w_alpha = 0.1;
  r->kappa_bounds[0] = 0.8;
  r->kappa_bounds[1] = 1.2;
  r->log_d_bounds[0] = 2.0;
  r->log_d_bounds[1] = 10.0;
  r->log_alpha_bounds[0] = 5.0;
  r->log_alpha_bounds[1] = 12.0;
  r->grid_points = 5;
  r->refinements = 4;
  r->shrink = 0.3;
  r->polish_iterations = 20000;
  r->threads = 0;
  return FW2_OK;
}

fw2_status fw2_fit_relaxation(const fw2_fit_request *r, fw2_fit_result *out) {
  if (!r || !out) {
    fw2::set_global_error("fw2_fit_relaxation: null argument");
    return FW2_EINVAL;
  }
  const int N = r->n_relax, D = 2 + 4 * N;
  if (N < 1 || N > FW2_FIT_MAX_RELAX || !(r->alpha0 > 0) || !(r->y > 0 && r->y < 3) || !(r->c0 > 0) ||
      !(r->f_lo > 0 && r->f_hi > r->f_lo) || r->n_freq < 3 || !(r->w_alpha >= 0 && r->w_alpha <= 1) ||
      r->grid_points < 1 || r->refinements < 0 || !(r->shrink > 0 && r->shrink < 1) || r->polish_iterations < 0 ||
      !(r->kappa_bounds[0] > 0 && r->kappa_bounds[1] >= r->kappa_bounds[0]) ||
      !(r->log_d_bounds[1] >= r->log_d_bounds[0]) || !(r->log_alpha_bounds[1] >= r->log_alpha_bounds[0])) {
    fw2::set_global_error("fw2_fit_relaxation: argument out of range");
    return FW2_EINVAL;
  }
  if (std::pow((double)r->grid_points, (double)D) > 2e9) {
    fw2::set_global_error("fw2_fit_relaxation: grid_points^(2 + 4N) exceeds 2e9 evaluations per search");
    return FW2_EINVAL;
  }
  // target: alpha0 f^y [dB/cm, f in MHz] and its Kramers-Kronig phase
  // velocity in the nearly-local form, c0 at f_ref (band centre by default)
  Target T;
  T.N = N;
  T.c0 = r->c0;
  T.w_alpha = r->w_alpha;
  const double f_ref = r->f_ref > 0 ? r->f_ref : 0.5 * (r->f_lo + r->f_hi);
  const double wr = 2 * kPi * f_ref;
  const double a0 = r->alpha0 * kNpPerDb * 100.0 / std::pow(2 * kPi * 1e6, r->y);  // Np/m per (rad/s)^y
  for (int i = 0; i < r->n_freq; ++i) {
    const double f = r->f_lo + (r->f_hi - r->f_lo) * i / (r->n_freq - 1);
    const double w = 2 * kPi * f;
    T.w.push_back(w);
    T.att.push_back(r->alpha0 * std::pow(f / 1e6, r->y));
    const double inv = std::fabs(r->y - 1.0) < 1e-12
                           ? 1.0 / r->c0 - (2.0 / kPi) * a0 * std::log(w / wr)
                           : 1.0 / r->c0 + a0 * std::tan(kPi * r->y / 2.0) * (std::pow(w, r->y - 1) - std::pow(wr, r->y - 1));
    T.c.push_back(1.0 / inv);
  }
  T.var_att = variance(T.att);
  T.var_c = variance(T.c);
  if (!(T.var_att > 0) || !(T.var_c > 0)) {
    fw2::set_global_error("fw2_fit_relaxation: target without variance over the band");
    return FW2_EINVAL;
  }
  std::vector<double> lo(D), hi(D);
  lo[0] = lo[1] = r->kappa_bounds[0];
  hi[0] = hi[1] = r->kappa_bounds[1];
  for (int d = 2; d < 2 + 2 * N; ++d) { lo[d] = r->log_d_bounds[0]; hi[d] = r->log_d_bounds[1]; }
  for (int d = 2 + 2 * N; d < D; ++d) { lo[d] = r->log_alpha_bounds[0]; hi[d] = r->log_alpha_bounds[1]; }
  int threads = r->threads > 0 ? r->threads : (int)std::thread::hardware_concurrency();
  threads = std::max(1, std::min(threads, 256));
  long long evals = 0;
  std::vector<double> centre(D), width(D), best;
  for (int d = 0; d < D; ++d) {
    centre[d] = 0.5 * (lo[d] + hi[d]);
    width[d] = hi[d] - lo[d];
  }
  double bj = INFINITY;
  std::vector<double> bx;
  for (int level = 0; level <= r->refinements; ++level) {
    const double j = grid_level(T, D, r->grid_points, centre.data(), width.data(), lo.data(), hi.data(), threads,
                                best, evals);
    if (j < bj) {
      bj = j;
      bx = best;
    }
    if (bx.empty()) break;
    centre = bx;
    for (int d = 0; d < D; ++d) width[d] *= 1.0 - r->shrink;
  }
  if (bx.empty()) {
    fw2::set_global_error("fw2_fit_relaxation: no finite cost on the grid");
    return FW2_EUNSTABLE;
  }
  std::memset(out, 0, sizeof *out);
  out->J_grid = bj;
  if (r->polish_iterations > 0) bj = std::min(bj, polish(T, D, lo.data(), hi.data(), bx, evals, r->polish_iterations));
  out->J = cost(T, bx.data());
  const Params p = unpack(bx.data(), N);
  out->kappa1 = p.k1;
  out->kappa2 = p.k2;
  for (int n = 0; n < N; ++n) {
    out->d1[n] = p.d1[n];
    out->d2[n] = p.d2[n];
    out->alpha1[n] = p.a1[n];
    out->alpha2[n] = p.a2[n];
  }
  out->f_ref = f_ref;
  double ea = 0, ec = 0;
  for (size_t i = 0; i < T.w.size(); ++i) {
    double a, c;
    model_at(p, N, T.c0, T.w[i], a, c);
    if (T.w[i] >= 2 * kPi * 2e6 - 1e-6) ea = std::max(ea, std::fabs(a / T.att[i] - 1.0));
    ec = std::max(ec, std::fabs(c / T.c[i] - 1.0));
  }
  out->max_att_rel_err = ea;
  out->max_phase_rel_err = ec;
  out->evaluations = evals;
  return FW2_OK;
}

fw2_status fw2_relaxation_curves(const fw2_fit_result *p, int32_t n_relax, double c0, const double *freqs,
                                 int64_t n, double *att_db_cm, double *c) {
  if (!p || !freqs || !att_db_cm || !c || n < 0 || n_relax < 1 || n_relax > FW2_FIT_MAX_RELAX || !(c0 > 0)) {
    fw2::set_global_error("fw2_relaxation_curves: bad argument");
    return FW2_EINVAL;
  }
  Params q{};
  q.k1 = p->kappa1;
  q.k2 = p->kappa2;
  for (int k = 0; k < n_relax; ++k) {
    q.d1[k] = p->d1[k];
    q.d2[k] = p->d2[k];
    q.a1[k] = p->alpha1[k];
    q.a2[k] = p->alpha2[k];
  }
  for (int64_t i = 0; i < n; ++i) model_at(q, n_relax, c0, 2 * kPi * freqs[i], att_db_cm[i], c[i]);
  return FW2_OK;
}

}  // extern "C"
