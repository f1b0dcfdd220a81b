// Host-side pieces of the library: error reporting, basis normalisation, the
// Boys-function table, and the least-squares Laplace quadrature (Eq. laplace).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "host.h"

namespace ltjk {

static thread_local char g_err[512] = "";

int set_error(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}
const char *last_error() { return g_err; }

// ------------------------------------------------------------ normalisation
static double double_factorial(int n) {
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

// Contracted coefficients: c_k N_k with N_k = (2a/pi)^{3/4} (4a)^{l/2} / sqrt((2l-1)!!),
// then scaled so that the contracted x^l function has unit self-overlap.
void normalise_shell(int l, int np, const double *exps, const double *coefs, double *out) {
  const double pi = 3.14159265358979323846;
  const double dfl = double_factorial(2 * l - 1);
  for (int k = 0; k < np; ++k)
    out[k] = coefs[k] * std::pow(2.0 * exps[k] / pi, 0.75) * std::pow(4.0 * exps[k], 0.5 * l) /
             std::sqrt(dfl);
  double s = 0.0;
  for (int i = 0; i < np; ++i)
    for (int j = 0; j < np; ++j) {
      const double g = exps[i] + exps[j];
      s += out[i] * out[j] * std::pow(pi / g, 1.5) * dfl / std::pow(2.0 * g, l);
    }
  const double f = 1.0 / std::sqrt(s);
  for (int k = 0; k < np; ++k) out[k] *= f;
}

// ------------------------------------------------------------ Boys table
// F_m(T_k) = int_0^1 u^{2m} exp(-T_k u^2) du by composite Gauss-Legendre
// quadrature (4 panels x 32 nodes), nodes from Newton's method on P_32.
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
  x.resize(n);
  w.resize(n);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void boys_table(int rows, int cols, double step, double *tab) {
  std::vector<double> gx, gw;
  gauss_legendre(32, gx, gw);
  const int panels = 4;
  std::vector<double> u, wu;
  for (int p = 0; p < panels; ++p)
    for (int i = 0; i < 32; ++i) {
      const double a = double(p) / panels, b = double(p + 1) / panels;
      u.push_back(0.5 * (b - a) * gx[i] + 0.5 * (a + b));
      wu.push_back(0.5 * (b - a) * gw[i]);
    }
  for (int k = 0; k < rows; ++k) {
    const double T = k * step;
    for (int m = 0; m < cols; ++m) {
      double s = 0.0;
      for (size_t i = 0; i < u.size(); ++i)
        s += wu[i] * std::pow(u[i], 2 * m) * std::exp(-T * u[i] * u[i]);
      tab[k * cols + m] = s;
    }
  }
}

// ------------------------------------------------------ Laplace quadrature
// Fit sum_q w_q exp(-t_q x) ~ 1/x in the least-squares sense on the relative
// residual r_s = 1 - x_s sum_q w_q exp(-t_q x_s).  The problem is scale
// invariant, so it is solved on [1, R], R = xmax/xmin.  Parameters are
// (log t, log w) (positivity); the solver is Levenberg-Marquardt with column
// scaling, each step from a Householder QR of the scaled Jacobian followed by
// the damped triangular system.  Points are added one at a time (continuation
// in n); nearby solutions warm-start new ranges.
namespace {

struct LapFit {
  std::vector<double> xs;
  int n = 0;
  double lt_lo = -30, lt_hi = 7;  // bounds on log t (normalised problem)
  double cost(const std::vector<double> &th, std::vector<double> *r) const {
    const int m = (int)xs.size();
    for (int q = 0; q < n; ++q)
      if (!(th[q] > lt_lo && th[q] < lt_hi && th[n + q] > -80.0 && th[n + q] < 20.0)) return 1e300;
    double c = 0.0;
    if (r) r->resize(m);
    for (int s = 0; s < m; ++s) {
      double v = 0.0;
      for (int q = 0; q < n; ++q) v += std::exp(th[n + q] - std::exp(th[q]) * xs[s]);
      double rr = 1.0 - xs[s] * v;
      if (r) (*r)[s] = rr;
      c += rr * rr;
    }
    return std::isfinite(c) ? c : 1e300;
  }
  // Jacobian J[s][k], k < n: d r/d log t_q; k >= n: d r/d log w_q
  void jac(const std::vector<double> &th, std::vector<double> &J) const {
    const int m = (int)xs.size(), p = 2 * n;
    J.assign((size_t)m * p, 0.0);
    for (int s = 0; s < m; ++s)
      for (int q = 0; q < n; ++q) {
        const double t = std::exp(th[q]);
        const double e = std::exp(th[n + q] - t * xs[s]);  // w e^{-t x}
        J[(size_t)s * p + q] = xs[s] * xs[s] * t * e;
        J[(size_t)s * p + n + q] = -xs[s] * e;
      }
  }
};

// Householder QR of the m x p matrix A (row-major), in place; returns R (p x p,
// upper) and applies Q^T to b.
void householder_qr(int m, int p, std::vector<double> &A, std::vector<double> &b,
                    std::vector<double> &R) {
  for (int k = 0; k < p; ++k) {
    double nrm = 0.0;
    for (int i = k; i < m; ++i) nrm += A[(size_t)i * p + k] * A[(size_t)i * p + k];
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    const double akk = A[(size_t)k * p + k];
    const double alpha = akk > 0 ? -nrm : nrm;
    // v = a_k - alpha e_k, stored in column k rows k..m-1
    A[(size_t)k * p + k] = akk - alpha;
    double vnorm2 = 0.0;
    for (int i = k; i < m; ++i) vnorm2 += A[(size_t)i * p + k] * A[(size_t)i * p + k];
    if (vnorm2 == 0.0) {
      A[(size_t)k * p + k] = alpha;
      continue;
    }
    for (int j = k + 1; j < p; ++j) {
      double d = 0.0;
      for (int i = k; i < m; ++i) d += A[(size_t)i * p + k] * A[(size_t)i * p + j];
      d = 2.0 * d / vnorm2;
      for (int i = k; i < m; ++i) A[(size_t)i * p + j] -= d * A[(size_t)i * p + k];
    }
    double d = 0.0;
    for (int i = k; i < m; ++i) d += A[(size_t)i * p + k] * b[i];
    d = 2.0 * d / vnorm2;
    for (int i = k; i < m; ++i) b[i] -= d * A[(size_t)i * p + k];
    A[(size_t)k * p + k] = alpha;
    for (int i = k + 1; i < m; ++i) A[(size_t)i * p + k] = 0.0;
  }
  R.assign((size_t)p * p, 0.0);
  for (int i = 0; i < p; ++i)
    for (int j = i; j < p; ++j) R[(size_t)i * p + j] = A[(size_t)i * p + j];
}

// Solve min |R x - c|^2 + lam |x|^2 for upper-triangular R (p x p) by a second QR.
std::vector<double> damped_solve(int p, const std::vector<double> &R, const std::vector<double> &c,
                                 double lam) {
  const int m = 2 * p;
  std::vector<double> A((size_t)m * p, 0.0), b(m, 0.0), R2;
  for (int i = 0; i < p; ++i) {
    for (int j = 0; j < p; ++j) A[(size_t)i * p + j] = R[(size_t)i * p + j];
    b[i] = c[i];
    A[(size_t)(p + i) * p + i] = std::sqrt(lam);
  }
  householder_qr(m, p, A, b, R2);
  std::vector<double> x(p, 0.0);
  for (int i = p - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < p; ++j) s -= R2[(size_t)i * p + j] * x[j];
    const double d = R2[(size_t)i * p + i];
    x[i] = d != 0.0 ? s / d : 0.0;
  }
  return x;
}

void lm_refine(const LapFit &F, std::vector<double> &th, int max_iter) {
  const int m = (int)F.xs.size(), p = 2 * F.n;
  std::vector<double> r, J, R, d(p);
  double cost = F.cost(th, &r);
  if (cost >= 1e300) return;  // start outside the parameter bounds
  double lam = 1e-3;
  for (int it = 0; it < max_iter; ++it) {
    F.jac(th, J);
    for (int k = 0; k < p; ++k) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += J[(size_t)i * p + k] * J[(size_t)i * p + k];
      d[k] = s > 1e-300 ? std::sqrt(s) : 1e-150;
      for (int i = 0; i < m; ++i) J[(size_t)i * p + k] /= d[k];
    }
    std::vector<double> b(m);
    for (int i = 0; i < m; ++i) b[i] = -r[i];
    householder_qr(m, p, J, b, R);
    std::vector<double> c(b.begin(), b.begin() + p);
    bool ok = false;
    double dec = 0.0, stepmax = 0.0;
    for (int trial = 0; trial < 50; ++trial) {
      std::vector<double> step = damped_solve(p, R, c, lam);
      std::vector<double> th2(p);
      stepmax = 0.0;
      for (int k = 0; k < p; ++k) {
        th2[k] = th[k] + step[k] / d[k];
        stepmax = std::max(stepmax, std::fabs(step[k] / d[k]));
      }
      std::vector<double> r2;
      const double c2 = F.cost(th2, &r2);
      if (c2 < cost) {
        dec = (cost - c2) / cost;
        th = th2;
        r = r2;
        cost = c2;
        lam = std::max(lam / 3.0, 1e-30);
        ok = true;
        break;
      }
      lam = std::max(lam * 4.0, 1e-14);
    }
    if (!ok) break;
    if (dec < 1e-13 && stepmax < 1e-9) break;
  }
}

double max_rel_error(const std::vector<double> &t, const std::vector<double> &w, double xmin,
                     double xmax, int ncheck) {
  double err = 0.0;
  const double lr = std::log(xmax / xmin);
  for (int s = 0; s < ncheck; ++s) {
    const double x = xmin * std::exp(lr * s / (ncheck - 1));
    double v = 0.0;
    for (size_t q = 0; q < t.size(); ++q) v += w[q] * std::exp(-t[q] * x);
    const double d = std::fabs(x * v - 1.0);
    if (!(d <= err)) err = d;  // propagates NaN
  }
  return err;
}

}  // namespace

// Sort the k nodes (and their weights) ascending.
static void sort_nodes(std::vector<double> &th, int k) {
  std::vector<int> ord(k);
  for (int q = 0; q < k; ++q) ord[q] = q;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return th[a] < th[b]; });
  std::vector<double> th2(2 * k);
  for (int q = 0; q < k; ++q) {
    th2[q] = th[ord[q]];
    th2[k + q] = th[k + ord[q]];
  }
  th = th2;
}

// Continuation in the number of points: from the best k-1 point fit, try a new
// node beyond the largest exponent, below the smallest, and in the widest gap;
// keep the candidate with the lowest cost after refinement.
static std::vector<double> fit_continuation(LapFit &F, double R, int n) {
  std::vector<double> th = {std::log(1.0 / std::sqrt(R)), 0.0};
  F.n = 1;
  lm_refine(F, th, 300);
  for (int k = 2; k <= n; ++k) {
    const int km = k - 1;
    std::vector<double> lt(th.begin(), th.begin() + km), lw(th.begin() + km, th.end());
    std::vector<std::vector<double>> cands;
    const double step = km > 1 ? lt[km - 1] - lt[km - 2] : std::log(3.0);
    const double step0 = km > 1 ? lt[1] - lt[0] : std::log(3.0);
    {  // beyond the largest
      auto t2 = lt, w2 = lw;
      t2.push_back(lt[km - 1] + step);
      w2.push_back(lw[km - 1] + std::log(0.5));
      cands.push_back(t2);
      cands.back().insert(cands.back().end(), w2.begin(), w2.end());
    }
    {  // below the smallest
      auto t2 = lt, w2 = lw;
      t2.push_back(lt[0] - step0);
      w2.push_back(lw[0] - step0);
      cands.push_back(t2);
      cands.back().insert(cands.back().end(), w2.begin(), w2.end());
    }
    if (km > 1) {  // split the widest gap
      int g = 0;
      for (int q = 1; q + 1 < km; ++q)
        if (lt[q + 1] - lt[q] > lt[g + 1] - lt[g]) g = q;
      auto t2 = lt, w2 = lw;
      t2.push_back(0.5 * (lt[g] + lt[g + 1]));
      w2.push_back(0.5 * (lw[g] + lw[g + 1]) + std::log(0.5));
      w2[g] += std::log(0.75);
      w2[g + 1] += std::log(0.75);
      cands.push_back(t2);
      cands.back().insert(cands.back().end(), w2.begin(), w2.end());
    }
    F.n = k;
    double best = 1e300;
    std::vector<double> best_th;
    for (auto &c : cands) {
      lm_refine(F, c, 300);
      const double cc = F.cost(c, nullptr);
      if (cc < best) {
        best = cc;
        best_th = c;
      }
    }
    th = best_th;
    sort_nodes(th, k);
  }
  return th;
}

int laplace_quadrature(double xmin, double xmax, int n, double *t_out, double *w_out,
                       double *err_out) {
  if (!(xmin > 0) || !(xmax > xmin) || !std::isfinite(xmax) || n < 1 || n > 32 || !t_out || !w_out)
    return set_error(LTJK_EINVAL, "laplace_quadrature: need 0 < xmin < xmax and 1 <= n <= 32");
  // Cache of normalised solutions per n, keyed by log R: an exact hit is
  // reused, a nearby one warm-starts the refinement.
  static std::mutex mu;
  static std::map<int, std::map<double, std::vector<double>>> cache;
  const double R = xmax / xmin, lR = std::log(R);
  std::vector<double> th;
  bool exact = false;
  {
    std::lock_guard<std::mutex> g(mu);
    auto &m = cache[n];
    auto it = m.lower_bound(lR);
    const std::vector<double> *near = nullptr;
    double dist = 1e300;
    if (it != m.end()) {
      dist = it->first - lR;
      near = &it->second;
      if (dist == 0.0) exact = true;
    }
    if (!exact && it != m.begin()) {
      auto jt = std::prev(it);
      if (lR - jt->first < dist) {
        dist = lR - jt->first;
        near = &jt->second;
      }
    }
    if (near && dist < 0.5) th = *near;
  }
  if (!exact) {
    LapFit F;
    const int m = 1000;
    for (int s = 0; s < m; ++s) F.xs.push_back(std::exp(lR * s / (m - 1)));
    F.lt_lo = std::log(1e-6 / R);
    F.lt_hi = std::log(1e3);
    std::vector<double> cold;
    if (!th.empty()) {
      F.n = n;
      lm_refine(F, th, 300);
      sort_nodes(th, n);
    }
    if (th.empty() || F.cost(th, nullptr) >= 1e300) th = fit_continuation(F, R, n);
    std::lock_guard<std::mutex> g(mu);
    cache[n][lR] = th;
  }
  std::vector<double> t(n), w(n);
  for (int q = 0; q < n; ++q) {
    t[q] = std::exp(th[q]) / xmin;
    w[q] = std::exp(th[n + q]) / xmin;
    t_out[q] = t[q];
    w_out[q] = w[q];
  }
  const double err = max_rel_error(t, w, xmin, xmax, 100000);
  if (!std::isfinite(err)) return set_error(LTJK_EINVAL, "laplace_quadrature: fit failed");
  if (err_out) *err_out = err;
  return LTJK_OK;
}

// ------------------------------------------------ minimax (Remez exchange)
// Best uniform relative approximation on [1, R]: the error e(x) = 1 - x sum w
// e^{-t x} of the optimum equioscillates at 2n+1 points.  Starting from the
// least-squares fit: (1) locate the 2n+1 alternating extrema of e on a fine
// log grid (split at sign changes, largest |e| in each piece); (2) solve
// e(x_i) = s_i E for (log t, log w, E) by damped Newton with Gaussian
// elimination; repeat until the levelled E equals the maximum error.
namespace {

double rel_err(const std::vector<double> &t, const std::vector<double> &w, double x) {
  double v = 0.0;
  for (size_t q = 0; q < t.size(); ++q) v += w[q] * std::exp(-t[q] * x);
  return 1.0 - x * v;
}

bool alternation(const std::vector<double> &t, const std::vector<double> &w, double R, int n,
                 std::vector<double> &pts, std::vector<double> &sg, double *emax) {
  const int ng = 20000;
  const double lr = std::log(R);
  pts.clear();
  sg.clear();
  *emax = 0.0;
  double best = -1.0, bx = 1.0;
  int cur = 0;
  for (int k = 0; k < ng; ++k) {
    const double x = std::exp(lr * k / (ng - 1)), e = rel_err(t, w, x);
    const int s = e > 0 ? 1 : (e < 0 ? -1 : cur);
    *emax = std::max(*emax, std::fabs(e));
    if (k > 0 && s != cur && cur != 0) {
      pts.push_back(bx);
      sg.push_back(cur);
      best = -1.0;
    }
    cur = s;
    if (std::fabs(e) > best) {
      best = std::fabs(e);
      bx = x;
    }
  }
  pts.push_back(bx);
  sg.push_back(cur);
  return (int)pts.size() == 2 * n + 1;
}

bool solve_dense(int m, std::vector<double> &A, std::vector<double> &b) {
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(A[(size_t)r * m + c]) > std::fabs(A[(size_t)piv * m + c])) piv = r;
    if (A[(size_t)piv * m + c] == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < m; ++k) std::swap(A[(size_t)c * m + k], A[(size_t)piv * m + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < m; ++r) {
      const double f = A[(size_t)r * m + c] / A[(size_t)c * m + c];
      if (f == 0.0) continue;
      for (int k = c; k < m; ++k) A[(size_t)r * m + k] -= f * A[(size_t)c * m + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = m - 1; r >= 0; --r) {
    double v = b[r];
    for (int k = r + 1; k < m; ++k) v -= A[(size_t)r * m + k] * b[k];
    b[r] = v / A[(size_t)r * m + r];
  }
  return true;
}

// Remez on [1, R] from (t, w); returns false (inputs untouched) on failure.
bool remez(double R, int n, std::vector<double> &t, std::vector<double> &w) {
  std::vector<double> tt = t, ww = w, pts, sg;
  double emax = 0.0, E = 0.0;
  bool ok = false;
  for (int it = 0; it < 60; ++it) {
    if (!alternation(tt, ww, R, n, pts, sg, &emax)) break;
    E = 0.0;
    for (int i = 0; i <= 2 * n; ++i) E += std::fabs(rel_err(tt, ww, pts[i]));
    E /= 2 * n + 1;
    if (it > 0 && emax <= E * (1.0 + 1e-6)) {
      ok = true;
      break;
    }
    // Newton on F_i = e(x_i) - s_i E over theta = (log t, log w, E)
    const int m = 2 * n + 1;
    std::vector<double> th(m);
    for (int q = 0; q < n; ++q) {
      th[q] = std::log(tt[q]);
      th[n + q] = std::log(ww[q]);
    }
    th[2 * n] = E;
    auto resid = [&](const std::vector<double> &x, std::vector<double> &F) {
      std::vector<double> t2(n), w2(n);
      for (int q = 0; q < n; ++q) {
        t2[q] = std::exp(x[q]);
        w2[q] = std::exp(x[n + q]);
      }
      double s = 0.0;
      for (int i = 0; i < m; ++i) {
        F[i] = rel_err(t2, w2, pts[i]) - sg[i] * x[2 * n];
        s += F[i] * F[i];
      }
      return s;
    };
    std::vector<double> F(m);
    double f0 = resid(th, F);
    for (int nt = 0; nt < 30 && f0 > 0; ++nt) {
      std::vector<double> Jm((size_t)m * m), rhs(m);
      for (int i = 0; i < m; ++i) {
        const double x = pts[i];
        for (int q = 0; q < n; ++q) {
          const double tq = std::exp(th[q]), wq = std::exp(th[n + q]), ex = std::exp(-tq * x);
          Jm[(size_t)i * m + q] = x * x * wq * tq * ex;  // d e / d log t
          Jm[(size_t)i * m + n + q] = -x * wq * ex;      // d e / d log w
        }
        Jm[(size_t)i * m + 2 * n] = -sg[i];
        rhs[i] = -F[i];
      }
      if (!solve_dense(m, Jm, rhs)) break;
      double lam = 1.0, f1 = 0.0;
      std::vector<double> th2(m), F2(m);
      for (int ls = 0; ls < 30; ++ls, lam *= 0.5) {
        for (int k = 0; k < m; ++k) th2[k] = th[k] + lam * rhs[k];
        f1 = resid(th2, F2);
        if (std::isfinite(f1) && f1 < f0) break;
      }
      if (!(std::isfinite(f1) && f1 < f0)) break;
      th = th2;
      F = F2;
      f0 = f1;
    }
    for (int q = 0; q < n; ++q) {
      tt[q] = std::exp(th[q]);
      ww[q] = std::exp(th[n + q]);
    }
  }
  if (!ok) return false;
  for (double v : tt)
    if (!(v > 0) || !std::isfinite(v)) return false;
  std::vector<int> ord(n);
  for (int q = 0; q < n; ++q) ord[q] = q;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return tt[a] < tt[b]; });
  for (int q = 0; q < n; ++q) {
    t[q] = tt[ord[q]];
    w[q] = ww[ord[q]];
  }
  return true;
}

}  // namespace

int laplace_minimax(double xmin, double xmax, int n, double *t_out, double *w_out,
                    double *err_out, int *converged) {
  int rc = laplace_quadrature(xmin, xmax, n, t_out, w_out, nullptr);
  if (rc) return rc;
  const double R = xmax / xmin;
  std::vector<double> t(n), w(n);
  for (int q = 0; q < n; ++q) {
    t[q] = t_out[q] * xmin;
    w[q] = w_out[q] * xmin;
  }
  const bool ok = remez(R, n, t, w);
  if (converged) *converged = ok ? 1 : 0;
  std::vector<double> tt(n), wt(n);
  for (int q = 0; q < n; ++q) {
    tt[q] = t[q] / xmin;
    wt[q] = w[q] / xmin;
    t_out[q] = tt[q];
    w_out[q] = wt[q];
  }
  if (err_out) *err_out = max_rel_error(tt, wt, xmin, xmax, 100000);
  return LTJK_OK;
}

}  // namespace ltjk
