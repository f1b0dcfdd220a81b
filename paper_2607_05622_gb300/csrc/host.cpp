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
// invariant, so it is solved on [1, R], R = xmax/xmin.  The residual is linear
// in the weights, so they are eliminated by variable projection (Golub and
// Pereyra, SIAM J. Numer. Anal. 10, 413 (1973)): for exponents t the weights
// are the linear least-squares solution (Householder QR), and
// Levenberg-Marquardt runs on log t alone, with the Jacobian of the projected
// residual by forward differences.  Points are added one at a time
// (continuation in n, trying a node beyond the largest exponent, below the
// smallest and in the widest gap, keeping the lowest cost with positive
// weights).  Once no added node lowers the cost (the fit has reached the
// limit double precision allows on this range), the remaining nodes are
// placed in the widest gaps with a negligible weight, so the requested n is
// honoured without a worse fit.  Nearby solutions warm-start
// new ranges.
namespace {

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

// Solve A x = b (m x m, row-major) by Gaussian elimination with partial
// pivoting; b is overwritten by x.  Returns false for a singular A.
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

// The normalised problem on [1, R]: sample points and bounds on log t.
struct LapFit {
  std::vector<double> xs;
  double lt_lo = -30, lt_hi = 7;
  // Weights of the exponents t = exp(th) by linear least squares, the
  // residual and its squared norm; 1e300 outside the bounds or for a
  // numerically singular basis.
  double project(const std::vector<double> &th, std::vector<double> *w, std::vector<double> *r) const {
    const int m = (int)xs.size(), n = (int)th.size();
    for (double v : th)
      if (!(v > lt_lo && v < lt_hi)) return 1e300;
    std::vector<double> A((size_t)m * n), b(m, 1.0), R, cn(n, 0.0);
    for (int s = 0; s < m; ++s)
      for (int q = 0; q < n; ++q) A[(size_t)s * n + q] = xs[s] * std::exp(-std::exp(th[q]) * xs[s]);
    const std::vector<double> A0 = A;
    // columns scaled to unit norm before the factorisation: the rank test then
    // sees the angles between the basis functions, not their sizes (a large t
    // gives a column of tiny norm that is still well determined)
    for (int s = 0; s < m; ++s)
      for (int q = 0; q < n; ++q) cn[q] += A[(size_t)s * n + q] * A[(size_t)s * n + q];
    for (int q = 0; q < n; ++q) {
      if (!(cn[q] > 0.0)) return 1e300;
      cn[q] = std::sqrt(cn[q]);
    }
    for (int s = 0; s < m; ++s)
      for (int q = 0; q < n; ++q) A[(size_t)s * n + q] /= cn[q];
    householder_qr(m, n, A, b, R);
    double dmax = 0.0, dmin = 1e300;
    for (int q = 0; q < n; ++q) {
      const double d = std::fabs(R[(size_t)q * n + q]);
      dmax = std::max(dmax, d);
      dmin = std::min(dmin, d);
    }
    if (!(dmin > 1e-15 * dmax)) return 1e300;
    std::vector<double> ww(n);
    for (int i = n - 1; i >= 0; --i) {
      double v = b[i];
      for (int j = i + 1; j < n; ++j) v -= R[(size_t)i * n + j] * ww[j];
      ww[i] = v / R[(size_t)i * n + i];
    }
    for (int q = 0; q < n; ++q) ww[q] /= cn[q];
    double c = 0.0;
    std::vector<double> rr(m);
    for (int s = 0; s < m; ++s) {
      double v = 1.0;
      for (int q = 0; q < n; ++q) v -= A0[(size_t)s * n + q] * ww[q];
      rr[s] = v;
      c += v * v;
    }
    if (!std::isfinite(c)) return 1e300;
    if (w) *w = ww;
    if (r) *r = rr;
    return c;
  }
};

// Levenberg-Marquardt on the exponents (log t) with the linear unknowns
// projected out by `proj(th, &lin, &r)` (returns |r|^2, 1e300 when infeasible);
// Marquardt scaling by diag(J^T J), J by forward differences; a step is taken
// only if it lowers the cost.  th and lin are updated in place; returns the
// final cost.
template <typename Proj>
double varpro_lm(const Proj &proj, std::vector<double> &th, std::vector<double> &w, int max_iter) {
  const int n = (int)th.size();
  std::vector<double> r, rp;
  double cost = proj(th, &w, &r);
  if (cost >= 1e300) return cost;
  const int m = (int)r.size();
  std::vector<double> J((size_t)m * n);
  double lam = 1e-3;
  for (int it = 0; it < max_iter; ++it) {
    for (int k = 0; k < n; ++k) {  // forward (else backward) differences
      std::vector<double> tp = th;
      double h = 1e-7;
      tp[k] += h;
      if (proj(tp, nullptr, &rp) >= 1e300) {
        tp[k] = th[k] - h;
        h = -h;
        if (proj(tp, nullptr, &rp) >= 1e300) return cost;
      }
      for (int s = 0; s < m; ++s) J[(size_t)s * n + k] = (rp[s] - r[s]) / h;
    }
    std::vector<double> H((size_t)n * n, 0.0), g(n, 0.0);
    for (int s = 0; s < m; ++s)
      for (int a = 0; a < n; ++a) {
        const double ja = J[(size_t)s * n + a];
        g[a] += ja * r[s];
        for (int b = 0; b <= a; ++b) H[(size_t)a * n + b] += ja * J[(size_t)s * n + b];
      }
    for (int a = 0; a < n; ++a)
      for (int b = a + 1; b < n; ++b) H[(size_t)a * n + b] = H[(size_t)b * n + a];
    bool ok = false;
    double dec = 0.0, stepmax = 0.0;
    for (int trial = 0; trial < 40; ++trial) {
      std::vector<double> A = H, step(n);
      for (int a = 0; a < n; ++a) {
        A[(size_t)a * n + a] += lam * (H[(size_t)a * n + a] + 1e-300);
        step[a] = -g[a];
      }
      if (!solve_dense(n, A, step)) {
        lam *= 4.0;
        continue;
      }
      std::vector<double> th2(n), w2, r2;
      stepmax = 0.0;
      for (int a = 0; a < n; ++a) {
        th2[a] = th[a] + step[a];
        stepmax = std::max(stepmax, std::fabs(step[a]));
      }
      const double c2 = proj(th2, &w2, &r2);
      if (c2 < cost) {
        dec = (cost - c2) / cost;
        th = th2;
        w = w2;
        r = r2;
        cost = c2;
        lam = std::max(lam / 3.0, 1e-20);
        ok = true;
        break;
      }
      lam *= 4.0;
    }
    if (!ok || (dec < 1e-15 && stepmax < 1e-12)) break;
  }
  return cost;
}

// Sort exponents ascending, carrying their weights.
void sort_pairs(std::vector<double> &th, std::vector<double> &w) {
  std::vector<int> ord(th.size());
  for (size_t q = 0; q < th.size(); ++q) ord[q] = (int)q;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return th[a] < th[b]; });
  std::vector<double> t2(th.size()), w2(w.size());
  for (size_t q = 0; q < th.size(); ++q) {
    t2[q] = th[ord[q]];
    w2[q] = w[ord[q]];
  }
  th = t2;
  w = w2;
}

bool all_positive(const std::vector<double> &w) {
  for (double v : w)
    if (!(v > 0.0)) return false;
  return !w.empty();
}

// Continuation in the number of points up to n; th/w receive the active
// nodes (log t, ascending) and their weights.  A non-empty th on entry is an
// earlier step of this same continuation (same F, fewer nodes, ascending),
// which it resumes from unchanged, so the result does not depend on whether
// the earlier steps were cached.  path, when given, receives the active nodes
// after every accepted step, keyed by their number.
void fit_continuation(const LapFit &F, double R, int n, std::vector<double> &th, std::vector<double> &w,
                      std::map<int, std::vector<double>> *path) {
  auto proj = [&F](const std::vector<double> &x, std::vector<double> *ww, std::vector<double> *rr) {
    return F.project(x, ww, rr);
  };
  double cost = th.empty() ? 1e300 : F.project(th, &w, nullptr);
  if (cost >= 1e300) {
    th = {std::log(1.0 / std::sqrt(R))};
    cost = varpro_lm(proj, th, w, 300);
  }
  if (path) (*path)[(int)th.size()] = th;
  while ((int)th.size() < n) {
    const int km = (int)th.size();
    const double step = km > 1 ? th[km - 1] - th[km - 2] : std::log(3.0);
    const double step0 = km > 1 ? th[1] - th[0] : std::log(3.0);
    std::vector<std::vector<double>> cands;
    cands.push_back(th);
    cands.back().push_back(th[km - 1] + step);  // beyond the largest
    cands.push_back(th);
    cands.back().push_back(th[0] - step0);  // below the smallest
    if (km > 1) {  // split the widest gap
      int gq = 0;
      for (int q = 1; q + 1 < km; ++q)
        if (th[q + 1] - th[q] > th[gq + 1] - th[gq]) gq = q;
      cands.push_back(th);
      cands.back().push_back(0.5 * (th[gq] + th[gq + 1]));
    }
    double best = cost;
    std::vector<double> bth, bw;
    for (auto &c : cands) {
      std::sort(c.begin(), c.end());
      std::vector<double> wc;
      const double cc = varpro_lm(proj, c, wc, 300);
      if (cc < best && all_positive(wc)) {
        best = cc;
        bth = c;
        bw = wc;
      }
    }
    if (bth.empty()) break;  // no added node lowers the cost: the fit has converged in n
    th = bth;
    w = bw;
    sort_pairs(th, w);
    cost = best;
    if (path) (*path)[(int)th.size()] = th;
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

// Complete n nodes: the ones a fit could not use go to the geometric midpoint
// of the widest gap (ordinary exponents, so their pseudo-densities are of
// ordinary size) with a weight of 1e-16 of the smallest.  lt holds log t.
static void fill_nodes(std::vector<double> &lt, std::vector<double> &lw, int n) {
  double wmin = 1e300;
  for (double v : lw) wmin = std::min(wmin, v);
  while ((int)lt.size() < n) {
    int g = 0;
    if (lt.size() > 1) {
      for (size_t q = 1; q + 1 < lt.size(); ++q)
        if (lt[q + 1] - lt[q] > lt[g + 1] - lt[g]) g = (int)q;
      lt.push_back(0.5 * (lt[g] + lt[g + 1]));
    } else {
      lt.push_back(lt[0] + std::log(3.0));
    }
    lw.push_back(1e-16 * wmin);
    sort_pairs(lt, lw);
  }
}

int laplace_quadrature(double xmin, double xmax, int n, double *t_out, double *w_out,
                       double *err_out) {
  if (!(xmin > 0) || !(xmax > xmin) || !std::isfinite(xmax) || n < 1 || n > 32 || !t_out || !w_out)
    return set_error(LTJK_EINVAL, "laplace_quadrature: need 0 < xmin < xmax and 1 <= n <= 32");
  // The fit is made on [1, Rg] with log Rg = log R rounded up to a multiple of
  // 1/8 (Rg / R < 1.14; a fit on the wider range is valid on the requested
  // one), so the nodes depend only on n and that cell, not on the order of
  // earlier requests.  Every step of a continuation is cached under its cell
  // and its number of points: a request resumes the continuation from the
  // largest cached step at or below n, which gives what a fresh continuation
  // would.
  static std::mutex mu;
  static std::map<std::pair<long, int>, std::vector<double>> cache;
  const double R = xmax / xmin;
  const long cell = std::max(1L, (long)std::ceil(8.0 * std::log(R) - 1e-12));
  const double lRg = cell / 8.0, Rg = std::exp(lRg);
  std::vector<double> th, w;
  bool hit = false;
  {
    std::lock_guard<std::mutex> g(mu);
    for (int k = n; k >= 1 && !hit && th.empty(); --k) {
      auto it = cache.find({cell, k});
      if (it == cache.end()) continue;
      th = it->second;
      hit = k == n;
    }
  }
  LapFit F;
  const int m = 500;
  for (int s = 0; s < m; ++s) F.xs.push_back(std::exp(lRg * s / (m - 1)));
  F.lt_lo = std::log(1e-6 / Rg);
  F.lt_hi = std::log(1e3);
  if (hit) {
    F.project(th, &w, nullptr);
  } else {
    std::map<int, std::vector<double>> path;
    fit_continuation(F, Rg, n, th, w, &path);
    std::lock_guard<std::mutex> g(mu);
    for (const auto &kv : path) cache.emplace(std::make_pair(cell, kv.first), kv.second);
    // a continuation that stopped below n has converged in the number of
    // points: its fit is also the answer for every count up to n
    for (int k = (int)th.size() + 1; k <= n; ++k) cache.emplace(std::make_pair(cell, k), th);
  }
  std::vector<double> lt = th, lw = w;
  fill_nodes(lt, lw, n);
  std::vector<double> t(n), wt(n);
  for (int q = 0; q < n; ++q) {
    t[q] = std::exp(lt[q]) / xmin;
    wt[q] = lw[q] / xmin;
    t_out[q] = t[q];
    w_out[q] = wt[q];
  }
  const double err = max_rel_error(t, wt, xmin, xmax, 100000);
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

// Lawson's iteration (iteratively reweighted least squares, each sample's
// weight multiplied by |e(x_s)| after every fit) on the 500-point grid of
// [1, R]: it moves the least-squares fit towards the best uniform
// approximation, so that the error acquires the 2n+1 alternating extrema the
// exchange starts from.  th (log t) and w are updated in place.
void lawson(double R, std::vector<double> &th, std::vector<double> &w, int iters) {
  const int m = 500, n = (int)th.size();
  const double lr = std::log(R), lt_lo = std::log(1e-6 / R), lt_hi = std::log(1e3);
  std::vector<double> xs(m), om(m, 1.0 / m);
  for (int s = 0; s < m; ++s) xs[s] = std::exp(lr * s / (m - 1));
  for (int it = 0; it < iters; ++it) {
    auto proj = [&](const std::vector<double> &x, std::vector<double> *ww, std::vector<double> *rr) {
      for (double v : x)
        if (!(v > lt_lo && v < lt_hi)) return 1e300;
      std::vector<double> A((size_t)m * n), b(m), Rm;
      for (int s = 0; s < m; ++s) {
        const double sq = std::sqrt(om[s]);
        b[s] = sq;
        for (int q = 0; q < n; ++q) A[(size_t)s * n + q] = sq * xs[s] * std::exp(-std::exp(x[q]) * xs[s]);
      }
      const std::vector<double> A0 = A, b0 = b;
      householder_qr(m, n, A, b, Rm);
      double dmax = 0.0, dmin = 1e300;
      for (int q = 0; q < n; ++q) {
        dmax = std::max(dmax, std::fabs(Rm[(size_t)q * n + q]));
        dmin = std::min(dmin, std::fabs(Rm[(size_t)q * n + q]));
      }
      if (!(dmin > 1e-15 * dmax)) return 1e300;
      std::vector<double> sol(n);
      for (int i = n - 1; i >= 0; --i) {
        double v = b[i];
        for (int j = i + 1; j < n; ++j) v -= Rm[(size_t)i * n + j] * sol[j];
        sol[i] = v / Rm[(size_t)i * n + i];
      }
      double c = 0.0;
      std::vector<double> res(m);
      for (int s = 0; s < m; ++s) {
        double v = b0[s];
        for (int q = 0; q < n; ++q) v -= A0[(size_t)s * n + q] * sol[q];
        res[s] = v;  // weighted residual
        c += v * v;
      }
      if (!std::isfinite(c)) return 1e300;
      if (ww) *ww = sol;
      if (rr) *rr = res;
      return c;
    };
    std::vector<double> th2 = th, w2;
    if (varpro_lm(proj, th2, w2, 30) >= 1e300 || !all_positive(w2)) return;
    th = th2;
    w = w2;
    double tot = 0.0;
    for (int s = 0; s < m; ++s) {
      double v = 0.0;
      for (int q = 0; q < n; ++q) v += w[q] * std::exp(-std::exp(th[q]) * xs[s]);
      om[s] *= std::fabs(1.0 - xs[s] * v);
      tot += om[s];
    }
    if (!(tot > 0.0)) return;
    for (double &v : om) v /= tot;
  }
}

// Remez on [1, R] from (t, w); returns false (inputs untouched) on failure.
// Each exchange solves e(x_i) = s_i E at the 2n+1 alternation points by
// variable projection: for exponents t the equations are linear in (w, E),
// solved in the least-squares sense by Householder QR, and Levenberg-Marquardt
// on log t drives their residual to zero.
bool remez(double R, int n, std::vector<double> &t, std::vector<double> &w) {
  std::vector<double> th(n), ww = w, pts, sg;
  for (int q = 0; q < n; ++q) th[q] = std::log(t[q]);
  lawson(R, th, ww, 20);
  const double lt_lo = std::log(1e-6 / R), lt_hi = std::log(1e3);
  double emax = 0.0, E = 0.0;
  bool ok = false;
  for (int it = 0; it < 60; ++it) {
    std::vector<double> tt(n);
    for (int q = 0; q < n; ++q) tt[q] = std::exp(th[q]);
    if (!alternation(tt, ww, R, n, pts, sg, &emax)) break;
    if (it > 0 && emax <= std::fabs(E) * (1.0 + 1e-6)) {
      ok = true;
      break;
    }
    const int m = 2 * n + 1, p = n + 1;
    auto proj = [&](const std::vector<double> &x, std::vector<double> *lin, std::vector<double> *rr) {
      for (double v : x)
        if (!(v > lt_lo && v < lt_hi)) return 1e300;
      std::vector<double> A((size_t)m * p), b(m, 1.0), Rm;
      for (int i = 0; i < m; ++i) {
        for (int q = 0; q < n; ++q) A[(size_t)i * p + q] = pts[i] * std::exp(-std::exp(x[q]) * pts[i]);
        A[(size_t)i * p + n] = sg[i];
      }
      const std::vector<double> A0 = A;
      householder_qr(m, p, A, b, Rm);
      double dmax = 0.0, dmin = 1e300;
      for (int q = 0; q < p; ++q) {
        dmax = std::max(dmax, std::fabs(Rm[(size_t)q * p + q]));
        dmin = std::min(dmin, std::fabs(Rm[(size_t)q * p + q]));
      }
      if (!(dmin > 1e-15 * dmax)) return 1e300;
      std::vector<double> sol(p);
      for (int i = p - 1; i >= 0; --i) {
        double v = b[i];
        for (int j = i + 1; j < p; ++j) v -= Rm[(size_t)i * p + j] * sol[j];
        sol[i] = v / Rm[(size_t)i * p + i];
      }
      double c = 0.0;
      std::vector<double> res(m);
      for (int i = 0; i < m; ++i) {
        double v = 1.0;
        for (int q = 0; q < p; ++q) v -= A0[(size_t)i * p + q] * sol[q];
        res[i] = v;
        c += v * v;
      }
      if (!std::isfinite(c)) return 1e300;
      if (lin) *lin = sol;
      if (rr) *rr = res;
      return c;
    };
    std::vector<double> lin;
    if (varpro_lm(proj, th, lin, 200) >= 1e300 || lin.size() != (size_t)p) break;
    ww.assign(lin.begin(), lin.begin() + n);
    E = lin[n];
    if (!all_positive(ww)) break;
  }
  if (!ok) return false;
  std::vector<double> tt(n);
  for (int q = 0; q < n; ++q) {
    tt[q] = std::exp(th[q]);
    if (!(tt[q] > 0) || !std::isfinite(tt[q])) return false;
  }
  sort_pairs(tt, ww);
  t = tt;
  w = ww;
  return true;
}

}  // namespace

int laplace_minimax(double xmin, double xmax, int n, double *t_out, double *w_out,
                    double *err_out, int *converged) {
  int rc = laplace_quadrature(xmin, xmax, n, t_out, w_out, nullptr);
  if (rc) return rc;
  const double R = xmax / xmin;
  // the exchange runs on the nodes the least-squares fit uses; the others
  // (negligible weight) are completed afterwards as in the least-squares grid
  double wmax = 0.0;
  for (int q = 0; q < n; ++q) wmax = std::max(wmax, w_out[q]);
  std::vector<double> t, w;
  for (int q = 0; q < n; ++q)
    if (w_out[q] > 1e-12 * wmax) {
      t.push_back(t_out[q] * xmin);
      w.push_back(w_out[q] * xmin);
    }
  const bool ok = remez(R, (int)t.size(), t, w);
  if (converged) *converged = ok ? 1 : 0;
  if (ok) {
    std::vector<double> lt(t.size());
    for (size_t q = 0; q < t.size(); ++q) lt[q] = std::log(t[q]);
    fill_nodes(lt, w, n);
    for (int q = 0; q < n; ++q) {
      t_out[q] = std::exp(lt[q]) / xmin;
      w_out[q] = w[q] / xmin;
    }
  }
  std::vector<double> tt(t_out, t_out + n), wt(w_out, w_out + n);
  if (err_out) *err_out = max_rel_error(tt, wt, xmin, xmax, 100000);
  return LTJK_OK;
}

}  // namespace ltjk
