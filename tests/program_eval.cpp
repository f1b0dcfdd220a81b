// Test infrastructure: evaluates contracted Cartesian shell quartets on the CPU
// by interpreting the library's generated recurrence programs (the programs
// the integral kernels run: Obara-Saika vertical steps level by level, the
// accumulation, the horizontal steps and the output block), with this file's
// own Boys function and primitive set-up.  The tests compare its blocks with
// the oracle's McMurchie-Davidson blocks, which pins the program generator on
// the CPU.  pe_quartet_f32 runs the same programs in binary32 (the mixed
// mode's error model); pe_quartet_gen, compiled with LTJK_GEN_HEADER, runs
// the straight-line source the class generator emits.  Compiled by the tests
// themselves (g++), never by the library build.
#include <algorithm>
#include <map>
#include <cmath>
#include <vector>

#include "ltjk_internal.h"

using namespace ltjk;

namespace {

const ProgramSet &programs() {
  static ProgramSet ps;
  static bool built = false;
  if (!built) {
    build_programs(ps);
    built = true;
  }
  return ps;
}

// F_m(T), m = 0..mmax: the convergent series e^{-T} sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1))
// evaluated for F_mmax and descended; for large T the erf form and upward recursion.
template <typename R>
void boys(int mmax, R Tr, R *F) {
  const long double T = Tr;
  if (T < 30.0L) {
    long double term = 1.0L / (2 * mmax + 1), sum = term;
    for (int k = 1; k < 400; ++k) {
      term *= 2.0L * T / (2 * mmax + 2 * k + 1);
      sum += term;
      if (term < 1e-22L * sum) break;
    }
    const long double e = std::exp(-T);
    long double f = e * sum;
    F[mmax] = (R)f;
    for (int m = mmax - 1; m >= 0; --m) {
      f = (2.0L * T * f + e) / (2 * m + 1);
      F[m] = (R)f;
    }
  } else {
    const long double e = std::exp(-T), pi = 3.141592653589793238462643383279503L;
    long double f = 0.5L * std::sqrt(pi / T) * std::erf(std::sqrt(T));
    F[0] = (R)f;
    for (int m = 0; m < mmax; ++m) {
      f = ((2 * m + 1) * f - e) / (2.0L * T);
      F[m + 1] = (R)f;
    }
  }
}

}  // namespace

extern "C" int pe_init() {
  try {
    programs();
  } catch (...) {
    return -1;
  }
  return 0;
}

namespace {

// Base values [00|00]^(m) (base[m], m = 0..ltot), the CoefSlot coefficients
// and the n/(2 zeta), n/(2 eta), n/(2 (zeta+eta)) tables of the primitive
// quartet (a, b | c, d) with full contraction coefficients ca..cd.
template <typename R>
void setup_primitive(const ClassProg &p, const R *A, const R *B, const R *C, const R *D, R a, R b, R c,
                     R d, R coef, R *base, R *cf, R *h) {
  const R zeta = a + b, eta = c + d, rho = zeta * eta / (zeta + eta);
  R P[3], Q[3], W[3], ab2 = 0, cd2 = 0, pq2 = 0;
  for (int x = 0; x < 3; ++x) {
    P[x] = (a * A[x] + b * B[x]) / zeta;
    Q[x] = (c * C[x] + d * D[x]) / eta;
    W[x] = (zeta * P[x] + eta * Q[x]) / (zeta + eta);
    ab2 += (A[x] - B[x]) * (A[x] - B[x]);
    cd2 += (C[x] - D[x]) * (C[x] - D[x]);
    pq2 += (P[x] - Q[x]) * (P[x] - Q[x]);
  }
  std::vector<R> F(p.ltot + 1);
  boys<R>(p.ltot, rho * pq2, F.data());
  const R pre = 2.0 * std::pow((R)3.141592653589793238462643383279503L, (R)2.5) / (zeta * eta * std::sqrt(zeta + eta)) *
                     std::exp(-a * b / zeta * ab2 - c * d / eta * cd2) * coef;
  for (int m = 0; m <= p.ltot; ++m) base[m] = pre * F[m];
  for (int x = 0; x < 3; ++x) {
    cf[kPAx + x] = P[x] - A[x];
    cf[kQCx + x] = Q[x] - C[x];
    cf[kWPx + x] = W[x] - P[x];
    cf[kWQx + x] = W[x] - Q[x];
  }
  cf[kHalfZeta] = 0.5 / zeta;
  cf[kHalfEta] = 0.5 / eta;
  cf[kRhoZeta] = rho / zeta;
  cf[kRhoEta] = rho / eta;
  cf[kHalfSum] = 0.5 / (zeta + eta);
  cf[kWA] = 2.0 * a;  // derivative channels: 2 alpha, 2 beta, 2 gamma
  cf[kWB] = 2.0 * b;
  cf[kWC] = 2.0 * c;
  for (int n = 0; n < p.nh; ++n) {
    h[n] = 0.5 * n / zeta;
    h[p.nh + n] = 0.5 * n / eta;
    h[2 * p.nh + n] = 0.5 * n / (zeta + eta);
  }
}

}  // namespace

// Shells s = 0..3 (l_0 >= l_1, l_2 >= l_3): centres ctr[3s..], np[s] primitives with
// exponents and full contraction coefficients (those multiplying the raw
// Gaussian x^l e^{-a r^2}) concatenated in shell order.  out [n0][n1][n2][n3].
// deriv = 0: the value block [n0][n1][n2][n3]; deriv = 1: the nine derivative
// tiles d/dA_x .. d/dC_z, each [n0][n1][n2][n3], concatenated.
namespace {

template <typename R>
int quartet_pt(const ProgramSet &ps, const ClassProg &p, const double *ctr_d, const int *np,
               const double *exps_d, const double *coefs_d, double *out) {
  int nprim = 0;
  for (int s = 0; s < 4; ++s) nprim += np[s];
  const std::vector<R> ctr(ctr_d, ctr_d + 12), exps(exps_d, exps_d + nprim), coefs(coefs_d, coefs_d + nprim);
  const R *A = ctr.data(), *B = A + 3, *C = A + 6, *D = A + 9;
  int off[5] = {0};
  for (int s = 0; s < 4; ++s) off[s + 1] = off[s] + np[s];
  std::vector<R> acc(p.acc_total + p.hrr_size + 1, 0.0), v(p.vrr_size), cf(kNumCoef), h(3 * p.nh);
  for (int i = off[0]; i < off[1]; ++i)
    for (int j = off[1]; j < off[2]; ++j)
      for (int k = off[2]; k < off[3]; ++k)
        for (int l = off[3]; l < off[4]; ++l) {
          v[0] = 0;
          setup_primitive(p, A, B, C, D, exps[i], exps[j], exps[k], exps[l],
                          coefs[i] * coefs[j] * coefs[k] * coefs[l], v.data() + 1, cf.data(), h.data());
          for (int L = 0; L < p.nvrr_level; ++L)
            for (int s = ps.levels[p.vrr_level0 + L]; s < ps.levels[p.vrr_level0 + L + 1]; ++s) {
              const VrrInstr &in = ps.vrr[s];
              R t = cf[kPAx + 3 * in.kind + in.dir] * v[in.s0] + cf[kWPx + 3 * in.kind + in.dir] * v[in.s1];
              if (in.n1) t += h[in.kind * p.nh + in.n1] * (v[in.s2] - cf[kRhoZeta + in.kind] * v[in.s3]);
              if (in.n2) t += h[2 * p.nh + in.n2] * v[in.s4];
              v[in.tgt] = t;
            }
          for (int s = p.acc_begin; s < p.acc_begin + p.nacc; ++s) {
            const AccInstr &in = ps.acc[s];
            acc[in.acc] += (in.chan == 0 ? (R)1 : cf[kWA + in.chan - 1]) * v[in.slot];
          }
        }
  R X[2][3];
  for (int x = 0; x < 3; ++x) {
    X[0][x] = A[x] - B[x];
    X[1][x] = C[x] - D[x];
  }
  const std::vector<R> acc0(acc.begin(), acc.begin() + p.acc_total);
  for (int tile = 0; tile < p.ntile; ++tile) {
    const TileProg &T = ps.tiles[p.tile_begin + tile];
    std::copy(acc0.begin(), acc0.end(), acc.begin());
    acc[p.acc_total] = 0;
    for (int L = 0; L < T.nhrr_level; ++L)
      for (int s = ps.levels[T.hrr_level0 + L]; s < ps.levels[T.hrr_level0 + L + 1]; ++s) {
        const HrrInstr &in = ps.hrr[s];
        const R c = in.kind < 2 ? X[in.kind][in.dir] : -(R)in.dir;
        acc[in.tgt] = c * acc[in.s1] + acc[in.s0];
      }
    for (int o = 0; o < T.nout; ++o) out[(size_t)T.store_off + o] = (double)acc[T.out_base + o];
  }
  return 0;
}

template <typename R>
int quartet_t(int la, int lb, int lc, int ld, int deriv, const double *ctr_d, const int *np,
              const double *exps_d, const double *coefs_d, double *out) {
  const ProgramSet &ps = programs();
  if (la < lb || lc < ld) return -1;
  return quartet_pt<R>(ps, ps.progs[quartet_index(la, lb, lc, ld, deriv)], ctr_d, np, exps_d, coefs_d, out);
}

}  // namespace

// Derivative programs of classes with an f shell, which the library does not
// generate (its gradient stops at d): built here one class at a time with the
// library's generator and validated by its checks, then interpreted as above
// in binary64.  *ntile receives the class's tile count (nine (centre,
// direction) tiles, each split over ranges of a's components where it
// would overflow the 16-bit slots).  out as pe_quartet_d with deriv = 1;
// pe_quartet_fderiv_ld runs the same program in long double.
namespace {
template <typename R>
int fderiv_t(int la, int lb, int lc, int ld, const double *ctr, const int *np,
             const double *exps, const double *coefs, double *out, int *ntile) {
  if (la < lb || lc < ld) return -1;
  static std::map<int, std::pair<ProgramSet, ClassProg>> cache;
  const int key = ((la * 4 + lb) * 4 + lc) * 4 + ld;
  auto it = cache.find(key);
  if (it == cache.end()) {
    std::pair<ProgramSet, ClassProg> e;
    try {
      build_one_program(e.first, la, lb, lc, ld, 1, e.second);
      validate_program(e.first, e.second);
    } catch (...) {
      return -2;
    }
    it = cache.emplace(key, std::move(e)).first;
  }
  *ntile = it->second.second.ntile;
  return quartet_pt<R>(it->second.first, it->second.second, ctr, np, exps, coefs, out);
}
}  // namespace

extern "C" int pe_quartet_fderiv(int la, int lb, int lc, int ld, const double *ctr, const int *np,
                                 const double *exps, const double *coefs, double *out, int *ntile) {
  return fderiv_t<double>(la, lb, lc, ld, ctr, np, exps, coefs, out, ntile);
}

extern "C" int pe_quartet_fderiv_ld(int la, int lb, int lc, int ld, const double *ctr, const int *np,
                                    const double *exps, const double *coefs, double *out, int *ntile) {
  return fderiv_t<long double>(la, lb, lc, ld, ctr, np, exps, coefs, out, ntile);
}

extern "C" int pe_quartet_d(int la, int lb, int lc, int ld, int deriv, const double *ctr, const int *np,
                            const double *exps, const double *coefs, double *out) {
  return quartet_t<double>(la, lb, lc, ld, deriv, ctr, np, exps, coefs, out);
}

// The same programs with every step in long double (64-bit significand on
// x86, 113 bits on Arm): the rounding of a class's recurrences falls ~2^-11
// (or more) below binary64's, which separates a wrong program from a badly
// conditioned quartet.
extern "C" int pe_quartet_ld(int la, int lb, int lc, int ld, int deriv, const double *ctr, const int *np,
                             const double *exps, const double *coefs, double *out) {
  return quartet_t<long double>(la, lb, lc, ld, deriv, ctr, np, exps, coefs, out);
}


#ifdef LTJK_GEN_HEADER
// The same quartet through the straight-line source the generator emits for
// the class (tests/codegen_emit.cpp writes LTJK_GEN_HEADER): one call of the
// class's _vrr per primitive quartet, one of its _hrr on the accumulators.
#include LTJK_GEN_HEADER
extern "C" int pe_quartet_gen(int la, int lb, int lc, int ld, const double *ctr, const int *np,
                              const double *exps, const double *coefs, double *out) {
  const GenClass *g = nullptr;
  for (const GenClass &c : kGenClasses)
    if (c.la == la && c.lb == lb && c.lc == lc && c.ld == ld) g = &c;
  if (!g) return -1;
  const ProgramSet &ps = programs();
  const ClassProg &p = ps.progs[quartet_index(la, lb, lc, ld, LTJK_GEN_DERIV)];
  const double *A = ctr, *B = ctr + 3, *C = ctr + 6, *D = ctr + 9;
  int off[5] = {0};
  for (int s = 0; s < 4; ++s) off[s + 1] = off[s] + np[s];
  std::vector<double> acc(p.acc_total, 0.0), base(p.ltot + 1), cf(kNumCoef), h(3 * p.nh);
  for (int i = off[0]; i < off[1]; ++i)
    for (int j = off[1]; j < off[2]; ++j)
      for (int k = off[2]; k < off[3]; ++k)
        for (int l = off[3]; l < off[4]; ++l) {
          setup_primitive(p, A, B, C, D, exps[i], exps[j], exps[k], exps[l],
                          coefs[i] * coefs[j] * coefs[k] * coefs[l], base.data(), cf.data(), h.data());
          g->vrr(base.data(), cf.data(), h.data(), acc.data());
        }
  double X[6];
  for (int x = 0; x < 3; ++x) {
    X[x] = A[x] - B[x];
    X[3 + x] = C[x] - D[x];
  }
  g->hrr(acc.data(), X, out);
  return 0;
}
#endif

extern "C" int pe_quartet(int la, int lb, int lc, int ld, const double *ctr, const int *np,
                          const double *exps, const double *coefs, double *out) {
  return pe_quartet_d(la, lb, lc, ld, 0, ctr, np, exps, coefs, out);
}

// The same quartet with the recurrences in IEEE binary32, in the operation
// order of the integral kernel's single-precision class: base values and
// coefficients computed in binary64 and rounded once to binary32, each
// vertical step as fused multiply-adds (PA v0, + WP v1, + n/2zeta (v2 -
// rho/zeta v3), + n/2(zeta+eta) v4), the accumulation over primitive quartets
// and the horizontal steps as binary32 fused multiply-adds.  Used to measure
// the error of single-precision quartets against the oracle's blocks, from
// which the mixed-precision tolerance is derived.
extern "C" int pe_quartet_f32(int la, int lb, int lc, int ld, int deriv, const double *ctr, const int *np,
                              const double *exps, const double *coefs, double *out) {
  const ProgramSet &ps = programs();
  if (la < lb || lc < ld) return -1;
  const ClassProg &p = ps.progs[quartet_index(la, lb, lc, ld, deriv)];
  const double *A = ctr, *B = ctr + 3, *C = ctr + 6, *D = ctr + 9;
  int off[5] = {0};
  for (int s = 0; s < 4; ++s) off[s + 1] = off[s] + np[s];
  std::vector<float> acc(p.acc_total + p.hrr_size + 1, 0.0f), v(p.vrr_size), cf(kNumCoef), h(3 * p.nh);
  std::vector<double> F(p.ltot + 1);
  for (int i = off[0]; i < off[1]; ++i)
    for (int j = off[1]; j < off[2]; ++j)
      for (int k = off[2]; k < off[3]; ++k)
        for (int l = off[3]; l < off[4]; ++l) {
          const double a = exps[i], b = exps[j], c = exps[k], d = exps[l];
          const double zeta = a + b, eta = c + d, rho = zeta * eta / (zeta + eta);
          double P[3], Q[3], W[3], ab2 = 0, cd2 = 0, pq2 = 0;
          for (int x = 0; x < 3; ++x) {
            P[x] = (a * A[x] + b * B[x]) / zeta;
            Q[x] = (c * C[x] + d * D[x]) / eta;
            W[x] = (zeta * P[x] + eta * Q[x]) / (zeta + eta);
            ab2 += (A[x] - B[x]) * (A[x] - B[x]);
            cd2 += (C[x] - D[x]) * (C[x] - D[x]);
            pq2 += (P[x] - Q[x]) * (P[x] - Q[x]);
          }
          boys(p.ltot, rho * pq2, F.data());
          const double pre = 2.0 * std::pow(M_PI, 2.5) / (zeta * eta * std::sqrt(zeta + eta)) *
                             std::exp(-a * b / zeta * ab2 - c * d / eta * cd2) * coefs[i] * coefs[j] *
                             coefs[k] * coefs[l];
          v[0] = 0.0f;
          for (int m = 0; m <= p.ltot; ++m) v[1 + m] = (float)(pre * F[m]);
          for (int x = 0; x < 3; ++x) {
            cf[kPAx + x] = (float)(P[x] - A[x]);
            cf[kQCx + x] = (float)(Q[x] - C[x]);
            cf[kWPx + x] = (float)(W[x] - P[x]);
            cf[kWQx + x] = (float)(W[x] - Q[x]);
          }
          cf[kRhoZeta] = (float)(rho / zeta);
          cf[kRhoEta] = (float)(rho / eta);
          cf[kWA] = (float)(2.0 * a);
          cf[kWB] = (float)(2.0 * b);
          cf[kWC] = (float)(2.0 * c);
          for (int n = 0; n < p.nh; ++n) {
            h[n] = (float)(0.5 * n / zeta);
            h[p.nh + n] = (float)(0.5 * n / eta);
            h[2 * p.nh + n] = (float)(0.5 * n / (zeta + eta));
          }
          for (int L = 0; L < p.nvrr_level; ++L)
            for (int s = ps.levels[p.vrr_level0 + L]; s < ps.levels[p.vrr_level0 + L + 1]; ++s) {
              const VrrInstr &in = ps.vrr[s];
              float t = cf[kPAx + 3 * in.kind + in.dir] * v[in.s0];
              t = std::fma(cf[kWPx + 3 * in.kind + in.dir], v[in.s1], t);
              if (in.n1) t = std::fma(h[in.kind * p.nh + in.n1], std::fma(-cf[kRhoZeta + in.kind], v[in.s3], v[in.s2]), t);
              if (in.n2) t = std::fma(h[2 * p.nh + in.n2], v[in.s4], t);
              v[in.tgt] = t;
            }
          for (int s = p.acc_begin; s < p.acc_begin + p.nacc; ++s) {
            const AccInstr &in = ps.acc[s];
            acc[in.acc] = std::fma(in.chan == 0 ? 1.0f : cf[kWA + in.chan - 1], v[in.slot], acc[in.acc]);
          }
        }
  float X[2][3];
  for (int x = 0; x < 3; ++x) {
    X[0][x] = (float)(A[x] - B[x]);
    X[1][x] = (float)(C[x] - D[x]);
  }
  const std::vector<float> acc0(acc.begin(), acc.begin() + p.acc_total);
  for (int tile = 0; tile < p.ntile; ++tile) {
    const TileProg &T = ps.tiles[p.tile_begin + tile];
    std::copy(acc0.begin(), acc0.end(), acc.begin());
    acc[p.acc_total] = 0.0f;
    for (int L = 0; L < T.nhrr_level; ++L)
      for (int s = ps.levels[T.hrr_level0 + L]; s < ps.levels[T.hrr_level0 + L + 1]; ++s) {
        const HrrInstr &in = ps.hrr[s];
        const float c = in.kind < 2 ? X[in.kind][in.dir] : -float(in.dir);
        acc[in.tgt] = std::fma(c, acc[in.s1], acc[in.s0]);
      }
    for (int o = 0; o < T.nout; ++o) out[(size_t)T.store_off + o] = acc[T.out_base + o];
  }
  return 0;
}
