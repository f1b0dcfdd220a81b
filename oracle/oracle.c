/*
 * oracle.c -- plain, slow FP64 CPU oracle for the AO-direct J/K build of the
 * Laplace-transform method and for its nuclear-gradient adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this file.  The
 * product path (the CUDA library) never does, and this file shares no code,
 * header, table or helper with it.
 *
 * What it computes, each written out from its definition:
 *   - Cartesian contracted Gaussian basis functions with the normalisation
 *     convention of the library (primitive normalised for the x^l component,
 *     contracted x^l function renormalised to unit self-overlap).
 *   - Electron-repulsion integrals (mu nu|kappa rho) in chemist notation
 *     (paper, "Notation and conventions") by the McMurchie-Davidson Hermite
 *     scheme: Hermite expansion coefficients E^{ij}_t of each Gaussian product
 *     and Hermite Coulomb integrals R^n_{tuv} built from Boys values.  This is a
 *     different integral scheme from the Obara-Saika/Head-Gordon-Pople
 *     recurrence of the CUDA kernels.
 *   - The Boys function F_m(T) from its power series (T < 30) or from
 *     erf with upward recursion (T >= 30), in long double.
 *   - Schwarz factors Q_ab = max sqrt|(mu nu|mu nu)|, mu in a, nu in b.
 *   - J[D]_{mu nu} = sum (mu nu|kappa rho) D_{kappa rho} and
 *     K[D]_{mu nu} = sum (mu kappa|nu rho) D_{kappa rho} for non-symmetric D
 *     (Eq. jkbuild), by visiting every AO-canonical integral once and applying
 *     each of its distinct index permutations explicitly (no degeneracy
 *     weights).
 *   - The gradient of E = sum_r [cJ J(P_r,Q_r) + cK K(P_r,Q_r)] with
 *     J(A,B) = sum (mu nu|kappa rho) A_{mu nu} B_{kappa rho} and
 *     K(A,B) = sum (mu kappa|nu rho) A_{mu nu} B_{kappa rho} (Eq. jkderiv):
 *     derivative integrals of all four centres explicitly, from the
 *     Gaussian derivative rule d/dA_x g = 2 alpha g(l_x+1) - l_x g(l_x-1).
 *
 * Parity pins (tests/test_oracle_*.py): closed-form (ss|ss) and the 1/R limit,
 * brute-force numerical quadrature of single integrals, 8-fold symmetry,
 * Cauchy-Schwarz, J/K identities, finite differences of the energy and
 * translational invariance of the gradient.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LMAX 4              /* largest shell angular momentum handled  */
#define ORC_LMAX_D (ORC_LMAX + 1) /* after one derivative raise              */
#define ORC_LTOT (4 * ORC_LMAX_D)
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
  int natoms;
  const double *coords;   /* [natoms][3] bohr */
  int nshells;
  const int *sh_atom;     /* [nshells] */
  const int *sh_l;        /* [nshells] */
  const int *sh_nprim;    /* [nshells] */
  const double *exps;     /* concatenated primitive exponents */
  const double *coefs;    /* concatenated raw contraction coefficients */
} orc_basis;

/* Derived bookkeeping (computed once per call). */
typedef struct {
  const orc_basis *b;
  int nao;
  int *ao0;       /* first AO of each shell */
  int *p0;        /* first primitive of each shell */
  double *ncoef;  /* normalised coefficient of each primitive */
} orc_ctx;

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* Component order within a shell: lexicographic, descending l_x, then l_y. */
static void cart_list(int l, int (*c)[3]) {
  int n = 0;
  for (int lx = l; lx >= 0; --lx)
    for (int ly = l - lx; ly >= 0; --ly) {
      c[n][0] = lx; c[n][1] = ly; c[n][2] = l - lx - ly; ++n;
    }
}
static int cart_index(int lx, int ly, int lz) {
  int l = lx + ly + lz;
  return (l - lx) * (l - lx + 1) / 2 + lz;
}

static double dfact(int n) { /* n!! with (-1)!! = 1 */
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

/* ---------------------------------------------------------------- Boys */
/* F_m(T) = int_0^1 u^{2m} exp(-T u^2) du, m = 0..mmax. */
void orc_boys(int mmax, double Td, double *out) {
  long double T = Td;
  if (Td < 30.0) {
    /* Series for the top order, F_m(T) = e^{-T} sum_k (2T)^k / prod_{j=0..k}(2m+2j+1),
       then the exact downward relation F_m = (2T F_{m+1} + e^{-T}) / (2m+1). */
    long double term = 1.0L / (2 * mmax + 1), sum = term;
    for (int k = 1; k < 400; ++k) {
      term *= 2.0L * T / (2 * mmax + 2 * k + 1);
      sum += term;
      if (term < 1e-22L * sum) break;
    }
    long double emt = expl(-T);
    long double f = emt * sum;
    out[mmax] = (double)f;
    for (int m = mmax - 1; m >= 0; --m) {
      f = (2.0L * T * f + emt) / (2 * m + 1);
      out[m] = (double)f;
    }
  } else {
    /* F_0 = (1/2) sqrt(pi/T) erf(sqrt T); upward F_{m+1} = ((2m+1)F_m - e^{-T}) / (2T). */
    long double emt = expl(-T);
    long double f = 0.5L * sqrtl(3.14159265358979323846264338327950288L / T) * erfl(sqrtl(T));
    out[0] = (double)f;
    for (int m = 0; m < mmax; ++m) {
      f = ((2 * m + 1) * f - emt) / (2.0L * T);
      out[m + 1] = (double)f;
    }
  }
}

/* ------------------------------------------------- McMurchie-Davidson */
/* Hermite expansion coefficients of the 1D product (x-A)^i e^{-a(x-A)^2} (x-B)^j e^{-b(x-B)^2}
   = sum_t E[i][j][t] Lambda_t(x; p, P):
     E^{00}_0 = exp(-ab/p XAB^2),
     E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + XPA E^{ij}_t + (t+1) E^{ij}_{t+1},
     E^{i,j+1}_t = E^{ij}_{t-1}/(2p) + XPB E^{ij}_t + (t+1) E^{ij}_{t+1}. */
#define EDIM (ORC_LMAX_D + 1)
#define ETDIM (2 * ORC_LMAX_D + 1)
static void hermite_E(int imax, int jmax, double a, double b, double XAB,
                      double E[EDIM][EDIM][ETDIM]) {
  double p = a + b;
  double XPA = -b / p * XAB, XPB = a / p * XAB;
  memset(E, 0, sizeof(double) * EDIM * EDIM * ETDIM);
  E[0][0][0] = exp(-a * b / p * XAB * XAB);
  for (int i = 0; i <= imax; ++i) {
    for (int j = 0; j <= jmax; ++j) {
      if (i == 0 && j == 0) continue;
      if (j == 0) { /* raise i from (i-1, 0) */
        for (int t = 0; t <= i + j; ++t) {
          double v = XPA * E[i - 1][j][t];
          if (t > 0) v += E[i - 1][j][t - 1] / (2 * p);
          if (t + 1 <= i - 1 + j) v += (t + 1) * E[i - 1][j][t + 1];
          E[i][j][t] = v;
        }
      } else { /* raise j from (i, j-1) */
        for (int t = 0; t <= i + j; ++t) {
          double v = XPB * E[i][j - 1][t];
          if (t > 0) v += E[i][j - 1][t - 1] / (2 * p);
          if (t + 1 <= i + j - 1) v += (t + 1) * E[i][j - 1][t + 1];
          E[i][j][t] = v;
        }
      }
    }
  }
}

/* Hermite Coulomb integrals R_{tuv} = R^0_{tuv}(alpha, PQ), t+u+v <= L, stored in a
   (L+1)^3 cube R[(t*(L+1)+u)*(L+1)+v]:
     R^n_{000} = (-2 alpha)^n F_n(alpha |PQ|^2),
     R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X_PQ R^{n+1}_{t,u,v}  (same for u, v). */
static void hermite_R(int L, double alpha, const double PQ[3], double *R, double *work) {
  const int D = L + 1;
  double F[ORC_LTOT + 2];
  double T = alpha * (PQ[0] * PQ[0] + PQ[1] * PQ[1] + PQ[2] * PQ[2]);
  orc_boys(L, T, F);
  double *prev = R, *cur = work;
  if (L % 2 == 0) { prev = work; cur = R; } /* so that the n = 0 level lands in R */
  for (int n = L; n >= 0; --n) {
    int top = L - n;
    cur[0] = pow(-2.0 * alpha, n) * F[n];
    for (int t = 0; t <= top; ++t)
      for (int u = 0; u <= top - t; ++u)
        for (int v = 0; v <= top - t - u; ++v) {
          if (t == 0 && u == 0 && v == 0) continue;
          double val;
          if (t > 0) {
            val = PQ[0] * prev[((t - 1) * D + u) * D + v];
            if (t > 1) val += (t - 1) * prev[((t - 2) * D + u) * D + v];
          } else if (u > 0) {
            val = PQ[1] * prev[(t * D + u - 1) * D + v];
            if (u > 1) val += (u - 1) * prev[(t * D + u - 2) * D + v];
          } else {
            val = PQ[2] * prev[(t * D + u) * D + v - 1];
            if (v > 1) val += (v - 1) * prev[(t * D + u) * D + v - 2];
          }
          cur[(t * D + u) * D + v] = val;
        }
    double *tmp = prev; prev = cur; cur = tmp;
  }
}

/* Primitive Cartesian integral block over the unnormalised primitives
   (x-A_x)^{ax}.. e^{-a|r-A|^2} etc., out[((i*nb + j)*nc + k)*nd + l]. */
void orc_eri_prim(int la, int lb, int lc, int ld, double a, double b, double c, double d,
                  const double *A, const double *B, const double *C, const double *Dc,
                  double *out) {
  int ca[64][3], cb[64][3], cc[64][3], cd[64][3];
  cart_list(la, ca); cart_list(lb, cb); cart_list(lc, cc); cart_list(ld, cd);
  int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
  double p = a + b, q = c + d, alpha = p * q / (p + q);
  double P[3], Q[3], PQ[3];
  double Eab[3][EDIM][EDIM][ETDIM], Ecd[3][EDIM][EDIM][ETDIM];
  for (int x = 0; x < 3; ++x) {
    P[x] = (a * A[x] + b * B[x]) / p;
    Q[x] = (c * C[x] + d * Dc[x]) / q;
    PQ[x] = P[x] - Q[x];
    hermite_E(la, lb, a, b, A[x] - B[x], Eab[x]);
    hermite_E(lc, ld, c, d, C[x] - Dc[x], Ecd[x]);
  }
  int L = la + lb + lc + ld;
  const int RD = L + 1;
  double *R = malloc(sizeof(double) * 2 * RD * RD * RD);
  hermite_R(L, alpha, PQ, R, R + RD * RD * RD);
  double pref = 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q));
  int Lab = la + lb;
  /* H[k][l][t][u][v] = sum_{tau nu phi} (-1)^{tau+nu+phi} E^{cd} R_{t+tau,u+nu,v+phi} */
  int nhab = (Lab + 1) * (Lab + 1) * (Lab + 1);
  double *H = malloc(sizeof(double) * nc * nd * nhab);
  for (int k = 0; k < nc; ++k)
    for (int l = 0; l < nd; ++l) {
      const int *ck = cc[k], *cl = cd[l];
      for (int t = 0; t <= Lab; ++t)
        for (int u = 0; u <= Lab - t; ++u)
          for (int v = 0; v <= Lab - t - u; ++v) {
            double s = 0.0;
            for (int tau = 0; tau <= ck[0] + cl[0]; ++tau)
              for (int nu = 0; nu <= ck[1] + cl[1]; ++nu)
                for (int phi = 0; phi <= ck[2] + cl[2]; ++phi) {
                  double e = Ecd[0][ck[0]][cl[0]][tau] * Ecd[1][ck[1]][cl[1]][nu] *
                             Ecd[2][ck[2]][cl[2]][phi];
                  double sign = ((tau + nu + phi) & 1) ? -1.0 : 1.0;
                  s += sign * e * R[((t + tau) * RD + (u + nu)) * RD + (v + phi)];
                }
            H[((k * nd + l) * (Lab + 1) + t) * (Lab + 1) * (Lab + 1) + u * (Lab + 1) + v] = s;
          }
    }
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j) {
      const int *ci = ca[i], *cj = cb[j];
      for (int k = 0; k < nc; ++k)
        for (int l = 0; l < nd; ++l) {
          double s = 0.0;
          for (int t = 0; t <= ci[0] + cj[0]; ++t)
            for (int u = 0; u <= ci[1] + cj[1]; ++u)
              for (int v = 0; v <= ci[2] + cj[2]; ++v) {
                double e = Eab[0][ci[0]][cj[0]][t] * Eab[1][ci[1]][cj[1]][u] *
                           Eab[2][ci[2]][cj[2]][v];
                s += e * H[((k * nd + l) * (Lab + 1) + t) * (Lab + 1) * (Lab + 1) + u * (Lab + 1) + v];
              }
          out[((i * nb + j) * nc + k) * nd + l] = pref * s;
        }
    }
  free(H); free(R);
}

/* --------------------------------------------------------------- basis */
/* Normalised contraction coefficients: primitive factor
   N(alpha,l) = (2 alpha/pi)^{3/4} (4 alpha)^{l/2} / sqrt((2l-1)!!)
   times the raw coefficient, then the whole x^l function scaled to unit
   self-overlap, S = sum_kl c_k c_l N_k N_l (pi/(a_k+a_l))^{3/2} (2l-1)!!/(2(a_k+a_l))^l. */
void orc_norm_coefs(int nshells, const int *sh_l, const int *sh_nprim, const double *exps,
                    const double *coefs, double *out) {
  int p0 = 0;
  for (int s = 0; s < nshells; ++s) {
    int l = sh_l[s], np = sh_nprim[s];
    for (int k = 0; k < np; ++k) {
      double a = exps[p0 + k];
      out[p0 + k] = coefs[p0 + k] * pow(2.0 * a / M_PI, 0.75) * pow(4.0 * a, 0.5 * l) /
                    sqrt(dfact(2 * l - 1));
    }
    double S = 0.0;
    for (int k = 0; k < np; ++k)
      for (int m = 0; m < np; ++m) {
        double g = exps[p0 + k] + exps[p0 + m];
        S += out[p0 + k] * out[p0 + m] * pow(M_PI / g, 1.5) * dfact(2 * l - 1) / pow(2.0 * g, l);
      }
    double f = 1.0 / sqrt(S);
    for (int k = 0; k < np; ++k) out[p0 + k] *= f;
    p0 += np;
  }
}

static void ctx_init(orc_ctx *c, const orc_basis *b) {
  c->b = b;
  c->ao0 = malloc(sizeof(int) * (b->nshells + 1));
  c->p0 = malloc(sizeof(int) * (b->nshells + 1));
  int nao = 0, np = 0;
  for (int s = 0; s < b->nshells; ++s) {
    c->ao0[s] = nao; c->p0[s] = np;
    nao += ncart(b->sh_l[s]); np += b->sh_nprim[s];
  }
  c->ao0[b->nshells] = nao; c->p0[b->nshells] = np;
  c->nao = nao;
  c->ncoef = malloc(sizeof(double) * np);
  orc_norm_coefs(b->nshells, b->sh_l, b->sh_nprim, b->exps, b->coefs, c->ncoef);
}
static void ctx_free(orc_ctx *c) { free(c->ao0); free(c->p0); free(c->ncoef); }

int orc_nao(const orc_basis *b) {
  int n = 0;
  for (int s = 0; s < b->nshells; ++s) n += ncart(b->sh_l[s]);
  return n;
}

static const double *shell_center(const orc_ctx *c, int s) {
  return c->b->coords + 3 * c->b->sh_atom[s];
}

/* Contracted block (ab|cd) with angular momenta given explicitly, out sized for them. */
static void contracted_block(const orc_ctx *c, int sa, int sb, int sc, int sd, double *out,
                             double *scratch) {
  const orc_basis *b = c->b;
  int la = b->sh_l[sa], lb = b->sh_l[sb], lc = b->sh_l[sc], ld = b->sh_l[sd];
  int n = ncart(la) * ncart(lb) * ncart(lc) * ncart(ld);
  memset(out, 0, sizeof(double) * n);
  const double *A = shell_center(c, sa), *B = shell_center(c, sb), *C = shell_center(c, sc),
               *D = shell_center(c, sd);
  for (int i = 0; i < b->sh_nprim[sa]; ++i)
    for (int j = 0; j < b->sh_nprim[sb]; ++j)
      for (int k = 0; k < b->sh_nprim[sc]; ++k)
        for (int l = 0; l < b->sh_nprim[sd]; ++l) {
          int pi = c->p0[sa] + i, pj = c->p0[sb] + j, pk = c->p0[sc] + k, pl = c->p0[sd] + l;
          orc_eri_prim(la, lb, lc, ld, b->exps[pi], b->exps[pj], b->exps[pk], b->exps[pl], A, B,
                       C, D, scratch);
          double w = c->ncoef[pi] * c->ncoef[pj] * c->ncoef[pk] * c->ncoef[pl];
          for (int t = 0; t < n; ++t) out[t] += w * scratch[t];
        }
}

#define MAXBLK (15 * 15 * 15 * 15)

/* Public: contracted block of one shell quartet, out[((i*nb+j)*nc+k)*nd+l]. */
void orc_shell_quartet(const orc_basis *b, int sa, int sb, int sc, int sd, double *out) {
  orc_ctx c; ctx_init(&c, b);
  double *scr = malloc(sizeof(double) * MAXBLK);
  contracted_block(&c, sa, sb, sc, sd, out, scr);
  free(scr); ctx_free(&c);
}

/* Full AO tensor out[((mu*N+nu)*N+ka)*N+rho] (small bases only). Every ordered
   shell quartet is evaluated directly; no permutational symmetry is used. */
void orc_eri_tensor(const orc_basis *b, double *out) {
  orc_ctx c; ctx_init(&c, b);
  int N = c.nao, ns = b->nshells;
#pragma omp parallel
  {
    double *blk = malloc(sizeof(double) * MAXBLK), *scr = malloc(sizeof(double) * MAXBLK);
#pragma omp for schedule(dynamic)
    for (int sa = 0; sa < ns; ++sa)
      for (int sb = 0; sb < ns; ++sb)
        for (int sc = 0; sc < ns; ++sc)
          for (int sd = 0; sd < ns; ++sd) {
            contracted_block(&c, sa, sb, sc, sd, blk, scr);
            int na = ncart(b->sh_l[sa]), nb = ncart(b->sh_l[sb]), nc = ncart(b->sh_l[sc]),
                nd = ncart(b->sh_l[sd]);
            for (int i = 0; i < na; ++i)
              for (int j = 0; j < nb; ++j)
                for (int k = 0; k < nc; ++k)
                  for (int l = 0; l < nd; ++l) {
                    size_t mu = c.ao0[sa] + i, nu = c.ao0[sb] + j, ka = c.ao0[sc] + k,
                           rho = c.ao0[sd] + l;
                    out[((mu * N + nu) * N + ka) * N + rho] = blk[((i * nb + j) * nc + k) * nd + l];
                  }
          }
    free(blk); free(scr);
  }
  ctx_free(&c);
}

/* Schwarz factors Q[sa*ns+sb] = max_{mu in a, nu in b} sqrt|(mu nu|mu nu)| for all ordered pairs. */
void orc_schwarz(const orc_basis *b, double *Q) {
  orc_ctx c; ctx_init(&c, b);
  int ns = b->nshells;
#pragma omp parallel
  {
    double *blk = malloc(sizeof(double) * MAXBLK), *scr = malloc(sizeof(double) * MAXBLK);
#pragma omp for schedule(dynamic)
    for (int sa = 0; sa < ns; ++sa)
      for (int sb = 0; sb < ns; ++sb) {
        contracted_block(&c, sa, sb, sa, sb, blk, scr);
        int na = ncart(b->sh_l[sa]), nb = ncart(b->sh_l[sb]);
        double m = 0.0;
        for (int i = 0; i < na; ++i)
          for (int j = 0; j < nb; ++j) {
            double v = fabs(blk[((i * nb + j) * na + i) * nb + j]);
            if (v > m) m = v;
          }
        Q[sa * ns + sb] = sqrt(m);
      }
    free(blk); free(scr);
  }
  ctx_free(&c);
}

/* Distinct index permutations of one integral (mu nu|ka rho): the images under
   mu<->nu, ka<->rho and (mu nu)<->(ka rho), duplicates removed. */
static int distinct_images(int mu, int nu, int ka, int rho, int img[8][4]) {
  int cand[8][4] = {{mu, nu, ka, rho}, {nu, mu, ka, rho}, {mu, nu, rho, ka}, {nu, mu, rho, ka},
                    {ka, rho, mu, nu}, {rho, ka, mu, nu}, {ka, rho, nu, mu}, {rho, ka, nu, mu}};
  int n = 0;
  for (int t = 0; t < 8; ++t) {
    int dup = 0;
    for (int s = 0; s < n && !dup; ++s)
      dup = img[s][0] == cand[t][0] && img[s][1] == cand[t][1] && img[s][2] == cand[t][2] &&
            img[s][3] == cand[t][3];
    if (!dup) { memcpy(img[n], cand[t], sizeof(int) * 4); ++n; }
  }
  return n;
}

/* J[q][mu][nu] = sum (mu nu|ka rho) D[q][ka][rho], K[q][mu][nu] = sum (mu ka|nu rho) D[q][ka][rho]
   over all AO indices (Eq. jkbuild).  Integrals are visited once each in canonical
   form: mu>=nu, ka>=rho, and the bra shell pair ranked at or above the ket shell pair,
   ties (the same shell pair) broken by mu*(mu+1)/2+nu >= ka*(ka+1)/2+rho.  Every
   distinct permuted image of a visited integral is then applied explicitly.  Shell quartets whose
   Schwarz product Q_ab Q_cd is below tau are skipped (tau <= 0: none). */
void orc_jk(const orc_basis *b, int nd, const double *D, double tau, double *J, double *K) {
  orc_ctx c; ctx_init(&c, b);
  int N = c.nao, ns = b->nshells;
  size_t NN = (size_t)N * N;
  double *Q = malloc(sizeof(double) * ns * ns);
  if (tau > 0) orc_schwarz(b, Q);
  memset(J, 0, sizeof(double) * nd * NN);
  memset(K, 0, sizeof(double) * nd * NN);
  int npair = ns * (ns + 1) / 2;
  int *pa = malloc(sizeof(int) * npair), *pb = malloc(sizeof(int) * npair);
  for (int a = 0, t = 0; a < ns; ++a)
    for (int bb = 0; bb <= a; ++bb, ++t) { pa[t] = a; pb[t] = bb; }
#pragma omp parallel
  {
    double *Jt = calloc(nd * NN, sizeof(double)), *Kt = calloc(nd * NN, sizeof(double));
    double *blk = malloc(sizeof(double) * MAXBLK), *scr = malloc(sizeof(double) * MAXBLK);
#pragma omp for schedule(dynamic)
    for (int P = 0; P < npair; ++P)
      for (int Qp = 0; Qp <= P; ++Qp) {
        int sa = pa[P], sb = pb[P], sc = pa[Qp], sd = pb[Qp];
        if (tau > 0 && Q[sa * ns + sb] * Q[sc * ns + sd] < tau) continue;
        contracted_block(&c, sa, sb, sc, sd, blk, scr);
        int na = ncart(b->sh_l[sa]), nb = ncart(b->sh_l[sb]), nc = ncart(b->sh_l[sc]),
            ndd = ncart(b->sh_l[sd]);
        for (int i = 0; i < na; ++i)
          for (int j = 0; j < nb; ++j)
            for (int k = 0; k < nc; ++k)
              for (int l = 0; l < ndd; ++l) {
                int mu = c.ao0[sa] + i, nu = c.ao0[sb] + j, ka = c.ao0[sc] + k, rho = c.ao0[sd] + l;
                if (mu < nu || ka < rho) continue;
                if (P == Qp && mu * (mu + 1) / 2 + nu < ka * (ka + 1) / 2 + rho) continue;
                double v = blk[((i * nb + j) * nc + k) * ndd + l];
                int img[8][4];
                int nimg = distinct_images(mu, nu, ka, rho, img);
                for (int s = 0; s < nimg; ++s) {
                  int p = img[s][0], qq = img[s][1], r = img[s][2], u = img[s][3];
                  /* image (p q|r u): J[p][q] += v D[r][u];  K[p][r] += v D[q][u] */
                  for (int d = 0; d < nd; ++d) {
                    Jt[d * NN + (size_t)p * N + qq] += v * D[d * NN + (size_t)r * N + u];
                    Kt[d * NN + (size_t)p * N + r] += v * D[d * NN + (size_t)qq * N + u];
                  }
                }
              }
      }
#pragma omp critical
    {
      for (size_t t = 0; t < nd * NN; ++t) { J[t] += Jt[t]; K[t] += Kt[t]; }
    }
    free(Jt); free(Kt); free(blk); free(scr);
  }
  free(pa); free(pb); free(Q);
  ctx_free(&c);
}

/* Sampled blocks straight from the definition, for full-size parity checks:
   Jblk[q][i][j] = J[q][mu][nu] for mu in shell sa, nu in shell sb, summing over every
   ordered ket shell pair (c,d);  Kblk[q][i][k] = K[q][mu][nu] for mu in sa, nu in sc,
   summing over every ordered pair of shells (b,d) in (mu b|nu d).  Schwarz rule as in orc_jk. */
void orc_j_block(const orc_basis *b, int nd, const double *D, double tau, int sa, int sb,
                 double *Jblk) {
  orc_ctx c; ctx_init(&c, b);
  int N = c.nao, ns = b->nshells;
  size_t NN = (size_t)N * N;
  double *Q = malloc(sizeof(double) * ns * ns);
  if (tau > 0) orc_schwarz(b, Q);
  int na = ncart(b->sh_l[sa]), nb = ncart(b->sh_l[sb]);
  memset(Jblk, 0, sizeof(double) * nd * na * nb);
#pragma omp parallel
  {
    double *acc = calloc(nd * na * nb, sizeof(double));
    double *blk = malloc(sizeof(double) * MAXBLK), *scr = malloc(sizeof(double) * MAXBLK);
#pragma omp for schedule(dynamic)
    for (int sc = 0; sc < ns; ++sc)
      for (int sd = 0; sd < ns; ++sd) {
        if (tau > 0 && Q[sa * ns + sb] * Q[sc * ns + sd] < tau) continue;
        contracted_block(&c, sa, sb, sc, sd, blk, scr);
        int nc = ncart(b->sh_l[sc]), ndd = ncart(b->sh_l[sd]);
        for (int i = 0; i < na; ++i)
          for (int j = 0; j < nb; ++j)
            for (int k = 0; k < nc; ++k)
              for (int l = 0; l < ndd; ++l) {
                double v = blk[((i * nb + j) * nc + k) * ndd + l];
                size_t kr = (size_t)(c.ao0[sc] + k) * N + c.ao0[sd] + l;
                for (int d = 0; d < nd; ++d) acc[(d * na + i) * nb + j] += v * D[d * NN + kr];
              }
      }
#pragma omp critical
    for (int t = 0; t < nd * na * nb; ++t) Jblk[t] += acc[t];
    free(acc); free(blk); free(scr);
  }
  free(Q); ctx_free(&c);
}

void orc_k_block(const orc_basis *b, int nd, const double *D, double tau, int sa, int sc,
                 double *Kblk) {
  orc_ctx c; ctx_init(&c, b);
  int N = c.nao, ns = b->nshells;
  size_t NN = (size_t)N * N;
  double *Q = malloc(sizeof(double) * ns * ns);
  if (tau > 0) orc_schwarz(b, Q);
  int na = ncart(b->sh_l[sa]), nc = ncart(b->sh_l[sc]);
  memset(Kblk, 0, sizeof(double) * nd * na * nc);
#pragma omp parallel
  {
    double *acc = calloc(nd * na * nc, sizeof(double));
    double *blk = malloc(sizeof(double) * MAXBLK), *scr = malloc(sizeof(double) * MAXBLK);
#pragma omp for schedule(dynamic)
    for (int sb = 0; sb < ns; ++sb)
      for (int sd = 0; sd < ns; ++sd) {
        if (tau > 0 && Q[sa * ns + sb] * Q[sc * ns + sd] < tau) continue;
        contracted_block(&c, sa, sb, sc, sd, blk, scr); /* (mu ka|nu rho), mu in a, nu in c */
        int nb = ncart(b->sh_l[sb]), ndd = ncart(b->sh_l[sd]);
        for (int i = 0; i < na; ++i)
          for (int j = 0; j < nb; ++j)
            for (int k = 0; k < nc; ++k)
              for (int l = 0; l < ndd; ++l) {
                double v = blk[((i * nb + j) * nc + k) * ndd + l];
                size_t kr = (size_t)(c.ao0[sb] + j) * N + c.ao0[sd] + l;
                for (int d = 0; d < nd; ++d) acc[(d * na + i) * nc + k] += v * D[d * NN + kr];
              }
      }
#pragma omp critical
    for (int t = 0; t < nd * na * nc; ++t) Kblk[t] += acc[t];
    free(acc); free(blk); free(scr);
  }
  free(Q); ctx_free(&c);
}

/* ------------------------------------------------------------ gradient */
/* Derivative of the contracted block (ab|cd) with respect to the three Cartesian
   coordinates of the centre of shell position `which` (0..3), each centre treated
   explicitly: for primitive g of exponent e and component (lx,ly,lz),
   d g / d X_x = 2 e g(lx+1) - lx g(lx-1).  out[x][n] for x = 0,1,2. */
static void deriv_block(const orc_ctx *c, const int sh[4], int which, double *out, double *up,
                        double *dn) {
  const orc_basis *b = c->b;
  int L[4], nL[4];
  for (int t = 0; t < 4; ++t) { L[t] = b->sh_l[sh[t]]; nL[t] = ncart(L[t]); }
  int n = nL[0] * nL[1] * nL[2] * nL[3];
  memset(out, 0, sizeof(double) * 3 * n);
  const double *X[4];
  for (int t = 0; t < 4; ++t) X[t] = shell_center(c, sh[t]);
  int Lu[4], Ld[4];
  for (int t = 0; t < 4; ++t) { Lu[t] = L[t]; Ld[t] = L[t]; }
  Lu[which] += 1; Ld[which] -= 1;
  int nu_[4], nd_[4];
  for (int t = 0; t < 4; ++t) { nu_[t] = ncart(Lu[t]); nd_[t] = Ld[t] >= 0 ? ncart(Ld[t]) : 0; }
  int cmp[4][64][3];
  for (int t = 0; t < 4; ++t) cart_list(L[t], cmp[t]);
  for (int i = 0; i < b->sh_nprim[sh[0]]; ++i)
    for (int j = 0; j < b->sh_nprim[sh[1]]; ++j)
      for (int k = 0; k < b->sh_nprim[sh[2]]; ++k)
        for (int l = 0; l < b->sh_nprim[sh[3]]; ++l) {
          int pidx[4] = {c->p0[sh[0]] + i, c->p0[sh[1]] + j, c->p0[sh[2]] + k, c->p0[sh[3]] + l};
          double e[4];
          for (int t = 0; t < 4; ++t) e[t] = b->exps[pidx[t]];
          double w = c->ncoef[pidx[0]] * c->ncoef[pidx[1]] * c->ncoef[pidx[2]] * c->ncoef[pidx[3]];
          orc_eri_prim(Lu[0], Lu[1], Lu[2], Lu[3], e[0], e[1], e[2], e[3], X[0], X[1], X[2], X[3],
                       up);
          if (Ld[which] >= 0)
            orc_eri_prim(Ld[0], Ld[1], Ld[2], Ld[3], e[0], e[1], e[2], e[3], X[0], X[1], X[2],
                         X[3], dn);
          for (int a0 = 0; a0 < nL[0]; ++a0)
            for (int a1 = 0; a1 < nL[1]; ++a1)
              for (int a2 = 0; a2 < nL[2]; ++a2)
                for (int a3 = 0; a3 < nL[3]; ++a3) {
                  int comp[4] = {a0, a1, a2, a3};
                  int oi = ((a0 * nL[1] + a1) * nL[2] + a2) * nL[3] + a3;
                  for (int x = 0; x < 3; ++x) {
                    int idx_u[4], idx_d[4], ok_d = 1;
                    for (int t = 0; t < 4; ++t) {
                      int lx = cmp[t][comp[t]][0], ly = cmp[t][comp[t]][1], lz = cmp[t][comp[t]][2];
                      if (t == which) {
                        int r[3] = {lx, ly, lz};
                        r[x] += 1;
                        idx_u[t] = cart_index(r[0], r[1], r[2]);
                        r[x] -= 2;
                        if (r[x] < 0) ok_d = 0; else idx_d[t] = cart_index(r[0], r[1], r[2]);
                      } else {
                        idx_u[t] = comp[t]; idx_d[t] = comp[t];
                      }
                    }
                    int ui = ((idx_u[0] * nu_[1] + idx_u[1]) * nu_[2] + idx_u[2]) * nu_[3] + idx_u[3];
                    double v = 2.0 * e[which] * up[ui];
                    if (ok_d) {
                      int lcomp = cmp[which][comp[which]][x];
                      int di = ((idx_d[0] * nd_[1] + idx_d[1]) * nd_[2] + idx_d[2]) * nd_[3] + idx_d[3];
                      v -= lcomp * dn[di];
                    }
                    out[x * n + oi] += w * v;
                  }
                }
        }
}

/* grad[atom][x] = d/dR_{atom,x} sum_r [cJ J(P_r,Q_r) + cK K(P_r,Q_r)]
   = sum over every ordered AO quadruple of (mu nu|ka rho)^x G_{mu nu ka rho},
   G = sum_r [cJ P_r[mu][nu] Q_r[ka][rho] + cK P_r[mu][ka] Q_r[nu][rho]].
   Every ordered shell quartet is visited; each of the four centres is differentiated.
   If atom_filter >= 0, only quartets with a shell on that atom are visited and only
   that atom's row of grad is complete (the others are partial). */
void orc_grad(const orc_basis *b, int nterms, const double *P, const double *Qd, double cJ,
              double cK, int atom_filter, double *grad) {
  orc_ctx c; ctx_init(&c, b);
  int N = c.nao, ns = b->nshells;
  size_t NN = (size_t)N * N;
  memset(grad, 0, sizeof(double) * 3 * b->natoms);
  int MAXB = 21 * 21 * 21 * 21; /* raised-shell blocks (up to g on one index) */
#pragma omp parallel
  {
    double *g = calloc(3 * b->natoms, sizeof(double));
    double *dblk = malloc(sizeof(double) * 3 * MAXBLK);
    double *up = malloc(sizeof(double) * MAXB), *dn = malloc(sizeof(double) * MAXB);
    double *G = malloc(sizeof(double) * MAXBLK);
#pragma omp for schedule(dynamic) collapse(2)
    for (int sa = 0; sa < ns; ++sa)
      for (int sb = 0; sb < ns; ++sb)
        for (int sc = 0; sc < ns; ++sc)
          for (int sd = 0; sd < ns; ++sd) {
            int sh[4] = {sa, sb, sc, sd};
            if (atom_filter >= 0) {
              int hit = 0;
              for (int t = 0; t < 4; ++t) hit |= b->sh_atom[sh[t]] == atom_filter;
              if (!hit) continue;
            }
            int nL[4];
            for (int t = 0; t < 4; ++t) nL[t] = ncart(b->sh_l[sh[t]]);
            int n = nL[0] * nL[1] * nL[2] * nL[3];
            for (int i = 0; i < nL[0]; ++i)
              for (int j = 0; j < nL[1]; ++j)
                for (int k = 0; k < nL[2]; ++k)
                  for (int l = 0; l < nL[3]; ++l) {
                    size_t mu = c.ao0[sa] + i, nu = c.ao0[sb] + j, ka = c.ao0[sc] + k,
                           rho = c.ao0[sd] + l;
                    double s = 0.0;
                    for (int r = 0; r < nterms; ++r) {
                      s += cJ * P[r * NN + mu * N + nu] * Qd[r * NN + ka * N + rho];
                      s += cK * P[r * NN + mu * N + ka] * Qd[r * NN + nu * N + rho];
                    }
                    G[((i * nL[1] + j) * nL[2] + k) * nL[3] + l] = s;
                  }
            for (int w = 0; w < 4; ++w) {
              int atom = b->sh_atom[sh[w]];
              if (atom_filter >= 0 && atom != atom_filter) continue;
              deriv_block(&c, sh, w, dblk, up, dn);
              for (int x = 0; x < 3; ++x) {
                double s = 0.0;
                for (int t = 0; t < n; ++t) s += dblk[x * n + t] * G[t];
                g[3 * atom + x] += s;
              }
            }
          }
#pragma omp critical
    for (int t = 0; t < 3 * b->natoms; ++t) grad[t] += g[t];
    free(g); free(dblk); free(up); free(dn); free(G);
  }
  ctx_free(&c);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
