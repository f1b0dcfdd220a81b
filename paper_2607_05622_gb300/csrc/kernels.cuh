// Device code: Boys function, the warp-cooperative recurrence interpreter for
// contracted shell quartets, and the fused J/K digestion and gradient
// contraction.  Included by context.cu only.
#pragma once
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "ltjk_internal.h"

namespace ltjk {

// ------------------------------------------------------------------ Boys
// F_m(T) = int_0^1 u^{2m} exp(-T u^2) du.  For T < kBoysTmax: Taylor expansion
// about the nearest tabulated point T_k (dF_m/dT = -F_{m+1}), with the table
// holding F_{m+j}(T_k)/j! so that each order costs kBoysTaylor-1 FMAs.  Low
// orders (mmax <= 4) are all expanded directly; higher ones expand F_mmax and
// descend with F_m = (2T F_{m+1} + e^{-T}) / (2m+1).  For T >= kBoysTmax:
// F_0 = (1/2) sqrt(pi/T) (erf(sqrt T) = 1 in double precision there) and
// F_{m+1} = ((2m+1) F_m - e^{-T}) / (2T).  The table is filled on the host by
// Gauss-Legendre quadrature of the defining integral.
constexpr double kBoysStep = 0.05;
constexpr double kBoysInvStep = 20.0;
constexpr double kBoysTmax = 40.0;
constexpr int kBoysRows = 801;                 // T_k = k * step, k = 0..800
constexpr int kBoysTaylor = 8;                 // terms; |T - T_k| <= 0.025
constexpr int kBoysM = kBoysMaxM + 1;          // orders tabulated
constexpr int kBoysRaw = kBoysMaxM + kBoysTaylor;  // orders needed to fill the table

__constant__ double c_inv_odd[kBoysRaw + 2];   // 1/(2m+1)
__constant__ double c_half_n[kNhMax];  // n/2

__device__ __forceinline__ double boys_taylor(const double *__restrict__ row, double x) {
  double f = __ldg(row + kBoysTaylor - 1);
#pragma unroll
  for (int j = kBoysTaylor - 2; j >= 0; --j) f = fma(f, x, __ldg(row + j));
  return f;
}

__device__ __forceinline__ void boys_eval(int mmax, double T, const double *__restrict__ tab,
                                          double *F) {
  if (T < kBoysTmax) {
    const int k = __double2int_rn(T * kBoysInvStep);
    const double x = k * kBoysStep - T;  // -(T - T_k)
    const double *row = tab + (size_t)k * kBoysM * kBoysTaylor;
    if (mmax <= 4) {
      for (int m = 0; m <= mmax; ++m) F[m] = boys_taylor(row + m * kBoysTaylor, x);
    } else {
      F[mmax] = boys_taylor(row + mmax * kBoysTaylor, x);
      const double e = exp(-T), T2 = 2.0 * T;
      for (int m = mmax - 1; m >= 0; --m) F[m] = fma(T2, F[m + 1], e) * c_inv_odd[m];
    }
  } else {
    const double e = exp(-T), inv2T = 0.5 / T;
    F[0] = 0.88622692545275801365 * rsqrt(T);  // (1/2) sqrt(pi/T)
    for (int m = 0; m < mmax; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) * inv2T;
  }
}

__device__ __forceinline__ dflt df_load(const float2 *p) {
  const float2 v = __ldg(p);
  return dflt(v.x, v.y);
}

// ----------------------------------------------- double-float Boys function
// F_m(T) = int_0^1 u^{2m} exp(-T u^2) du on the FP32 pipe.  For T < 60:
// Taylor expansion about the nearest point T_k = k/16 of a table of
// F_{m+j}(T_k)/j! and e^{-T_k}/j! (j < 7, |T - T_k| <= 1/32, truncation below
// 6e-15 relative); low orders (m <= 1) are expanded directly, higher ones
// expand F_mmax and e^{-T} and descend with F_m = (2T F_{m+1} + e^{-T})/(2m+1)
// (stable downwards).  For T >= 60: F_0 = (1/2) sqrt(pi/T) and
// F_{m+1} = (2m+1)/(2T) F_m, the e^{-T} terms (below e^{-60} = 9e-27 of F_0,
// under 1e-14 relative up to m = 14) dropped.  No exp() call: the table
// carries the exponential.
constexpr int kBoysDfTaylor = 7;
constexpr int kBoysDfRows = 961;                  // T_k = k/16, k = 0..960
constexpr int kBoysDfOrders = kBoysMaxM + 1;      // F_0 .. F_kBoysMaxM, then e^{-T}
constexpr int kBoysDfRow = (kBoysDfOrders + 1) * kBoysDfTaylor;  // float2 per row
constexpr float kBoysDfTmax = 60.0f;

__device__ __forceinline__ dflt df_horner7(const float2 *__restrict__ c, dflt x) {
  dflt f = df_load(c + kBoysDfTaylor - 1);
#pragma unroll
  for (int j = kBoysDfTaylor - 2; j >= 0; --j) f = fma(f, x, df_load(c + j));
  return f;
}

template <int MMAX>
__device__ __forceinline__ void boys_df(dflt T, const float2 *__restrict__ tab, dflt *F) {
  if (T.hi < kBoysDfTmax) {
    const int k = min(max(__float2int_rn(T.hi * 16.0f), 0), kBoysDfRows - 1);
    // x = T_k - T: the leading difference is exact (Sterbenz), then renormalised
    const float xh = __fsub_rn((float)k * 0.0625f, T.hi);
    const float s = __fadd_rn(xh, -T.lo);
    const float bb = __fsub_rn(s, xh);
    const dflt x(s, __fadd_rn(__fsub_rn(xh, __fsub_rn(s, bb)), __fsub_rn(-T.lo, bb)));
    const float2 *row = tab + (size_t)k * kBoysDfRow;
    if (MMAX <= 1) {
#pragma unroll
      for (int m = 0; m <= MMAX; ++m) F[m] = df_horner7(row + m * kBoysDfTaylor, x);
    } else {
      F[MMAX] = df_horner7(row + MMAX * kBoysDfTaylor, x);
      const dflt e = df_horner7(row + kBoysDfOrders * kBoysDfTaylor, x);
      const dflt T2(2.0f * T.hi, 2.0f * T.lo);
#pragma unroll
      for (int m = MMAX - 1; m >= 0; --m) F[m] = fma(T2, F[m + 1], e) * dflt(1.0 / (2 * m + 1));
    }
  } else {
    const dflt r = df_recip(T);
    F[0] = df_sqrt(r) * dflt(0.88622692545275801365);  // (1/2) sqrt(pi)
#pragma unroll
    for (int m = 0; m < MMAX; ++m) F[m + 1] = df_mulf(F[m] * r, 0.5f * (2 * m + 1));
  }
}

// Runtime-order variant for the interpreted kernel's set-up.
__device__ __forceinline__ void boys_df_rt(int mmax, dflt T, const float2 *__restrict__ tab, dflt *F) {
  if (T.hi < kBoysDfTmax) {
    const int k = min(max(__float2int_rn(T.hi * 16.0f), 0), kBoysDfRows - 1);
    const float xh = __fsub_rn((float)k * 0.0625f, T.hi);
    const float s = __fadd_rn(xh, -T.lo);
    const float bb = __fsub_rn(s, xh);
    const dflt x(s, __fadd_rn(__fsub_rn(xh, __fsub_rn(s, bb)), __fsub_rn(-T.lo, bb)));
    const float2 *row = tab + (size_t)k * kBoysDfRow;
    if (mmax <= 1) {
      for (int m = 0; m <= mmax; ++m) F[m] = df_horner7(row + m * kBoysDfTaylor, x);
    } else {
      F[mmax] = df_horner7(row + mmax * kBoysDfTaylor, x);
      const dflt e = df_horner7(row + kBoysDfOrders * kBoysDfTaylor, x);
      const dflt T2(2.0f * T.hi, 2.0f * T.lo);
      for (int m = mmax - 1; m >= 0; --m) F[m] = fma(T2, F[m + 1], e) * dflt(c_inv_odd[m]);
    }
  } else {
    const dflt r = df_recip(T);
    F[0] = df_sqrt(r) * dflt(0.88622692545275801365);
    for (int m = 0; m < mmax; ++m) F[m + 1] = df_mulf(F[m] * r, 0.5f * (2 * m + 1));
  }
}

// --------------------------------------------------------------- layouts
struct DevBasis {
  // shells
  const double *sh_ctr;  // [nshells][3]
  const int *sh_l, *sh_ao, *sh_atom;
  // shell pairs (a, b) sorted by class, then by Schwarz factor (descending)
  const int2 *pair_sh;   // shells (a, b), l_a >= l_b
  const int *pair_pp0;   // first primitive pair
  const int *pair_npp;   // number of primitive pairs kept
  // primitive pairs
  const double *pp_zeta, *pp_inv_zeta, *pp_P, *pp_pref, *pp_a, *pp_b;  // pp_P: [npp][3]
  const float2 *pp2;     // the same as double-float pairs: [npp][8] = zeta, 1/zeta, P, pref, alpha, beta
  const float2 *ctr2;    // shell centres as double-float pairs [nshells][3]
  const double *boys;    // [kBoysRows][kBoysCols]
  // class-specialised kernel: primitive pairs as double-float [npp][kPrimDf] =
  // zeta, 1/zeta, P[3], P - A[3], prefactor (A the centre of the pair's first
  // shell), the same in binary64 [npp][kPrimDf], and the double-float Boys table
  const float2 *ppg2;
  const double *ppg;
  const float2 *boys2;
  int nao;
};

struct DevProgs {
  const VrrInstr *vrr;
  const HrrInstr *hrr;
  const AccInstr *acc;
  const int *levels;
  const TileProg *tiles;
};

// Work item: bra pair, ket pairs [k0, k0 + nk) (absolute pair indices).
struct WorkItem {
  int bra, k0, nk, pad;
};

enum Mode { kStore = 0, kJK = 1, kGrad = 2 };

struct JKArgs {
  // q-innermost layouts: X[(mu*N + nu)*nd + q]
  const double *D;   // densities
  const double *S;   // D + D^T
  const float *D32;  // FP32 copies for the FP32 quartets (mixed precision)
  const float *S32;
  const dflt *D2;    // double-float copies for the double-float quartets
  const dflt *S2;
  double *J;         // half-Coulomb accumulator (symmetrised afterwards)
  double *K;
  const double *scale;  // per density: the power of two the copies were scaled by
  int nd;
  // store mode
  double *out;
  const long long *out_off;  // per work item: offset of its first block
  // gradient
  const double *P, *Q;  // q-innermost term stacks, nd = nterms
  double cJ, cK;
  double *grad;         // [natoms][3]
};

// One job of a launch: a context's basis and buffers and its slice of the
// class's work list.  A launch carries up to kMaxJobs jobs by value in its
// parameter block, so work items of several requests share one kernel.
constexpr int kMaxJobs = 24;
struct JobDesc {
  DevBasis B;
  JKArgs a;
  const WorkItem *items;
  int nitems;
  int first;  // index of this job's first item in the launch
};
struct JobTable {
  int njobs;
  int total;
  JobDesc j[kMaxJobs];
};

// Per-primitive-quartet table entry layout (Real units):
//   [0 .. ltot]           base values [00|00]^(m)
//   [ltot+1 .. +kNumCoef) coefficients (CoefSlot order)
//   then hz[0..nh), he[0..nh), hs[0..nh): n/(2 zeta), n/(2 eta), n/(2(zeta+eta))
__host__ __device__ inline int pt_stride(const ClassProg &p) { return p.ltot + 1 + kNumCoef + 3 * p.nh; }

struct ClassLaunch {
  ClassProg p;
  int G;        // primitive-quartet groups per warp (S = 32 / G lanes each)
  int warps;    // warps per CTA
  int smem_per_warp;  // bytes
  int T;        // primitive-table entries (set-up of T primitive quartets at a time)
  int P;        // primitive quartets per group in the vertical recurrence (1 or 2)
  int split;    // warps per work item: warp sub takes kets sub, sub + split, ...
};

// The digestion tabulates its output offsets in the dead primitive table: ten
// placements x ceil(nx ny / 4) groups x 4 outputs of int2, nx ny the largest
// product of two of the quartet's component counts (at least 36, the d x d
// table, so lighter classes keep the table they were tuned with).
__host__ __device__ inline size_t digest_table_bytes(const ClassProg &p) {
  int l = p.la > p.lb ? p.la : p.lb;
  l = l > p.lc ? l : p.lc;
  l = l > p.ld ? l : p.ld;
  int nn = ncart(l) * ncart(l);
  nn = nn > 36 ? nn : 36;
  return (size_t)10 * ((nn + 3) / 4) * 4 * 8;
}
// Reals of the primitive table: T entries, and never less than the digestion's
// offset table.
__host__ __device__ inline int ptab_reals(const ClassProg &p, int T, size_t real_bytes) {
  const int t = T * pt_stride(p);
  const int d = (int)((digest_table_bytes(p) + real_bytes - 1) / real_bytes);
  return t > d ? t : d;
}
// Shared memory one warp needs for class program p with G groups and a T-entry
// primitive table, in bytes: primitive table, G accumulator sets and the work
// region (Real: P G vertical regions, or the horizontal slots if larger),
// then for the gradient the Gamma block of one quartet (double).
__host__ __device__ inline size_t gamma_offset(const ClassProg &p, int G, int T, int P, size_t real_bytes) {
  int work = P * G * p.vrr_size > p.hrr_size ? P * G * p.vrr_size : p.hrr_size;
  size_t b = (size_t)(ptab_reals(p, T, real_bytes) + G * p.acc_total + work) * real_bytes;
  return (b + 15) / 16 * 16;
}
__host__ __device__ inline size_t warp_smem_bytes(const ClassProg &p, int G, int T, int P, size_t real_bytes) {
  size_t b = gamma_offset(p, G, T, P, real_bytes);
  if (p.deriv) b += (size_t)p.nout * sizeof(double);
  return (b + 15) / 16 * 16;
}

// ------------------------------------------- stage 1: one primitive quartet
// Base values [00|00]^(m) = 2 pi^{5/2} K_AB K_CD c.. / (zeta eta sqrt(zeta+eta))
// F_m(rho |PQ|^2) and the Obara-Saika coefficients of primitive pairs ia
// (bra) and ic (ket), written to the table entry e.
template <typename Real>
__device__ __forceinline__ void stage1(const DevBasis &B, const ClassProg &p, Real *e, int ia, int ic,
                                       int2 sab, int2 scd);

// IEEE FP64 throughout.
template <>
__device__ __forceinline__ void stage1<double>(const DevBasis &B, const ClassProg &p, double *e, int ia,
                                               int ic, int2 sab, int2 scd) {
  const double *A = B.sh_ctr + 3 * sab.x, *C = B.sh_ctr + 3 * scd.x;
  const double zeta = B.pp_zeta[ia], eta = B.pp_zeta[ic];
  const double izeta = B.pp_inv_zeta[ia], ieta = B.pp_inv_zeta[ic];
  const double *P = B.pp_P + 3 * ia, *Q = B.pp_P + 3 * ic;
  const double isum = 1.0 / (zeta + eta);
  const double rho = zeta * eta * isum;
  double PQ2 = 0.0, W[3];
  for (int x = 0; x < 3; ++x) {
    double d = P[x] - Q[x];
    PQ2 = fma(d, d, PQ2);
    W[x] = (zeta * P[x] + eta * Q[x]) * isum;
  }
  double F[kBoysMaxM + 1];
  boys_eval(p.ltot, rho * PQ2, B.boys, F);
  const double pre = B.pp_pref[ia] * B.pp_pref[ic] * sqrt(isum);
  for (int m = 0; m <= p.ltot; ++m) e[m] = pre * F[m];
  double *cf = e + p.ltot + 1;
  for (int x = 0; x < 3; ++x) {
    cf[kPAx + x] = P[x] - A[x];
    cf[kQCx + x] = Q[x] - C[x];
    cf[kWPx + x] = W[x] - P[x];
    cf[kWQx + x] = W[x] - Q[x];
  }
  cf[kHalfZeta] = 0.5 * izeta;
  cf[kHalfEta] = 0.5 * ieta;
  cf[kRhoZeta] = rho * izeta;
  cf[kRhoEta] = rho * ieta;
  cf[kHalfSum] = 0.5 * isum;
  cf[kWA] = 2.0 * B.pp_a[ia];
  cf[kWB] = 2.0 * B.pp_b[ia];
  cf[kWC] = 2.0 * B.pp_a[ic];
  double *h = cf + kNumCoef;
  const int nh = p.nh;
  for (int n = 0; n < nh; ++n) {
    h[n] = c_half_n[n] * izeta;
    h[nh + n] = c_half_n[n] * ieta;
    h[2 * nh + n] = c_half_n[n] * isum;
  }
}

template <typename Real>
__device__ __forceinline__ Real df_cvt(dflt x);
template <>
__device__ __forceinline__ dflt df_cvt<dflt>(dflt x) { return x; }
template <>
__device__ __forceinline__ float df_cvt<float>(dflt x) { return df_to_float(x); }

// Double-float throughout on the FP32 pipe, the Boys function included.
template <typename Real>
__device__ __forceinline__ void stage1(const DevBasis &B, const ClassProg &p, Real *e, int ia, int ic,
                                       int2 sab, int2 scd) {
  const float2 *pa = B.pp2 + 8 * ia, *pc = B.pp2 + 8 * ic;
  const float2 *A = B.ctr2 + 3 * sab.x, *C = B.ctr2 + 3 * scd.x;
  const dflt zeta = df_load(pa + 0), eta = df_load(pc + 0);
  const dflt izeta = df_load(pa + 1), ieta = df_load(pc + 1);
  const dflt isum = df_recip(zeta + eta);
  const dflt rho = zeta * eta * isum;
  dflt PQ2(0.0f, 0.0f), P[3], Q[3];
  for (int x = 0; x < 3; ++x) {
    P[x] = df_load(pa + 2 + x);
    Q[x] = df_load(pc + 2 + x);
    const dflt d = P[x] - Q[x];
    PQ2 = fma(d, d, PQ2);
  }
  dflt F[kBoysMaxM + 1];
  boys_df_rt(p.ltot, rho * PQ2, B.boys2, F);
  const dflt pre = df_load(pa + 5) * df_load(pc + 5) * df_sqrt(isum);
  for (int m = 0; m <= p.ltot; ++m) e[m] = df_cvt<Real>(pre * F[m]);
  Real *cf = e + p.ltot + 1;
  for (int x = 0; x < 3; ++x) {
    const dflt W = (zeta * P[x] + eta * Q[x]) * isum;
    cf[kPAx + x] = df_cvt<Real>(P[x] - df_load(A + x));
    cf[kQCx + x] = df_cvt<Real>(Q[x] - df_load(C + x));
    cf[kWPx + x] = df_cvt<Real>(W - P[x]);
    cf[kWQx + x] = df_cvt<Real>(W - Q[x]);
  }
  cf[kHalfZeta] = df_cvt<Real>(df_mulf(izeta, 0.5f));
  cf[kHalfEta] = df_cvt<Real>(df_mulf(ieta, 0.5f));
  cf[kRhoZeta] = df_cvt<Real>(rho * izeta);
  cf[kRhoEta] = df_cvt<Real>(rho * ieta);
  cf[kHalfSum] = df_cvt<Real>(df_mulf(isum, 0.5f));
  if (p.deriv) {
    cf[kWA] = df_cvt<Real>(df_mulf(df_load(pa + 6), 2.0f));
    cf[kWB] = df_cvt<Real>(df_mulf(df_load(pa + 7), 2.0f));
    cf[kWC] = df_cvt<Real>(df_mulf(df_load(pc + 6), 2.0f));
  }
  Real *h = cf + kNumCoef;
  const int nh = p.nh;
  for (int n = 0; n < nh; ++n) {
    const float hn = 0.5f * (float)n;
    h[n] = df_cvt<Real>(df_mulf(izeta, hn));
    h[nh + n] = df_cvt<Real>(df_mulf(ieta, hn));
    h[2 * nh + n] = df_cvt<Real>(df_mulf(isum, hn));
  }
}

// Vertical recurrence and accumulation of nchunk primitive-table entries,
// NP per group at a time: group g runs entries r0 + j G + g, j < NP, and each
// lane applies every step it decodes to all NP of them (NP independent
// chains per instruction load).  Regions: entry j of group g at
// work + (j G + g) vrr_size.
template <typename Real, int NP>
__device__ __forceinline__ void vrr_multi(const DevProgs &PR, const ClassProg &p, int G, int S, int g, int s,
                                          int nh, int stride, const Real *ptab, Real *work, Real *my_acc,
                                          int nchunk) {
  for (int r0 = 0; r0 < nchunk; r0 += NP * G) {
    const Real *cf[NP], *h[NP];
    Real *v[NP];
    bool act[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const int loc = r0 + j * G + g;
      act[j] = loc < nchunk;
      const Real *e = ptab + (act[j] ? loc : r0 + g) * stride;
      cf[j] = e + p.ltot + 1;
      h[j] = cf[j] + kNumCoef;
      v[j] = work + (j * G + g) * p.vrr_size;
    }
    if (act[0]) {
#pragma unroll
      for (int j = 0; j < NP; ++j)
        for (int t = s; t <= p.ltot + 1; t += S) v[j][t] = t == 0 ? zero_real<Real>() : cf[j][t - 1 - (p.ltot + 1)];
    }
    __syncwarp();
    for (int L = 0; L < p.nvrr_level; ++L) {
      const int i0 = PR.levels[p.vrr_level0 + L], i1 = PR.levels[p.vrr_level0 + L + 1];
      if (act[0]) {
        // steps of one level never read each other's targets, so every
        // source is read before any target of the level is written; the
        // optional operands are read only by the steps that use them
        for (int k = i0 + s; k < i1; k += S) {
          const VrrInstr in = PR.vrr[k];
          const int c0 = kPAx + 3 * in.kind + in.dir;
          Real t[NP];
#pragma unroll
          for (int j = 0; j < NP; ++j) t[j] = cf[j][c0] * v[j][in.s0];
#pragma unroll
          for (int j = 0; j < NP; ++j) t[j] = fma(cf[j][kWPx - kPAx + c0], v[j][in.s1], t[j]);
          if (in.n1) {
            const int hn = in.kind * nh + in.n1, rk = kRhoZeta + in.kind;
#pragma unroll
            for (int j = 0; j < NP; ++j) t[j] = fma(h[j][hn], fma(-cf[j][rk], v[j][in.s3], v[j][in.s2]), t[j]);
          }
          if (in.n2) {
            const int hn = 2 * nh + in.n2;
#pragma unroll
            for (int j = 0; j < NP; ++j) t[j] = fma(h[j][hn], v[j][in.s4], t[j]);
          }
#pragma unroll
          for (int j = 0; j < NP; ++j) v[j][in.tgt] = t[j];
        }
      }
      __syncwarp();
    }
    if (act[0]) {
      for (int k = p.acc_begin + s; k < p.acc_begin + p.nacc; k += S) {
        const AccInstr a = PR.acc[k];
        Real x = my_acc[a.acc];
#pragma unroll
        for (int j = 0; j < NP; ++j)
          if (act[j]) x = fma(a.chan == 0 ? Real(1) : cf[j][kWA + a.chan - 1], v[j][a.slot], x);
        my_acc[a.acc] = x;
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------ one contracted quartet
// Computes the contracted block(s) of quartet (bra pair ip | ket pair jp) into
// the warp's shared memory and returns a pointer to the output block (nout
// Reals, row-major [na][nb][nc][nd], or 9 such blocks for derivatives).
template <typename Real>
__device__ Real *quartet_block(const DevBasis &B, const DevProgs &PR, const ClassProg &p, int G, int T,
                               int P, Real *sm, int ip, int jp, int lane) {
  const int S = 32 / G, g = lane / S, s = lane % S;
  const int stride = pt_stride(p), nh = p.nh;
  Real *ptab = sm;                              // [T][stride] (and the digestion's table)
  Real *accs = ptab + ptab_reals(p, T, sizeof(Real));  // [G][acc_total]; group 0's last
  Real *acc0 = accs + (G - 1) * p.acc_total;
  Real *work = acc0 + p.acc_total;              // VRR regions / HRR slots
  Real *my_acc = accs + (G - 1 - g) * p.acc_total;
  Real *my_vrr = work + g * p.vrr_size;

  const int2 sab = B.pair_sh[ip], scd = B.pair_sh[jp];
  const int pp0 = B.pair_pp0[ip], npp = B.pair_npp[ip];
  const int qq0 = B.pair_pp0[jp], nqq = B.pair_npp[jp];
  const int npq = npp * nqq;

  for (int t = lane; t < G * p.acc_total; t += 32) accs[t] = zero_real<Real>();

  for (int c0 = 0; c0 < npq; c0 += T) {
    // stage 1: base values and coefficients, one primitive quartet per lane
    const int pq = c0 + lane;
    if (lane < T && pq < npq) {
      const int ia = pp0 + pq / nqq, ic = qq0 + pq % nqq;
      stage1<Real>(B, p, ptab + lane * stride, ia, ic, sab, scd);
    }
    __syncwarp();
    // stage 2: recurrences.  P = 2: 2G primitive quartets at a time, each
    // lane applying every step it decodes to two of them (vrr_multi; two
    // chains per instruction load measured 5 % faster on the double-float
    // and binary32 classes than P = 1, four chains 2 % slower than two).
    // P = 1: G at a time, each lane taking two steps of one quartet per
    // iteration (the smallest vertical regions: the binary64 f classes,
    // bound by the FP64 pipe, keep their occupancy).
    const int nchunk = min(T, npq - c0);
    if (P == 2) {
      vrr_multi<Real, 2>(PR, p, G, S, g, s, nh, stride, ptab, work, my_acc, nchunk);
    } else {
      for (int r0 = 0; r0 < nchunk; r0 += G) {
        const int loc = r0 + g;
        const bool active = loc < nchunk;
        const Real *e = ptab + loc * stride;
        const Real *cf = e + p.ltot + 1;
        const Real *h = cf + kNumCoef;
        if (active) {
          for (int t = s; t <= p.ltot + 1; t += S) my_vrr[t] = t == 0 ? zero_real<Real>() : e[t - 1];
        }
        __syncwarp();
        for (int L = 0; L < p.nvrr_level; ++L) {
          const int i0 = PR.levels[p.vrr_level0 + L], i1 = PR.levels[p.vrr_level0 + L + 1];
          if (active) {
            // two independent steps per lane per iteration (every source of
            // both is read before either target is written)
            for (int k = i0 + s; k < i1; k += 2 * S) {
              const bool two = k + S < i1;
              const VrrInstr ia = PR.vrr[k];
              const VrrInstr ib = PR.vrr[two ? k + S : k];
              const Real a0 = my_vrr[ia.s0], a1 = my_vrr[ia.s1];
              const Real b0 = my_vrr[ib.s0], b1 = my_vrr[ib.s1];
              Real ta = cf[kPAx + 3 * ia.kind + ia.dir] * a0;
              Real tb = cf[kPAx + 3 * ib.kind + ib.dir] * b0;
              ta = fma(cf[kWPx + 3 * ia.kind + ia.dir], a1, ta);
              tb = fma(cf[kWPx + 3 * ib.kind + ib.dir], b1, tb);
              if (ia.n1) ta = fma(h[ia.kind * nh + ia.n1], fma(-cf[kRhoZeta + ia.kind], my_vrr[ia.s3], my_vrr[ia.s2]), ta);
              if (ib.n1) tb = fma(h[ib.kind * nh + ib.n1], fma(-cf[kRhoZeta + ib.kind], my_vrr[ib.s3], my_vrr[ib.s2]), tb);
              if (ia.n2) ta = fma(h[2 * nh + ia.n2], my_vrr[ia.s4], ta);
              if (ib.n2) tb = fma(h[2 * nh + ib.n2], my_vrr[ib.s4], tb);
              my_vrr[ia.tgt] = ta;
              if (two) my_vrr[ib.tgt] = tb;
            }
          }
          __syncwarp();
        }
        if (active) {
          for (int k = p.acc_begin + s; k < p.acc_begin + p.nacc; k += S) {
            const AccInstr a = PR.acc[k];
            Real w = a.chan == 0 ? Real(1) : cf[kWA + a.chan - 1];
            my_acc[a.acc] = fma(w, my_vrr[a.slot], my_acc[a.acc]);
          }
        }
        __syncwarp();
      }
    }
  }
  // reduce the group accumulators into group 0's
  if (G > 1) {
    for (int t = lane; t < p.acc_total; t += 32) {
      Real v = acc0[t];
      for (int gg = 1; gg < G; ++gg) v += accs[(G - 1 - gg) * p.acc_total + t];
      acc0[t] = v;
    }
  }
  __syncwarp();
  return acc0;
}

// Horizontal recurrence of one output tile on the contracted accumulators acc0
// (followed in memory by the work region); returns the tile's output block.
template <typename Real>
__device__ Real *hrr_tile(const DevBasis &B, const DevProgs &PR, const ClassProg &p, int tile,
                          Real *acc0, int ip, int jp, int lane) {
  const TileProg T = PR.tiles[p.tile_begin + tile];
  const int2 sab = B.pair_sh[ip], scd = B.pair_sh[jp];
  const double *A = B.sh_ctr + 3 * sab.x, *Bc = B.sh_ctr + 3 * sab.y;
  const double *C = B.sh_ctr + 3 * scd.x, *Dc = B.sh_ctr + 3 * scd.y;
  if (lane == 0) acc0[p.acc_total] = zero_real<Real>();  // zero slot
  __syncwarp();
  Real X[2][3];
  for (int x = 0; x < 3; ++x) {
    X[0][x] = from_double<Real>(A[x] - Bc[x]);
    X[1][x] = from_double<Real>(C[x] - Dc[x]);
  }
  for (int L = 0; L < T.nhrr_level; ++L) {
    const int i0 = PR.levels[T.hrr_level0 + L], i1 = PR.levels[T.hrr_level0 + L + 1];
    for (int k = i0 + lane; k < i1; k += 64) {  // two independent steps per lane
      const bool two = k + 32 < i1;
      const HrrInstr ia = PR.hrr[k];
      const HrrInstr ib = PR.hrr[two ? k + 32 : k];
      const Real ca = ia.kind < 2 ? X[ia.kind][ia.dir] : -Real(ia.dir);
      const Real cb = ib.kind < 2 ? X[ib.kind][ib.dir] : -Real(ib.dir);
      const Real ta = fma(ca, acc0[ia.s1], acc0[ia.s0]);
      const Real tb = fma(cb, acc0[ib.s1], acc0[ib.s0]);
      acc0[ia.tgt] = ta;
      if (two) acc0[ib.tgt] = tb;
    }
    __syncwarp();
  }
  return acc0 + T.out_base;
}

// Index sets of the ten digestion placements (Eq. quartet_scatter with every
// permutational image of the unique quartet applied, non-symmetric D):
// out(row,col) += w * sum_{u,v} I * M(row2, col2); indices 0..3 = a, b, c, d.
struct Placement {
  int orow, ocol, srow, scol, isJ;
};
__constant__ Placement c_place[10] = {
    {0, 1, 2, 3, 1}, {2, 3, 0, 1, 1},  // J half: Jh[ab] += I S[cd], Jh[cd] += I S[ab]
    {0, 2, 1, 3, 0}, {1, 2, 0, 3, 0}, {0, 3, 1, 2, 0}, {1, 3, 0, 2, 0},
    {2, 0, 3, 1, 0}, {3, 0, 2, 1, 0}, {2, 1, 3, 0, 0}, {3, 1, 2, 0, 0}};

template <typename Real>
__device__ __forceinline__ const Real *digest_operand(const JKArgs &a, bool isJ);
template <>
__device__ __forceinline__ const double *digest_operand<double>(const JKArgs &a, bool isJ) {
  return isJ ? a.S : a.D;
}
template <>
__device__ __forceinline__ const float *digest_operand<float>(const JKArgs &a, bool isJ) {
  return isJ ? a.S32 : a.D32;
}
template <>
__device__ __forceinline__ const dflt *digest_operand<dflt>(const JKArgs &a, bool isJ) {
  return isJ ? a.S2 : a.D2;
}

// One placement of the digestion, out(x, y) += sum_{u<nu, v<nv} I[x sr + y sc +
// u su + v sv] M(u, v), for every output (x, y) of the nout = nr x nc block and
// every density.  Lanes run over (output group, density) units, four outputs per
// group sharing each density load (four independent accumulation chains), so a
// warp stays full when the number of densities is not a multiple of 32.
// Double-float sums use the compensated accumulator (AccOf<dflt>).  The
// sums stay runtime loops: unrolled per block shape, the double-float code of
// the ten placements outgrows the instruction cache and stalls every warp on
// the SM, the recurrence's included.
// tab[grp*4 + j] = (integral offset, output offset without the density) of
// output j of group grp, tabulated once per quartet by digest_jk.
template <typename Real>
__device__ __forceinline__ void digest_place(const Real *__restrict__ I, const Real *__restrict__ Mblk,
                                             double *__restrict__ Tblk, int nd, size_t mrow, int nout,
                                             const int2 *tab, int su, int sv, int nu, int nv, int lane) {
  const int ngrp = (nout + 3) >> 2;
  int q = lane, grp = 0;
  while (q >= nd) { q -= nd; ++grp; }
  while (grp < ngrp) {
    const int o0 = grp << 2, cnt = min(4, nout - o0);
    const Real *Ib[4];
    size_t to[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int2 t = tab[o0 + j];
      Ib[j] = I + t.x;
      to[j] = (size_t)(unsigned)t.y + q;
    }
    using Acc = typename AccOf<Real>::type;
    Acc acc0 = acc_zero(Real()), acc1 = acc0, acc2 = acc0, acc3 = acc0;
    const Real *Mu = Mblk + q;
    for (int u = 0; u < nu; ++u, Mu += mrow) {
      const int iu = u * su;
      for (int v = 0; v < nv; ++v) {
        const Real m = ldg(Mu + (size_t)v * nd);
        const int iv = iu + v * sv;
        acc0 = acc_fma(acc0, Ib[0][iv], m);
        acc1 = acc_fma(acc1, Ib[1][iv], m);
        acc2 = acc_fma(acc2, Ib[2][iv], m);
        acc3 = acc_fma(acc3, Ib[3][iv], m);
      }
    }
    red_add(Tblk + to[0], acc0);
    if (cnt > 1) red_add(Tblk + to[1], acc1);
    if (cnt > 2) red_add(Tblk + to[2], acc2);
    if (cnt > 3) red_add(Tblk + to[3], acc3);
    q += 32;
    while (q >= nd) { q -= nd; ++grp; }
  }
}

// The ten placements of one quartet (or of one output tile of it: off[0] and
// n[0] then give the tile's range of a, and I its sub-block).  tab is scratch
// shared memory of the warp (its primitive table, dead between the
// recurrences of two kets) for the per-output offsets of every placement,
// digest_table_bytes of the class; the primitive table is never smaller.
// The output offsets x*N*nd + y*nd fit 32 bits for every size the build accepts.
template <typename Real>
__device__ void digest_jk(const JKArgs &a, const Real *I, const int off[4], const int n[4], int N,
                          int2 *tab, int lane) {
  const int str[4] = {n[1] * n[2] * n[3], n[2] * n[3], n[3], 1};
  const int nd = a.nd;
  const size_t mrow = (size_t)N * nd;  // stride of one AO row in the q-innermost layout
  int base[11];
  base[0] = 0;
  for (int pl = 0; pl < 10; ++pl) {
    const Placement P = c_place[pl];
    const bool on = P.isJ ? a.J != nullptr : a.K != nullptr;
    base[pl + 1] = base[pl] + (on ? ((n[P.orow] * n[P.ocol] + 3) >> 2) * 4 : 0);
  }
  for (int e = lane; e < base[10]; e += 32) {
    int pl = 0;
    while (e >= base[pl + 1]) ++pl;
    const Placement P = c_place[pl];
    const int r = e - base[pl], o0 = r & ~3, j = r & 3;
    const int nout = n[P.orow] * n[P.ocol], nc = n[P.ocol];
    const int o = o0 + (j < min(4, nout - o0) ? j : 0);
    const int x = o / nc, y = o - x * nc;
    tab[e] = make_int2(x * str[P.orow] + y * str[P.ocol], (int)((size_t)x * mrow + (size_t)y * nd));
  }
  __syncwarp();
  for (int pl = 0; pl < 10; ++pl) {
    const Placement P = c_place[pl];
    if (base[pl + 1] == base[pl]) continue;
    const Real *M = digest_operand<Real>(a, P.isJ);
    double *T = P.isJ ? a.J : a.K;
    const Real *Mblk = M + ((size_t)off[P.srow] * N + off[P.scol]) * nd;
    double *Tblk = T + ((size_t)off[P.orow] * N + off[P.ocol]) * nd;
    digest_place<Real>(I, Mblk, Tblk, nd, mrow, n[P.orow] * n[P.ocol], tab + base[pl], str[P.srow],
                       str[P.scol], n[P.srow], n[P.scol], lane);
  }
  __syncwarp();  // the table region is the next ket's primitive table
}

// Gamma of one quartet for the gradient: the sum over the distinct images of
// G_{mu nu ka rho} = sum_r [cJ P_r[mu][nu] Q_r[ka][rho] + cK P_r[mu][ka] Q_r[nu][rho]]
// (Eq. jkderiv), times the degeneracy weight w, into gam[ijkl].  The J images
// pair the symmetric sums, read from a.S = P + P^T and a.D = Q + Q^T (same
// q-innermost layout as a.P, a.Q).
__device__ void gamma_block(const JKArgs &a, double *gam, const int off[4], const int n[4],
                            double w, int N, int lane) {
  const int nq = n[0] * n[1] * n[2] * n[3];
  const int nt = a.nd;
  // L lanes per element, each over terms r = sub, sub + L, ... (consecutive
  // lanes read consecutive terms: the term index is innermost in P and Q),
  // then a butterfly sum inside the L-lane group; 32 / L elements per pass.
  // Light classes have only a few elements per quartet, so lanes over
  // elements alone left most of the warp idle through all the terms.
  const int L = nt >= 32 ? 32 : nt > 16 ? 32 : nt > 8 ? 16 : nt > 4 ? 8 : nt > 2 ? 4 : nt > 1 ? 2 : 1;
  const int E = 32 / L, sub = lane % L, eg = lane / L;
  for (int e0 = 0; e0 < nq; e0 += E) {
    const int e = e0 + eg;
    double g = 0.0;
    if (e < nq) {
      const int l = e % n[3], k = (e / n[3]) % n[2], j = (e / (n[3] * n[2])) % n[1],
                i = e / (n[3] * n[2] * n[1]);
      const size_t mu = off[0] + i, nu = off[1] + j, ka = off[2] + k, rho = off[3] + l;
      for (int r = sub; r < nt; r += L) {
        const double *P = a.P + r, *Q = a.Q + r;
#define PX(x, y) __ldg(P + ((x) * N + (y)) * nt)
#define QX(x, y) __ldg(Q + ((x) * N + (y)) * nt)
        // a zero coefficient skips its images (warp-uniform branches)
        if (a.cJ != 0.0) {
          const double *Ps = a.S + r, *Qs = a.D + r;
          const double gJ = __ldg(Ps + (mu * N + nu) * nt) * __ldg(Qs + (ka * N + rho) * nt) +
                            __ldg(Ps + (ka * N + rho) * nt) * __ldg(Qs + (mu * N + nu) * nt);
          g = fma(a.cJ, gJ, g);
        }
        if (a.cK != 0.0) {
          const double gK = PX(mu, ka) * QX(nu, rho) + PX(nu, ka) * QX(mu, rho) +
                            PX(mu, rho) * QX(nu, ka) + PX(nu, rho) * QX(mu, ka) +
                            PX(ka, mu) * QX(rho, nu) + PX(rho, mu) * QX(ka, nu) +
                            PX(ka, nu) * QX(rho, mu) + PX(rho, nu) * QX(ka, mu);
          g = fma(a.cK, gK, g);
        }
#undef PX
#undef QX
      }
    }
    for (int o = L >> 1; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
    if (sub == 0 && e < nq) gam[e] = w * g;
  }
}

// ------------------------------------------------------------- the kernel
// One warp per work item (bra pair, ket range); warps of a CTA are independent.
// 128 registers per thread: the J/K kernels also fit 80 or 96 without spills,
// but the extra warps do not make up for the lost scheduling freedom (measured
// 8 % slower on the 200-AO chain), and the gradient kernels spill below 128.
template <typename Real, int MODE>
__global__ void __launch_bounds__(128, 4) quartet_kernel(DevProgs PR, ClassLaunch CL,
                                                      const __grid_constant__ JobTable T) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const ClassProg &p = CL.p;
  unsigned char *wbase = smem_raw + (size_t)warp * CL.smem_per_warp;
  Real *sm = reinterpret_cast<Real *>(wbase);
  double *gam = reinterpret_cast<double *>(wbase + gamma_offset(p, CL.G, CL.T, CL.P, sizeof(Real)));
  const long long units = (long long)T.total * CL.split;
  for (long long u = (long long)blockIdx.x * CL.warps + warp; u < units; u += (long long)gridDim.x * CL.warps) {
    const int it = (int)(u / CL.split), sub = (int)(u % CL.split);
    int jb = 0;  // job holding item it (jobs are few; linear search in the parameter block)
    while (jb + 1 < T.njobs && it >= T.j[jb + 1].first) ++jb;
    const JobDesc &J = T.j[jb];
    const DevBasis &B = J.B;
    const JKArgs &a = J.a;
    const int N = B.nao;
    const int li = it - J.first;
    const WorkItem W = J.items[li];
    const int2 sab = B.pair_sh[W.bra];
    for (int kk = sub; kk < W.nk; kk += CL.split) {
      const int jp = W.k0 + kk;
      const int2 scd = B.pair_sh[jp];
      Real *acc0 = quartet_block<Real>(B, PR, p, CL.G, CL.T, CL.P, sm, W.bra, jp, lane);
      const int sh[4] = {sab.x, sab.y, scd.x, scd.y};
      int off[4], n[4];
      for (int t = 0; t < 4; ++t) {
        off[t] = B.sh_ao[sh[t]];
        n[t] = ncart(B.sh_l[sh[t]]);
      }
      double w = 1.0;
      float wf = 1.0f;
      if (sab.x == sab.y) { w *= 0.5; wf *= 0.5f; }
      if (scd.x == scd.y) { w *= 0.5; wf *= 0.5f; }
      if (W.bra == jp) { w *= 0.5; wf *= 0.5f; }
      if (MODE == kGrad) gamma_block(a, gam, off, n, w, N, lane);
      double g9 = 0.0;  // lane t < 9 keeps component t
      for (int tile = 0; tile < p.ntile; ++tile) {
        const TileProg TP = PR.tiles[p.tile_begin + tile];
        const Real *I = hrr_tile<Real>(B, PR, p, tile, acc0, W.bra, jp, lane);
        if (MODE == kStore) {
          const long long per_quartet = p.deriv ? (long long)p.ntile * p.nout : p.nout;
          double *o = a.out + a.out_off[li] + kk * per_quartet + TP.store_off;
          for (int t = lane; t < TP.nout; t += 32) o[t] = to_double(I[t]);
        } else if (MODE == kJK) {
          Real *Iw = const_cast<Real *>(I);
          for (int t = lane; t < TP.nout; t += 32) Iw[t] = scale_pow2(Iw[t], wf);  // degeneracy weight, once
          __syncwarp();
          // the tile is the block of a "shell" made of a's components [a0, a0 + na)
          const int offt[4] = {off[0] + TP.a0, off[1], off[2], off[3]};
          const int nt[4] = {TP.na, n[1], n[2], n[3]};
          digest_jk<Real>(a, I, offt, nt, N, reinterpret_cast<int2 *>(sm), lane);
        } else {
          double v = 0.0;
          for (int e = lane; e < p.nout; e += 32) v = fma(to_double(I[e]), gam[e], v);
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == tile) g9 = v;
        }
        __syncwarp();
      }
      if (MODE == kGrad) {
        // lanes 0..8 hold dE/dX for X = A_x..C_z; centre D by translational invariance
        const int x = lane % 3;
        const double gA = __shfl_sync(0xffffffffu, g9, x), gB = __shfl_sync(0xffffffffu, g9, 3 + x),
                     gC = __shfl_sync(0xffffffffu, g9, 6 + x);
        if (lane < 3) {
          atomicAdd(a.grad + 3 * B.sh_atom[sh[0]] + x, gA);
          atomicAdd(a.grad + 3 * B.sh_atom[sh[1]] + x, gB);
          atomicAdd(a.grad + 3 * B.sh_atom[sh[2]] + x, gC);
          atomicAdd(a.grad + 3 * B.sh_atom[sh[3]] + x, -(gA + gB + gC));
        }
      }
      __syncwarp();
    }
  }
}

// --------------------------------------------------------- layout kernels
// scale[q] = 2^-e with max_ij |D[q][i][j]| in [2^(e-1), 2^e): one block per
// density.  A zero or non-finite maximum gives scale 1 (so NaN and Inf still
// propagate to J and K).
__global__ void density_scales(const double *__restrict__ D, size_t NN, double *__restrict__ scale) {
  __shared__ double red[32];
  const double *Dq = D + (size_t)blockIdx.x * NN;
  double m = 0.0;
  for (size_t t = threadIdx.x; t < NN; t += blockDim.x) m = fmax(m, fabs(Dq[t]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) {
      // the exponent field of m gives e exactly: m = f 2^e with f in [1/2, 1)
      const long long b = __double_as_longlong(m);
      const int E = (int)((b >> 52) & 0x7FF);
      double s = 1.0;
      if (m > 0.0 && E > 0 && E < 0x7FF) {
        const int e = E - 1022;
        s = ldexp(1.0, -e);
      }
      scale[blockIdx.x] = s;
    }
  }
}

// [nd][N][N] -> q-innermost [(mu*N+nu)*nd + q] copies of s_q D and of
// s_q (D + D^T) (s_q = scale[q], 1 when scale is null): FP64 (Dq, Sq),
// double-float pairs (D2, S2) and FP32 (D32, S32); null = skip.
__global__ void to_qinner(const double *__restrict__ D, double *__restrict__ Dq,
                          double *__restrict__ Sq, float *__restrict__ Dq32,
                          float *__restrict__ Sq32, int nd, int N, dflt *__restrict__ D2 = nullptr,
                          dflt *__restrict__ S2 = nullptr, const double *__restrict__ scale = nullptr) {
  const size_t NN = (size_t)N * N;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < NN * nd;
       t += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(t % nd);
    const size_t mn = t / nd;
    const int mu = (int)(mn / N), nu = (int)(mn % N);
    const double s = scale ? scale[q] : 1.0;
    const double v = D[q * NN + mn] * s;
    const double sv = v + D[q * NN + (size_t)nu * N + mu] * s;
    if (Dq) Dq[t] = v;
    if (Sq) Sq[t] = sv;
    if (Dq32) Dq32[t] = (float)v;
    if (Sq32) Sq32[t] = (float)sv;
    if (D2) D2[t] = dflt(v);
    if (S2) S2[t] = dflt(sv);
  }
}

// J[q] = (Jh[q] + Jh[q]^T) / s_q and K[q] = Kq[q] / s_q from the q-innermost
// accumulators (s_q = scale[q], 1 when scale is null; dividing by a power of
// two is exact).
__global__ void from_qinner(const double *__restrict__ Jq, const double *__restrict__ Kq,
                            double *__restrict__ J, double *__restrict__ K, int nd, int N,
                            const double *__restrict__ scale = nullptr) {
  const size_t NN = (size_t)N * N;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < NN * nd;
       t += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(t / NN);
    const size_t mn = t % NN;
    const int mu = (int)(mn / N), nu = (int)(mn % N);
    const double inv = scale ? 1.0 / scale[q] : 1.0;
    if (J) J[t] = (Jq[mn * nd + q] + Jq[((size_t)nu * N + mu) * nd + q]) * inv;
    if (K) K[t] = Kq[mn * nd + q] * inv;
  }
}

// F[q] = (cJ (Jh[q] + Jh[q]^T) + cK Kq[q]) / s_q from the q-innermost
// accumulators (a null accumulator contributes nothing).
__global__ void from_qinner_fock(const double *__restrict__ Jq, const double *__restrict__ Kq,
                                 double *__restrict__ F, int nd, int N, const double *__restrict__ scale,
                                 double cJ, double cK) {
  const size_t NN = (size_t)N * N;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < NN * nd;
       t += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(t / NN);
    const size_t mn = t % NN;
    const int mu = (int)(mn / N), nu = (int)(mn % N);
    double v = 0.0;
    if (Jq) v = cJ * (Jq[mn * nd + q] + Jq[((size_t)nu * N + mu) * nd + q]);
    if (Kq) v = fma(cK, Kq[mn * nd + q], v);
    F[t] = v / scale[q];
  }
}

// Deterministic dot product <P, F> over n elements: block b sums its
// contiguous chunk in a fixed order into partial[b]; dot_final adds the
// partials in index order.
__global__ void dot_partial(const double *__restrict__ P, const double *__restrict__ F, size_t n,
                            double *__restrict__ partial) {
  __shared__ double red[32];
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
  double v = 0.0;
  for (size_t t = b0 + threadIdx.x; t < b1; t += blockDim.x) v = fma(P[t], F[t], v);
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
}
__global__ void dot_final(const double *__restrict__ partial, int nb, double *__restrict__ E) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double v = 0.0;
    for (int b = 0; b < nb; ++b) v += partial[b];
    *E = v;
  }
}

// --------------------------------------------------- arithmetic throughput
// Eight independent multiply-add chains per thread, `iters` steps each; the
// operands come from the launch so nothing folds, and the chains' sum is
// stored only when it matches an impossible value, so nothing is dead.
__device__ double g_alu_sink;
template <int KIND>
__global__ void __launch_bounds__(256) alu_peak_kernel(int iters, float b, float c) {
  const float t = (float)(threadIdx.x + 1) * 1e-7f;
  if (KIND == 0) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = t + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], b, c);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == -1.2345f) g_alu_sink = s;
  } else if (KIND == 1) {
    double x[8];
    const double bd = b, cd = c;
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = t + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = ::fma(x[k], bd, cd);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == -1.2345) g_alu_sink = s;
  } else if (KIND == 2) {
    dflt x[8];
    const dflt bd(b, b * 1e-9f), cd(c, c * 1e-9f);
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = dflt(t + k, 0.0f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fma(x[k], bd, cd);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k].hi + x[k].lo;
    if (s == -1.2345f) g_alu_sink = s;
  } else {
    DotAcc x[8];
    const dflt bd(b, b * 1e-9f), cd(c, c * 1e-9f);
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = DotAcc{t + k, 0.0f};
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = acc_fma(x[k], bd, cd);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k].hi + x[k].lo;
    if (s == -1.2345f) g_alu_sink = s;
  }
}

// ----------------------------------------------------- pseudo-densities
// Y[q*npair+p][i][a] = exp(t_q (eps_i - eps_a)) X[p][i][a]
__global__ void scale_amplitudes(const double *__restrict__ X, const double *__restrict__ eo,
                                 const double *__restrict__ ev, const double *__restrict__ t,
                                 double *__restrict__ Y, int nlap, int npair, int no, int nv) {
  const size_t per = (size_t)no * nv, total = per * npair * nlap;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const size_t qp = k / per, ia = k % per;
    const int q = (int)(qp / npair), p = (int)(qp % npair);
    const int i = (int)(ia / nv), aa = (int)(ia % nv);
    Y[k] = exp(t[q] * (eo[i] - ev[aa])) * X[(size_t)p * per + ia];
  }
}

// Batched FP64 GEMM with 16x16 tiles, C[b][m][n] = sum_k Aop(b)[m][k] Bop(b)[k][n],
// Aop[m][k] = A[k][m] when TRANSA else A[m][k]; Bop[k][n] = B[n][k] when TRANSB
// else B[k][n].  Row-major, leading dims lda/ldb/ldc.
template <bool TRANSB, bool TRANSA = false>
__global__ void gemm_f64(const double *__restrict__ A, long long strideA,
                         const double *__restrict__ Bm, long long strideB, double *__restrict__ C,
                         long long strideC, int M, int Nn, int Kd, int lda, int ldb, int ldc) {
  __shared__ double As[16][17], Bs[16][17];  // As[m][k], Bs[k][n]
  const int b = blockIdx.z;
  const double *Ab = A + b * strideA, *Bb = Bm + b * strideB;
  double *Cb = C + b * strideC;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int m0 = blockIdx.y * 16, n0 = blockIdx.x * 16;
  double acc = 0.0;
  for (int k0 = 0; k0 < Kd; k0 += 16) {
    if (TRANSA)  // thread (tx,ty) reads A[k0+ty][m0+tx] (coalesced in tx) -> As[m=tx][k=ty]
      As[tx][ty] = (k0 + ty < Kd && m0 + tx < M) ? Ab[(size_t)(k0 + ty) * lda + m0 + tx] : 0.0;
    else
      As[ty][tx] = (m0 + ty < M && k0 + tx < Kd) ? Ab[(size_t)(m0 + ty) * lda + k0 + tx] : 0.0;
    if (TRANSB)  // thread (tx,ty) reads B[n0+ty][k0+tx] (coalesced in tx) -> Bs[k=tx][n=ty]
      Bs[tx][ty] = (n0 + ty < Nn && k0 + tx < Kd) ? Bb[(size_t)(n0 + ty) * ldb + k0 + tx] : 0.0;
    else         // thread (tx,ty) reads B[k0+ty][n0+tx] -> Bs[k=ty][n=tx]
      Bs[ty][tx] = (k0 + ty < Kd && n0 + tx < Nn) ? Bb[(size_t)(k0 + ty) * ldb + n0 + tx] : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(As[ty][k], Bs[k][tx], acc);
    __syncthreads();
  }
  if (m0 + ty < M && n0 + tx < Nn) Cb[(size_t)(m0 + ty) * ldc + n0 + tx] = acc;
}

// M = cJ J + cK K, elementwise.
__global__ void combine_jk(const double *__restrict__ J, const double *__restrict__ K, double cJ,
                           double cK, double *__restrict__ M, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    M[t] = cJ * J[t] + cK * K[t];
}

}  // namespace ltjk
