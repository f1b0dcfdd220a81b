// Class-specialised J/K kernel for the light value classes (gen_class()).
//
// The interpreted kernel (kernels.cuh) spends most of a light quartet's time
// decoding recurrence steps, round-tripping shared-memory slots and running
// its class-agnostic digestion.  Here every class is its own kernel,
// instantiated from the straight-line recurrences that csrc/gen_main.cpp
// writes at build time:
//
//   * one thread per contracted quartet: a warp takes one work item (a bra
//     pair and up to 32 Schwarz-kept ket pairs of one class); each lane runs
//     the primitive quartets of its ket in registers -- set-up, Boys
//     function, vertical recurrence and accumulation (Obara-Saika), then the
//     horizontal recurrence (Head-Gordon-Pople) on the contracted values;
//   * the warp then digests its 32 integral blocks with compile-time block
//     sizes: lanes run over (ket, density) units, each unit applying the nine
//     placements that depend on the ket (Eq. quartet_scatter with every
//     permutational image of the unique quartet: the ket half of J and the
//     eight exchange images); the bra half of J is summed over all kets of the
//     item before its one atomic per output element and density.
//
// Arithmetic: Real = dflt (FP64 class: double-float set-up, recurrences and
// digestion), float (mixed mode's binary32 quartets: double-float set-up
// rounded to binary32) or double (IEEE binary64 throughout).  The Boys
// function is evaluated in double-float for dflt and float (binary64 class,
// about 2^-44 relative), in binary64 for double.  Accumulation across
// quartets is binary64 (atomics).  Included by context.cu only.
#pragma once
#include <type_traits>

#include "kernels.cuh"

#define LTJK_GEN_FN __device__ __forceinline__
#include "gen_classes.inc"

namespace ltjk {

constexpr int kPrimDf = 9;  // per primitive pair: zeta, 1/zeta, P[3], P - A[3], prefactor

// ------------------------------------------------- primitive quartet set-up
struct PrimDf {
  dflt zeta, izeta, P[3], PA[3], pref;
};
__device__ __forceinline__ PrimDf load_prim_df(const float2 *__restrict__ p) {
  PrimDf r;
  r.zeta = df_load(p + 0);
  r.izeta = df_load(p + 1);
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    r.P[x] = df_load(p + 2 + x);
    r.PA[x] = df_load(p + 5 + x);
  }
  r.pref = df_load(p + 8);
  return r;
}
struct Prim64 {
  double zeta, izeta, P[3], PA[3], pref;
};
__device__ __forceinline__ Prim64 load_prim_64(const double *__restrict__ p) {
  Prim64 r;
  r.zeta = __ldg(p + 0);
  r.izeta = __ldg(p + 1);
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    r.P[x] = __ldg(p + 2 + x);
    r.PA[x] = __ldg(p + 5 + x);
  }
  r.pref = __ldg(p + 8);
  return r;
}

// Base values base[m] = [00|00]^(m) = pref_a pref_c sqrt(1/(zeta+eta)) F_m(rho |PQ|^2)
// (the pair prefactors carry 2 pi^{5/2} K c c / zeta), the Obara-Saika
// coefficients cf[] (CoefSlot order: P - A, Q - C, W - P = -eta/(zeta+eta) (P - Q),
// W - Q = zeta/(zeta+eta) (P - Q), rho/zeta, rho/eta) and h[] = n/(2 zeta),
// n/(2 eta), n/(2 (zeta+eta)) for n < NH.  Entries a class does not read are
// dead code after inlining.
template <typename Real, int LTOT, int NH>
__device__ __forceinline__ void gen_setup_df(const PrimDf &a, const PrimDf &c, const float2 *boys,
                                             Real *base, Real *cf, Real *h) {
  const dflt isum = df_recip(a.zeta + c.zeta);
  const dflt es = c.zeta * isum;  // rho / zeta
  const dflt zs = a.zeta * isum;  // rho / eta
  dflt PQ[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) PQ[x] = a.P[x] - c.P[x];
  const dflt pq2 = fma(PQ[2], PQ[2], fma(PQ[1], PQ[1], PQ[0] * PQ[0]));
  dflt F[LTOT + 1];
  boys_df<LTOT>((a.zeta * es) * pq2, boys, F);
  const dflt pre = a.pref * c.pref * df_sqrt(isum);
#pragma unroll
  for (int m = 0; m <= LTOT; ++m) base[m] = df_cvt<Real>(pre * F[m]);
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    cf[kPAx + x] = df_cvt<Real>(a.PA[x]);
    cf[kQCx + x] = df_cvt<Real>(c.PA[x]);
    cf[kWPx + x] = df_cvt<Real>(-(es * PQ[x]));
    cf[kWQx + x] = df_cvt<Real>(zs * PQ[x]);
  }
  cf[kRhoZeta] = df_cvt<Real>(es);
  cf[kRhoEta] = df_cvt<Real>(zs);
#pragma unroll
  for (int n = 0; n < NH; ++n) {
    h[n] = df_cvt<Real>(df_mulf(a.izeta, 0.5f * n));
    h[NH + n] = df_cvt<Real>(df_mulf(c.izeta, 0.5f * n));
    h[2 * NH + n] = df_cvt<Real>(df_mulf(isum, 0.5f * n));
  }
}

template <int LTOT, int NH>
__device__ __forceinline__ void gen_setup_64(const Prim64 &a, const Prim64 &c, const double *boys,
                                             double *base, double *cf, double *h) {
  const double isum = 1.0 / (a.zeta + c.zeta);
  const double es = c.zeta * isum, zs = a.zeta * isum;
  double PQ[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) PQ[x] = a.P[x] - c.P[x];
  const double pq2 = fma(PQ[2], PQ[2], fma(PQ[1], PQ[1], PQ[0] * PQ[0]));
  double F[kBoysMaxM + 1];
  boys_eval(LTOT, (a.zeta * es) * pq2, boys, F);
  const double pre = a.pref * c.pref * sqrt(isum);
#pragma unroll
  for (int m = 0; m <= LTOT; ++m) base[m] = pre * F[m];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    cf[kPAx + x] = a.PA[x];
    cf[kQCx + x] = c.PA[x];
    cf[kWPx + x] = -(es * PQ[x]);
    cf[kWQx + x] = zs * PQ[x];
  }
  cf[kRhoZeta] = es;
  cf[kRhoEta] = zs;
#pragma unroll
  for (int n = 0; n < NH; ++n) {
    h[n] = 0.5 * n * a.izeta;
    h[NH + n] = 0.5 * n * c.izeta;
    h[2 * NH + n] = 0.5 * n * isum;
  }
}

// Classes whose contracted accumulators and output block live in shared
// memory (one column per lane) rather than in registers: with the recurrence
// temporaries, the accumulators of a total angular momentum of 4 or more,
// and of (pp|ps), would need 170-250 registers in double-float.
template <int LA, int LB, int LC, int LD>
constexpr bool kGenSmemAcc = LA + LB + LC + LD >= 4 || (LA == 1 && LB == 1 && LC == 1);

// Accumulate the contracted values [e0|f0] of quartet (bra pair ip | ket
// pair jp) into acc[AS * i] over all primitive quartets (acc zeroed first).
template <typename Real, int LA, int LB, int LC, int LD, int AS>
__device__ __forceinline__ void gen_contract(const DevBasis &B, int ip, int jp, Real *acc) {
  using G = GenClass<LA, LB, LC, LD>;
  constexpr int LT = G::kLtot, NH = G::kNh;
#pragma unroll
  for (int t = 0; t < G::kAcc; ++t) acc[AS * t] = zero_real<Real>();
  const int pp0 = __ldg(B.pair_pp0 + ip), npp = __ldg(B.pair_npp + ip);
  const int qq0 = __ldg(B.pair_pp0 + jp), nqq = __ldg(B.pair_npp + jp);
  for (int ia = pp0; ia < pp0 + npp; ++ia) {
    if constexpr (std::is_same<Real, double>::value) {
      const Prim64 pa = load_prim_64(B.ppg + (size_t)kPrimDf * ia);
      for (int ic = qq0; ic < qq0 + nqq; ++ic) {
        const Prim64 pc = load_prim_64(B.ppg + (size_t)kPrimDf * ic);
        double base[LT + 1], cf[kNumCoef], h[3 * NH];
        gen_setup_64<LT, NH>(pa, pc, B.boys, base, cf, h);
        G::template vrr<double, AS>(base, cf, h, acc);
      }
    } else {
      const PrimDf pa = load_prim_df(B.ppg2 + (size_t)kPrimDf * ia);
      for (int ic = qq0; ic < qq0 + nqq; ++ic) {
        const PrimDf pc = load_prim_df(B.ppg2 + (size_t)kPrimDf * ic);
        Real base[LT + 1], cf[kNumCoef], h[3 * NH];
        gen_setup_df<Real, LT, NH>(pa, pc, B.boys2, base, cf, h);
        G::template vrr<Real, AS>(base, cf, h, acc);
      }
    }
  }
}

// Horizontal recurrence of quartet (ip | jp): acc[AS * i] -> out[OS * o].
template <typename Real, int LA, int LB, int LC, int LD, int AS, int OS>
__device__ __forceinline__ void gen_transfer(const DevBasis &B, int ip, int jp, const Real *acc, Real *out) {
  const int2 sab = __ldg(B.pair_sh + ip), scd = __ldg(B.pair_sh + jp);
  Real X[6];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    if constexpr (std::is_same<Real, double>::value) {
      X[x] = __ldg(B.sh_ctr + 3 * sab.x + x) - __ldg(B.sh_ctr + 3 * sab.y + x);
      X[3 + x] = __ldg(B.sh_ctr + 3 * scd.x + x) - __ldg(B.sh_ctr + 3 * scd.y + x);
    } else {
      X[x] = df_cvt<Real>(df_load(B.ctr2 + 3 * sab.x + x) - df_load(B.ctr2 + 3 * sab.y + x));
      X[3 + x] = df_cvt<Real>(df_load(B.ctr2 + 3 * scd.x + x) - df_load(B.ctr2 + 3 * scd.y + x));
    }
  }
  GenClass<LA, LB, LC, LD>::template hrr<Real, AS, OS>(acc, X, out);
}

// ------------------------------------------------------------ digestion
// Placement of Eq. quartet_scatter: out(R, S) += sum_{t1 in T1, t2 in T2}
// I[r s t1 t2] M(t1, t2), shells named 0..3 = a, b, c, d of the quartet.
struct GenPlace {
  int orow, ocol, srow, scol;
};
// index 0: the ket half of J (against S = D + D^T); 1..8: the exchange images.
// The bra half of J, out (a, b) from S(c, d), is summed over the item's kets.
constexpr GenPlace kGenPlace[9] = {{2, 3, 0, 1}, {0, 2, 1, 3}, {1, 2, 0, 3}, {0, 3, 1, 2}, {1, 3, 0, 2},
                                   {2, 0, 3, 1}, {3, 0, 2, 1}, {2, 1, 3, 0}, {3, 1, 2, 0}};

// One placement for one (ket, density) unit.  Ik: the ket's integrals in the
// warp's shared block, element o at Ik[32 o]; Mb, Tb: the operand and output
// blocks at the unit's density (q-innermost layout, AO row stride mrow,
// column stride nd).  The operand block is read once into registers; every
// output element sums its N1 x N2 terms and is flushed with one atomic.
template <typename Real, int NR, int NS, int N1, int N2, int SR, int SS, int S1, int S2>
__device__ __forceinline__ void gen_place(const Real *__restrict__ Ik, const Real *__restrict__ Mb,
                                          double *__restrict__ Tb, size_t mrow, int nd) {
  using Acc = typename AccOf<Real>::type;
  Real m[N1 * N2];
#pragma unroll
  for (int t1 = 0; t1 < N1; ++t1)
#pragma unroll
    for (int t2 = 0; t2 < N2; ++t2) m[t1 * N2 + t2] = ldg(Mb + t1 * mrow + (size_t)t2 * nd);
  // output loops stay rolled: unrolled, the nine placements of a (pp|ps)
  // unit grew to ~70 KB of code and the warps stalled on instruction fetch
#pragma unroll 1
  for (int r = 0; r < NR; ++r) {
    const Real *Ir = Ik + 32 * r * SR;
    double *Tr = Tb + r * mrow;
#pragma unroll 1
    for (int s = 0; s < NS; ++s) {
      const Real *Irs = Ir + 32 * s * SS;
      Acc acc = acc_zero(Real());
#pragma unroll
      for (int t1 = 0; t1 < N1; ++t1)
#pragma unroll
        for (int t2 = 0; t2 < N2; ++t2) acc = acc_fma(acc, Irs[32 * (t1 * S1 + t2 * S2)], m[t1 * N2 + t2]);
      red_add(Tr + (size_t)s * nd, acc);
    }
  }
}

template <typename Real, int NA, int NB, int NC, int ND, int P>
__device__ __forceinline__ void gen_place_n(const Real *Ik, const Real *M, double *T, const int off[4],
                                            int N, size_t mrow, int nd, int q) {
  constexpr int n[4] = {NA, NB, NC, ND};
  constexpr int st[4] = {NB * NC * ND, NC * ND, ND, 1};
  constexpr GenPlace p = kGenPlace[P];
  const Real *Mb = M + ((size_t)off[p.srow] * N + off[p.scol]) * nd + q;
  double *Tb = T + ((size_t)off[p.orow] * N + off[p.ocol]) * nd + q;
  gen_place<Real, n[p.orow], n[p.ocol], n[p.srow], n[p.scol], st[p.orow], st[p.ocol], st[p.srow],
            st[p.scol]>(Ik, Mb, Tb, mrow, nd);
}

// ---------------------------------------------------------------- kernel
// Shared memory of one warp: the integral blocks of its 32 kets [NOUT][32],
// the kets' AO offsets [32], and (shared-memory classes) the contracted
// accumulators [NACC][32].
template <int NOUT, int NACC, typename Real>
__host__ __device__ constexpr size_t gen_warp_smem() {
  return ((size_t)(NOUT + NACC) * 32 * sizeof(Real) + 32 * sizeof(int2) + 15) / 16 * 16;
}

template <typename Real, int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(128, 4) gen_jk_kernel(const __grid_constant__ JobTable T) {
  constexpr int NA = (LA + 1) * (LA + 2) / 2, NB = (LB + 1) * (LB + 2) / 2;
  constexpr int NC = (LC + 1) * (LC + 2) / 2, ND = (LD + 1) * (LD + 2) / 2;
  constexpr int NOUT = NA * NB * NC * ND;
  constexpr bool SMEM = kGenSmemAcc<LA, LB, LC, LD>;
  constexpr int NACC = SMEM ? GenClass<LA, LB, LC, LD>::kAcc : 0;
  static_assert(NOUT == GenClass<LA, LB, LC, LD>::kOut, "generated block size");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  unsigned char *wbase = smem_raw + (size_t)warp * gen_warp_smem<NOUT, NACC, Real>();
  Real *Ism = reinterpret_cast<Real *>(wbase);                              // [NOUT][32]
  Real *Asm = Ism + NOUT * 32;                                              // [NACC][32]
  int2 *kinfo = reinterpret_cast<int2 *>(wbase + (size_t)(NOUT + NACC) * 32 * sizeof(Real));  // [32]
  for (int it = blockIdx.x * nwarps + warp; it < T.total; it += gridDim.x * nwarps) {
    int jb = 0;
    while (jb + 1 < T.njobs && it >= T.j[jb + 1].first) ++jb;
    const JobDesc &Jd = T.j[jb];
    const DevBasis &B = Jd.B;
    const JKArgs &a = Jd.a;
    const int N = B.nao, nd = a.nd;
    const WorkItem W = Jd.items[it - Jd.first];
    const int nk = W.nk;
    const int2 sab = __ldg(B.pair_sh + W.bra);
    const int a0 = __ldg(B.sh_ao + sab.x), b0 = __ldg(B.sh_ao + sab.y);
    if (lane < nk) {
      const int jp = W.k0 + lane;
      const int2 scd = __ldg(B.pair_sh + jp);
      float wf = 1.0f;  // degeneracy weight of the unique quartet
      if (sab.x == sab.y) wf *= 0.5f;
      if (scd.x == scd.y) wf *= 0.5f;
      if (W.bra == jp) wf *= 0.5f;
      if constexpr (SMEM) {
        gen_contract<Real, LA, LB, LC, LD, 32>(B, W.bra, jp, Asm + lane);
        gen_transfer<Real, LA, LB, LC, LD, 32, 32>(B, W.bra, jp, Asm + lane, Ism + lane);
#pragma unroll 4
        for (int o = 0; o < NOUT; ++o) Ism[32 * o + lane] = scale_pow2(Ism[32 * o + lane], wf);
      } else {
        Real acc[GenClass<LA, LB, LC, LD>::kAcc], out[NOUT];
        gen_contract<Real, LA, LB, LC, LD, 1>(B, W.bra, jp, acc);
        gen_transfer<Real, LA, LB, LC, LD, 1, 1>(B, W.bra, jp, acc, out);
#pragma unroll
        for (int o = 0; o < NOUT; ++o) Ism[32 * o + lane] = scale_pow2(out[o], wf);
      }
      kinfo[lane] = make_int2(__ldg(B.sh_ao + scd.x), __ldg(B.sh_ao + scd.y));
    }
    __syncwarp();
    const size_t mrow = (size_t)N * nd;
    using Acc = typename AccOf<Real>::type;
    if (a.J) {
      // bra half of J: Jh(a, b) += sum over the item's kets of I S(c, d)
      const Real *S = digest_operand<Real>(a, true);
      for (int u = lane; u < NA * NB * nd; u += 32) {
        const int o = u / nd, q = u - o * nd;
        const int x = o / NB, y = o - x * NB;
        Acc acc = acc_zero(Real());
        for (int k = 0; k < nk; ++k) {
          const int2 cd = kinfo[k];
          const Real *Sb = S + ((size_t)cd.x * N + cd.y) * nd + q;
          const Real *Ik = Ism + 32 * (o * NC * ND) + k;
#pragma unroll
          for (int uu = 0; uu < NC; ++uu)
#pragma unroll
            for (int vv = 0; vv < ND; ++vv)
              acc = acc_fma(acc, Ik[32 * (uu * ND + vv)], ldg(Sb + uu * mrow + (size_t)vv * nd));
        }
        red_add(a.J + ((size_t)(a0 + x) * N + b0 + y) * nd + q, acc);
      }
    }
    // the ket-dependent placements, lanes over (ket, density) units
    const Real *Dm = digest_operand<Real>(a, false), *Sm = digest_operand<Real>(a, true);
    for (int u = lane; u < nk * nd; u += 32) {
      const int k = u / nd, q = u - k * nd;
      const int2 cd = kinfo[k];
      const int off[4] = {a0, b0, cd.x, cd.y};
      const Real *Ik = Ism + k;
      if (a.J) gen_place_n<Real, NA, NB, NC, ND, 0>(Ik, Sm, a.J, off, N, mrow, nd, q);
      if (a.K) {
        gen_place_n<Real, NA, NB, NC, ND, 1>(Ik, Dm, a.K, off, N, mrow, nd, q);
        gen_place_n<Real, NA, NB, NC, ND, 2>(Ik, Dm, a.K, off, N, mrow, nd, q);
        gen_place_n<Real, NA, NB, NC, ND, 3>(Ik, Dm, a.K, off, N, mrow, nd, q);
        gen_place_n<Real, NA, NB, NC, ND, 4>(Ik, Dm, a.K, off, N, mrow, nd, q);
        gen_place_n<Real, NA, NB, NC, ND, 5>(Ik, Dm, a.K, off, N, mrow, nd, q);
        gen_place_n<Real, NA, NB, NC, ND, 6>(Ik, Dm, a.K, off, N, mrow, nd, q);
        gen_place_n<Real, NA, NB, NC, ND, 7>(Ik, Dm, a.K, off, N, mrow, nd, q);
        gen_place_n<Real, NA, NB, NC, ND, 8>(Ik, Dm, a.K, off, N, mrow, nd, q);
      }
    }
    __syncwarp();  // the shared block is the next item's
  }
}


}  // namespace ltjk
