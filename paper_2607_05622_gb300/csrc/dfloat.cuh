// Double-float arithmetic on the FP32 pipe, and float<->double conversions
// done with integer bit operations.
//
// GB300 runs FP64 FMAs at 1/58 of the FP32 rate, and its double<->float
// conversions share that slow unit.  The integral recurrences and the density
// digestion therefore run on pairs of floats (hi + lo, ~2^-44 relative per
// operation), using the error-free transformations of Knuth (TwoSum), Dekker
// (FastTwoSum) and the FMA-based TwoProduct, in the "sloppy" double-word
// addition of Hida, Li and Bailey (Library for double-double and quad-double
// arithmetic, 2001), written here for float words.  Every operation uses the
// explicitly rounded intrinsics so the compiler cannot contract or reorder it.
#pragma once
#include <cuda_runtime.h>

namespace ltjk {

// Exact float -> double (zero and subnormal floats map to signed zero).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sgn = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  unsigned hi = sgn | ((e + 896u) << 20) | (m >> 3);  // 1023 - 127 = 896
  unsigned lo = m << 29;
  if (e == 0u) {
    hi = sgn;
    lo = 0u;
  } else if (e == 0xFFu) {
    hi = sgn | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u);
  }
  return __hiloint2double((int)hi, (int)lo);
}

// double -> (hi, lo) floats with hi = x truncated to 24 bits and lo the next
// 24 bits of the remainder (|x - hi - lo| <= 2^-47 |x|), for 2^-126 <= |x| < 2^127;
// smaller magnitudes flush to zero (far below every tolerance here).
__device__ __forceinline__ void d2f_split(double x, float &hi, float &lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const int E = (int)((b >> 52) & 0x7FFu);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const int fe = E - 896;
  if (fe <= 0) {
    hi = 0.0f;
    lo = 0.0f;
    return;
  }
  hi = __uint_as_float(sgn | ((unsigned)fe << 23) | (unsigned)(m >> 29));
  // remainder: (m mod 2^29) * 2^(E - 1075)
  const unsigned r = (unsigned)(m & 0x1FFFFFFFull);
  const int pe = E - 1075 + 127;  // biased float exponent of 2^(E - 1075)
  float rl = 0.0f;
  if (r != 0u && pe >= 1) rl = __uint2float_rn(r) * __uint_as_float((unsigned)pe << 23);
  lo = sgn ? -rl : rl;
}

// float nearest to x (up to 2^-47 relative), for 2^-126 <= |x| < 2^127; tiny values flush to zero.
__device__ __forceinline__ float d2f_bits(double x) {
  float h, l;
  d2f_split(x, h, l);
  return __fadd_rn(h, l);
}

// hi + lo rounded to double with integer operations only (no FP64 add, which
// on this part costs as much as ~60 FP32 instructions).  hi converts exactly;
// lo is added as an integer number of units in the last place of that double
// (half-units rounded away from zero).  Requires |lo| < ulp(hi), which holds for
// every normalised double-float and for the split of a double; then the sum
// never carries out of the mantissa field, and the one borrow (hi a power of
// two, lo of opposite sign) is handled by counting in the half-size units of
// the binade below.
__device__ __forceinline__ double df_to_double(float hi, float lo) {
  const unsigned uh = __float_as_uint(hi), ul = __float_as_uint(lo);
  const int eh = (int)((uh >> 23) & 0xFFu), el = (int)((ul >> 23) & 0xFFu);
  if (eh == 0 || eh == 0xFF) return f2d_bits(hi);
  unsigned long long H = ((unsigned long long)(uh & 0x80000000u) << 32) |
                         ((unsigned long long)(eh + 896) << 52) |
                         ((unsigned long long)(uh & 0x7FFFFFu) << 29);
  if (el == 0) return __longlong_as_double((long long)H);
  const bool opp = ((uh ^ ul) & 0x80000000u) != 0u;
  int s = el - eh + 29;  // |lo| / ulp(H) = mantissa(lo) * 2^s
  if (opp && (uh & 0x7FFFFFu) == 0u) s += 1;
  const unsigned long long ml = (unsigned long long)((ul & 0x7FFFFFu) | 0x800000u);
  unsigned long long off = 0ull;
  if (s >= 0)
    off = ml << s;
  else if (s > -40)
    off = (ml + (1ull << (-s - 1))) >> (-s);
  H = opp ? H - off : H + off;
  return __longlong_as_double((long long)H);
}

struct dflt {
  float hi, lo;
  __device__ __forceinline__ dflt() {}
  __device__ __forceinline__ dflt(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit dflt(double x) { d2f_split(x, hi, lo); }
  __device__ __forceinline__ explicit dflt(int n) : hi((float)n), lo(0.0f) {}
  __device__ __forceinline__ explicit operator double() const { return df_to_double(hi, lo); }
};

// a + b, double-word (two-sum of the leading words, then renormalise)
__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, e);
  return dflt(h, __fsub_rn(e, __fsub_rn(h, s)));
}

// fma overloads for the built-in types (so that the double-float overload
// below does not hide them inside this namespace)
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float fma(float a, float b, float c) { return ::fmaf(a, b, c); }

// a * b + c
__device__ __forceinline__ dflt fma(dflt a, dflt b, dflt c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(p, c.hi);
  const float bb = __fsub_rn(s, p);
  float err = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.hi, bb));
  err = __fadd_rn(err, __fadd_rn(e, c.lo));
  const float h = __fadd_rn(s, err);
  return dflt(h, __fsub_rn(err, __fsub_rn(h, s)));
}

__device__ __forceinline__ dflt operator*(dflt a, dflt b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float h = __fadd_rn(p, e);
  return dflt(h, __fsub_rn(e, __fsub_rn(h, p)));
}
__device__ __forceinline__ dflt operator+(dflt a, dflt b) { return df_add(a, b); }
__device__ __forceinline__ dflt operator-(dflt a, dflt b) { return df_add(a, dflt(-b.hi, -b.lo)); }

// a * f for a float f (exact when f is a small power of two)
__device__ __forceinline__ dflt df_mulf(dflt a, float f) {
  const float p = __fmul_rn(a.hi, f);
  float e = __fmaf_rn(a.hi, f, -p);
  e = __fmaf_rn(a.lo, f, e);
  const float h = __fadd_rn(p, e);
  return dflt(h, __fsub_rn(e, __fsub_rn(h, p)));
}

// 1/a: float reciprocal refined by one double-word Newton step y + y (1 - a y)
__device__ __forceinline__ dflt df_recip(dflt a) {
  const float y0 = __frcp_rn(a.hi);
  const dflt y(y0, 0.0f);
  const dflt r = dflt(1.0f, 0.0f) - a * y;  // residual, small
  return df_add(y, df_mulf(r, y0));
}

// sqrt(a) for a > 0: float root refined by one double-word Newton step
__device__ __forceinline__ dflt df_sqrt(dflt a) {
  const float s0 = __fsqrt_rn(a.hi);
  const dflt s(s0, 0.0f);
  const dflt r = a - s * s;  // residual, small
  return df_add(s, df_mulf(r, __frcp_rn(2.0f * s0)));
}

__device__ __forceinline__ float df_to_float(dflt a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ dflt &operator+=(dflt &a, dflt b) { return a = df_add(a, b); }
__device__ __forceinline__ dflt operator-(dflt a) { return dflt(-a.hi, -a.lo); }
// scaling by a power of two is exact
__device__ __forceinline__ dflt &operator*=(dflt &a, dflt b) { return a = a * b; }

__device__ __forceinline__ dflt ldg(const dflt *p) {
  const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
  return dflt(v.x, v.y);
}
__device__ __forceinline__ double ldg(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ldg(const float *p) { return __ldg(p); }

// Conversions used by the templated kernels.
template <typename Real>
__device__ __forceinline__ Real from_double(double x);
template <>
__device__ __forceinline__ double from_double<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_double<float>(double x) { return d2f_bits(x); }
template <>
__device__ __forceinline__ dflt from_double<dflt>(double x) { return dflt(x); }

__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return f2d_bits(x); }
__device__ __forceinline__ double to_double(dflt x) { return (double)x; }

// Exact scaling by a power of two (the degeneracy weights 1, 1/2, 1/4, 1/8).
__device__ __forceinline__ double scale_pow2(double x, float w) { return x * (double)w; }
__device__ __forceinline__ float scale_pow2(float x, float w) { return x * w; }
__device__ __forceinline__ dflt scale_pow2(dflt x, float w) { return dflt(x.hi * w, x.lo * w); }

// Compensated dot-product accumulator for double-float operands (the
// accumulation of Ogita, Rump and Oishi's Dot2, SIAM J. Sci. Comput. 26, 1955
// (2005), with double-float inputs): the product's leading part is exact by
// FMA TwoProduct, the cross terms join its error, the leading parts are summed
// with Knuth's TwoSum, and all error terms go to `lo` unnormalised.  The only
// dependency from one term to the next is one add on hi and one on lo;
// acc_final renormalises once (~n^2 2^-48 relative for n terms).
struct DotAcc {
  float hi, lo;
};
template <typename Real>
struct AccOf {
  using type = Real;
};
template <>
struct AccOf<dflt> {
  using type = DotAcc;
};
__device__ __forceinline__ double acc_zero(double) { return 0.0; }
__device__ __forceinline__ float acc_zero(float) { return 0.0f; }
__device__ __forceinline__ DotAcc acc_zero(dflt) { return DotAcc{0.0f, 0.0f}; }
__device__ __forceinline__ double acc_fma(double acc, double a, double b) { return ::fma(a, b, acc); }
__device__ __forceinline__ float acc_fma(float acc, float a, float b) { return ::fmaf(a, b, acc); }
__device__ __forceinline__ DotAcc acc_fma(DotAcc acc, dflt a, dflt b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  return DotAcc{s, __fadd_rn(acc.lo, __fadd_rn(err, e))};
}
__device__ __forceinline__ double acc_final(double acc) { return acc; }
__device__ __forceinline__ double acc_final(float acc) { return f2d_bits(acc); }
__device__ __forceinline__ double acc_final(DotAcc acc) {
  // TwoSum renormalisation, then the integer conversion of the pair
  const float s = __fadd_rn(acc.hi, acc.lo);
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(acc.lo, bb));
  return df_to_double(s, err);
}

// Add an accumulated sum into a binary64 element with L2 reductions.  A
// double-float sum goes in as its two words, each converted exactly: the L2
// adds them in binary64, so no renormalisation or integer rounding of the
// pair is needed (two reductions instead of ~25 instructions of conversion).
__device__ __forceinline__ void red_add(double *p, double acc) { atomicAdd(p, acc); }
__device__ __forceinline__ void red_add(double *p, float acc) { atomicAdd(p, f2d_bits(acc)); }
__device__ __forceinline__ void red_add(double *p, DotAcc acc) {
  atomicAdd(p, f2d_bits(acc.hi));
  atomicAdd(p, f2d_bits(acc.lo));
}

template <typename Real>
__device__ __forceinline__ Real zero_real() { return Real(0); }
template <>
__device__ __forceinline__ dflt zero_real<dflt>() { return dflt(0.0f, 0.0f); }

}  // namespace ltjk
