// Double-float arithmetic and integer-only FP64 <-> (FP32, FP32) conversions
// for the sliced FP64 path.  A double-float pair (h, l) stands for h + l with
// |l| < ulp(h); products and sums use the error-free transformations of
// Dekker ("A floating-point technique for extending the available precision",
// Numer. Math. 18, 1971) and Knuth (TwoSum), with FMA for the product error,
// which keeps about 2^-47 relative accuracy per operation.  The conversions
// work on the bit patterns so that the FP64 pipe is not used.
#pragma once
#include <stdint.h>

namespace w2 {

// m * 2^x as FP64 (m truncated to 53 bits; below the normal range: signed zero;
// above it: signed infinity).
__device__ __forceinline__ double ll_to_double_scaled(long long v, int x) {
  if (v == 0) return 0.0;
  const unsigned long long sg = (unsigned long long)v & 0x8000000000000000ull;
  const unsigned long long m = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int top = 63 - __clzll((long long)m);
  const unsigned long long mant = top > 52 ? (m >> (top - 52)) : (m << (52 - top));
  const int be = top + x + 1023;
  if (be <= 0) return __longlong_as_double((long long)sg);
  if (be > 2046) return __longlong_as_double((long long)(sg | 0x7ff0000000000000ull));
  return __longlong_as_double((long long)(sg | ((unsigned long long)be << 52) | (mant & 0xfffffffffffffull)));
}

// s + e = a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b for |a| >= |b| (Dekker's Fast2Sum).
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// ph + pe ~ (xh + xl)(yh + yl): the exact product of the high parts plus the
// cross terms (the xl yl term is below 2^-48 of the product).
__device__ __forceinline__ void df_mul(float xh, float xl, float yh, float yl, float &ph, float &pe) {
  ph = __fmul_rn(xh, yh);
  pe = __fmaf_rn(xh, yh, -ph);
  pe = __fmaf_rn(xh, yl, pe);
  pe = __fmaf_rn(xl, yh, pe);
}

// (sh, se) += (ph, pe), leaving the pair unnormalised.
__device__ __forceinline__ void df_acc(float &sh, float &se, float ph, float pe) {
  float t;
  two_sum(sh, ph, sh, t);
  se = __fadd_rn(se, __fadd_rn(t, pe));
}

// FP64 -> (h, l): h is v truncated to 24 significant bits, l the next 24 bits
// rounded to nearest.  |v| below 2^-126 flushes to a signed zero (and l below
// the FP32 normal range to zero); Inf, NaN and |v| >= 2^128 give h = Inf/NaN.
__device__ __forceinline__ float2 df_split(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = b & 0xfffffffffffffull;
  const int fe = e - 896;  // FP32 biased exponent of v
  if (fe <= 0) return make_float2(__uint_as_float(sgn), 0.f);
  if (fe >= 255) return make_float2(__uint_as_float(sgn | 0x7f800000u | (e == 2047 && m ? 0x400000u : 0u)), 0.f);
  const float h = __uint_as_float(sgn | ((unsigned)fe << 23) | (unsigned)(m >> 29));
  const unsigned r = (unsigned)(m & 0x1fffffffu);  // the 29 bits below h, unit 2^(e - 1075)
  float l = 0.f;
  if (r) {
    const int p = 31 - __clz(r);
    const int el = p + fe - 52;  // FP32 biased exponent of l
    if (el > 0) {
      const unsigned mant = p <= 23 ? (r << (23 - p)) : ((r + (1u << (p - 24))) >> (p - 23));
      l = __uint_as_float(sgn | (((unsigned)(el - 1) << 23) + mant));  // a carry of mant moves the exponent
    }
  }
  return make_float2(h, l);
}

// (h, l) -> FP64 h + l (exact up to the last 2^-52; integer operations only:
// zero and subnormal parts count as zero, Inf and NaN pass through).
__device__ __forceinline__ double df_join_general(float h, float l) {
  unsigned hb = __float_as_uint(h), lb = __float_as_uint(l);
  int eh = (int)((hb >> 23) & 0xff), el = (int)((lb >> 23) & 0xff);
  if (el > eh) {  // not normalised (|l| > |h|): take the larger part as the base
    const unsigned tb = hb;
    hb = lb;
    lb = tb;
    const int te = eh;
    eh = el;
    el = te;
  }
  const unsigned long long sg = (unsigned long long)(hb >> 31) << 63;
  if (eh == 0) return __longlong_as_double((long long)sg);
  if (eh == 255)  // Inf or NaN: same class in FP64
    return __longlong_as_double((long long)(sg | 0x7ff0000000000000ull | ((hb & 0x7fffffu) ? 0x8000000000000ull : 0ull)));
  long long s = (long long)((hb & 0x7fffffu) | 0x800000u) * (1ll << 29);  // unit 2^(eh - 179)
  if (hb >> 31) s = -s;
  if (el != 0) {
    long long m = (long long)((lb & 0x7fffffu) | 0x800000u);
    if (lb >> 31) m = -m;
    const int d = eh - el;  // >= 0
    if (d <= 29)
      s += m * (1ll << (29 - d));
    else if (d < 29 + 25)
      s += m >> (d - 29);
  }
  return ll_to_double_scaled(s, eh - 179);
}

// The same for a normalised pair (|l| <= ulp(h) / 2, as Fast2Sum leaves it),
// the common case, in a few integer operations: h + l keeps h's exponent or
// drops it by one, so no leading-zero count is needed.
__device__ __forceinline__ double df_join(float h, float l) {
  const unsigned hb = __float_as_uint(h), lb = __float_as_uint(l);
  const int eh = (int)((hb >> 23) & 0xff), el = (int)((lb >> 23) & 0xff);
  const int d = eh - el;
  if (eh == 0 || eh == 255 || (el != 0 && d < 24)) return df_join_general(h, l);
  unsigned long long M = (unsigned long long)((hb & 0x7fffffu) | 0x800000u) << 29;  // 53 bits, unit 2^(eh - 179)
  if (el != 0 && d < 29 + 25) {
    const unsigned long long ml = (unsigned long long)((lb & 0x7fffffu) | 0x800000u);
    const unsigned long long lv = d <= 29 ? ml << (29 - d) : ml >> (d - 29);  // < 2^29
    M = ((hb ^ lb) >> 31) ? M - lv : M + lv;
  }
  int be = eh + 896;
  if (M < (1ull << 52)) {  // a borrow from a power of two: one place down
    M <<= 1;
    --be;
  }
  return __longlong_as_double((long long)(((unsigned long long)(hb >> 31) << 63) | ((unsigned long long)be << 52) |
                                          (M & 0xfffffffffffffull)));
}

}  // namespace w2
