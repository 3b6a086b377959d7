// Double-word ("double-FP32") arithmetic: a value is the unevaluated sum hi + lo of two floats.
//
// GB300 runs FP32 FMAs about 60x faster than FP64 FMAs, so the FP64-accurate operator kernels do
// their arithmetic on pairs of floats.  The building blocks are the error-free transformations
// TwoSum (Knuth, TAOCP vol. 2; Moller 1965), Fast2Sum (Dekker 1971) and the FMA-based TwoProd, as
// analysed for double-word arithmetic by Joldes, Muller and Popescu ("Tight and rigorous error
// bounds for basic building blocks of double-word arithmetic", ACM TOMS 44(2), 2017).
//
// The operators here are "lazy": the sum of the high parts is exact (TwoSum) and the low parts
// are added in FP32 without renormalising the pair afterwards.  The absolute error of each
// operation is then O(u^2 (|x| + |y|)) with u = 2^-24, which is what a sum of element
// contributions needs (the FP64 tolerance is relative to the norm of the whole result, not to
// each cancelled intermediate).  Pairs are renormalised only where they leave the kernel.
//
// All operations use the explicitly rounded intrinsics so the compiler cannot contract or
// reassociate them.
#pragma once

#include <stdint.h>

namespace dwa {

struct dw {
  float h, l;
};

__device__ __forceinline__ dw make(float h, float l = 0.0f) { return dw{h, l}; }

// TwoSum: s + t == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t) {
  s = __fadd_rn(a, b);
  const float ap = __fsub_rn(s, b);
  const float bp = __fsub_rn(s, ap);
  t = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// Fast2Sum (requires |a| >= |b| or a == 0): s + t == a + b exactly.
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &t) {
  s = __fadd_rn(a, b);
  t = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dw add(dw x, dw y) {
  float s, t;
  two_sum(x.h, y.h, s, t);
  return dw{s, __fadd_rn(__fadd_rn(x.l, y.l), t)};
}

__device__ __forceinline__ dw sub(dw x, dw y) {
  float s, t;
  two_sum(x.h, -y.h, s, t);
  return dw{s, __fadd_rn(__fsub_rn(x.l, y.l), t)};
}

__device__ __forceinline__ dw neg(dw x) { return dw{-x.h, -x.l}; }

// x * y; the lo*lo term (relative size u^2) is dropped.
__device__ __forceinline__ dw mul(dw x, dw y) {
  const float p = __fmul_rn(x.h, y.h);
  const float e = __fmaf_rn(x.h, y.h, -p);
  return dw{p, __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, e))};
}

// x / y (the division of Joldes, Muller and Popescu 2017, Alg. 17 "DWDivDW2"): quotient of the high
// parts, one correction step on the DW remainder.
__device__ __forceinline__ dw div(dw x, dw y) {
  const float th = __fdiv_rn(x.h, y.h);
  const float p = __fmul_rn(y.h, th);
  const float pe = __fmaf_rn(y.h, th, -p);
  const float pl = __fmaf_rn(y.l, th, pe);  // y * th = p + pl
  float s, t;
  two_sum(x.h, -p, s, t);
  const float rem = __fadd_rn(s, __fadd_rn(__fsub_rn(t, pl), x.l));
  const float tl = __fdiv_rn(rem, y.h);
  float zh, zl;
  fast_two_sum(th, tl, zh, zl);
  return dw{zh, zl};
}

// x * 2^k (exact for both parts in the normal range).
__device__ __forceinline__ dw scale(dw x, float pow2) { return dw{__fmul_rn(x.h, pow2), __fmul_rn(x.l, pow2)}; }

// Renormalise so that |lo| <= ulp(hi)/2.
__device__ __forceinline__ dw norm(dw x) {
  float s, t;
  two_sum(x.h, x.l, s, t);
  return dw{s, t};
}

// --------------------------------------------------------------------------- conversions ----

// double -> (hi, lo) with integer operations only (the FP64 pipe of GB300 is the scarce unit):
// hi keeps the leading 24 significand bits (truncated), lo is the remaining 29 bits rounded to a
// float; |x - (hi + lo)| <= 2^-48 |x|.  Zeros give a signed zero pair; other values outside
// [2^-74, 2^127) and non-finite values take the FP64 conversion path.
__device__ __forceinline__ dw split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned bh = (unsigned)(b >> 32), bl = (unsigned)b;
  const int e = (int)((bh >> 20) & 0x7ffu);
  if ((e != 0 && e < 949) || e > 1150) {  // rare: tiny non-zero or huge magnitudes
    const float h = __double2float_rz(x);
    return dw{h, __double2float_rn(x - (double)h)};
  }
  // zeros (and subnormal doubles, below 2^-1022) become a signed zero pair by selects, so that
  // lanes holding zeros do not diverge from the others
  const unsigned sign = bh & 0x80000000u;
  const unsigned mhi = ((bh & 0x000fffffu) << 3) | (bl >> 29);
  const unsigned hb = sign | ((unsigned)(e - 1023 + 127) << 23) | mhi;
  const unsigned rem = bl & 0x1fffffffu;
  const float lo = __fmul_rn(__uint2float_rn(rem), __uint_as_float((unsigned)(e - 1075 + 127) << 23));
  const unsigned lb = __float_as_uint(lo) | sign;
  return dw{__uint_as_float(e == 0 ? sign : hb), __uint_as_float(e == 0 ? sign : lb)};
}

// split() without its out-of-range path: exact for |x| in [2^-74, 2^127) (biased exponent e in
// [949, 1150]) and zeros; the biased exponent field is returned in e so that the caller can check
// the range itself (any other input gives an unspecified pair).
__device__ __forceinline__ dw split_fast(double x, unsigned &e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned bh = (unsigned)(b >> 32), bl = (unsigned)b;
  e = (bh >> 20) & 0x7ffu;
  const unsigned sign = bh & 0x80000000u;
  const unsigned hb = sign | ((e - 1023u + 127u) << 23) | ((bh & 0x000fffffu) << 3) | (bl >> 29);
  const float lo = __fmul_rn(__uint2float_rn(bl & 0x1fffffffu), __uint_as_float((e - 1075u + 127u) << 23));
  const unsigned lb = __float_as_uint(lo) | sign;
  return dw{__uint_as_float(e == 0u ? sign : hb), __uint_as_float(e == 0u ? sign : lb)};
}

// float -> double exactly by bit manipulation, without branches (lanes of a warp often differ in
// whether the low part of a pair is zero): normal floats are rebiased; zeros and subnormals give a
// signed zero (a subnormal low part is below 2^-126 of nothing that matters here), infinities and
// NaNs keep their class (exponent all ones, payload shifted like the mantissa).
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned sign = u & 0x80000000u, mant = u & 0x7fffffu;
  const unsigned ed = e == 0xffu ? 0x7ffu : e + 896u;
  unsigned hi = sign | (ed << 20) | (mant >> 3);
  unsigned lo = u << 29;
  hi = e == 0u ? sign : hi;
  lo = e == 0u ? 0u : lo;
  return __hiloint2double((int)hi, (int)lo);
}

// (hi, lo) -> nearest double: one FP64 add.
__device__ __forceinline__ double to_double(dw x) { return __dadd_rn(f2d(x.h), f2d(x.l)); }

// ------------------------------------------------------------ power-of-two range scaling ----
// The double-word kernels work in FP32's exponent range.  Inputs outside it are brought in by an
// exact power-of-two scaling (x * 2^-s before the split, y * 2^s after the final add); these helpers
// do that scaling and record the magnitude of the inputs a CTA has read.

// 2^k as a double, k in [-1022, 1023].
__device__ __forceinline__ double pow2d(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// v * 2^k exactly (up to FP64's own underflow and overflow), |k| <= 2044.  Normal values whose
// result stays normal take two integer operations on the exponent field; zeros, subnormals,
// non-finite values and results leaving the normal range take two FP64 multiplies.
__device__ __forceinline__ double ldexp_exact(double v, int k) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e != 0 && e != 0x7ff && e + k >= 1 && e + k <= 2046) return __longlong_as_double(b + ((long long)k << 52));
  const int k1 = k / 2, k2 = k - k1;
  return __dmul_rn(__dmul_rn(v, pow2d(k1)), pow2d(k2));
}

// float v * 2^k, |k| <= 252 (FP32 results keep FP32's range).
__device__ __forceinline__ float ldexpf_exact(float v, int k) {
  const int k1 = k / 2, k2 = k - k1;
  return __fmul_rn(__fmul_rn(v, __uint_as_float((unsigned)(k1 + 127) << 23)), __uint_as_float((unsigned)(k2 + 127) << 23));
}

// split(x * 2^-s): the scaled value as a pair.  Values that are below 2^-74 after the scaling
// (negligible next to the CTA's largest input, which the scaling brings to [1, 2)) become zero.
__device__ __forceinline__ dw split_scaled(double x, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffu);
  const int es = e - s;
  if (e == 0 || e == 0x7ff || es < 949 || es > 1150) {
    const double xs = ldexp_exact(x, -s);
    if (!(fabs(xs) >= 0x1p-74)) {  // also zeros; NaN stays NaN through the FP32 conversion below
      if (xs == xs) return dw{__uint_as_float((unsigned)(b >> 32) & 0x80000000u), 0.0f};
    }
    const float h = __double2float_rz(xs);
    return dw{h, __double2float_rn(xs - (double)h)};
  }
  const unsigned bh = (unsigned)(b >> 32), bl = (unsigned)b;
  const unsigned sign = bh & 0x80000000u;
  const unsigned mhi = ((bh & 0x000fffffu) << 3) | (bl >> 29);
  const unsigned hb = sign | ((unsigned)(es - 1023 + 127) << 23) | mhi;
  const unsigned rem = bl & 0x1fffffffu;
  const float lo = __fmul_rn(__uint2float_rn(rem), __uint_as_float((unsigned)(es - 1075 + 127) << 23));
  return dw{__uint_as_float(hb), __uint_as_float(__float_as_uint(lo) | sign)};
}

// split(x * 2^-s) for any s, one code path: s = 0 gives exactly split(x).  With s != 0, values
// below 2^-74 after the scaling become zero (see split_scaled).
__device__ __forceinline__ dw split_shift(double x, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffu);
  const int es = e - s;
  if ((e != 0 && (es < 949 || es > 1150)) || (e == 0 && s != 0)) {
    const double xs = s == 0 ? x : ldexp_exact(x, -s);
    if (s != 0 && !(fabs(xs) >= 0x1p-74) && xs == xs)
      return dw{__uint_as_float((unsigned)(b >> 32) & 0x80000000u), 0.0f};
    const float h = __double2float_rz(xs);
    return dw{h, __double2float_rn(xs - (double)h)};
  }
  const unsigned bh = (unsigned)(b >> 32), bl = (unsigned)b;
  const unsigned sign = bh & 0x80000000u;
  const unsigned mhi = ((bh & 0x000fffffu) << 3) | (bl >> 29);
  const unsigned hb = sign | ((unsigned)(es - 1023 + 127) << 23) | mhi;
  const unsigned rem = bl & 0x1fffffffu;
  const float lo = __fmul_rn(__uint2float_rn(rem), __uint_as_float((unsigned)(es - 1075 + 127) << 23));
  const unsigned lb = __float_as_uint(lo) | sign;
  return dw{__uint_as_float(e == 0 ? sign : hb), __uint_as_float(e == 0 ? sign : lb)};
}

// Magnitude record of the inputs a thread has read, in one register: the largest high word of |x|
// (exponent and leading mantissa bits, ordered like |x|), with bit 0 also set for any input whose
// low word is non-zero (so that inputs below 2^-1042, whose high word is zero, still count).
struct MagRec {
  unsigned key = 0u;
  __device__ __forceinline__ void add(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    key = max(key, ((unsigned)(b >> 32) & 0x7fffffffu) | ((unsigned)b != 0u ? 1u : 0u));
  }
};

// Exponent s with max |x| < 2^(s+1) and, for normal inputs, 2^s <= max |x| (inputs below 2^-1042 are
// given s = -1043); false when every input was zero or one of them was not finite.
__device__ __forceinline__ bool mag_exponent(unsigned key, int &s) {
  const int e = (int)(key >> 20);
  if (e == 0x7ff || key == 0u) return false;
  if (e != 0) s = e - 1023;
  else if (key > 1u) s = -1042 + (31 - __clz(key & 0xfffffu));
  else s = -1043;
  return true;
}

// Window of input magnitudes (exponent of the CTA's largest |x|) in which the double-word kernels
// keep FP64 accuracy without rescaling, given cell constants and spacings normalised at setup.
constexpr int kMagLo = -72, kMagHi = 40;

// Quick test on a thread's own record: some input was non-zero and the largest is outside the window
// (or not finite; the caller then looks at the whole CTA with mag_exponent).
__device__ __forceinline__ bool mag_outside(unsigned key) {
  const unsigned e = key >> 20;
  return key != 0u && (e < (unsigned)(1023 + kMagLo) || e > (unsigned)(1023 + kMagHi));
}

// Host/device-agnostic split of a double constant (setup and constants, not hot paths).
__host__ __device__ inline dw from_double_slow(double x) {
  const float h = (float)x;
  return dw{h, (float)(x - (double)h)};
}

}  // namespace dwa
