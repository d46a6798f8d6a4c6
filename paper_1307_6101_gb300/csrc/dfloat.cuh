// Double-FP32 ("double-single") arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, which carries about 48 significand bits.  The operations are
// the error-free transformations of Dekker (1971, "A floating-point technique for extending the
// available precision") and Knuth (TAOCP vol. 2, two-sum), with the exact product error taken
// from an FMA:
//   two_sum(a, b):       s = a + b, e = (a - (s - v)) + (b - v) with v = s - a   (s + e = a + b exactly)
//   fast_two_sum(a, b):  s = a + b, e = b - (s - a)                              (|a| >= |b|)
//   two_prod(a, b):      p = a * b, e = fma(a, b, -p)                            (p + e = a * b exactly)
// The sum below is the short ("sloppy") form: one two_sum of the leading parts, the trailing
// parts added in FP32, one renormalisation; its relative error is a few units of 2^-44 unless the
// leading parts cancel.  Used on GB300, whose FP64 rate is 1/64 of its FP32 rate, for the
// outer solver's operator and Gram-Schmidt products when the caller asks for it.
//
// Conversions from FP64 split the bit pattern with integer operations (no FP64 instruction):
// hi keeps the top 24 significand bits (truncation), lo the next 23 bits; magnitudes below
// 2^-80 lose lo and magnitudes below 2^-126 flush to zero (both far below the products that
// matter in the solver's vectors); magnitudes of 2^128 or more become infinite.
#pragma once

#include <cuda_runtime.h>

struct dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ __forceinline__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ constexpr dfl(int v) : hi(float(v)), lo(0.f) {}
  __host__ __device__ __forceinline__ constexpr dfl(float v) : hi(v), lo(0.f) {}
};

__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s, e);
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }

__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// c + a * b: the exact leading product, its error and the cross terms, then one sum with c
__device__ __forceinline__ dfl fma(dfl a, dfl b, dfl c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(c.hi, p);
  const float v = __fsub_rn(s, c.hi);
  float t = __fadd_rn(__fsub_rn(c.hi, __fsub_rn(s, v)), __fsub_rn(p, v));
  t = __fadd_rn(t, __fadd_rn(e, c.lo));
  return df_fast_two_sum(s, t);
}

__device__ __forceinline__ bool operator<(dfl a, dfl b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// FP64 -> double-FP32 by integer operations on the bit pattern
__device__ __forceinline__ dfl df_from_double(double x) {
  const long long bits = __double_as_longlong(x);
  const unsigned hw = (unsigned)((unsigned long long)bits >> 32), lw = (unsigned)bits;
  const int e = (int)((hw >> 20) & 0x7FFu);      // biased FP64 exponent
  const unsigned sign = hw & 0x80000000u;
  if (e <= 896) return dfl(0.f, 0.f);           // below the FP32 normal range (or zero)
  if (e >= 1151) return dfl(__int_as_float((int)(sign | 0x7F800000u)), 0.f);
  const unsigned fh = sign | ((unsigned)(e - 896) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  float lo = 0.f;
  const unsigned r = (lw & 0x1FFFFFFFu) >> 6;   // next 23 significand bits
  if (r != 0u && e >= 943) {
    // r * 2^(e - 1069) with r < 2^23 exact: r + 2^23 formed in the significand, 2^23 subtracted
    const float fr = __fsub_rn(__int_as_float((int)(0x4B000000u | r)), 8388608.0f);
    const float scale = __int_as_float((int)((unsigned)(e - 1069 + 127) << 23));
    lo = __int_as_float(__float_as_int(__fmul_rn(fr, scale)) ^ (int)sign);
  }
  return dfl(__int_as_float((int)fh), lo);
}

__device__ __forceinline__ double df_to_double(dfl a) { return __dadd_rn((double)a.hi, (double)a.lo); }
