// Double-float ("df64") arithmetic for the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats (a 48-bit significand,
// unit roundoff ~2^-48 = 3.6e-15 within float's exponent range).  The kernels
// use it where FP64 accuracy is required, because GB300 issues 64 times more
// FP32 than FP64 operations per clock.
//
// Building blocks (published error-free transformations, written here from
// their definitions):
//   TwoSum (Knuth): s = a + b, e = (a - (s - t)) + (b - t) with t = s - a;
//     s + e == a + b exactly.
//   TwoProd with FMA: p = a*b, e = fma(a, b, -p); p + e == a*b exactly.
// The multiply-add below follows the double-word product and sum of Joldes,
// Muller and Popescu (ACM TOMS 2017): the leading product with its exact error,
// the two cross terms by FMA (the lo*lo term, of relative size 2^-48, is
// dropped), then an exact TwoSum of the leading parts and one float add of the
// remaining tails.  The result is left unnormalised (lo may exceed half an ulp
// of hi after cancellation); every consumer accepts that, and the absolute
// error of a chain of n updates stays O(n * 2^-48 * sum |terms|).  No step
// relies on flush-to-zero or fast-math: the library is compiled without them.
#pragma once

#include <cuda_runtime.h>

namespace wq {

struct dd {
  float hi, lo;
};

__device__ __forceinline__ dd dd_from_double(double x) {
  const float h = (float)x;
  return dd{h, (float)(x - (double)h)};
}

// a*b + c
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) {
  const float ph = a.hi * b.hi;
  float pl = fmaf(a.hi, b.hi, -ph);
  pl = fmaf(a.hi, b.lo, pl);
  pl = fmaf(a.lo, b.hi, pl);
  const float sh = ph + c.hi;
  const float t = sh - ph;
  const float sl = (ph - (sh - t)) + (c.hi - t);
  return dd{sh, sl + (pl + c.lo)};
}

// a + b
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  const float sh = a.hi + b.hi;
  const float t = sh - a.hi;
  const float sl = (a.hi - (sh - t)) + (b.hi - t);
  return dd{sh, sl + (a.lo + b.lo)};
}

// Exact float -> double by bit manipulation on the integer pipe (normal
// numbers, zero, infinities and NaN; float subnormals, below 1.2e-38, are
// treated as zero).
__device__ __forceinline__ double float_to_double_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned s = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned hi_word, lo_word;
  if (e == 0u) {
    hi_word = s;
    lo_word = 0u;
  } else if (e == 0xffu) {
    hi_word = s | 0x7ff00000u | (m >> 3);
    lo_word = m << 29;
  } else {
    hi_word = s | ((e + 896u) << 20) | (m >> 3);
    lo_word = m << 29;
  }
  return __hiloint2double((int)hi_word, (int)lo_word);
}

// hi + lo rounded to double: both parts converted exactly, one FP64 add.
__device__ __forceinline__ double dd_to_double(dd a) {
  return float_to_double_bits(a.hi) + float_to_double_bits(a.lo);
}

// ---------------------------------------------------------------- packed pairs
// Two double-float values side by side for the packed FP32 instructions of
// sm_100 and later (add/sub/fma .f32x2: one instruction issues two lanes
// of FP32 work, halving the issue slots of the arithmetic): hi = (x.hi, y.hi)
// and lo = (x.lo, y.lo) as 64-bit register pairs.  dd2_fma performs dd_fma's
// operations lane by lane, so each lane's result has dd_fma's bits.
struct dd2 {
  unsigned long long hi, lo;
};

__device__ __forceinline__ unsigned long long f2_pack(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long r, float &x, float &y) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(r));
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ dd2 dd2_pack(dd x, dd y) { return dd2{f2_pack(x.hi, y.hi), f2_pack(x.lo, y.lo)}; }
__device__ __forceinline__ dd dd2_first(dd2 a) {
  float h0, h1, l0, l1;
  f2_unpack(a.hi, h0, h1);
  f2_unpack(a.lo, l0, l1);
  return dd{h0, l0};
}
__device__ __forceinline__ dd dd2_second(dd2 a) {
  float h0, h1, l0, l1;
  f2_unpack(a.hi, h0, h1);
  f2_unpack(a.lo, l0, l1);
  return dd{h1, l1};
}
__device__ __forceinline__ dd2 dd2_with_second(dd2 a, dd y) {
  float h0, h1, l0, l1;
  f2_unpack(a.hi, h0, h1);
  f2_unpack(a.lo, l0, l1);
  return dd2{f2_pack(h0, y.hi), f2_pack(l0, y.lo)};
}

// lane-wise a*b + c with dd_fma's operations and bits.  z must be a pair of
// zeros that the compiler cannot see as constants (a value read at run time).
// The leading product is formed as fma(a.hi, b.hi, z) rather than by a packed
// multiply: with a packed multiply (or a literal zero, which lets the compiler
// turn the FMA back into one) the generated code did not keep the product's
// rounding separate from the following add and subtract, and every lane came
// out wrong at single precision; with no packed multiply in the sequence each
// lane has dd_fma's bits (checked over 2^17 random lanes).
__device__ __forceinline__ dd2 dd2_fma(dd2 a, dd2 b, dd2 c, unsigned long long z) {
  const unsigned long long ph = f2_fma(a.hi, b.hi, z);
  unsigned long long pl = f2_fma(a.hi, b.hi, f2_sub(z, ph));
  pl = f2_fma(a.hi, b.lo, pl);
  pl = f2_fma(a.lo, b.hi, pl);
  const unsigned long long sh = f2_add(ph, c.hi);
  const unsigned long long t = f2_sub(sh, ph);
  const unsigned long long sl = f2_add(f2_sub(ph, f2_sub(sh, t)), f2_sub(c.hi, t));
  return dd2{sh, f2_add(sl, f2_add(pl, c.lo))};
}

// ---------------------------------------------------------------- generic helpers
// The row kernels are written once over an arithmetic type R (double, float
// or dd) through these helpers; OutT<R> is the band's storage type.
template <typename R> struct OutT { using type = R; };
template <> struct OutT<dd> { using type = double; };

template <typename R> __device__ __forceinline__ R r_zero() { return R(0); }
template <> __device__ __forceinline__ dd r_zero<dd>() { return dd{0.0f, 0.0f}; }

template <typename R> __device__ __forceinline__ R r_from_double(double x) { return (R)x; }
template <> __device__ __forceinline__ dd r_from_double<dd>(double x) { return dd_from_double(x); }

__device__ __forceinline__ double r_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ dd r_fma(dd a, dd b, dd c) { return dd_fma(a, b, c); }

__device__ __forceinline__ double r_add(double a, double b) { return a + b; }
__device__ __forceinline__ float r_add(float a, float b) { return a + b; }
__device__ __forceinline__ dd r_add(dd a, dd b) { return dd_add(a, b); }

__device__ __forceinline__ double r_shfl_xor(double a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
__device__ __forceinline__ float r_shfl_xor(float a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
__device__ __forceinline__ dd r_shfl_xor(dd a, int o) {
  return dd{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// A band-typed value (OutT<R>) in the arithmetic type R.
template <typename R> __device__ __forceinline__ R r_from_out(typename OutT<R>::type v) { return (R)v; }
template <> __device__ __forceinline__ dd r_from_out<dd>(double v) { return dd_from_double(v); }

__device__ __forceinline__ double r_out(double a) { return a; }
__device__ __forceinline__ float r_out(float a) { return a; }
__device__ __forceinline__ double r_out(dd a) { return dd_to_double(a); }

}  // namespace wq
