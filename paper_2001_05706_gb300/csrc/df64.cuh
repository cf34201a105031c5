// Double-float ("DF64") arithmetic: a real number held as the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, i.e. a 48-bit
// significand, computed entirely on the FP32 pipes.
//
// GB300 executes FP64 at 1/64 of its FP32 rate (two FP64 FMAs per clock per
// SM against 128 FP32 lanes), which makes the FP64 dslash FP64-ALU-bound at
// about a sixth of the HBM bandwidth.  The same operator in double-float
// arithmetic costs ~15 FP32 instructions per FP64 multiply-add but runs at
// several times the FP64 throughput, with a relative rounding error of about
// 2^-47 per operation (FP64: 2^-53) -- enough for residuals of 1e-10 and for
// the 1e-10 sign function of the overlap operator.  Storage is the same eight
// bytes per real as FP64 (hi, lo as two floats), so a DF64 field has the FP64
// word layout.
//
// The building blocks are the classical error-free transformations:
// Knuth's TwoSum (a + b = s + e exactly, six additions, no ordering
// precondition), Dekker's Fast2Sum (three additions, |a| >= |b|), and the
// FMA form of TwoProduct (a * b = p + e exactly, e = fma(a, b, -p)).  The
// operations below are the "sloppy" double-float sum (the two low parts are
// added without their own TwoSum: error bound relative to |a| + |b|) and the
// product with the lo * lo term dropped, as in the double-double literature
// (Dekker 1971; Hida, Li and Bailey 2001).  Every FP32 step uses an explicit
// _rn intrinsic so the compiler cannot contract it into an FMA or
// reassociate it.
#pragma once

#include <cuda_runtime.h>

namespace lqcd {
// The type and its operations live in a namespace of their own: calls with
// df arguments find them by argument-dependent lookup, while unqualified
// fma(float, float, float) elsewhere in namespace lqcd still resolves to the
// CUDA math function (an fma(df, df, df) declared in lqcd itself would hide
// it and, through df's converting constructors, capture float calls).
namespace dfmath {

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ constexpr df(float v) : hi(v), lo(0.0f) {}
  // round-to-nearest split of a double: hi = fl32(v), lo = fl32(v - hi)
  __host__ __device__ explicit df(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __device__ explicit operator float() const { return __fadd_rn(hi, lo); }
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df(s, e);
}

// s + e = a + b exactly, given |a| >= |b| or a == 0 (Dekker)
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df(s, e);
}

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }

__device__ __forceinline__ df operator+(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the leading product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// a * b + c with one renormalisation
__device__ __forceinline__ df fma(df a, df b, df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df s = df_two_sum(p, c.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

__device__ __forceinline__ df to_f(df v) { return v; }

// Compensated dot-product accumulator (the Dot2 scheme of Ogita, Rump and
// Oishi, 2005, with double-float operands): the leading FP32 sum s takes each
// exact leading product through TwoSum, while the rounding errors and the
// low-order product terms collect in e; one renormalisation at the end.  The
// dependency chain through s is one addition per product instead of a full
// double-float fma, and each product costs 12 FP32 operations instead of 15.
struct dfacc {
  float s, e;
};

__device__ __forceinline__ void dfacc_madd(dfacc &a, df x, df y) {  // a += x * y
  const float p = __fmul_rn(x.hi, y.hi);
  float pe = __fmaf_rn(x.hi, y.hi, -p);
  pe = __fmaf_rn(x.hi, y.lo, pe);
  pe = __fmaf_rn(x.lo, y.hi, pe);
  const df t = df_two_sum(a.s, p);
  a.s = t.hi;
  a.e = __fadd_rn(a.e, __fadd_rn(t.lo, pe));
}

__device__ __forceinline__ df dfacc_value(dfacc a) {
  const df t = df_two_sum(a.s, a.e);
  return t;
}

// acc + x with the low parts summed lazily: TwoSum of the leading parts, no
// renormalisation (|lo| may grow to a few ulp of hi over a handful of
// additions; the next multiplication or df operation absorbs it)
__device__ __forceinline__ df df_lazy_add(df acc, df x) {
  const df t = df_two_sum(acc.hi, x.hi);
  return df(t.hi, __fadd_rn(acc.lo, __fadd_rn(t.lo, x.lo)));
}

// s * a for s = +-1 (or any power of two): exact, two multiplications
__device__ __forceinline__ df sgn_mul(df s, df a) { return df(__fmul_rn(s.hi, a.hi), __fmul_rn(s.hi, a.lo)); }

}  // namespace dfmath
using dfmath::df;
using dfmath::dfacc;

}  // namespace lqcd
