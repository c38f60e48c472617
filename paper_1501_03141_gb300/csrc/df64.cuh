// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits (relative
// rounding error near 2^-47, against 2^-53 for FP64).  On GB300 the FP32
// pipe runs 64x the FP64 rate, so transforms in double-float cost a fraction
// of their FP64 form while keeping errors far below the 1e-10 residuals the
// Sternheimer refinement needs.
//
// The operations are the error-free transformations of Knuth (TwoSum: the
// exact rounding error of an addition, TAOCP vol. 2, Sec. 4.2.2) and Dekker
// (FastTwoSum for |a| >= |b|, and the exact product error, here one fused
// multiply-add; Dekker, Numer. Math. 18, 224 (1971)), combined as in
// double-single / double-double libraries: sum of the high parts with its
// exact error, low parts added, renormalised.  Every FP32 step is an _rn
// intrinsic so that the compiler can neither contract a multiply into a
// later add nor reassociate, either of which would break the exactness the
// algorithms rely on.
#pragma once

#include "common.cuh"

namespace pdep {

struct df {
  float hi, lo;
  df() = default;
  // from a double (constants are folded at compile time)
  __host__ __device__ constexpr df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ double to_double(df a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (Knuth's TwoSum, no ordering assumption)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df(s, e);
}
// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker's FastTwoSum)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }

__device__ __forceinline__ df operator+(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  const float l = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, l);
}
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);            // exact error of the product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ df& operator+=(df& a, df b) {
  a = a + b;
  return a;
}

// c + a b with one rounding of the exact product's error terms: the product's
// high part and c's high part are summed exactly (TwoSum), the product error
// (one FMA per cross term) and the low parts added, then renormalised
__device__ __forceinline__ df fma_df(df a, df b, df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df s = two_sum(p, c.hi);
  const float l = __fadd_rn(s.lo, __fadd_rn(e, c.lo));
  return fast_two_sum(s.hi, l);
}
// acc + a b in the arithmetic of the type (an FMA for float and double)
template <typename R>
__device__ __forceinline__ R mad(R a, R b, R acc) {
  return acc + a * b;
}
template <>
__device__ __forceinline__ df mad<df>(df a, df b, df acc) {
  return fma_df(a, b, acc);
}

// complex helpers the line FFTs need for df (the generic ones use __ldg and
// one shuffle per component)
template <>
__device__ __forceinline__ cpx<df> shfl_xor(cpx<df> a, int m) {
  return mk(df(__shfl_xor_sync(0xffffffffu, a.x.hi, m), __shfl_xor_sync(0xffffffffu, a.x.lo, m)),
            df(__shfl_xor_sync(0xffffffffu, a.y.hi, m), __shfl_xor_sync(0xffffffffu, a.y.lo, m)));
}
template <>
__device__ __forceinline__ cpx<df> shfl_idx(cpx<df> a, int lane) {
  return mk(df(__shfl_sync(0xffffffffu, a.x.hi, lane), __shfl_sync(0xffffffffu, a.x.lo, lane)),
            df(__shfl_sync(0xffffffffu, a.y.hi, lane), __shfl_sync(0xffffffffu, a.y.lo, lane)));
}

// Storage type of the vectors and grids a transform of compute type R reads
// and writes: double-float transforms read and write FP64 arrays.
template <typename R>
struct Io {
  using T = R;
};
template <>
struct Io<df> {
  using T = double;
};
template <typename R>
__device__ __forceinline__ R ld_io(const typename Io<R>::T* p) {
  return R(*p);
}
template <typename R>
__device__ __forceinline__ typename Io<R>::T io_of(R v) {
  return v;
}
template <>
__device__ __forceinline__ double io_of<df>(df v) {
  return to_double(v);
}
// to FP64 for the density accumulation
__device__ __forceinline__ double as_double(double v) { return v; }
__device__ __forceinline__ double as_double(float v) { return v; }
__device__ __forceinline__ double as_double(df v) { return to_double(v); }

}  // namespace pdep
