// Two-fold floating-point numbers: x = hi + lo with |lo| <= ulp(hi) / 2, an
// unevaluated sum of two numbers of a base type B, built from error-free
// transformations (Knuth's TwoSum, Dekker's Fast2Sum, the FMA-based exact
// product; the double-word algorithms of Joldes, Muller and Popescu, ACM
// TOMS 44 (2017)).
//
//   twofold<float>:  about 48 significant bits on the FP32 pipe (FP32
//                    exponent range), the library's FP32X2 precision;
//   twofold<double>: about 106 significant bits on the FP64 pipe, the
//                    library's FP64X2 precision.
//
// Addition is the "sloppy" double-word sum: its error is bounded by a small
// multiple of u^2 (|x| + |y|) (u = unit roundoff of B), not of u^2 |x + y|,
// which is the normwise accuracy an FFT needs.  Multiplication has relative
// error below 5 u^2.  Every base operation is an explicitly rounded
// intrinsic, so no FMA contraction or reassociation can break the
// error-free transformations.
#pragma once
#include <cuda_runtime.h>

namespace lbo {

__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename B>
struct twofold {
  B hi, lo;
  twofold() = default;
  __host__ __device__ constexpr twofold(B h, B l) : hi(h), lo(l) {}
  __host__ __device__ constexpr twofold(int v) : hi((B)v), lo((B)0) {}
  // from double: exact for B = double; for B = float the remainder after
  // rounding to float, so the pair carries the double's value to ~2^-48
  __host__ __device__ twofold(double v) : hi((B)v), lo((B)(v - (double)(B)v)) {}
  __host__ __device__ twofold(float v) : hi((B)v), lo((B)0) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

template <typename T>
struct is_twofold {
  static constexpr bool value = false;
};
template <typename B>
struct is_twofold<twofold<B>> {
  static constexpr bool value = true;
};

// s + e = a + b exactly
template <typename B>
__device__ __forceinline__ twofold<B> two_sum(B a, B b) {
  const B s = add_rn(a, b);
  const B bb = sub_rn(s, a);
  const B e = add_rn(sub_rn(a, sub_rn(s, bb)), sub_rn(b, bb));
  return twofold<B>(s, e);
}

// s + e = a + b exactly, for |a| >= |b| (or a = 0)
template <typename B>
__device__ __forceinline__ twofold<B> fast_two_sum(B a, B b) {
  const B s = add_rn(a, b);
  return twofold<B>(s, sub_rn(b, sub_rn(s, a)));
}

template <typename B>
__device__ __forceinline__ twofold<B> operator+(twofold<B> x, twofold<B> y) {
  const twofold<B> s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, add_rn(s.lo, add_rn(x.lo, y.lo)));
}

template <typename B>
__device__ __forceinline__ twofold<B> operator-(twofold<B> x) {
  return twofold<B>(-x.hi, -x.lo);
}

template <typename B>
__device__ __forceinline__ twofold<B> operator-(twofold<B> x, twofold<B> y) {
  return x + (-y);
}

template <typename B>
__device__ __forceinline__ twofold<B> operator*(twofold<B> x, twofold<B> y) {
  const B ph = mul_rn(x.hi, y.hi);
  const B pl = fma_rn(x.hi, y.hi, -ph);  // ph + pl = x.hi y.hi exactly
  const B t = fma_rn(x.hi, y.lo, mul_rn(x.lo, y.hi));
  return fast_two_sum(ph, add_rn(pl, t));
}

template <typename B>
__device__ __forceinline__ twofold<B>& operator+=(twofold<B>& x, twofold<B> y) {
  x = x + y;
  return x;
}

template <typename B>
__device__ __forceinline__ twofold<B>& operator*=(twofold<B>& x, twofold<B> y) {
  x = x * y;
  return x;
}

using f32x2 = twofold<float>;
using f64x2 = twofold<double>;

// A constant given as hi + lo doubles (lo the rounding remainder of the exact
// value): rounded to T, or kept as a pair for the two-fold types.
template <typename T>
__device__ __forceinline__ T kconst(double hi, double lo) {
  if constexpr (is_twofold<T>::value) {
    if constexpr (sizeof(T) == 16) return T(hi, lo);
    else return T(hi);  // float pair: the double hi carries more than its 48 bits
  } else {
    return (T)hi;
  }
}

}  // namespace lbo
