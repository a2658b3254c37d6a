// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// words with |lo| <= ulp(hi)/2, which carries a 48-bit significand (relative
// rounding about 2^-47, against 2^-53 for FP64) on the FP32 pipes.  The
// operations are built from error-free transformations:
//   TwoSum (Knuth, The Art of Computer Programming, Vol. 2, 4.2.2):
//     s = a + b,  e = (a - (s - v)) + (b - v),  v = s - a,      a + b = s + e exactly;
//   FastTwoSum (Dekker 1971), for |a| >= |b|:  s = a + b,  e = b - (s - a);
//   TwoProd with a fused multiply-add:  p = a b,  e = fma(a, b, -p),  a b = p + e exactly;
// and the double-word algorithms of Dekker (1971, "A floating-point technique
// for extending the available precision").  Every step is written with the
// round-to-nearest intrinsics, which the compiler never fuses into a
// multiply-add (a fused p would break the exactness of TwoProd's error term).
// Used as the elimination type of the wall-normal z solves (precision
// PF_MIXED_Z2F): the FP32 pipes do in a few dozen instructions what one FP64
// operation costs on a GPU whose FP64 rate is a small fraction of its FP32 rate.
#pragma once
#include <cmath>

namespace pf {
// (a namespace of its own: its functions reach DF arguments by argument-dependent
// lookup and hide no sqrt, fabs, exp2 or log2 of the enclosing code)
namespace dfa {

struct DF {
  float hi, lo;
  DF() = default;
  __host__ __device__ constexpr DF(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ DF(float x) : hi(x), lo(0.f) {}
  __host__ __device__ DF(int x) : DF((double)x) {}
  __host__ __device__ DF(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

#ifdef __CUDACC__
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), v = __fsub_rn(s, a);
  return DF(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v)));
}
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return DF(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// Dekker's addition: the leading words by TwoSum, the trailing ones added in
// FP32 (relative error about 2^-46 of the larger operand's magnitude: an
// absolute bound, which is what the eliminations' recurrences need)
__device__ __forceinline__ DF operator+(DF a, DF b) {
  const DF s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__device__ __forceinline__ DF operator*(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// three quotient digits: each a correctly rounded FP32 quotient of the current
// remainder by b's leading word
__device__ __forceinline__ DF operator/(DF a, DF b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  DF r = a - b * DF(q1);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  r = r - b * DF(q2);
  const float q3 = __fdiv_rn(r.hi, b.hi);
  return df_fast_two_sum(q1, q2) + DF(q3);
}
__device__ __forceinline__ DF& operator+=(DF& a, DF b) { return a = a + b; }
__device__ __forceinline__ DF& operator-=(DF& a, DF b) { return a = a - b; }
__device__ __forceinline__ DF& operator*=(DF& a, DF b) { return a = a * b; }
__device__ __forceinline__ DF& operator/=(DF& a, DF b) { return a = a / b; }
__device__ __forceinline__ bool operator<(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(DF a, DF b) { return b < a; }
__device__ __forceinline__ bool operator<=(DF a, DF b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(DF a, DF b) { return !(a < b); }
__device__ __forceinline__ bool operator==(DF a, DF b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(DF a, DF b) { return !(a == b); }
__device__ __forceinline__ DF fabs(DF a) { return a.hi < 0.f ? -a : a; }
// the few transcendental steps (once per thread in the closed-form factors) in FP64
__device__ __forceinline__ DF sqrt(DF a) { return DF(::sqrt((double)a)); }
__device__ __forceinline__ DF exp2(DF a) { return DF(::exp2((double)a)); }
__device__ __forceinline__ DF log2(DF a) { return DF(::log2((double)a)); }
#endif

}  // namespace dfa
using dfa::DF;
}  // namespace pf
