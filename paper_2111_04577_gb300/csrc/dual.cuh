// Forward-mode derivative arithmetic: a value and its derivative with respect
// to one scalar parameter (dual numbers, a + b e with e^2 = 0).  Running the
// whole time step on Dual instead of double gives dJ/dp for one parameter p by
// the chain rule, exactly up to FP64 rounding, through every operation of the
// step: the transforms, the z eliminations, the projection and the polymer
// eigen-decomposition.  Comparisons and branches act on the value.
//
// Wide<T> is the type a step keeps in FP64 whatever its field precision (the
// contact-line flux, the pressure's mean mode, reductions): double for float
// and double fields, Dual for Dual fields, so that derivatives pass through
// those FP64 parts too.
#pragma once
#include <cmath>

namespace pf {
namespace ad {

struct Dual {
  double v, d;  // value, derivative
  __host__ __device__ constexpr Dual() : v(0), d(0) {}
  __host__ __device__ constexpr Dual(double x) : v(x), d(0) {}
  __host__ __device__ constexpr Dual(double x, double dx) : v(x), d(dx) {}
  __host__ __device__ explicit operator double() const { return v; }
  __host__ __device__ explicit operator float() const { return (float)v; }
  __host__ __device__ Dual& operator+=(Dual b) {
    v += b.v;
    d += b.d;
    return *this;
  }
  __host__ __device__ Dual& operator-=(Dual b) {
    v -= b.v;
    d -= b.d;
    return *this;
  }
  __host__ __device__ Dual& operator*=(Dual b) {
    d = d * b.v + v * b.d;
    v *= b.v;
    return *this;
  }
  __host__ __device__ Dual& operator/=(Dual b) {
    const double q = v / b.v;
    d = (d - q * b.d) / b.v;
    v = q;
    return *this;
  }
};

__host__ __device__ inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__host__ __device__ inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__host__ __device__ inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__host__ __device__ inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__host__ __device__ inline Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
// comparisons on the value: the branch taken is the one the value takes
__host__ __device__ inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
__host__ __device__ inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
__host__ __device__ inline bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
__host__ __device__ inline bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
__host__ __device__ inline bool operator==(Dual a, Dual b) { return a.v == b.v; }
__host__ __device__ inline bool operator!=(Dual a, Dual b) { return a.v != b.v; }

// elementary functions: f(a) + f'(a) a.d e
__host__ __device__ inline Dual sqrt(Dual a) {
  const double s = ::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
__host__ __device__ inline Dual rsqrt(Dual a) {
  const double r = 1.0 / ::sqrt(a.v);
  return Dual(r, -0.5 * r * r * r * a.d);
}
__host__ __device__ inline Dual exp(Dual a) {
  const double e = ::exp(a.v);
  return Dual(e, e * a.d);
}
__host__ __device__ inline Dual expm1(Dual a) { return Dual(::expm1(a.v), ::exp(a.v) * a.d); }
__host__ __device__ inline Dual exp2(Dual a) {
  const double e = ::exp2(a.v);
  return Dual(e, e * 0.69314718055994530942 * a.d);
}
__host__ __device__ inline Dual log2(Dual a) { return Dual(::log2(a.v), a.d / (a.v * 0.69314718055994530942)); }
__host__ __device__ inline Dual fabs(Dual a) { return a.v < 0.0 ? -a : a; }
__host__ __device__ inline Dual fmax(Dual a, Dual b) { return a.v >= b.v ? a : b; }

}  // namespace ad

using ad::Dual;

template <class T>
struct WideOf {
  using type = double;
};
template <>
struct WideOf<Dual> {
  using type = Dual;
};
template <class T>
using Wide = typename WideOf<T>::type;

template <class T>
struct IsDual {
  static constexpr bool value = false;
};
template <>
struct IsDual<Dual> {
  static constexpr bool value = true;
};

}  // namespace pf
