// Shared device/host definitions of the dual-resolution phase-field library.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

namespace pf {

// ---------------------------------------------------------------------------
// complex value in registers / memory (interleaved re, im)
// ---------------------------------------------------------------------------
template <class T>
struct alignas(2 * sizeof(T)) cpx {
  T re, im;
};

template <class T>
__host__ __device__ __forceinline__ cpx<T> mk(T a, T b) {
  cpx<T> z;
  z.re = a;
  z.im = b;
  return z;
}
template <class T>
__host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <class T>
__host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <class T>
__host__ __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class T>
__host__ __device__ __forceinline__ cpx<T> scal(cpx<T> a, T s) { return mk(a.re * s, a.im * s); }
template <class T>
__host__ __device__ __forceinline__ cpx<T> conjg(cpx<T> a) { return mk(a.re, -a.im); }
// multiply by (sign * i): sign = +1 -> i z, sign = -1 -> -i z
template <class T>
__host__ __device__ __forceinline__ cpx<T> mul_si(cpx<T> a, int sign) {
  return sign > 0 ? mk(-a.im, a.re) : mk(a.im, -a.re);
}

// ---------------------------------------------------------------------------
// geometry handed to kernels by value
// ---------------------------------------------------------------------------
struct Dims {
  int nx, ny, nz;      // coarse cells
  int r, ry;           // refinement in x/z and in y (ry = 1 in 2D)
  int fnx, fny, fnz;   // fine cells
  int dim;             // 2 or 3
  double dx, h;        // coarse and fine spacing
};

// constants of the scheme (derived on the host in FP64)
struct Phys {
  double dt, gamma0;
  double eta, lam, mob, Ml, S, alpha, c;
  double cos_bot, cos_top;
  double rho1, rho2, rho0, mu_s1, mu_s2, mu_p1, lam_h, nu_m;
  double uw_bot, uw_top, gx, gy, gz;
  int visco;
};

// fine index helpers (x fastest)
__host__ __device__ __forceinline__ size_t fidx(const Dims& d, int i, int j, int k) {
  return ((size_t)k * d.fny + j) * d.fnx + i;
}
__host__ __device__ __forceinline__ size_t cidx(const Dims& d, int i, int j, int k) {
  return ((size_t)k * d.ny + j) * d.nx + i;
}
__host__ __device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ---------------------------------------------------------------------------
// FFT plan: mixed radix 2/3/4/5/7 Stockham stages, factor list on the host
// ---------------------------------------------------------------------------
struct FftPlan {
  int n;
  int ns;
  int radix[24];
};

}  // namespace pf

#define PF_CUDA_TRY(expr)                                                    \
  do {                                                                       \
    cudaError_t _e = (expr);                                                 \
    if (_e != cudaSuccess) {                                                 \
      throw pf::CudaError(_e, #expr, __FILE__, __LINE__);                    \
    }                                                                        \
  } while (0)

namespace pf {
struct CudaError {
  cudaError_t err;
  const char* expr;
  const char* file;
  int line;
  CudaError(cudaError_t e, const char* x, const char* f, int l) : err(e), expr(x), file(f), line(l) {}
};
}  // namespace pf
