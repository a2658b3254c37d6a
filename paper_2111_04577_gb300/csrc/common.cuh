// Shared device/host definitions of the dual-resolution phase-field library.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

#include "dual.cuh"

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
  int rs, rys;         // log2(r), log2(ry)
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
  double alpha_g;  // Giesekus mobility (0: Oldroyd-B)
  double uw_bot, uw_top, gx, gy, gz;
  int visco;
  int approach1;                    // Eq. NS11: polymer parameters linear in phi, tau = tau_p
  double mu_p2, lam_h2, alpha_g2;   // phase 2's polymer (approach 1)
  int weno;                         // WENO5-Z convective fluxes for phi and Theta (else central)
  double dw, kappa;                 // wall relaxation D_w of Eq. NS15 and D_w gamma0/dt
};

// Scheme constants converted once to the arithmetic type of the kernels, so
// that no FP64 operation is issued per cell on the FP32 path.
template <class T>
struct PhysT {
  T idt, irho0, inum, num;            // 1/dt, 1/rho0, 1/nu_m, nu_m
  T rho1, rho2, mu_s1, mu_s2;
  T uw2_bot, uw2_top;                 // 2 u_w (no-slip ghost)
  T cj_dx;                            // -(rho1 - rho2)/2 M / dx  (J per unit G difference)
  T gx, gy, gz;
  T ih, ih2, iD, iD2;                 // fine and coarse inverse spacings
  T ie2, lam;                         // 1/eta^2, lambda
  T dt, ilh, wtau;                    // dt, 1/lambda_H, mu_p/lambda_H
  T ag;                               // Giesekus mobility alpha (0: Oldroyd-B)
  Wide<T> gbot, gtop;                 // cos(theta_s)/(sqrt(2) eta) of the two walls (FP64, or carrying a derivative)
  Wide<T> ihw;                        // 1/h in FP64: the wall flux enters R and mu* as g/h
  // approach 1 (Eq. NS11): lambda_H, mu_p and alpha of the two phases, mixed
  // per coarse centre by the restricted phi; ilh, wtau and ag above unused
  T lh1, lh2, mp1, mp2, ag2;
  int ap1;
  int weno;  // WENO5-Z advection of phi and Theta (csrc/weno.cuh), else central
};

// Kernels over rows of a mesh use a 2D grid: blockIdx.x = row (y, z pair),
// blockIdx.y * blockDim.x + threadIdx.x = x.  No 64-bit index division.
struct RowIdx {
  int i, j, k, row;
};
__device__ __forceinline__ bool row_index_b(const int3 bid, int nxrow, int nyrow, RowIdx& r) {
  r.row = bid.x;
  r.i = bid.y * blockDim.x + threadIdx.x;
  if (r.i >= nxrow) return false;
  r.k = r.row / nyrow;
  r.j = r.row - r.k * nyrow;
  return true;
}
__device__ __forceinline__ bool row_index(int nxrow, int nyrow, RowIdx& r) {
  return row_index_b(make_int3(blockIdx.x, blockIdx.y, blockIdx.z), nxrow, nyrow, r);
}

// Exact quotient of 0 <= x < 2^22 by 1 <= d using a float reciprocal (one
// correction step); avoids the long integer-division sequence in index math.
__device__ __forceinline__ int qdiv(int x, int d, float invd) {
  int q = __float2int_rz((float)x * invd);
  const int r = x - q * d;
  if (r < 0) --q;
  else if (r >= d) ++q;
  return q;
}

// fine index helpers (x fastest)
__host__ __device__ __forceinline__ size_t fidx(const Dims& d, int i, int j, int k) {
  return ((size_t)k * d.fny + j) * d.fnx + i;
}
__host__ __device__ __forceinline__ size_t cidx(const Dims& d, int i, int j, int k) {
  return ((size_t)k * d.ny + j) * d.nx + i;
}
// Knuth's TwoSum (The Art of Computer Programming, Vol. 2, 4.2.2): s = fl(a + b)
// and e with s + e = a + b exactly, for any a, b, in round-to-nearest.
template <class T>
__host__ __device__ __forceinline__ void two_sum(T a, T b, T& s, T& e) {
  s = a + b;
  const T bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__host__ __device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ---------------------------------------------------------------------------
// FFT plan: mixed radix 2/3/4/5/7 Stockham stages, factor list on the host
// ---------------------------------------------------------------------------
struct FftPlan {
  int n;
  int ns;
  unsigned long long code;  // radix of stage s in bits [3s, 3s+3)
  __host__ __device__ __forceinline__ int radix(int s) const { return (int)((code >> (3 * s)) & 7ull); }
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
