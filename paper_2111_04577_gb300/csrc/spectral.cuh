// Batched transform-solve kernels: real FFT along x, complex FFT along y and
// the two-sided tridiagonal solves along the wall-normal z direction.
//
// Constant-coefficient problems (L - shift) x = rhs, L the second-order
// central Laplacian (Eqs. NS26, NS27, NS36, NS37), are diagonalised by the DFT
// along the periodic x and y axes (discrete eigenvalues
// -(4/h^2) sin^2(pi k/n)); what remains per (kx, ky) mode is a tridiagonal
// system along z with the wall condition in its end rows:
//   NEUMANN  cell unknowns, mirror ghost     end diagonal -1 - sigma  (phi, Psi, p')
//   DIRICH   cell unknowns, odd ghost        end diagonal -3 - sigma  (tangential u, v)
//   FACES    face unknowns, zero walls       end diagonal -2 - sigma  (w)
// (rows scaled by h^2, off-diagonals 1, interior diagonal -2 - sigma,
// sigma = (k^2 + shift) h^2).  The systems are diagonally dominant for
// sigma > 0, so elimination needs no pivoting.
//
// Layout of a spectral array: [z][y][kx] complex, kx = 0..nx/2 stored in a row
// of `pitch` entries (pitch even), y = 0..ny-1 (ny = 1 in 2D).
#pragma once
#include "fft.cuh"

namespace pf {

enum ZBc { Z_NEUMANN = 0, Z_DIRICH = 1, Z_FACES = 2 };

// ---------------------------------------------------------------------------
// forward real FFT along x: two real lines per complex transform
// Pro: T operator()(int line, int x) const  -- produces the input sample
// ---------------------------------------------------------------------------
template <class T, class Pro>
__global__ void k_rfft_x(Pro pro, cpx<T>* __restrict__ out, int n, int nlines, int pitch, FftPlan pl,
                         const cpx<T>* __restrict__ tw, int npair) {
  extern __shared__ unsigned char smraw[];
  cpx<T>* a = reinterpret_cast<cpx<T>*>(smraw);
  cpx<T>* b = a + (size_t)npair * n;
  const int pair0 = blockIdx.x * npair;
  for (int e = threadIdx.x; e < npair * n; e += blockDim.x) {
    const int m = e / n, x = e - (e / n) * n;
    const int l0 = 2 * (pair0 + m), l1 = l0 + 1;
    T va = 0, vb = 0;
    if (l0 < nlines) va = pro(l0, x);
    if (l1 < nlines) vb = pro(l1, x);
    a[e] = mk(va, vb);
  }
  __syncthreads();
  cpx<T>* z = fft_lines<T>(a, b, pl, tw, -1, npair, 1, n);
  const int nh = n / 2 + 1;
  for (int e = threadIdx.x; e < npair * nh; e += blockDim.x) {
    const int m = e / nh, k = e - (e / nh) * nh;
    const int l0 = 2 * (pair0 + m), l1 = l0 + 1;
    if (l0 >= nlines) continue;
    const cpx<T> zk = z[m * n + k];
    const cpx<T> zn = conjg(z[m * n + (k == 0 ? 0 : n - k)]);
    const cpx<T> A = scal(zk + zn, (T)0.5);
    const cpx<T> d = zk - zn;  // B = -i/2 d
    out[(size_t)l0 * pitch + k] = A;
    if (l1 < nlines) out[(size_t)l1 * pitch + k] = mk(d.im * (T)0.5, -d.re * (T)0.5);
  }
}

// ---------------------------------------------------------------------------
// inverse real FFT along x; Epi: void operator()(int line, int x, T value)
// value already multiplied by `scale`
// ---------------------------------------------------------------------------
template <class T, class Epi>
__global__ void k_irfft_x(const cpx<T>* __restrict__ in, Epi epi, int n, int nlines, int pitch, FftPlan pl,
                          const cpx<T>* __restrict__ tw, int npair, T scale) {
  extern __shared__ unsigned char smraw[];
  cpx<T>* a = reinterpret_cast<cpx<T>*>(smraw);
  cpx<T>* b = a + (size_t)npair * n;
  const int pair0 = blockIdx.x * npair;
  const int nh = n / 2;
  for (int e = threadIdx.x; e < npair * n; e += blockDim.x) {
    const int m = e / n, x = e - (e / n) * n;
    const int l0 = 2 * (pair0 + m), l1 = l0 + 1;
    const int k = x <= nh ? x : n - x;
    cpx<T> A = mk<T>(0, 0), B = mk<T>(0, 0);
    if (l0 < nlines) A = in[(size_t)l0 * pitch + k];
    if (l1 < nlines) B = in[(size_t)l1 * pitch + k];
    if (x > nh) {
      A = conjg(A);
      B = conjg(B);
    }
    a[e] = mk(A.re - B.im, A.im + B.re);  // A + i B
  }
  __syncthreads();
  cpx<T>* z = fft_lines<T>(a, b, pl, tw, +1, npair, 1, n);
  for (int e = threadIdx.x; e < npair * n; e += blockDim.x) {
    const int m = e / n, x = e - (e / n) * n;
    const int l0 = 2 * (pair0 + m), l1 = l0 + 1;
    const cpx<T> v = z[e];
    if (l0 < nlines) epi(l0, x, v.re * scale);
    if (l1 < nlines) epi(l1, x, v.im * scale);
  }
}

// ---------------------------------------------------------------------------
// complex FFT along y, in place, tile of TX kx-columns at one z level
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_fft_y(cpx<T>* __restrict__ data, int ny, int pitch, int ncol, FftPlan pl,
                        const cpx<T>* __restrict__ tw, int sign, int tx) {
  extern __shared__ unsigned char smraw[];
  cpx<T>* a = reinterpret_cast<cpx<T>*>(smraw);
  cpx<T>* b = a + (size_t)ny * tx;
  const int c0 = blockIdx.x * tx;
  cpx<T>* base = data + (size_t)blockIdx.y * ny * pitch;
  for (int e = threadIdx.x; e < ny * tx; e += blockDim.x) {
    const int y = e / tx, c = e - (e / tx) * tx;
    a[e] = (c0 + c < ncol) ? base[(size_t)y * pitch + c0 + c] : mk<T>(0, 0);
  }
  __syncthreads();
  cpx<T>* z = fft_lines<T>(a, b, pl, tw, sign, tx, tx, 1);
  for (int e = threadIdx.x; e < ny * tx; e += blockDim.x) {
    const int y = e / tx, c = e - (e / tx) * tx;
    if (c0 + c < ncol) base[(size_t)y * pitch + c0 + c] = z[e];
  }
}

// ---------------------------------------------------------------------------
// z solves.  One CTA: TX kx-columns at one ky; thread t handles column t/2,
// component t%2 (real and imaginary parts are independent real systems).
// Solve 1: (L - shift1) x = scale * rhs, eliminated bottom-up then substituted
// top-down.  With `two`, the result x feeds solve 2, (L - shift2) y = x, whose
// elimination runs top-down while solve 1 substitutes, so the pair costs three
// sweeps.  The factor sequence of the symmetric end rows is the same read in
// either direction, which solve 2 reuses when shift2 == shift1.
// TC: arithmetic type of the elimination (FP64 on request).
// ---------------------------------------------------------------------------
struct ZSolve {
  int rows;        // unknowns along z
  int ny, pitch, ncol;
  int bc;
  int two;         // 0: single solve; 1: pair
  int same;        // shift2 == shift1
  int skip_zero;   // the (0,0) column is handled by k_zero_mode
  double h2, shift1, shift2, scale;
};

template <class TC>
__device__ __forceinline__ TC zdiag(int k, int rows, int bc, TC sig) {
  if (bc == Z_FACES || (k > 0 && k < rows - 1)) return (TC)-2 - sig;
  return (bc == Z_NEUMANN ? (TC)-1 : (TC)-3) - sig;
}

template <class T, class TC>
__global__ void k_zsolve(cpx<T>* __restrict__ data, const double* __restrict__ eigx,
                         const double* __restrict__ eigy, ZSolve zs, int tx) {
  extern __shared__ unsigned char smraw[];
  const int R = zs.rows;
  const int nt = 2 * tx;
  TC* cp = reinterpret_cast<TC*>(smraw);            // R x tx  (factor 1/b')
  TC* dp = cp + (size_t)R * tx;                      // R x nt  (modified rhs)
  TC* cq = dp + (size_t)R * nt;                      // R x tx  (solve-2 factors, if !same)
  const int t = threadIdx.x;
  const int c = t >> 1, part = t & 1;
  const int ky = blockIdx.y;
  int col = blockIdx.x * tx + c;
  // inactive lanes keep participating in __syncwarp but touch no memory
  const bool active = col < zs.ncol && !(zs.skip_zero && col == 0 && ky == 0);
  if (!active) col = 0;
  const size_t zstride = (size_t)zs.ny * zs.pitch * 2;  // in T units
  T* base = reinterpret_cast<T*>(data) + ((size_t)ky * zs.pitch + col) * 2 + part;
  const TC k2 = (TC)(-(eigx[col] + eigy[ky]));
  const TC h2 = (TC)zs.h2;
  const TC sg1 = (k2 + (TC)zs.shift1) * h2;
  const TC rs = (TC)(zs.h2 * zs.scale);
  // phase A: bottom-up elimination of solve 1
  TC cprev = 0, dprev = 0;
  for (int k = 0; k < R; ++k) {
    const TC r = active ? (TC)base[(size_t)k * zstride] * rs : (TC)0;
    const TC bk = zdiag<TC>(k, R, zs.bc, sg1) - cprev;
    const TC m = (TC)1 / bk;
    const TC dk = (r - dprev) * m;
    if (part == 0) cp[(size_t)k * tx + c] = m;
    dp[(size_t)k * nt + t] = dk;
    cprev = m;
    dprev = dk;
  }
  if (!zs.two) {
    __syncwarp();
    TC x = 0;
    for (int k = R - 1; k >= 0; --k) {
      x = dp[(size_t)k * nt + t] - (k < R - 1 ? cp[(size_t)k * tx + c] * x : (TC)0);
      if (active) base[(size_t)k * zstride] = (T)x;
    }
    return;
  }
  TC* c2 = cp;
  if (!zs.same) {
    const TC sg2 = (k2 + (TC)zs.shift2) * h2;
    TC cc = 0;
    for (int k = 0; k < R; ++k) {
      const TC m = (TC)1 / (zdiag<TC>(k, R, zs.bc, sg2) - cc);
      if (part == 0) cq[(size_t)k * tx + c] = m;
      cc = m;
    }
    c2 = cq;
  }
  __syncwarp();
  // phase B: substitute solve 1 top-down; eliminate solve 2 in the same order
  TC x = 0, q = 0;
  for (int k = R - 1; k >= 0; --k) {
    x = dp[(size_t)k * nt + t] - (k < R - 1 ? cp[(size_t)k * tx + c] * x : (TC)0);
    const TC m2 = c2[(size_t)(R - 1 - k) * tx + c];
    q = (x * h2 - (k < R - 1 ? q : (TC)0)) * m2;
    dp[(size_t)k * nt + t] = q;
  }
  // phase C: substitute solve 2 bottom-up
  TC y = 0;
  for (int k = 0; k < R; ++k) {
    y = dp[(size_t)k * nt + t] - (k > 0 ? c2[(size_t)(R - 1 - k) * tx + c] * y : (TC)0);
    if (active) base[(size_t)k * zstride] = (T)y;
  }
}

// The (kx, ky) = (0, 0) column of a pure Neumann Poisson problem is singular
// (constants).  Solved in FP64 with the last row replaced by x = 0, then the
// mean is removed -- the zero mode set to zero, as in Eq. NS37's solver.
template <class T>
__global__ void k_zero_mode(cpx<T>* __restrict__ data, int rows, int ny, int pitch, double h2, double scale,
                            double* __restrict__ work) {
  if (threadIdx.x > 1 || blockIdx.x != 0) return;
  const int part = threadIdx.x;
  const size_t zstride = (size_t)ny * pitch * 2;
  T* base = reinterpret_cast<T*>(data) + part;
  double* cp = work + (size_t)part * 2 * rows;
  double* dp = cp + rows;
  double cprev = 0, dprev = 0;
  for (int k = 0; k < rows; ++k) {
    double r = (double)base[(size_t)k * zstride] * h2 * scale;
    double bk = ((k == 0 || k == rows - 1) ? -1.0 : -2.0) - cprev;
    if (k == rows - 1) {
      bk = 1.0;
      r = 0.0;
      dprev = 0.0;
    }
    const double m = 1.0 / bk;
    cp[k] = (k == rows - 1) ? 0.0 : m;
    dp[k] = (r - dprev) * m;
    cprev = m;
    dprev = dp[k];
  }
  double x = 0, sum = 0;
  for (int k = rows - 1; k >= 0; --k) {
    x = dp[k] - (k < rows - 1 ? cp[k] * x : 0.0);
    dp[k] = x;
    sum += x;
  }
  const double mean = sum / rows;
  for (int k = 0; k < rows; ++k) base[(size_t)k * zstride] = (T)(dp[k] - mean);
}

}  // namespace pf
