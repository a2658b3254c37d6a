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

// Copy n elements global -> shared (or back) with U independent loads in
// flight per thread before the first store.
template <int U, class V, class Src, class Dst>
__device__ __forceinline__ void staged_copy(int n, Src src, Dst dst) {
  const int nth = blockDim.x;
  for (int b = threadIdx.x; b < n; b += nth * U) {
    V tmp[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = b + u * nth;
      if (e < n) tmp[u] = src(e);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = b + u * nth;
      if (e < n) dst(e, tmp[u]);
    }
  }
}


// ---------------------------------------------------------------------------
// forward real FFT along x: two real lines per complex transform
// Pro: T operator()(int line, int x) const  -- produces the input sample
// ---------------------------------------------------------------------------
template <class T, class Pro>
__device__ __forceinline__ void k_rfft_x_b(Pro pro, cpx<T>* __restrict__ out, int n, int nlines, int pitch, FftPlan pl, const cpx<T>* __restrict__ tw, int npair, const int3 bid, unsigned char* smraw) {
  cpx<T>* a = reinterpret_cast<cpx<T>*>(smraw);
  cpx<T>* b = a + (size_t)npair * n;
  const int pair0 = bid.x * npair;
  for (int m = 0; m < npair; ++m) {
    const int l0 = 2 * (pair0 + m), l1 = l0 + 1;
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
      T va = 0, vb = 0;
      if (l0 < nlines) va = pro(l0, x);
      if (l1 < nlines) vb = pro(l1, x);
      a[m * n + x] = mk(va, vb);
    }
  }
  __syncthreads();
  cpx<T>* z = fft_lines<T>(a, b, pl, tw, -1, npair, 1, n);
  const int nh = n / 2 + 1;
  for (int m = 0; m < npair; ++m) {
    const int l0 = 2 * (pair0 + m), l1 = l0 + 1;
    if (l0 >= nlines) break;
    for (int k = threadIdx.x; k < nh; k += blockDim.x) {
      const cpx<T> zk = z[m * n + k];
      const cpx<T> zn = conjg(z[m * n + (k == 0 ? 0 : n - k)]);
      const cpx<T> A = scal(zk + zn, (T)0.5);
      const cpx<T> dd = zk - zn;  // B = -i/2 dd
      out[(size_t)l0 * pitch + k] = A;
      if (l1 < nlines) out[(size_t)l1 * pitch + k] = mk(dd.im * (T)0.5, -dd.re * (T)0.5);
    }
  }
}

template <class T, class Pro>
__global__ void k_rfft_x(Pro pro, cpx<T>* __restrict__ out, int n, int nlines, int pitch, FftPlan pl, const cpx<T>* __restrict__ tw, int npair) {
  extern __shared__ __align__(16) unsigned char smraw[];
  k_rfft_x_b(pro, out, n, nlines, pitch, pl, tw, npair, make_int3(blockIdx.x, blockIdx.y, blockIdx.z), smraw);
}

// ---------------------------------------------------------------------------
// inverse real FFT along x; Epi: void operator()(int line, int x, T value)
// value already multiplied by `scale`
// ---------------------------------------------------------------------------
// Asynchronous global -> shared copy of one element (cp.async, no register
// staging); completed by cp_async_wait_all.
template <class T>
__device__ __forceinline__ void cp_async_elem(T* sdst, const T* gsrc) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8 || sizeof(T) == 16, "4-, 8- or 16-byte elements");
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gsrc), "n"((int)sizeof(T)) : "memory");
}
// 16-byte variant that bypasses L1 (streamed planes); both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// An epilogue with kNPre > 0 names kNPre arrays (pre(j), row length pre_n())
// whose elements at (line, x) it combines with the transform output
// (apply(line, x, value, staged values, stride)); the kernel copies them into
// shared memory with cp.async before the transform, so their latency hides
// behind it.
template <class T, class Epi>
__device__ __forceinline__ void k_irfft_x_b(const cpx<T>* __restrict__ in, Epi epi, int n, int nlines, int pitch, FftPlan pl, const cpx<T>* __restrict__ tw, int npair, T scale, const int3 bid, unsigned char* smraw) {
  constexpr int NP = Epi::kNPre;
  cpx<T>* a = reinterpret_cast<cpx<T>*>(smraw);
  cpx<T>* b = a + (size_t)npair * n;
  T* pre = reinterpret_cast<T*>(b + (size_t)npair * n);  // [npair][2 lines][NP arrays][n]
  const int pair0 = bid.x * npair;
  const int nh = n / 2;
  if constexpr (NP > 0) {
    for (int m = 0; m < npair; ++m)
      for (int li = 0; li < 2; ++li) {
        const int l = 2 * (pair0 + m) + li;
        if (l >= nlines) continue;
        for (int j = 0; j < NP; ++j) {
          const T* src = epi.pre(j) + (size_t)l * epi.pre_n();
          T* dst = pre + ((size_t)(m * 2 + li) * NP + j) * n;
          for (int x = threadIdx.x; x < n; x += blockDim.x) cp_async_elem(dst + x, src + x);
        }
      }
    cp_async_commit();
  }
  for (int m = 0; m < npair; ++m) {
    const int l0 = 2 * (pair0 + m), l1 = l0 + 1;
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
      const int k = x <= nh ? x : n - x;
      cpx<T> A = mk<T>(0, 0), B = mk<T>(0, 0);
      if (l0 < nlines) A = in[(size_t)l0 * pitch + k];
      if (l1 < nlines) B = in[(size_t)l1 * pitch + k];
      if (x > nh) {
        A = conjg(A);
        B = conjg(B);
      }
      a[m * n + x] = mk(A.re - B.im, A.im + B.re);  // A + i B
    }
  }
  __syncthreads();
  cpx<T>* z = fft_lines<T>(a, b, pl, tw, +1, npair, 1, n);
  if constexpr (NP > 0) {
    cp_async_wait_all();
    __syncthreads();
  }
  for (int m = 0; m < npair; ++m) {
    const int l0 = 2 * (pair0 + m), l1 = l0 + 1;
    if (l0 >= nlines) break;
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
      const cpx<T> v = z[m * n + x];
      if constexpr (NP > 0) {
        const T* p0 = pre + ((size_t)(m * 2) * NP) * n;
        epi.apply(l0, x, v.re * scale, p0 + x, n);
        if (l1 < nlines) epi.apply(l1, x, v.im * scale, p0 + (size_t)NP * n + x, n);
      } else {
        epi(l0, x, v.re * scale);
        if (l1 < nlines) epi(l1, x, v.im * scale);
      }
    }
  }
}

// shared memory of k_irfft_x for epilogue Epi
template <class T, class Epi>
inline size_t irfft_x_smem(int n, int npair) {
  return (size_t)npair * n * (2 * sizeof(cpx<T>) + 2 * Epi::kNPre * sizeof(T));
}

template <class T, class Epi>
__global__ void k_irfft_x(const cpx<T>* __restrict__ in, Epi epi, int n, int nlines, int pitch, FftPlan pl, const cpx<T>* __restrict__ tw, int npair, T scale) {
  extern __shared__ __align__(16) unsigned char smraw[];
  k_irfft_x_b(in, epi, n, nlines, pitch, pl, tw, npair, scale, make_int3(blockIdx.x, blockIdx.y, blockIdx.z), smraw);
}

// ---------------------------------------------------------------------------
// complex FFT along y, in place, tile of TX kx-columns at one z level
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void k_fft_y_b(cpx<T>* __restrict__ data, int ny, int pitch, int ncol, FftPlan pl, const cpx<T>* __restrict__ tw, int sign, int tx, const int3 bid, unsigned char* smraw) {
  cpx<T>* a = reinterpret_cast<cpx<T>*>(smraw);
  cpx<T>* b = a + (size_t)ny * tx;
  const int c0 = bid.x * tx;
  cpx<T>* base = data + (size_t)bid.y * ny * pitch;
  const float itx = 1.0f / (float)tx;
  staged_copy<8, cpx<T>>(
      ny * tx,
      [&](int e) {
        const int y = qdiv(e, tx, itx), c = e - y * tx;
        return (c0 + c < ncol) ? base[(size_t)y * pitch + c0 + c] : mk<T>(0, 0);
      },
      [&](int e, cpx<T> v) { a[e] = v; });
  __syncthreads();
  cpx<T>* z = fft_lines<T>(a, b, pl, tw, sign, tx, tx, 1);
  for (int e = threadIdx.x; e < ny * tx; e += blockDim.x) {
    const int y = qdiv(e, tx, itx), c = e - y * tx;
    if (c0 + c < ncol) base[(size_t)y * pitch + c0 + c] = z[e];
  }
}

template <class T>
__global__ void k_fft_y(cpx<T>* __restrict__ data, int ny, int pitch, int ncol, FftPlan pl, const cpx<T>* __restrict__ tw, int sign, int tx) {
  extern __shared__ __align__(16) unsigned char smraw[];
  k_fft_y_b(data, ny, pitch, ncol, pl, tw, sign, tx, make_int3(blockIdx.x, blockIdx.y, blockIdx.z), smraw);
}

// ---------------------------------------------------------------------------
// z solves of the batched sweep's persistent kernel.  TX must be a multiple of
// 16: the 2 TX solver lanes then form whole warps, which the __syncwarp of the
// solve phase requires.
// One CTA: a tile of TX kx-columns x all z rows at one ky, staged
// in shared memory with coalesced row loads; thread t < 2 TX then solves column
// t/2, component t%2 (real and imaginary parts are independent real systems)
// sequentially along z in shared memory, and the tile is stored back.
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
  double dshift1, dshift2;  // derivatives of the shifts (used when TC carries derivatives)
  // FP32 eliminations: -(lambda_x + lambda_y) per (ky, kx) mode ([ny][ncol]) and h^2,
  // the shifts and h^2 scale, rounded to float on the host from the same FP64 values
  const float* k2f;
  float h2f, s1f, s2f, rsf;
};

// a shift in the elimination type: with Dual, its derivative as well
template <class TC>
__device__ __forceinline__ TC zshift(double s, double ds) {
  (void)ds;
  return (TC)s;
}
template <>
__device__ __forceinline__ Dual zshift<Dual>(double s, double ds) {
  return Dual(s, ds);
}

template <class TC>
__device__ __forceinline__ TC recip(TC x) { return (TC)1 / x; }
template <>
__device__ __forceinline__ float recip<float>(float x) { return __frcp_rn(x); }

template <class TC>
__device__ __forceinline__ TC zdiag(int k, int rows, int bc, TC sig) {
  if (bc == Z_FACES || (k > 0 && k < rows - 1)) return (TC)-2 - sig;
  return (bc == Z_NEUMANN ? (TC)-1 : (TC)-3) - sig;
}

template <class T, class TC>
__device__ __forceinline__ void k_zsolve_b(cpx<T>* __restrict__ data, const double* __restrict__ eigx, const double* __restrict__ eigy, ZSolve zs, int tx, const int3 bid, unsigned char* smraw) {
  // shared memory: the tile (R rows x tx complex), then the factors
  const int R = zs.rows;
  cpx<T>* tile = reinterpret_cast<cpx<T>*>(smraw);   // R x tx, row k at tile + k*tx
  TC* cp = reinterpret_cast<TC*>(tile + (size_t)R * tx);  // R x tx  (1/b' of solve 1)
  TC* cq = cp + (size_t)R * tx;                            // R x tx  (solve-2 factors, if !same)
  const int ky = bid.y;
  const int col0 = bid.x * tx;
  const int ncol = min(tx, zs.ncol - col0);
  cpx<T>* gbase = data + (size_t)ky * zs.pitch + col0;
  const size_t zstride = (size_t)zs.ny * zs.pitch;
  // stage the tile: rows of tx contiguous complex values (coalesced)
  const float itx = 1.0f / (float)tx;
  staged_copy<8, cpx<T>>(
      R * tx,
      [&](int e) {
        const int k = qdiv(e, tx, itx), c = e - k * tx;
        const bool mean_mode = zs.skip_zero && col0 + c == 0 && ky == 0;  // k_zero_mode's column
        return c < ncol && !mean_mode ? gbase[(size_t)k * zstride + c] : mk<T>(0, 0);
      },
      [&](int e, cpx<T> v) { tile[e] = v; });
  __syncthreads();
  const int t = threadIdx.x;
  const int c = t >> 1, part = t & 1;
  const int col = col0 + c;
  const bool active = c < ncol && !(zs.skip_zero && col == 0 && ky == 0);
  if (t < 2 * tx) {
    T* v = reinterpret_cast<T*>(tile + c) + part;  // component `part` of column c; row stride 2*tx
    const int vs = 2 * tx;
    const TC k2 = (TC)(-(eigx[active ? col : 0] + eigy[ky]));
    const TC h2 = (TC)zs.h2;
    const TC sg1 = (k2 + zshift<TC>(zs.shift1, zs.dshift1)) * h2;
    const TC rs = (TC)(zs.h2 * zs.scale);
    // phase A: elimination of solve 1 (top row k = 0 first), modified rhs in place.
    // The factor recurrence m_k = 1/(b - m_{k-1}) is stationary once two
    // successive values agree bit for bit (constant interior diagonal), so
    // from there on it is reused without recomputation -- exactly.
    TC cprev = 0, dprev = 0;
    bool stat = false;
#pragma unroll 4
    for (int k = 0; k < R; ++k) {
      const TC r = (TC)v[(size_t)k * vs] * rs;
      TC m = cprev;
      if (!stat || k == R - 1) {
        m = recip<TC>(zdiag<TC>(k, R, zs.bc, sg1) - cprev);
        stat = (k > 0 && k < R - 1 && m == cprev);
      }
      const TC dk = (r - dprev) * m;
      if (part == 0) cp[(size_t)k * tx + c] = m;
      v[(size_t)k * vs] = (T)dk;
      cprev = m;
      dprev = dk;
    }
    TC* c2 = cp;
    if (zs.two && !zs.same) {
      const TC sg2 = (k2 + zshift<TC>(zs.shift2, zs.dshift2)) * h2;
      TC cc = 0;
      for (int k = 0; k < R; ++k) {
        const TC m = recip<TC>(zdiag<TC>(k, R, zs.bc, sg2) - cc);
        if (part == 0) cq[(size_t)k * tx + c] = m;
        cc = m;
      }
      c2 = cq;
    }
    __syncwarp();
    if (!zs.two) {
      TC x = 0;
#pragma unroll 4
      for (int k = R - 1; k >= 0; --k) {
        x = (TC)v[(size_t)k * vs] - (k < R - 1 ? cp[(size_t)k * tx + c] * x : (TC)0);
        v[(size_t)k * vs] = (T)x;
      }
    } else {
      // phase B: back substitution of solve 1 (bottom-up); solve 2 eliminated in the same order
      TC x = 0, qv = 0;
#pragma unroll 4
      for (int k = R - 1; k >= 0; --k) {
        x = (TC)v[(size_t)k * vs] - (k < R - 1 ? cp[(size_t)k * tx + c] * x : (TC)0);
        const TC m2 = c2[(size_t)(R - 1 - k) * tx + c];
        qv = (x * h2 - (k < R - 1 ? qv : (TC)0)) * m2;
        v[(size_t)k * vs] = (T)qv;
      }
      // phase C: back substitution of solve 2 (top-down)
      TC y = 0;
#pragma unroll 4
      for (int k = 0; k < R; ++k) {
        y = (TC)v[(size_t)k * vs] - (k > 0 ? c2[(size_t)(R - 1 - k) * tx + c] * y : (TC)0);
        v[(size_t)k * vs] = (T)y;
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < R * tx; e += blockDim.x) {
    const int k = qdiv(e, tx, itx), cc = e - k * tx;
    const int colc = col0 + cc;
    if (cc < ncol && !(zs.skip_zero && colc == 0 && ky == 0)) gbase[(size_t)k * zstride + cc] = tile[e];
  }
}

// The (kx, ky) = (0, 0) column of a pure Neumann Poisson problem is singular
// (constants).  Row k of it says f_{k+1/2} - f_{k-1/2} = h^2 r_k for the
// face differences f_{k+1/2} = x_{k+1} - x_k, with f = 0 through both walls;
// so f is the running sum of h^2 r and x the running sum of f (the last row
// is the compatibility condition and is dropped).  The mean of x is then
// removed: the zero mode set to zero, as in Eq. NS37's solver.  FP64, no
// division; one thread per real/imaginary part.
template <class T>
__device__ __forceinline__ void k_zero_mode_b(cpx<T>* __restrict__ data, int rows, int ny, int pitch, double h2, double scale, Wide<T>* __restrict__ work, const int3 bid, unsigned char* smraw) {
  using W = Wide<T>;
  if (threadIdx.x > 1 || bid.x != 0) return;
  const int part = threadIdx.x;
  const size_t zstride = (size_t)ny * pitch * 2;
  T* base = reinterpret_cast<T*>(data) + part;
  W* xs = work + (size_t)part * rows;
  const double hs = h2 * scale;
  W f = 0.0, x = 0.0, sum = 0.0;
  for (int k = 0; k < rows; ++k) {
    xs[k] = x;
    sum += x;
    f += (W)base[(size_t)k * zstride] * hs;
    x += f;
  }
  const W mean = sum / (double)rows;
  for (int k = 0; k < rows; ++k) base[(size_t)k * zstride] = (T)(xs[k] - mean);
}

// The same solve with the column staged in shared memory: every thread loads
// rows in parallel, one thread per real/imaginary part runs the two running
// sums there, and the mean-free result is written back in parallel.
// smem: 2 * rows elements of Wide<T>.
template <class T>
__global__ void k_zero_mode_smem(cpx<T>* __restrict__ data, int rows, int ny, int pitch, double h2, double scale) {
  using W = Wide<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  W* col = reinterpret_cast<W*>(smraw);  // [2][rows]
  __shared__ W mean[2];
  const size_t zstride = (size_t)ny * pitch * 2;
  T* base = reinterpret_cast<T*>(data);
  for (int e = threadIdx.x; e < 2 * rows; e += blockDim.x) {
    const int part = e / rows, k = e - part * rows;
    col[e] = (W)base[(size_t)k * zstride + part];
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    W* c = col + (size_t)threadIdx.x * rows;
    const double hs = h2 * scale;
    W f = 0.0, x = 0.0, sum = 0.0;
    for (int k = 0; k < rows; ++k) {
      const W r = c[k];
      c[k] = x;
      sum += x;
      f += r * hs;
      x += f;
    }
    mean[threadIdx.x] = sum / (double)rows;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * rows; e += blockDim.x) {
    const int part = e / rows, k = e - part * rows;
    base[(size_t)k * zstride + part] = (T)(col[e] - mean[part]);
  }
}

template <class T>
__global__ void k_zero_mode(cpx<T>* __restrict__ data, int rows, int ny, int pitch, double h2, double scale, Wide<T>* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char smraw[];
  k_zero_mode_b(data, rows, ny, pitch, h2, scale, work, make_int3(blockIdx.x, blockIdx.y, blockIdx.z), smraw);
}

}  // namespace pf
