// Register-resident FFT of power-of-two lines (64 <= N <= 4096) for the
// periodic directions of the transform solves (Sections 3.2.1-3.2.2).
//
// The same self-sorting (Stockham) factorisation as fft.cuh: stage s combines
// sub-transforms of length L into length L*P; with M = N/(L*P), butterfly
// bf = (j, k), j = bf / M, k = bf % M, gathers z_c = w_N^{c j M} Y[j M P + k + c M]
// and writes the length-P DFT of z to Y'[(j + L q) M + k].  Here a line is
// owned by NT = N/E threads, each holding E (8 or 16) elements in registers, and the
// small radix (2 or 4, when log2 N is not a multiple of 3) goes first, the
// radix-8 stages after it:
//  - on entry thread t holds x[t + NT c], c = 0..E-1, which is exactly the input
//    of the first stage's butterflies (bf = t + NT i, j = 0), so the first
//    stage reads registers loaded straight from global memory;
//  - stages exchange through one shared buffer of N complex per line, in place
//    (every thread reads its inputs, barrier, then writes);
//  - the last (radix-8) stage has M = 1, so its outputs Y'[t + NT c] stay in
//    registers in natural order for the epilogue.
// Two shared-memory round trips for N = 512 instead of four, and one buffer
// instead of two.  Every thread of the CTA must call reg_fft together (the
// stages use __syncthreads()).
#pragma once
#include <type_traits>

#include "spectral.cuh"

namespace pf {

template <int N>
struct RegFftShape {
  static constexpr int log2n() {
    int l = 0;
    for (int n = N; n > 1; n >>= 1) ++l;
    return l;
  }
  static constexpr int NT = N / 8;
  static constexpr int P0 = log2n() % 3 == 0 ? 8 : (log2n() % 3 == 1 ? 2 : 4);  // first radix
  static_assert(N >= 64 && N <= 4096 && (N & (N - 1)) == 0, "power of two in [64, 4096]");
};

// Shared-memory slot of element i of a line: one pad element after every 8, so
// that the strided accesses of the radix-8 stages (8t + c, 64j + k + 8c) fall
// in distinct banks.  A line buffer holds fft_pad_len(N) elements.
// (PAD = false: element i at slot i.)
template <bool PAD = true>
__host__ __device__ constexpr int fft_pad(int i) { return PAD ? i + (i >> 3) : i; }
__host__ __device__ constexpr int fft_pad_len(int n) { return n + n / 8; }

template <class T, int P>
__device__ __forceinline__ void reg_dft(cpx<T>* z, int sign) {
  if constexpr (P == 8) dft8<T>(z, sign);
  else dft_small<T, P>(z, sign);
}

// one stage; FIRST: inputs already in registers; LAST: outputs stay in registers.
// E elements a thread (8 or 16): NT = N/E threads a line, E/P butterflies a stage.
// sm element i sits at sm[fft_pad(i) * ss] (ss = 1 for a line buffer of its own; the
// y transform interleaves its columns, ss = columns per CTA, so that the
// threads of a warp, which are consecutive columns, hit consecutive banks).
template <class T, int N, int E, int L, int P, bool FIRST, bool PAD>
__device__ __forceinline__ void reg_stage(cpx<T> (&v)[E], cpx<T>* __restrict__ sm, const cpx<T>* __restrict__ tw,
                                          int sign, int t, int ss) {
  constexpr int NT = N / E, M = N / (L * P), NB = E / P;
  constexpr bool LAST = L * P == N;
  if constexpr (!FIRST) {
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int bf = t + NT * i, j = bf / M, k = bf % M;
#pragma unroll
      for (int c = 0; c < P; ++c) v[i + NB * c] = sm[fft_pad<PAD>(j * M * P + k + c * M) * ss];
    }
    if constexpr (!LAST) __syncthreads();  // every read of this stage before the in-place writes
  }
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int bf = t + NT * i, j = bf / M, k = bf % M;
    cpx<T> z[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      cpx<T> a = v[i + NB * c];
      if (!FIRST && c > 0) {
        cpx<T> w = tw[c * j * M];
        if (sign > 0) w.im = -w.im;
        a = a * w;
      }
      z[c] = a;
    }
    reg_dft<T, P>(z, sign);
    if constexpr (LAST) {
      // M = 1: dst = j + L q = t + NT (i + NB q)
#pragma unroll
      for (int q = 0; q < P; ++q) v[i + NB * q] = z[q];
    } else {
#pragma unroll
      for (int q = 0; q < P; ++q) sm[fft_pad<PAD>((j + L * q) * M + k) * ss] = z[q];
    }
  }
  if constexpr (!LAST) __syncthreads();
}

template <class T, int N, int E, int L, bool PAD>
__device__ __forceinline__ void reg_rest(cpx<T> (&v)[E], cpx<T>* sm, const cpx<T>* tw, int sign, int t, int ss) {
  if constexpr (L < N) {
    reg_stage<T, N, E, L, 8, false, PAD>(v, sm, tw, sign, t, ss);
    reg_rest<T, N, E, L * 8, PAD>(v, sm, tw, sign, t, ss);
  }
}

// Whole transform of one line: thread t (0 <= t < N/E) holds x[t + NT c] in
// v[c] on entry and X[t + NT q] in v[q] on exit; sm is the line's N-element
// shared buffer, element i at sm[fft_pad(i) * ss] (its contents are undefined
// afterwards); tw[m] = exp(-2 pi i m/N).
template <class T, int N, int E = 8, bool PAD = true>
__device__ __forceinline__ void reg_fft(cpx<T> (&v)[E], cpx<T>* sm, const cpx<T>* tw, int sign, int t, int ss = 1) {
  using S = RegFftShape<N>;
  reg_stage<T, N, E, 1, S::P0, true, PAD>(v, sm, tw, sign, t, ss);
  reg_rest<T, N, E, S::P0, PAD>(v, sm, tw, sign, t, ss);
}

// ---------------------------------------------------------------------------
// Forward real FFT along x, two real lines per complex transform (as
// k_rfft_x in spectral.cuh): a CTA of NT * LPC threads owns LPC line pairs.
// smem: LPC * fft_pad_len(N) complex.  FP32 is held to 48 registers (five
// 256-thread CTAs per SM instead of four), which measured faster.
// ---------------------------------------------------------------------------
template <class T, int N, class Pro>
__global__ void __launch_bounds__(1024) __maxnreg__(sizeof(T) == 4 ? 48 : 64) k_rfft_x_reg(Pro pro, cpx<T>* __restrict__ out, int nlines, int pitch,
                                                     const cpx<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int NT = N / 8;
  const int m = threadIdx.x / NT, t = threadIdx.x % NT;
  const int lpc = blockDim.x / NT;
  const int l0 = 2 * (blockIdx.x * lpc + m), l1 = l0 + 1;
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw) + (size_t)m * fft_pad_len(N);
  cpx<T> v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int x = t + NT * c;
    v[c] = mk<T>(l0 < nlines ? pro(l0, x) : (T)0, l1 < nlines ? pro(l1, x) : (T)0);
  }
  reg_fft<T, N>(v, sm, tw, -1, t);
  __syncthreads();  // the last stage's reads of sm are done
#pragma unroll
  for (int q = 0; q < 8; ++q) sm[fft_pad(t + NT * q)] = v[q];
  __syncthreads();
  if (l0 >= nlines) return;
  for (int k = t; k <= N / 2; k += NT) {
    const cpx<T> zk = sm[fft_pad(k)];
    const cpx<T> zn = conjg(sm[fft_pad(k == 0 ? 0 : N - k)]);
    out[(size_t)l0 * pitch + k] = scal(zk + zn, (T)0.5);
    const cpx<T> dd = zk - zn;  // B = -i/2 dd
    if (l1 < nlines) out[(size_t)l1 * pitch + k] = mk(dd.im * (T)0.5, -dd.re * (T)0.5);
  }
}

// ---------------------------------------------------------------------------
// Inverse real FFT along x (as k_irfft_x): the input A + iB of each line pair
// is built in registers from the two half spectra, the output goes from
// registers to the epilogue.  An epilogue with kNPre > 0 has its kNPre arrays
// copied into shared memory by cp.async before the transform (smem after the
// line buffers: LPC * 2 * kNPre * N elements of T).  Line buffers: LPC * N complex.
// ---------------------------------------------------------------------------
template <class T, int N, class Epi>
__global__ void __launch_bounds__(1024) k_irfft_x_reg(const cpx<T>* __restrict__ in, Epi epi, int nlines, int pitch,
                                                      const cpx<T>* __restrict__ tw, T scale) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int NT = N / 8;
  constexpr int NP = Epi::kNPre;
  const int m = threadIdx.x / NT, t = threadIdx.x % NT;
  const int lpc = blockDim.x / NT;
  const int l0 = 2 * (blockIdx.x * lpc + m), l1 = l0 + 1;
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw) + (size_t)m * N;  // unpadded line buffers
  // [line of the pair][array][N]
  T* pre = reinterpret_cast<T*>(reinterpret_cast<cpx<T>*>(smraw) + (size_t)lpc * N) + (size_t)m * 2 * NP * N;
  if constexpr (NP > 0) {
#pragma unroll
    for (int li = 0; li < 2; ++li) {
      const int l = l0 + li;
      if (l >= nlines) continue;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const T* src = epi.pre(j) + (size_t)l * epi.pre_n();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int x = t + NT * q;
          cp_async_elem(pre + (size_t)(li * NP + j) * N + x, src + x);
        }
      }
    }
    cp_async_commit();
  }
  cpx<T> v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int x = t + NT * c;
    const int k = x <= N / 2 ? x : N - x;
    cpx<T> A = mk<T>(0, 0), B = mk<T>(0, 0);
    if (l0 < nlines) A = in[(size_t)l0 * pitch + k];
    if (l1 < nlines) B = in[(size_t)l1 * pitch + k];
    if (x > N / 2) {
      A = conjg(A);
      B = conjg(B);
    }
    v[c] = mk(A.re - B.im, A.im + B.re);  // A + i B
  }
  reg_fft<T, N, 8, false>(v, sm, tw, +1, t);  // unpadded here: fewer registers measured faster
  if constexpr (NP > 0) cp_async_wait_all();  // this thread's own copies
  if (l0 >= nlines) return;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int x = t + NT * q;
    if constexpr (NP > 0) {
      epi.apply(l0, x, v[q].re * scale, pre + x, N);
      if (l1 < nlines) epi.apply(l1, x, v[q].im * scale, pre + (size_t)NP * N + x, N);
    } else {
      epi(l0, x, v[q].re * scale);
      if (l1 < nlines) epi(l1, x, v[q].im * scale);
    }
  }
}

// ---------------------------------------------------------------------------
// Complex FFT along y, in place (as k_fft_y): a CTA of NT * TXC threads
// (NT = N/E) owns TXC consecutive kx columns of one z level; thread (t, col) =
// threadIdx (t * TXC + col), so each warp reads rows of TXC contiguous values.
// smem: TXC * fft_pad_len(N) complex.  FP32 lines of 512 and more are
// compiled for two 512-thread CTAs per SM (64 registers, a few spilled): the
// transform waits on DRAM, and twice the resident warps measured faster; the
// shorter lines measured faster without the cap.
// ---------------------------------------------------------------------------
template <class T, int N, int E>
__global__ void __launch_bounds__(512, (sizeof(T) == 4 && N >= 512) ? 2 : 1) k_fft_y_reg(cpx<T>* __restrict__ data, int pitch, int ncol,
                                                   const cpx<T>* __restrict__ tw, int sign) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int NT = N / E;
  const int txc = blockDim.x / NT;
  const int col = threadIdx.x % txc, t = threadIdx.x / txc;
  const int c = blockIdx.x * txc + col;
  const bool in = c < ncol;
  cpx<T>* base = data + (size_t)blockIdx.y * N * pitch + c;
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw) + col;  // columns interleaved: element i at sm[i * txc]
  cpx<T> v[E];
#pragma unroll
  for (int q = 0; q < E; ++q) v[q] = in ? base[(size_t)(t + NT * q) * pitch] : mk<T>(0, 0);
  reg_fft<T, N, E>(v, sm, tw, sign, t, txc);
  if (!in) return;
#pragma unroll
  for (int q = 0; q < E; ++q) base[(size_t)(t + NT * q) * pitch] = v[q];
}

}  // namespace pf

namespace pf {

// sizes with a register-resident kernel
__host__ __device__ inline bool reg_fft_size(int n) { return n >= 64 && n <= 1024 && (n & (n - 1)) == 0; }

// call f(std::integral_constant<int, N>{}) for the runtime size n (one of reg_fft_size)
template <class F>
inline void reg_fft_dispatch(int n, F&& f) {
  switch (n) {
    case 64: f(std::integral_constant<int, 64>{}); break;
    case 128: f(std::integral_constant<int, 128>{}); break;
    case 256: f(std::integral_constant<int, 256>{}); break;
    case 512: f(std::integral_constant<int, 512>{}); break;
    default: f(std::integral_constant<int, 1024>{}); break;
  }
}

}  // namespace pf
