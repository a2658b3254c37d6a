// Shared-memory mixed-radix Stockham FFT used by the transform solves.
//
// The paper solves its constant-coefficient Helmholtz/Poisson problems with
// an FFT-based direct solver along the periodic directions (Section 3.2.1 and
// 3.2.2, the FFT solver of the CaNS code).  Here every periodic line is
// transformed in shared memory by a CTA-wide self-sorting (Stockham)
// mixed-radix FFT.  Stage t combines sub-transforms of length L into length
// L*p: with M = n/(L*p), butterfly (j, k), j < L, k < M, gathers
//   z_c = w_{L p}^{c j} * Y[j*M*p + k + c*M],   c = 0..p-1
// and writes the length-p DFT of z to Y'[(j + L*q)*M + k], q = 0..p-1.
// The input is in natural order and so is the output.  w_m = exp(-2 pi i/m)
// for a forward transform, its conjugate for an inverse one (no 1/n scaling).
#pragma once
#include "common.cuh"

namespace pf {

// cos/sin(2 pi m/p) for the odd radices (exact values of the roots of unity)
__device__ __forceinline__ double root_cos(int p, int m) {
  if (p == 3) return -0.5;
  if (p == 5) return (m == 1 || m == 4) ? 0.30901699437494742 : -0.80901699437494742;
  // p == 7
  if (m == 1 || m == 6) return 0.62348980185873353;
  if (m == 2 || m == 5) return -0.22252093395631440;
  return -0.90096886790241913;
}
__device__ __forceinline__ double root_sin(int p, int m) {
  double s;
  if (p == 3) s = 0.86602540378443865;
  else if (p == 5) s = (m == 1 || m == 4) ? 0.95105651629515357 : 0.58778525229247313;
  else s = (m == 1 || m == 6) ? 0.78183148246802981 : ((m == 2 || m == 5) ? 0.97492791218182361 : 0.43388373911755812);
  return (2 * m > p) ? -s : s;
}

// length-p DFT in registers; sign = -1 forward, +1 inverse
template <class T, int P>
__device__ __forceinline__ void dft_small(cpx<T>* z, int sign) {
  if constexpr (P == 2) {
    cpx<T> a = z[0], b = z[1];
    z[0] = a + b;
    z[1] = a - b;
  } else if constexpr (P == 4) {
    cpx<T> s02 = z[0] + z[2], d02 = z[0] - z[2];
    cpx<T> s13 = z[1] + z[3], d13 = z[1] - z[3];
    cpx<T> r = mul_si(d13, sign);
    z[0] = s02 + s13;
    z[2] = s02 - s13;
    z[1] = d02 + r;
    z[3] = d02 - r;
  } else {
    constexpr int H = (P - 1) / 2;
    cpx<T> sp[H], sm[H];
#pragma unroll
    for (int c = 1; c <= H; ++c) {
      sp[c - 1] = z[c] + z[P - c];
      sm[c - 1] = z[c] - z[P - c];
    }
    cpx<T> out[P];
    cpx<T> s0 = z[0];
#pragma unroll
    for (int c = 0; c < H; ++c) s0 = s0 + sp[c];
    out[0] = s0;
#pragma unroll
    for (int q = 1; q < P; ++q) {
      cpx<T> acc = z[0];
      cpx<T> accs = mk<T>(0, 0);
#pragma unroll
      for (int c = 1; c <= H; ++c) {
        int m = (c * q) % P;
        T cs = (T)root_cos(P, m), sn = (T)root_sin(P, m);
        acc = acc + scal(sp[c - 1], cs);
        accs = accs + scal(sm[c - 1], sn);
      }
      out[q] = acc + mul_si(accs, sign);
    }
#pragma unroll
    for (int q = 0; q < P; ++q) z[q] = out[q];
  }
}

// length-8 DFT (split into two length-4 DFTs of the even and odd samples)
template <class T>
__device__ __forceinline__ void dft8(cpx<T>* z, int sign) {
  cpx<T> e[4] = {z[0], z[2], z[4], z[6]};
  cpx<T> o[4] = {z[1], z[3], z[5], z[7]};
  dft_small<T, 4>(e, sign);
  dft_small<T, 4>(o, sign);
  const T r = (T)0.70710678118654752440;
  // w^q = exp(sign * 2 pi i q/8), q = 1, 2, 3
  const cpx<T> o1 = mk<T>(r * (o[1].re - sign * o[1].im), r * (o[1].im + sign * o[1].re));
  const cpx<T> o2 = mul_si(o[2], sign);
  const cpx<T> o3 = mk<T>(r * (-o[3].re - sign * o[3].im), r * (-o[3].im + sign * o[3].re));
  z[0] = e[0] + o[0];
  z[4] = e[0] - o[0];
  z[1] = e[1] + o1;
  z[5] = e[1] - o1;
  z[2] = e[2] + o2;
  z[6] = e[2] - o2;
  z[3] = e[3] + o3;
  z[7] = e[3] - o3;
}

// Stockham stage with compile-time size, radix and sub-transform length (all
// powers of two): index arithmetic reduces to shifts and masks.
template <class T, int N, int P, int L>
__device__ __forceinline__ void fft_stage_c(const cpx<T>* __restrict__ in, cpx<T>* __restrict__ out,
                                            const cpx<T>* __restrict__ tw, int sign, int nl, int es, int ls,
                                            int tid, int nth) {
  constexpr int M = N / (L * P);
  constexpr int NBF = N / P;
  const int total = NBF * nl;
  const float inl = 1.0f / (float)nl;
  for (int id = tid; id < total; id += nth) {
    int l, bf;
    if (es == 1) {
      l = id / NBF;
      bf = id - l * NBF;
    } else {
      bf = qdiv(id, nl, inl);
      l = id - bf * nl;
    }
    const int j = bf / M, k = bf - j * M;
    const cpx<T>* src = in + (size_t)l * ls;
    cpx<T>* dst = out + (size_t)l * ls;
    cpx<T> z[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      cpx<T> v = src[(size_t)(j * M * P + k + c * M) * es];
      if (L > 1 && c > 0) {
        cpx<T> w = tw[c * j * M];
        if (sign > 0) w.im = -w.im;
        v = v * w;
      }
      z[c] = v;
    }
    if constexpr (P == 8) dft8<T>(z, sign);
    else dft_small<T, P>(z, sign);
#pragma unroll
    for (int q = 0; q < P; ++q) dst[(size_t)((j + L * q) * M + k) * es] = z[q];
  }
}

// radix-8 stages, then one radix-4 or radix-2 stage if N is not a power of 8
template <class T, int N, int L>
__device__ __forceinline__ cpx<T>* fft_pow2_run(cpx<T>* in, cpx<T>* out, const cpx<T>* tw, int sign, int nl, int es,
                                                int ls) {
  if constexpr (L >= N) {
    return in;
  } else {
    constexpr int REM = N / L;
    constexpr int P = REM % 8 == 0 ? 8 : (REM % 4 == 0 ? 4 : 2);
    fft_stage_c<T, N, P, L>(in, out, tw, sign, nl, es, ls, threadIdx.x, blockDim.x);
    __syncthreads();
    return fft_pow2_run<T, N, L * P>(out, in, tw, sign, nl, es, ls);
  }
}

template <class T>
__device__ __forceinline__ cpx<T>* fft_pow2(cpx<T>* a, cpx<T>* b, int n, const cpx<T>* tw, int sign, int nl, int es,
                                            int ls) {
  switch (n) {
    case 64: return fft_pow2_run<T, 64, 1>(a, b, tw, sign, nl, es, ls);
    case 128: return fft_pow2_run<T, 128, 1>(a, b, tw, sign, nl, es, ls);
    case 256: return fft_pow2_run<T, 256, 1>(a, b, tw, sign, nl, es, ls);
    case 512: return fft_pow2_run<T, 512, 1>(a, b, tw, sign, nl, es, ls);
    case 1024: return fft_pow2_run<T, 1024, 1>(a, b, tw, sign, nl, es, ls);
    default: return nullptr;
  }
}

// One Stockham stage of radix P over nl lines.  Element n of line l sits at
// base[l*ls + n*es].  tw[m] = exp(-2 pi i m/n), m < n.
template <class T, int P>
__device__ void fft_stage(const cpx<T>* __restrict__ in, cpx<T>* __restrict__ out, int n, int L,
                          const cpx<T>* __restrict__ tw, int sign, int nl, int es, int ls, int tid,
                          int nth) {
  const int M = n / (L * P);
  const int nbf = n / P;
  const int total = nbf * nl;
  const float iM = 1.0f / (float)M, inbf = 1.0f / (float)nbf, inl = 1.0f / (float)nl;
  for (int id = tid; id < total; id += nth) {
    int l, bf;
    if (es == 1) {
      l = qdiv(id, nbf, inbf);
      bf = id - l * nbf;
    } else {
      bf = qdiv(id, nl, inl);
      l = id - bf * nl;
    }
    const int j = qdiv(bf, M, iM), k = bf - j * M;
    const cpx<T>* src = in + (size_t)l * ls;
    cpx<T>* dst = out + (size_t)l * ls;
    cpx<T> z[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      cpx<T> v = src[(size_t)(j * M * P + k + c * M) * es];
      if (c > 0 && j > 0) {
        cpx<T> w = tw[c * j * M];
        if (sign > 0) w.im = -w.im;
        v = v * w;
      }
      z[c] = v;
    }
    dft_small<T, P>(z, sign);
#pragma unroll
    for (int q = 0; q < P; ++q) dst[(size_t)((j + L * q) * M + k) * es] = z[q];
  }
}

// Whole transform.  a holds the input; b is scratch of the same size.  Returns
// the buffer holding the result.  Ends with __syncthreads().
template <class T>
__device__ cpx<T>* fft_lines(cpx<T>* a, cpx<T>* b, const FftPlan& pl, const cpx<T>* tw, int sign, int nl,
                             int es, int ls) {
  const int tid = threadIdx.x, nth = blockDim.x;
  if (pl.n >= 64 && pl.n <= 1024 && (pl.n & (pl.n - 1)) == 0) return fft_pow2<T>(a, b, pl.n, tw, sign, nl, es, ls);
  int L = 1;
  cpx<T>* in = a;
  cpx<T>* out = b;
  for (int s = 0; s < pl.ns; ++s) {
    const int p = pl.radix(s);
    switch (p) {
      case 2: fft_stage<T, 2>(in, out, pl.n, L, tw, sign, nl, es, ls, tid, nth); break;
      case 3: fft_stage<T, 3>(in, out, pl.n, L, tw, sign, nl, es, ls, tid, nth); break;
      case 4: fft_stage<T, 4>(in, out, pl.n, L, tw, sign, nl, es, ls, tid, nth); break;
      case 5: fft_stage<T, 5>(in, out, pl.n, L, tw, sign, nl, es, ls, tid, nth); break;
      default: fft_stage<T, 7>(in, out, pl.n, L, tw, sign, nl, es, ls, tid, nth); break;
    }
    __syncthreads();
    L *= p;
    cpx<T>* t = in;
    in = out;
    out = t;
  }
  return in;
}

}  // namespace pf
