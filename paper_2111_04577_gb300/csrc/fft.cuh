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
