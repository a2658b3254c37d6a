// Wall-normal tridiagonal solves of the transform solvers (Eqs. NS26-NS27,
// NS36-NS37 after the DFT along x and y), parallel along z.
//
// Per (kx, ky) mode and real/imaginary part, the system along z (rows scaled
// by h^2: off-diagonals 1, diagonal D_k = -2 - sigma inside, the boundary
// value at the two end rows, sigma = (k^2 + shift) h^2) is solved by LU:
//   factors   m_k = 1 / (D_k - m_{k-1}),             m_{-1} = 0
//   forward   d_k = m_k (r_k - d_{k-1})              (r = scale h^2 rhs)
//   backward  x_k = d_k - m_k x_{k+1}
// and, for the pair (L - shift2) y = h^2 x of the CH step, solve 2 is
// eliminated from the last row down while solve 1 substitutes, with the
// factors g_k = m2_{R-1-k} of the mirrored recurrence (the end rows are the
// same at both walls):
//   q_k = g_k (h^2 x_k - q_{k+1}),   y_k = q_k - g_k y_{k-1}.
// Every step above is a first-order linear recurrence z_k = a_k z_prev + b_k.
// The rows are cut into segments of ZSEG = 16; thread (lane, segment) keeps its
// 16 values in registers, runs each recurrence over its segment from a zero
// start while multiplying up a_k, then adds the carried-in value times the
// running product once the segment ends of all earlier segments are combined.
// The factors have a closed form (LuClosed below), so every thread forms those
// of its own rows.
// A lane is one real component of one kx column; consecutive lanes are
// consecutive reals of a row, so every row of a segment is one coalesced
// access per warp.  The segment length is fixed, so the arithmetic of a
// column does not depend on the columns per CTA.
#pragma once
#include <cstddef>
#include <type_traits>

#include "df.cuh"
#include "spectral.cuh"

namespace pf {

constexpr int ZSEG = 16;

// the primal value of a factor (the value itself, or a dual number's value)
template <class TC>
__device__ __forceinline__ TC zs_val(TC x) { return x; }
__device__ __forceinline__ double zs_val(Dual x) { return x.v; }
__device__ __forceinline__ double zs_val(DF x) { return (double)x; }

// the per-row division of the FP32 factors: a fast divide (within 2 ulp; the
// operands are ratios of order one), where a correctly rounded one costs several
// times the instructions on every row of every solve; wider types divide exactly
template <class TC>
__device__ __forceinline__ TC zs_div(TC a, TC b) { return a / b; }
template <>
__device__ __forceinline__ float zs_div<float>(float a, float b) { return __fdividef(a, b); }

template <class TC>
__device__ __forceinline__ TC zs_exp2(TC x) { return exp2(x); }
template <>
__device__ __forceinline__ float zs_exp2<float>(float x) { return exp2f(x); }
template <class TC>
__device__ __forceinline__ TC zs_log2(TC x) { return log2(x); }
template <>
__device__ __forceinline__ float zs_log2<float>(float x) { return log2f(x); }

// LU factors of the z system in closed form.  With the interior diagonal
// D = -2 - sigma, the pivots are ratios U_{k+1}/U_k of U_{k+1} = D U_k - U_{k-1},
// U_0 = 1, U_1 = D_0 (the end-row diagonal), so with the roots l1 (|l1| > 1) and
// l2 = 1/l1 of x^2 - D x + 1, rho = l2/l1 and beta = (l1 - D_0)/(D_0 - l2):
//   m_k = U_k / U_{k+1} = (1/l1) (1 + beta rho^k) / (1 + beta rho^{k+1}),  k < R-1,
// and the last row, whose diagonal is the other end row, m_{R-1} = 1/(D_0 - m_{R-2}).
// D^2 - 4 is formed as sigma (sigma + 4) to avoid cancellation.  (sigma = 0, the
// singular Poisson mode, gives NaN; that column is not stored.)
template <class TC>
struct LuClosed {
  TC il1, beta, lr, d0;
  int R;
  __device__ __forceinline__ LuClosed(int rows, int bc, TC sg) : R(rows) {
    const TC D = (TC)-2 - sg;
    d0 = zdiag<TC>(0, rows, bc, sg);
    const TC l1 = (D - sqrt(sg * (sg + (TC)4))) * (TC)0.5;
    const TC l2 = (TC)1 / l1;
    il1 = l2;
    beta = (l1 - d0) / (d0 - l2);
    lr = zs_log2<TC>(l2 / l1);
  }
  __device__ __forceinline__ TC interior(int k) const {
    const TC pk = zs_exp2<TC>((TC)k * lr);
    const TC pk1 = zs_exp2<TC>((TC)(k + 1) * lr);
    return il1 * ((TC)1 + beta * pk) / ((TC)1 + beta * pk1);
  }
  __device__ __forceinline__ TC m(int k) const {
    if (R == 1) return (TC)1 / d0;
    if (k < R - 1) return interior(k);
    return (TC)1 / (d0 - interior(R - 2));
  }
};

// smem (TC): f1[R][tx], f2[R][tx] (pair with two shifts), car[4 phases][2][S][L]
template <class T, class TC>
__global__ void __launch_bounds__(512, sizeof(TC) == 4 ? 2 : 1) k_zsolve_seg(cpx<T>* __restrict__ data, const double* __restrict__ eigx,
                                                     const double* __restrict__ eigy, const ZSolve zs, const int tx) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int R = zs.rows;
  const int L = 2 * tx;
  const int S = (R + ZSEG - 1) / ZSEG;
  const int lane = threadIdx.x % L, s = threadIdx.x / L;
  const int c = lane >> 1;
  const int ky = blockIdx.y;
  const int col0 = blockIdx.x * tx;
  const int col = col0 + c;
  const bool in = col < zs.ncol;
  const bool dual = zs.two && !zs.same;
  TC* f1 = reinterpret_cast<TC*>(smraw);
  TC* f2 = dual ? f1 + (size_t)R * tx : f1;
  TC* car = f1 + (size_t)R * tx * (dual ? 2 : 1);  // [4][2][S][L]
  TC* ccol = car + (size_t)8 * S * L;               // (8-byte factors) [2][tx][6], see below
  const int k0 = s * ZSEG;
  const int nk = max(0, min(ZSEG, R - k0));
  // ---- loads first: the rows of this lane, in flight during the factor phase ----
  T* gcol = reinterpret_cast<T*>(data + (size_t)ky * zs.pitch + col0) + lane;
  const size_t zstride = (size_t)zs.ny * zs.pitch * 2;  // reals between rows
  // the (0,0) column of a Poisson solve belongs to k_zero_mode (which may run
  // at the same time): neither read nor written here
  const bool keep = in && !(zs.skip_zero && col == 0 && ky == 0);
  TC v[ZSEG];
  {
    const T* gp = gcol + (size_t)k0 * zstride;
#pragma unroll
    for (int j = 0; j < ZSEG; ++j) {
      v[j] = (keep && j < nk) ? (TC)*gp : (TC)0;
      gp += zstride;
    }
  }
  // FP32 eliminations take -(lambda_x + lambda_y), h^2, the shifts and h^2 scale as
  // floats formed on the host by the same roundings: no FP64 instruction (a burst
  // of conversions at every CTA's start on GB300's slow FP64 pipe) in the kernel
  TC k2, h2, s1, s2, rs;
  if constexpr (std::is_same<TC, float>::value) {
    if (zs.k2f) {
      k2 = zs.k2f[(size_t)ky * zs.ncol + (in ? col : col0)];
      h2 = zs.h2f;
      s1 = zs.s1f;
      s2 = zs.s2f;
      rs = zs.rsf;
    }
  }
  if (!std::is_same<TC, float>::value || !zs.k2f) {
    k2 = (TC)(-(eigx[in ? col : col0] + eigy[ky]));
    h2 = (TC)zs.h2;
    s1 = zshift<TC>(zs.shift1, zs.dshift1);
    s2 = zshift<TC>(zs.shift2, zs.dshift2);
    rs = (TC)(zs.h2 * zs.scale);
  }
  const TC sg1 = (k2 + s1) * h2;
  const TC sg2 = (k2 + s2) * h2;
  // ---- factors in closed form: the two lanes of a column share the rows ----
  // Each lane forms rows k0 + part, k0 + part + 2, ...; rho^k is advanced by
  // rho^2 from row to row instead of being raised afresh.  In FP64, from row kc
  // on, |beta rho^k| <= 2^-60: 1 + beta rho^k rounds to 1 and the interior
  // factor is 1/l1 exactly, so it is stored without the division, and a warp
  // whose rows all have it takes it from a register in the passes below.
  const int part = lane & 1;
  // (the convergence row: a row estimate with one row of margin)
  auto conv_row = [&](const LuClosed<TC>& lu) {
    using S = decltype(zs_val(lu.beta));
    const S lthr = (S)-60;  // log2 of the threshold
    const S ab = fabs(zs_val(lu.beta)), lr = zs_val(lu.lr);
    if (ab == (S)0) return 0;
    const S la = log2(ab);
    if (la <= lthr) return 0;
    if (!(lr < (S)-1e-6)) return R;
    const S k = ceil((lthr - la) / lr) + (S)1;
    return k >= (S)R ? R : (int)k;
  };
  // stores the factors of this lane's rows; returns the convergence row kc and 1/l1.
  // (Only 8-byte factors -- FP64, double-float -- skip the division and take the
  // constant passes: there a division costs far more than the registers the extra
  // paths take; the FP32 form would spill.  They also form a column's constants
  // once, in one thread, and every segment its rho^k by powers of rho: the
  // closed form's square root, logarithm and exponentials run at the FP64 rate
  // and would otherwise be repeated by all segments of the column.)
  constexpr bool kConst = sizeof(TC) == 8;  // FP64 and double-float
  if constexpr (kConst) {
    if (s == 0 && part == 0)
      for (int w = 0; w < (dual ? 2 : 1); ++w) {
        const LuClosed<TC> lu(R, zs.bc, w == 0 ? sg1 : sg2);
        TC* cst = ccol + ((size_t)w * tx + c) * 6;
        cst[0] = lu.il1;
        cst[1] = lu.beta;
        cst[2] = zs_exp2<TC>(lu.lr);  // rho
        cst[3] = lu.d0;
        cst[4] = R == 1 ? (TC)1 / lu.d0 : (TC)1 / (lu.d0 - lu.interior(R - 2));  // the last row
        cst[5] = (TC)conv_row(lu);
      }
    __syncthreads();
  }
  auto ipow = [](TC x, int n) {
    TC r = (TC)1;
    while (n) {
      if (n & 1) r *= x;
      x *= x;
      n >>= 1;
    }
    return r;
  };
  auto factors = [&](TC sg, TC* f, TC& il, int w) {
    TC beta, rho, d0, mlast;
    int kc;
    if constexpr (kConst) {
      const TC* cst = ccol + ((size_t)w * tx + c) * 6;
      il = cst[0];
      beta = cst[1];
      rho = cst[2];
      d0 = cst[3];
      mlast = cst[4];
      kc = (int)zs_val(cst[5]);
    } else {
      const LuClosed<TC> lu(R, zs.bc, sg);
      il = lu.il1;
      beta = lu.beta;
      rho = zs_exp2<TC>(lu.lr);
      d0 = lu.d0;
      mlast = R == 1 ? (TC)1 / lu.d0 : (TC)1 / (lu.d0 - lu.interior(R - 2));
      kc = R;
    }
    (void)d0;
    const TC rho2 = rho * rho;
    TC pk;  // rho^k
    if constexpr (kConst) pk = ipow(rho, k0 + part);
    else {
      const LuClosed<TC> lu(R, zs.bc, sg);
      pk = zs_exp2<TC>((TC)(k0 + part) * lu.lr);
    }
    for (int j = part; j < nk; j += 2) {
      const int k = k0 + j;
      TC m;
      if (k < R - 1) {
        if (k >= kc) m = il;
        else m = zs_div<TC>(il * ((TC)1 + beta * pk), (TC)1 + beta * pk * rho);
      } else {
        m = mlast;
      }
      f[(size_t)k * tx + c] = m;
      pk *= rho2;
    }
    return kc;
  };
  TC il1, il2;
  const int kc1 = factors(sg1, f1, il1, 0);
  int kc2 = kc1;
  il2 = il1;
  if (dual) kc2 = factors(sg2, f2, il2, 1);
  // segments whose rows all take the constant factor, per solve (solve 2 reads
  // its factors mirrored, g_k = m2_{R-1-k}), decided for the whole warp so that
  // the passes below do not diverge
  bool c1 = false, c2 = false;
  if constexpr (kConst) {
    const unsigned wmask = __activemask();
    const bool full_seg = nk == ZSEG;
    c1 = __all_sync(wmask, full_seg && k0 >= kc1 && k0 + nk - 1 <= R - 2);
    c2 = __all_sync(wmask, full_seg && k0 >= 1 && k0 + nk - 1 <= R - 1 - kc2);
  }
  __syncthreads();
  // carried-in value of a linear recurrence, from the (product, last) pairs of the earlier segments
  auto carry_fwd = [&](const TC* cp) -> TC {
    const TC* cz = cp + (size_t)S * L;
    TC g = 0;
    for (int t = 0; t < s; ++t) g = cp[(size_t)t * L + lane] * g + cz[(size_t)t * L + lane];
    return g;
  };
  auto carry_bwd = [&](const TC* cp) -> TC {
    const TC* cz = cp + (size_t)S * L;
    TC g = 0;
    for (int t = S - 1; t > s; --t) g = cp[(size_t)t * L + lane] * g + cz[(size_t)t * L + lane];
    return g;
  };
  TC* cA = car;
  TC* cB = car + (size_t)2 * S * L;
  TC* cC = car + (size_t)4 * S * L;
  TC* cD = car + (size_t)6 * S * L;
  // Every pass below runs between barriers; a full segment (all but possibly
  // the last) takes a copy of the loop without the row-count predicate, and a
  // segment of constant factors one that takes them from a register.
  const bool full = nk == ZSEG;
  auto pass = [&](bool cst, auto&& body) {
    if constexpr (kConst) {
      if (full && cst) {
        body(std::true_type{}, std::true_type{});
        return;
      }
    }
    if (full) body(std::true_type{}, std::false_type{});
    else body(std::false_type{}, std::false_type{});
  };
  const TC* m1 = f1 + c;                         // m_k at m1[k * tx]
  const TC* g2 = f2 + (size_t)(R - 1) * tx + c;  // g_k = m2_{R-1-k} at g2[-k * tx]
  auto M1 = [&](auto C, int k) -> TC {
    if constexpr (decltype(C)::value) return il1;
    else return m1[(size_t)k * tx];
  };
  auto G2 = [&](auto C, int k) -> TC {
    if constexpr (decltype(C)::value) return il2;
    else return g2[-(ptrdiff_t)k * tx];
  };
  // ---- solve 1, forward: d_k = -m_k d_{k-1} + m_k r_k ----
  pass(c1, [&](auto F, auto C) {
    constexpr bool FULL = decltype(F)::value;
    TC z = 0, P = 1;
#pragma unroll
    for (int j = 0; j < ZSEG; ++j)
      if (FULL || j < nk) {
        const TC m = M1(C, k0 + j);
        z = m * (v[j] * rs - z);
        v[j] = z;
        P *= -m;
      }
    cA[(size_t)s * L + lane] = P;
    cA[(size_t)(S + s) * L + lane] = z;
  });
  __syncthreads();
  // ---- fix-up of solve 1 forward, then solve 1 backward: x_k = -m_k x_{k+1} + d_k ----
  pass(c1, [&](auto F, auto C) {
    constexpr bool FULL = decltype(F)::value;
    const TC g = carry_fwd(cA);
    TC p = 1;
#pragma unroll
    for (int j = 0; j < ZSEG; ++j)
      if (FULL || j < nk) {
        p *= -M1(C, k0 + j);
        v[j] += p * g;
      }
    TC z = 0, P = 1;
#pragma unroll
    for (int j = ZSEG - 1; j >= 0; --j)
      if (FULL || j < nk) {
        const TC m = M1(C, k0 + j);
        z = v[j] - m * z;
        v[j] = z;
        P *= -m;
      }
    cB[(size_t)s * L + lane] = P;
    cB[(size_t)(S + s) * L + lane] = z;
  });
  __syncthreads();
  auto store = [&](auto F) {
    constexpr bool FULL = decltype(F)::value;
    if (!keep) return;
    T* gp = gcol + (size_t)k0 * zstride;
#pragma unroll
    for (int j = 0; j < ZSEG; ++j)
      if (FULL || j < nk) {
        gp[0] = (T)v[j];
        gp += zstride;
      }
  };
  if (!zs.two) {
    pass(c1, [&](auto F, auto C) {
      constexpr bool FULL = decltype(F)::value;
      const TC g = carry_bwd(cB);
      TC p = 1;
#pragma unroll
      for (int j = ZSEG - 1; j >= 0; --j)
        if (FULL || j < nk) {
          p *= -M1(C, k0 + j);
          v[j] += p * g;
        }
      store(F);
    });
    return;
  }
  // ---- finish solve 1 and run solve 2's elimination in the same backward pass ----
  pass(c1 && c2, [&](auto F, auto C) {
    constexpr bool FULL = decltype(F)::value;
    const TC g = carry_bwd(cB);
    TC p = 1, z = 0, P = 1;
#pragma unroll
    for (int j = ZSEG - 1; j >= 0; --j)
      if (FULL || j < nk) {
        const int k = k0 + j;
        p *= -M1(C, k);
        const TC x = v[j] + p * g;
        const TC gk = G2(C, k);
        z = gk * (h2 * x - z);
        v[j] = z;
        P *= -gk;
      }
    cC[(size_t)s * L + lane] = P;
    cC[(size_t)(S + s) * L + lane] = z;
  });
  __syncthreads();
  // ---- fix-up of solve 2's elimination, then its forward substitution: y_k = -g_k y_{k-1} + q_k ----
  pass(c2, [&](auto F, auto C) {
    constexpr bool FULL = decltype(F)::value;
    const TC g = carry_bwd(cC);
    TC p = 1;
#pragma unroll
    for (int j = ZSEG - 1; j >= 0; --j)
      if (FULL || j < nk) {
        p *= -G2(C, k0 + j);
        v[j] += p * g;
      }
    TC z = 0, P = 1;
#pragma unroll
    for (int j = 0; j < ZSEG; ++j)
      if (FULL || j < nk) {
        const TC gk = G2(C, k0 + j);
        z = v[j] - gk * z;
        v[j] = z;
        P *= -gk;
      }
    cD[(size_t)s * L + lane] = P;
    cD[(size_t)(S + s) * L + lane] = z;
  });
  __syncthreads();
  pass(c2, [&](auto F, auto C) {
    constexpr bool FULL = decltype(F)::value;
    const TC g = carry_fwd(cD);
    TC p = 1;
#pragma unroll
    for (int j = 0; j < ZSEG; ++j)
      if (FULL || j < nk) {
        p *= -G2(C, k0 + j);
        v[j] += p * g;
      }
    store(F);
  });
}

// shared memory of k_zsolve_seg in bytes
template <class TC>
inline size_t zsolve_seg_smem(int rows, int tx, bool dual) {
  const int S = (rows + ZSEG - 1) / ZSEG;
  return sizeof(TC) * ((size_t)rows * tx * (dual ? 2 : 1) + (size_t)8 * S * 2 * tx + (sizeof(TC) == 8 ? 12 * tx : 0));
}

}  // namespace pf
