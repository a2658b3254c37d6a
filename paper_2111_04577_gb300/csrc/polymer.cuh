// Log-conformation Oldroyd-B update on coarse centres (Section 3.2.3).
//
// RH of Eq. NS41 with alpha = 0 and the relaxation acting toward Theta = 0:
//   RH = -div(u Theta) + (Omega Theta - Theta Omega) + 2 B + (e^{-Theta} - I)/lambda_H,
// Omega and B from the decomposition of Eqs. NS21-NS24 with
// Theta = R diag(theta) R^T, lambda = e^theta, M~ = R^T (grad u)^T R.
// In the eigenbasis RH~ = R^T (RH + div(u Theta)) R is symmetric with
//   RH~_aa = 2 m_aa + (e^{-theta_a} - 1)/lambda_H,
//   RH~_ab = omega_ab (theta_b - theta_a)
//          = (lambda_b m_ab + lambda_a m_ba) (theta_b - theta_a)/(lambda_b - lambda_a),
// evaluated as (e^d m_ab + m_ba) d/expm1(d), d = theta_b - theta_a, which is
// finite as d -> 0 and equals there the equal-eigenvalue limit m_ab + m_ba
// (Omega = 0, B = sym(grad u^T), the zero-stress rule after Eq. NS24).
// RK2-TVD: Theta1 = Theta^n + dt RH(Theta^n) (Eq. NS42); Theta^{n+1} =
// Theta^n/2 + (Theta1 + dt RH(Theta1))/2 (Eq. NS44); tau_p = (mu_p/lambda_H)
// (R e^Lambda R^T - I) (Eq. NS46); the momentum equation receives
// tau = (1 + phi)/2 tau_p (Eq. NS12, droplet phase viscoelastic).
#pragma once
#include "common.cuh"

namespace pf {

template <class T>
__device__ __forceinline__ T dexpm1(T d);
template <>
__device__ __forceinline__ float dexpm1<float>(float d) {  // d / expm1(d)
  if (fabsf(d) < 1e-3f) return 1.f - 0.5f * d + d * d * (1.f / 12.f);
  return d / expm1f(d);
}
template <>
__device__ __forceinline__ double dexpm1<double>(double d) {
  if (fabs(d) < 1e-6) return 1.0 - 0.5 * d + d * d * (1.0 / 12.0);
  return d / expm1(d);
}

template <class T>
__device__ __forceinline__ T fexp(T x) { return exp(x); }
template <>
__device__ __forceinline__ float fexp<float>(float x) { return __expf(x); }

// one Jacobi rotation zeroing A[p][q] (A symmetric, full storage), V <- V J
template <class T, int N>
__device__ __forceinline__ void jacobi_rot(T A[N][N], T V[N][N], int p, int q) {
  const T apq = A[p][q];
  if (apq == (T)0) return;
  const T th = (A[q][q] - A[p][p]) / (2 * apq);
  const T ath = fabs(th);
  // t = sgn(th)/(|th| + sqrt(th^2 + 1)), the smaller root; 1/(2 th) when th^2 would overflow
  T t = ath > (T)1e15 ? (T)0.5 / ath : (T)1 / (ath + sqrt(ath * ath + (T)1));
  if (th < 0) t = -t;
  const T c = (T)1 / sqrt(t * t + (T)1), s = t * c;
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const T arp = A[r][p], arq = A[r][q];
    A[r][p] = c * arp - s * arq;
    A[r][q] = s * arp + c * arq;
  }
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const T apr = A[p][r], aqr = A[q][r];
    A[p][r] = c * apr - s * aqr;
    A[q][r] = s * apr + c * aqr;
  }
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const T vrp = V[r][p], vrq = V[r][q];
    V[r][p] = c * vrp - s * vrq;
    V[r][q] = s * vrp + c * vrq;
  }
}

// symmetric eigen-decomposition A = V diag(w) V^T by cyclic Jacobi rotations
template <class T, int N>
__device__ __forceinline__ void eig_sym(T A[N][N], T w[N], T V[N][N]) {
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int b = 0; b < N; ++b) V[a][b] = (a == b) ? (T)1 : (T)0;
  const T eps2 = sizeof(T) == 4 ? (T)1e-14 : (T)1e-30;
#pragma unroll 1
  for (int sweep = 0; sweep < (sizeof(T) == 4 ? 6 : 10); ++sweep) {
    T off = 0, dia = 0;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      dia += A[a][a] * A[a][a];
#pragma unroll
      for (int b = a + 1; b < N; ++b) off += A[a][b] * A[a][b];
    }
    if (off <= eps2 * dia || off == (T)0) break;
    if (N == 2) {
      jacobi_rot<T, N>(A, V, 0, 1);
    } else {
      jacobi_rot<T, N>(A, V, 0, 1);
      jacobi_rot<T, N>(A, V, 0, N - 1);
      jacobi_rot<T, N>(A, V, 1, N - 1);
    }
  }
#pragma unroll
  for (int a = 0; a < N; ++a) w[a] = A[a][a];
}

template <class T>
struct PolyIn {
  const T *u, *v, *w;  // u^{n+1} (w with both wall faces)
  const T* phic;       // restricted phi^{n+1} at centres
  const T* th[6];      // Theta to take RH of (component-major)
  const T* base[6];    // Theta^n (stage 2 only)
  T* out[6];           // Theta1 (stage 1) or Theta^{n+1} (stage 2)
  T* tau[6];           // weighted tau^{n+1} (stage 2)
};

// component maps: 2D (x, z) comps xx, xz, zz; 3D xx, yy, zz, xy, xz, yz
template <int N>
__device__ __forceinline__ int comp_of(int a, int b) {
  if (N == 2) return (a == b) ? (a == 0 ? 0 : 2) : 1;
  if (a == b) return a;
  const int s = a + b;  // (0,1) -> 3, (0,2) -> 4, (1,2) -> 5
  return s == 1 ? 3 : (s == 2 ? 4 : 5);
}

template <class T, int N>
__device__ __forceinline__ void k_polymer_b(PolyIn<T> P, Dims d, PhysT<T> q, int stage, const int3 bid, unsigned char* smraw) {
  const int plane = d.nx * d.ny;
  const T iD = q.iD;
  const T dt = q.dt, ilh = q.ilh;
  constexpr int NC = N == 2 ? 3 : 6;
  RowIdx x;
  if (!row_index_b(bid, d.nx, d.ny, x)) return;
  {
    const int i = x.i, j = x.j, k = x.k;
    const int id = x.row * d.nx + i;
    auto C = [&](int ii, int jj, int kk) { return (kk * d.ny + wrap(jj, d.ny)) * d.nx + wrap(ii, d.nx); };
    // velocity gradient L[a][b] = du_a/dx_b (Eq. NS23 uses its transpose convention)
    auto uc = [&](int ii, int jj, int kk) -> T {  // centre-averaged u, ghosts at walls
      if (kk < 0) return q.uw2_bot - (T)0.5 * (P.u[C(ii, jj, 0)] + P.u[C(ii + 1, jj, 0)]);
      if (kk >= d.nz) return q.uw2_top - (T)0.5 * (P.u[C(ii, jj, d.nz - 1)] + P.u[C(ii + 1, jj, d.nz - 1)]);
      return (T)0.5 * (P.u[C(ii, jj, kk)] + P.u[C(ii + 1, jj, kk)]);
    };
    auto vc = [&](int ii, int jj, int kk) -> T {
      if (kk < 0) return -(T)0.5 * (P.v[C(ii, jj, 0)] + P.v[C(ii, jj + 1, 0)]);
      if (kk >= d.nz) return -(T)0.5 * (P.v[C(ii, jj, d.nz - 1)] + P.v[C(ii, jj + 1, d.nz - 1)]);
      return (T)0.5 * (P.v[C(ii, jj, kk)] + P.v[C(ii, jj + 1, kk)]);
    };
    auto wc = [&](int ii, int jj, int kk) -> T { return (T)0.5 * (P.w[C(ii, jj, kk)] + P.w[C(ii, jj, kk + 1)]); };
    T L[N][N];
    const T dudx = (P.u[C(i + 1, j, k)] - P.u[id]) * iD;
    const T dwdz = (P.w[id + plane] - P.w[id]) * iD;
    const T dudz = (uc(i, j, k + 1) - uc(i, j, k - 1)) * (T)0.5 * iD;
    const T dwdx = (wc(i + 1, j, k) - wc(i - 1, j, k)) * (T)0.5 * iD;
    if (N == 2) {
      L[0][0] = dudx; L[0][1] = dudz;
      L[1][0] = dwdx; L[1][N - 1] = dwdz;
    } else {
      L[0][0] = dudx;
      L[0][1] = (uc(i, j + 1, k) - uc(i, j - 1, k)) * (T)0.5 * iD;
      L[0][N - 1] = dudz;
      L[1][0] = (vc(i + 1, j, k) - vc(i - 1, j, k)) * (T)0.5 * iD;
      L[1][1] = (P.v[C(i, j + 1, k)] - P.v[id]) * iD;
      L[1][N - 1] = (vc(i, j, k + 1) - vc(i, j, k - 1)) * (T)0.5 * iD;
      L[N - 1][0] = dwdx;
      L[N - 1][1] = (wc(i, j + 1, k) - wc(i, j - 1, k)) * (T)0.5 * iD;
      L[N - 1][N - 1] = dwdz;
    }
    // advection div(u Theta), central conservative fluxes, no wall flux
    T adv[NC];
    {
      const T ul = P.u[id], ur = P.u[C(i + 1, j, k)];
      const T wb = P.w[id], wt = P.w[id + plane];
      const int xm = C(i - 1, j, k), xp = C(i + 1, j, k);
#pragma unroll
      for (int cq = 0; cq < NC; ++cq) {
        const T t0 = P.th[cq][id];
        T a = (ur * (t0 + P.th[cq][xp]) - ul * (P.th[cq][xm] + t0));
        if (k + 1 < d.nz) a += wt * (t0 + P.th[cq][id + plane]);
        if (k > 0) a -= wb * (P.th[cq][id - plane] + t0);
        if (N == 3) {
          const T vl = P.v[id], vr = P.v[C(i, j + 1, k)];
          a += vr * (t0 + P.th[cq][C(i, j + 1, k)]) - vl * (P.th[cq][C(i, j - 1, k)] + t0);
        }
        adv[cq] = (T)0.5 * iD * a;
      }
    }
    // eigen-decomposition of Theta at the cell
    T A[N][N], th[N], R[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int b = 0; b < N; ++b) A[a][b] = P.th[comp_of<N>(a, b)][id];
    eig_sym<T, N>(A, th, R);
    // M~ = R^T L R
    T LR[N][N], Mt[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int b = 0; b < N; ++b) {
        T s = 0;
#pragma unroll
        for (int c = 0; c < N; ++c) s += L[a][c] * R[c][b];
        LR[a][b] = s;
      }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int b = 0; b < N; ++b) {
        T s = 0;
#pragma unroll
        for (int c = 0; c < N; ++c) s += R[c][a] * LR[c][b];
        Mt[a][b] = s;
      }
    // RH in the eigenbasis
    T H[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
      H[a][a] = 2 * Mt[a][a] + (fexp<T>(-th[a]) - (T)1) * ilh;
#pragma unroll
      for (int b = a + 1; b < N; ++b) {
        const T dd = th[b] - th[a];
        T o;
        if (dd > 0) o = (Mt[a][b] + fexp<T>(-dd) * Mt[b][a]) * dexpm1<T>(-dd);
        else o = (fexp<T>(dd) * Mt[a][b] + Mt[b][a]) * dexpm1<T>(dd);
        H[a][b] = o;
        H[b][a] = o;
      }
    }
    // back to the physical basis: R H R^T
    T HR[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int b = 0; b < N; ++b) {
        T s = 0;
#pragma unroll
        for (int c = 0; c < N; ++c) s += H[a][c] * R[b][c];
        HR[a][b] = s;
      }
    T newth[NC];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int b = a; b < N; ++b) {
        T s = 0;
#pragma unroll
        for (int c = 0; c < N; ++c) s += R[a][c] * HR[c][b];
        const int cq = comp_of<N>(a, b);
        const T rh = s - adv[cq];
        const T t0 = P.th[cq][id];
        newth[cq] = stage == 1 ? t0 + dt * rh : (T)0.5 * P.base[cq][id] + (T)0.5 * (t0 + dt * rh);
      }
#pragma unroll
    for (int cq = 0; cq < NC; ++cq) P.out[cq][id] = newth[cq];
    if (stage == 2) {
      // tau = (1 + phi)/2 (mu_p/lambda_H) (R e^theta R^T - I)
#pragma unroll
      for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) A[a][b] = newth[comp_of<N>(a, b)];
      eig_sym<T, N>(A, th, R);
      const T wgt = (T)0.5 * ((T)1 + P.phic[id]) * q.wtau;
#pragma unroll
      for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = a; b < N; ++b) {
          T s = 0;
#pragma unroll
          for (int c = 0; c < N; ++c) s += R[a][c] * fexp<T>(th[c]) * R[b][c];
          P.tau[comp_of<N>(a, b)][id] = wgt * (s - (a == b ? (T)1 : (T)0));
        }
    }
  }
}

template <class T, int N>
__global__ void k_polymer(PolyIn<T> P, Dims d, PhysT<T> q, int stage) {
  extern __shared__ __align__(16) unsigned char smraw[];
  k_polymer_b<T, N>(P, d, q, stage, make_int3(blockIdx.x, blockIdx.y, blockIdx.z), smraw);
}

}  // namespace pf
