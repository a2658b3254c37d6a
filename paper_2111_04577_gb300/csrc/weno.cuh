// WENO5-Z convective fluxes (Borges et al. 2008), the paper's scheme for the
// advection of phi in the CH step (Section 3.2.1) and of Theta in the
// log-conformation update (text before Eq. NS40); selected by
// pf_params.advection = 1 (0 keeps the central second-order flux).
//
// The face value at i+1/2 from the left (upwind for a face velocity >= 0) is
// the WENO-Z blend of the three third-order candidates on cells i-2..i+2:
//   q0 = (2 v_{i-2} - 7 v_{i-1} + 11 v_i)/6,  q1 = (-v_{i-1} + 5 v_i + 2 v_{i+1})/6,
//   q2 = (2 v_i + 5 v_{i+1} - v_{i+2})/6,
// with the Jiang-Shu smoothness indicators b_k, tau5 = |b0 - b2| and the
// weights a_k = d_k (1 + tau5/(b_k + eps)), (d0, d1, d2) = (1/10, 6/10, 3/10);
// for a negative face velocity the mirror stencil (cells i+3..i-1) gives it.
// The flux through the face is the face velocity times that value, and the
// term is the divergence of those fluxes (conservative).  Periodic axes wrap;
// at the walls the face flux is zero and the stencils read mirror ghosts
// v_{-1-m} = v_m, v_{n+m} = v_{n-1-m}.  eps = 1e-40 in FP64; FP32 takes 1e-30,
// the smallest normal-range value that keeps b_k + eps > 0 when the kernels
// flush subnormals (a flat stencil then has tau5 = 0 and ideal weights).
#pragma once

#include "ch.cuh"
#include "common.cuh"

namespace pf {

template <class T>
__device__ __forceinline__ T weno_eps() { return (T)1e-40; }
template <>
__device__ __forceinline__ float weno_eps<float>() { return 1e-30f; }

// face value at i+1/2 from the stencil (v_{i-2}, ..., v_{i+2})
template <class T>
__device__ __forceinline__ T weno5z_left(T vm2, T vm1, T v0, T vp1, T vp2) {
  const T s6 = (T)(1.0 / 6.0);
  const T q0 = ((T)2 * vm2 - (T)7 * vm1 + (T)11 * v0) * s6;
  const T q1 = (-vm1 + (T)5 * v0 + (T)2 * vp1) * s6;
  const T q2 = ((T)2 * v0 + (T)5 * vp1 - vp2) * s6;
  const T e0 = vm2 - (T)2 * vm1 + v0, f0 = vm2 - (T)4 * vm1 + (T)3 * v0;
  const T e1 = vm1 - (T)2 * v0 + vp1, f1 = vm1 - vp1;
  const T e2 = v0 - (T)2 * vp1 + vp2, f2 = (T)3 * v0 - (T)4 * vp1 + vp2;
  const T c13 = (T)(13.0 / 12.0), c14 = (T)0.25;
  const T b0 = c13 * e0 * e0 + c14 * f0 * f0;
  const T b1 = c13 * e1 * e1 + c14 * f1 * f1;
  const T b2 = c13 * e2 * e2 + c14 * f2 * f2;
  const T t5 = fabs(b0 - b2);
  const T eps = weno_eps<T>();
  const T a0 = (T)0.1 * ((T)1 + t5 / (b0 + eps));
  const T a1 = (T)0.6 * ((T)1 + t5 / (b1 + eps));
  const T a2 = (T)0.3 * ((T)1 + t5 / (b2 + eps));
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// upwind flux through the face between s2 and s3 of the six cells s0..s5
// (i-2..i+3 for the face i+1/2), face velocity uf
template <class T>
__device__ __forceinline__ T weno_flux(T uf, T s0, T s1, T s2, T s3, T s4, T s5) {
  return uf >= (T)0 ? uf * weno5z_left(s0, s1, s2, s3, s4) : uf * weno5z_left(s5, s4, s3, s2, s1);
}

__device__ __forceinline__ int weno_pmod(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}
// mirror ghost index across the walls of an axis of n cells (n >= 3)
__device__ __forceinline__ int zmirror(int k, int n) { return k < 0 ? -1 - k : (k >= n ? 2 * n - 1 - k : k); }

// div(u q) at cell (i, j, k) of an nx x ny x nz mesh (row-major, x fastest),
// spacing 1/ih: Q(i, j, k) returns q, UF(i, j, k) the velocity of the left x
// face of cell i, VF the lower y face (3D), WF the lower z face (k = 0..nz;
// the two wall faces carry no flux).
template <class T, class Q, class UF, class VF, class WF>
__device__ __forceinline__ T weno_div(int i, int j, int k, int nx, int ny, int nz, int dim, T ih, Q&& qf, UF&& uf,
                                      VF&& vf, WF&& wf) {
  T s[7];
  // x: cells i-3..i+3 (periodic)
#pragma unroll
  for (int o = 0; o < 7; ++o) s[o] = qf(weno_pmod(i + o - 3, nx), j, k);
  T div = weno_flux(uf(weno_pmod(i + 1, nx), j, k), s[1], s[2], s[3], s[4], s[5], s[6]) -
          weno_flux(uf(i, j, k), s[0], s[1], s[2], s[3], s[4], s[5]);
  if (dim == 3) {
#pragma unroll
    for (int o = 0; o < 7; ++o) s[o] = qf(i, weno_pmod(j + o - 3, ny), k);
    div += weno_flux(vf(i, weno_pmod(j + 1, ny), k), s[1], s[2], s[3], s[4], s[5], s[6]) -
           weno_flux(vf(i, j, k), s[0], s[1], s[2], s[3], s[4], s[5]);
  }
  // z: walls, mirror ghosts
#pragma unroll
  for (int o = 0; o < 7; ++o) s[o] = qf(i, j, zmirror(k + o - 3, nz));
  if (k + 1 < nz) div += weno_flux(wf(i, j, k + 1), s[1], s[2], s[3], s[4], s[5], s[6]);
  if (k > 0) div -= weno_flux(wf(i, j, k), s[0], s[1], s[2], s[3], s[4], s[5]);
  return div * ih;
}

// div(u* phi*) on the fine mesh with the prolonged extrapolated velocity
// (Eq. dual1) and phi* = 2 phi^n - phi^{n-1} (stored values), into A.
template <class T>
__global__ void k_weno_adv_fine(FineView<T> f, CoarseVel<T> v, T* __restrict__ A, Dims d, PhysT<T> q) {
  RowIdx x;
  if (!row_index(d.fnx, d.fny, x)) return;
  const size_t plane = (size_t)d.fnx * d.fny;
  auto qf = [&](int i, int j, int k) { return f.star((size_t)k * plane + (size_t)j * d.fnx + i); };
  auto uf = [&](int i, int j, int k) { return v.uface(d, i, j, k); };
  auto vf = [&](int i, int j, int k) { return v.vface(d, i, j, k); };
  auto wf = [&](int i, int j, int k) { return v.wface(d, i, j, k); };
  A[(size_t)x.row * d.fnx + x.i] = weno_div<T>(x.i, x.j, x.k, d.fnx, d.fny, d.fnz, d.dim, q.ih, qf, uf, vf, wf);
}

// div(u Theta_c) of one Theta component on the coarse mesh with the face
// velocities u, v, w (w with both wall faces)
template <class T>
__device__ __forceinline__ T weno_div_coarse(const T* __restrict__ th, const T* __restrict__ u, const T* __restrict__ v,
                                             const T* __restrict__ w, int i, int j, int k, const Dims& d, T iD) {
  const size_t plane = (size_t)d.nx * d.ny;
  auto at = [&](int ii, int jj, int kk) { return (size_t)kk * plane + (size_t)jj * d.nx + ii; };
  auto qf = [&](int ii, int jj, int kk) { return th[at(ii, jj, kk)]; };
  auto uf = [&](int ii, int jj, int kk) { return u[at(ii, jj, kk)]; };
  auto vf = [&](int ii, int jj, int kk) { return v[at(ii, jj, kk)]; };
  auto wf = [&](int ii, int jj, int kk) { return w[at(ii, jj, kk)]; };
  return weno_div<T>(i, j, k, d.nx, d.ny, d.nz, d.dim, iD, qf, uf, vf, wf);
}

}  // namespace pf
