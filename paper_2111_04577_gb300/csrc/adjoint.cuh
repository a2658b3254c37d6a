// Hand-written discrete adjoint of the Cahn-Hilliard step (velocity held fixed).
//
// Forward step in increment form (see ch.cuh; Eqs. NS25-NS34):
//   phi* = 2 phi^n - phi^{n-1}
//   w_b = 1.5 phi*_0 - 0.5 phi*_1,  g_b = cos(theta_b)(1 - w_b^2)/(sqrt(2) eta)   (top alike)
//   mu*  = F(phi*) - L_N phi* - B(g),        F(x) = x (x^2 - 1)/eta^2, B(g) = g/h on the wall layers
//   R    = a1 (phi^{n-1} - phi^n) - a2 A(phi*) + L_N mu*,   a1 = 1/(M lambda dt), a2 = 1/(M lambda)
//   eps  = (L_N - c)^{-1} R,  delta = (L_N + alpha)^{-1} eps,  phi^{n+1} = phi* + delta
// Reverse (all operators symmetric; A(phi) = D(u) phi is linear for fixed u):
//   eps_bar = (L_N + alpha)^{-1} phi_bar^{n+1},     alpha_bar = -<eps_bar, delta>
//   R_bar   = (L_N - c)^{-1} eps_bar,               c_bar     =  <R_bar, eps>
//   mu_bar  = L_N R_bar
//   phi*_bar = phi_bar^{n+1} - a2 D^T R_bar + F'(phi*) mu_bar - L_N mu_bar + (wall terms of g)
//   g_bar_b = -mu_bar_0/h,  w_bar_b = g_bar_b cos(theta_b)(-2 w_b)/(sqrt(2) eta)
//   theta_bar += sum_b g_bar_b (-sin theta_b)(1 - w_b^2)/(sqrt(2) eta)
//   phi_bar^n += 2 phi*_bar - a1 R_bar,  phi_bar^{n-1} += -phi*_bar + a1 R_bar
//   M_bar += -(a1/M) <R_bar, phi^{n-1} - phi^n> + (a2/M) <R_bar, A> + c_bar dc/dM + alpha_bar dalpha/dM
#pragma once
#include "ch.cuh"

namespace pf {

// phi* and the advection A(phi*) (central conservative fluxes, prolonged velocity)
template <class T>
__global__ void k_adj_prep(FineView<T> f, CoarseVel<T> vel, T* __restrict__ phis, T* __restrict__ adv, Dims d,
                           PhysT<T> q) {
  RowIdx x;
  if (!row_index(d.fnx, d.fny, x)) return;
  const int i = x.i, j = x.j, k = x.k;
  const size_t id = (size_t)x.row * d.fnx + i;
  const size_t plane = (size_t)d.fnx * d.fny;
  const int ip = wrap(i + 1, d.fnx), im = wrap(i - 1, d.fnx);
  const T c0 = f.star(id);
  T a = vel.uface(d, ip, j, k) * (c0 + f.star(id - i + ip)) - vel.uface(d, i, j, k) * (f.star(id - i + im) + c0);
  if (d.dim == 3) {
    const int jp = wrap(j + 1, d.fny), jm = wrap(j - 1, d.fny);
    a += vel.vface(d, i, jp, k) * (c0 + f.star(fidx(d, i, jp, k))) - vel.vface(d, i, j, k) * (f.star(fidx(d, i, jm, k)) + c0);
  }
  if (k + 1 < d.fnz) a += vel.wface(d, i, j, k + 1) * (c0 + f.star(id + plane));
  if (k > 0) a -= vel.wface(d, i, j, k) * (f.star(id - plane) + c0);
  phis[id] = c0;
  adv[id] = a * (T)0.5 * q.ih;
}

// out = L_N a + s b  (periodic x, y; mirror ghosts at the walls)
template <class T>
__global__ void k_lapN_axpy(const T* __restrict__ a, const T* __restrict__ b, T s, T* __restrict__ out, Dims d,
                            PhysT<T> q) {
  RowIdx x;
  if (!row_index(d.fnx, d.fny, x)) return;
  const int i = x.i, j = x.j, k = x.k;
  const size_t id = (size_t)x.row * d.fnx + i;
  const size_t plane = (size_t)d.fnx * d.fny;
  const T c0 = a[id];
  T lap = a[id - i + wrap(i + 1, d.fnx)] + a[id - i + wrap(i - 1, d.fnx)] - 2 * c0;
  if (d.dim == 3) lap += a[fidx(d, i, wrap(j + 1, d.fny), k)] + a[fidx(d, i, wrap(j - 1, d.fny), k)] - 2 * c0;
  lap += (k + 1 < d.fnz ? a[id + plane] : c0) + (k > 0 ? a[id - plane] : c0) - 2 * c0;
  out[id] = lap * q.ih2 + (b ? s * b[id] : (T)0);
}

// one stencil pass for both: lap = L_N a, out_l = lap, out_s = lap + s a
template <class T>
__global__ void k_lapN_two(const T* __restrict__ a, T s, T* __restrict__ out_l, T* __restrict__ out_s, Dims d,
                           PhysT<T> q) {
  RowIdx x;
  if (!row_index(d.fnx, d.fny, x)) return;
  const int i = x.i, j = x.j, k = x.k;
  const size_t id = (size_t)x.row * d.fnx + i;
  const size_t plane = (size_t)d.fnx * d.fny;
  const T c0 = a[id];
  T lap = a[id - i + wrap(i + 1, d.fnx)] + a[id - i + wrap(i - 1, d.fnx)] - 2 * c0;
  if (d.dim == 3) lap += a[fidx(d, i, wrap(j + 1, d.fny), k)] + a[fidx(d, i, wrap(j - 1, d.fny), k)] - 2 * c0;
  lap += (k + 1 < d.fnz ? a[id + plane] : c0) + (k > 0 ? a[id - plane] : c0) - 2 * c0;
  const T L = lap * q.ih2;
  out_l[id] = L;
  out_s[id] = L + s * c0;
}

// out = x + y
template <class T>
__global__ void k_add(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = a[i] + b[i];
}

// out = x - y
template <class T>
__global__ void k_sub(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

// FP64 partial dot products of up to 4 pairs; with y2b, the third pair's y is
// y2 - y2b (formed in T)
template <class T>
__global__ void k_dots(const T* __restrict__ x0, const T* __restrict__ y0, const T* __restrict__ x1,
                       const T* __restrict__ y1, const T* __restrict__ x2, const T* __restrict__ y2,
                       const T* __restrict__ x3, const T* __restrict__ y3, size_t n, double* __restrict__ partial,
                       const T* __restrict__ y2b = nullptr) {
  __shared__ double sh[4][256];
  double a[4] = {0, 0, 0, 0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    a[0] += (double)x0[i] * (double)y0[i];
    a[1] += (double)x1[i] * (double)y1[i];
    a[2] += (double)x2[i] * (double)(y2b ? (T)(y2[i] - y2b[i]) : y2[i]);
    a[3] += (double)x3[i] * (double)y3[i];
  }
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) partial[(size_t)blockIdx.x * 4 + q] = sh[q][0];
}

// phi*_bar at every fine cell, then the new adjoint state:
//   an_new = acur + 2 phi*_bar - a1 R_bar     (adjoint of phi^n, complete)
//   acur_new = -phi*_bar + a1 R_bar           (partial adjoint of phi^{n-1})
// thb_col receives, per bottom column, g_bar_b d g_b/d theta_b.
template <class T>
__global__ void k_adj_phibar(const T* __restrict__ phis, const T* __restrict__ rbar, const T* __restrict__ mubar,
                             const T* __restrict__ pbar_next, const T* __restrict__ acur, T* __restrict__ an_new,
                             T* __restrict__ acur_new, double* __restrict__ thb_col, CoarseVel<T> vel, Dims d,
                             Phys p, PhysT<T> q, T a1, T a2, const double* __restrict__ gbx = nullptr) {
  RowIdx x;
  if (!row_index(d.fnx, d.fny, x)) return;
  const int i = x.i, j = x.j, k = x.k;
  const size_t id = (size_t)x.row * d.fnx + i;
  const size_t plane = (size_t)d.fnx * d.fny;
  const int ip = wrap(i + 1, d.fnx), im = wrap(i - 1, d.fnx);
  // -a2 D^T R_bar: [u_{+}(a_i - a_{i+1}) + u_{-}(a_{i-1} - a_i)] / (2h) with a = -a2 R_bar
  const T r0 = rbar[id];
  T dt = vel.uface(d, ip, j, k) * (r0 - rbar[id - i + ip]) + vel.uface(d, i, j, k) * (rbar[id - i + im] - r0);
  if (d.dim == 3) {
    const int jp = wrap(j + 1, d.fny), jm = wrap(j - 1, d.fny);
    dt += vel.vface(d, i, jp, k) * (r0 - rbar[fidx(d, i, jp, k)]) + vel.vface(d, i, j, k) * (rbar[fidx(d, i, jm, k)] - r0);
  }
  if (k + 1 < d.fnz) dt += vel.wface(d, i, j, k + 1) * (r0 - rbar[id + plane]);
  if (k > 0) dt += vel.wface(d, i, j, k) * (rbar[id - plane] - r0);
  T sb = pbar_next[id] - a2 * dt * (T)0.5 * q.ih;
  // F'(phi*) mu_bar - L_N mu_bar
  const T c0 = phis[id];
  const T m0 = mubar[id];
  T lap = mubar[id - i + ip] + mubar[id - i + im] - 2 * m0;
  if (d.dim == 3) lap += mubar[fidx(d, i, wrap(j + 1, d.fny), k)] + mubar[fidx(d, i, wrap(j - 1, d.fny), k)] - 2 * m0;
  lap += (k + 1 < d.fnz ? mubar[id + plane] : m0) + (k > 0 ? mubar[id - plane] : m0) - 2 * m0;
  sb += (3 * c0 * c0 - 1) * q.ie2 * m0 - lap * q.ih2;
  // wall terms: g depends on w = 1.5 phi*_0 - 0.5 phi*_1 (and the top mirror)
  const double s2eta = 1.4142135623730951 * p.eta;
  const size_t col = (size_t)j * d.fnx + i;
  if (k <= 1) {
    const size_t b0 = col, b1 = plane + col;  // cells 0 and 1 of this column
    const double w = 1.5 * (double)phis[b0] - 0.5 * (double)phis[b1];
    // gbx: the wall flux's adjoint from elsewhere in the step (G's wall term, coupled sweep)
    const double gbar = -(double)mubar[b0] / d.h + (gbx ? gbx[col] : 0.0);
    const double wbar = gbar * p.cos_bot * (-2.0 * w) / s2eta;
    sb += (T)(k == 0 ? 1.5 * wbar : -0.5 * wbar);
    if (k == 0) thb_col[col] = gbar * (-sqrt(fmax(0.0, 1.0 - p.cos_bot * p.cos_bot))) * (1.0 - w * w) / s2eta;
  }
  if (k >= d.fnz - 2) {
    const size_t t0 = (size_t)(d.fnz - 1) * plane + col, t1 = (size_t)(d.fnz - 2) * plane + col;
    const double w = 1.5 * (double)phis[t0] - 0.5 * (double)phis[t1];
    const double gbar = -(double)mubar[t0] / d.h + (gbx ? gbx[plane + col] : 0.0);
    const double wbar = gbar * p.cos_top * (-2.0 * w) / s2eta;
    sb += (T)(k == d.fnz - 1 ? 1.5 * wbar : -0.5 * wbar);
  }
  const T ar = a1 * r0;
  an_new[id] = acur[id] + 2 * sb - ar;
  acur_new[id] = -sb + ar;
}

// FP64 partial sums of a double array
static __global__ void k_sum_d(const double* __restrict__ a, size_t n, double* __restrict__ partial) {
  __shared__ double sh[256];
  double s = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) s += a[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// seed: d(wetted length)/d phi, or d(z-centroid)/d phi = (z - zc)/(2 D)
template <class T>
__global__ void k_obj_seed(T* __restrict__ out, Dims d, int which, double zc, double D) {
  RowIdx x;
  if (!row_index(d.fnx, d.fny, x)) return;
  const int k = x.k;
  const size_t id = (size_t)x.row * d.fnx + x.i;
  double v = 0.0;
  if (which == 0) {
    const double hw = d.dim == 3 ? d.h * d.h : d.h;
    if (k == 0) v += 0.75 * hw;
    if (k == 1) v -= 0.25 * hw;
  } else {
    v = (((double)k + 0.5) * d.h - zc) / (2.0 * D);
  }
  out[id] = (T)v;
}

}  // namespace pf
