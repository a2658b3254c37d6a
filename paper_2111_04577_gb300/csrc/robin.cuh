// Dynamic contact angle, D_w > 0 (Eq. NS15; its discrete form Eq. NS34).
//
// The wall flux of phi^{n+1} holds the BDF2 time derivative at the wall
// (Eq. NS31), implicit in phi^{n+1}, and the wall advection:
//   g = n.grad(phi^{n+1}) = E - kappa phi_w^{n+1},   kappa = D_w gamma0/dt,
//   E = -f_w'(phi*_w)/lambda - D_w u_w d_x phi*_w + (D_w/dt) phi_hat_w,
// every wall value the extrapolation 1.5 v_0 - 0.5 v_1, u_w the wall's x
// velocity (no slip), d_x the central difference along the wall.  Eq. NS33
// passes c g to Psi, so the pair of solves sees a Robin condition on both.
//
// In the increment form delta = phi^{n+1} - phi* of the step the right side
// is formed with the flux g* = E - kappa phi*_w of phi* (the kernels form the
// static flux g0 = -f_w'(phi*_w)/lambda; k_robin_rhs adds -L_N B(g* - g0),
// the only place the flux enters the right side).  delta then has the flux
// b = -kappa w(delta) at each wall (w the wall extrapolation): the paired
// z solve gives delta0 for homogeneous Neumann walls, and
//   delta = delta0 + b_bot D(k) + b_top D(R-1-k)
// per Fourier mode, where D is the response of the pair to a unit flux at the
// bottom wall (computed once on the host in FP64; the top wall's is its mirror
// image).  With s = w_bot(D), x = w_top(D), the two fluxes solve
//   (1 + kappa s) b_bot + kappa x b_top = -kappa w_bot(delta0),
//   kappa x b_bot + (1 + kappa s) b_top = -kappa w_top(delta0).
// After the step k_robin_flux stores the flux of phi^{n+1}, g = E - kappa
// w(phi^{n+1}), which the chemical potential (Eq. NS5) takes.
#pragma once

#include "ch.cuh"
#include "common.cuh"

namespace pf {

// Per wall column (both walls): E into gE, and g* - g0 into dg.  phi* is
// formed in T exactly as the right-side kernels form it, so that g0 cancels;
// the remaining terms take FP64 values with the compensated remainders.
template <class T>
__global__ void k_robin_wall(FineView<T> f, Wide<T>* __restrict__ gE, Wide<T>* __restrict__ dg, Dims d, Phys p,
                             PhysT<T> q, double dw, double kappa) {
  using W = Wide<T>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= d.fnx) return;
  const size_t plane = (size_t)d.fnx * d.fny;
  const size_t cols = plane;
  for (int wall = 0; wall < 2; ++wall) {
    const int k0 = wall == 0 ? 0 : d.fnz - 1, k1 = wall == 0 ? 1 : d.fnz - 2;
    const W cg = wall == 0 ? q.gbot : q.gtop;
    const double uw = wall == 0 ? p.uw_bot : p.uw_top;
    auto full = [&](const T* a, const T* lo, size_t o) { return lo ? (W)a[o] + (W)lo[o] : (W)a[o]; };
    // wall values of phi* (full precision) at column ii
    auto wstar = [&](int ii) {
      const size_t o0 = (size_t)k0 * plane + (size_t)j * d.fnx + ii, o1 = (size_t)k1 * plane + (size_t)j * d.fnx + ii;
      const W s0 = 2.0 * full(f.pn, f.ln, o0) - full(f.po, f.lo, o0);
      const W s1 = 2.0 * full(f.pn, f.ln, o1) - full(f.po, f.lo, o1);
      return 1.5 * s0 - 0.5 * s1;
    };
    const size_t o0 = (size_t)k0 * plane + (size_t)j * d.fnx + i, o1 = (size_t)k1 * plane + (size_t)j * d.fnx + i;
    const W g0 = wall_g(cg, (W)((T)2 * f.pn[o0] - f.po[o0]), (W)((T)2 * f.pn[o1] - f.po[o1]));
    const W h0 = 2.0 * full(f.pn, f.ln, o0) - 0.5 * full(f.po, f.lo, o0);
    const W h1 = 2.0 * full(f.pn, f.ln, o1) - 0.5 * full(f.po, f.lo, o1);
    const W what = 1.5 * h0 - 0.5 * h1;
    const W ws = wstar(i);
    const W dxw = (wstar(i + 1 == d.fnx ? 0 : i + 1) - wstar(i == 0 ? d.fnx - 1 : i - 1)) * (0.5 / d.h);
    const W tail = -dw * uw * dxw + (dw / p.dt) * what;  // E - g0
    const size_t c = (size_t)wall * cols + (size_t)j * d.fnx + i;
    gE[c] = g0 + tail;
    dg[c] = tail - kappa * ws;  // g* - g0
  }
}

// R += -L_N B(g* - g0) on the layers next to the walls (B: the flux over h on
// the wall layer, zero elsewhere; L_N with mirror walls, periodic x and y)
template <class T>
__global__ void k_robin_rhs(T* __restrict__ R, const Wide<T>* __restrict__ dg, Dims d, PhysT<T> q) {
  using W = Wide<T>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= d.fnx) return;
  const size_t plane = (size_t)d.fnx * d.fny;
  const int R1 = d.fnz - 1;
  const double ih = 1.0 / d.h, ih2 = ih * ih;
  auto Bv = [&](int k, int ii, int jj) -> W {  // B at (ii, jj, k)
    const size_t col = (size_t)jj * d.fnx + ii;
    W b = 0.0;
    if (k == 0) b += dg[col] * ih;
    if (k == R1) b += dg[plane + col] * ih;
    return b;
  };
  const int ip = i + 1 == d.fnx ? 0 : i + 1, im = i == 0 ? d.fnx - 1 : i - 1;
  const int jp = j + 1 == d.fny ? 0 : j + 1, jm = j == 0 ? d.fny - 1 : j - 1;
  const int ks[4] = {0, 1, R1 - 1, R1};
  for (int a = 0; a < 4; ++a) {
    const int k = ks[a];
    if (k < 0 || k > R1) continue;
    bool dup = false;
    for (int b = 0; b < a; ++b) dup |= ks[b] == k;
    if (dup) continue;
    const W c0 = Bv(k, i, j);
    W lap = Bv(k, ip, j) + Bv(k, im, j) - 2.0 * c0;
    if (d.dim == 3) lap += Bv(k, i, jp) + Bv(k, i, jm) - 2.0 * c0;
    const W up = k < R1 ? Bv(k + 1, i, j) : c0, dn = k > 0 ? Bv(k - 1, i, j) : c0;
    lap = (lap + up + dn - 2.0 * c0) * ih2;
    const size_t o = (size_t)k * plane + (size_t)j * d.fnx + i;
    R[o] = (T)((W)R[o] - lap);
  }
}

// delta = delta0 + b_bot D(k) + b_top D(R-1-k) on the paired solve's output
// (spectral, rows of ny x pitch complex; one thread per real component of a
// kx column).  D: [R][ny][ncol]; sx: [ny][ncol][2] = (s, x).
template <class T, class TC>
__global__ void k_robin_correct(cpx<T>* __restrict__ data, int rows, int ny, int pitch, int ncol, const TC* __restrict__ D,
                                const TC* __restrict__ sx, TC kappa) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x, ky = blockIdx.y;
  const int col = t >> 1, part = t & 1;
  if (col >= ncol) return;
  T* base = reinterpret_cast<T*>(data + (size_t)ky * pitch + col) + part;
  const size_t zs = (size_t)ny * pitch * 2;
  const TC y0 = (TC)base[0], y1 = (TC)base[zs];
  const TC ya = (TC)base[(size_t)(rows - 1) * zs], yb = (TC)base[(size_t)(rows - 2) * zs];
  const TC wb = (TC)1.5 * y0 - (TC)0.5 * y1, wt = (TC)1.5 * ya - (TC)0.5 * yb;
  const size_t m = (size_t)ky * ncol + col;
  const TC a = (TC)1 + kappa * sx[2 * m], bq = kappa * sx[2 * m + 1];
  const TC det = a * a - bq * bq;
  const TC bb = -kappa * (a * wb - bq * wt) / det, bt = -kappa * (a * wt - bq * wb) / det;
  const size_t dstride = (size_t)ny * ncol;
  for (int k = 0; k < rows; ++k) {
    const TC corr = bb * D[(size_t)k * dstride + m] + bt * D[(size_t)(rows - 1 - k) * dstride + m];
    base[(size_t)k * zs] = (T)((TC)base[(size_t)k * zs] + corr);
  }
}

// the flux of phi^{n+1} at each wall column: g = E - kappa w(phi^{n+1})
template <class T>
__global__ void k_robin_flux(const T* __restrict__ pn, const T* __restrict__ ln, const Wide<T>* __restrict__ gE,
                             Wide<T>* __restrict__ gwall, Dims d, double kappa) {
  using W = Wide<T>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= d.fnx) return;
  const size_t plane = (size_t)d.fnx * d.fny;
  for (int wall = 0; wall < 2; ++wall) {
    const int k0 = wall == 0 ? 0 : d.fnz - 1, k1 = wall == 0 ? 1 : d.fnz - 2;
    const size_t o0 = (size_t)k0 * plane + (size_t)j * d.fnx + i, o1 = (size_t)k1 * plane + (size_t)j * d.fnx + i;
    const W v0 = ln ? (W)pn[o0] + (W)ln[o0] : (W)pn[o0];
    const W v1 = ln ? (W)pn[o1] + (W)ln[o1] : (W)pn[o1];
    const size_t c = (size_t)wall * plane + (size_t)j * d.fnx + i;
    gwall[c] = gE[c] - kappa * (1.5 * v0 - 0.5 * v1);
  }
}

}  // namespace pf
