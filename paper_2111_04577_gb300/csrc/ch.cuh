// Cahn-Hilliard kernels on the phase-field (fine) mesh.
//
// Section 3.2.1: BDF2 with extrapolation (Eqs. NS31, NS32), the stabilised
// scheme Eq. NS25 split into the Helmholtz pair Eqs. NS26-NS27 with the wall
// conditions Eqs. NS33-NS34 (D_w = 0), the divergence-free prolongation of the
// extrapolated velocity (Eq. dual1) and the chemical potential Eq. NS5.
//
// Increment form.  With phi^{n+1} = phi* + delta and Psi = (L + alpha) phi* +
// eps, the two solves of Eqs. NS26-NS27 become
//   (L_N - c) eps   = R,   (L_N + alpha) delta = eps,
//   R = (phi^{n-1} - phi^n)/(M lambda dt) - div(u* phi*)/(M lambda) + L_N mu*,
//   mu* = f(phi*) - (L_N phi* + B(g)),
// an exact algebraic rewrite (alpha^2 + (S/eta^2) alpha + gamma0/(M lambda dt) = 0
// from Eq. NS29, and gamma0 phi* - phi_hat = phi^n - phi^{n-1}).  The right side
// and the solution are O(increment) instead of O(phi/(M lambda dt)), which keeps
// FP32 storage accurate.  L_N: Laplacian with homogeneous-Neumann wall ghosts;
// B(g) = g/h on the wall layers, g = n.grad(phi) of the contact-angle law
// (Eq. NS34), evaluated in FP64 at phi*_w = 1.5 phi*_0 - 0.5 phi*_1.
#pragma once
#include "common.cuh"

namespace pf {

template <class T>
struct FineView {
  const T* pn;   // phi^n
  const T* po;   // phi^{n-1}
  __device__ __forceinline__ T star(size_t i) const { return (T)2 * pn[i] - po[i]; }
};

// Contact-angle flux (Eqs. NS15-NS16, NS34 with D_w = 0), FP64.
__device__ __forceinline__ double wall_g(double cth, double p0, double p1, double eta) {
  const double w = 1.5 * p0 - 0.5 * p1;
  return cth * (1.0 - w * w) / (1.4142135623730951 * eta);
}

// mu* = f(phi*) - (L_N phi* + B(g)); also stores g per wall column.
template <class T>
__global__ void k_ch_mu(FineView<T> f, T* __restrict__ mu, double* __restrict__ gwall, Dims d, Phys p, PhysT<T> q) {
  RowIdx x;
  if (!row_index(d.fnx, d.fny, x)) return;
  const int i = x.i, j = x.j, k = x.k;
  const size_t id = (size_t)x.row * d.fnx + i;
  const T c0 = f.star(id);
  T lap = f.star(id - i + wrap(i + 1, d.fnx)) + f.star(id - i + wrap(i - 1, d.fnx)) - 2 * c0;
  if (d.dim == 3) lap += f.star(fidx(d, i, wrap(j + 1, d.fny), k)) + f.star(fidx(d, i, wrap(j - 1, d.fny), k)) - 2 * c0;
  const size_t plane = (size_t)d.fnx * d.fny;
  const T zp = (k + 1 < d.fnz) ? f.star(id + plane) : c0;
  const T zm = (k > 0) ? f.star(id - plane) : c0;
  lap = (lap + zp + zm - 2 * c0) * q.ih2;
  T B = 0;
  const size_t col = (size_t)j * d.fnx + i;
  if (k == 0) {
    const double g = wall_g(p.cos_bot, (double)c0, (double)zp, p.eta);
    gwall[col] = g;
    B += (T)(g / d.h);
  }
  if (k == d.fnz - 1) {
    const double g = wall_g(p.cos_top, (double)c0, (double)zm, p.eta);
    gwall[plane + col] = g;
    B += (T)(g / d.h);
  }
  mu[id] = c0 * (c0 * c0 - 1) * q.ie2 - (lap + B);
}

// Prolonged extrapolated velocity (Eq. dual1) on the fine faces.
template <class T>
struct CoarseVel {
  const T *un, *uo, *vn, *vo, *wn, *wo;  // coarse, levels n and n-1
  __device__ __forceinline__ T us(size_t i) const { return (T)2 * un[i] - uo[i]; }
  __device__ __forceinline__ T vs(size_t i) const { return (T)2 * vn[i] - vo[i]; }
  __device__ __forceinline__ T ws(size_t i) const { return (T)2 * wn[i] - wo[i]; }
  // fine x-face I (left face of fine cell I), fine row (J, K)
  __device__ __forceinline__ T uface(const Dims& d, int I, int J, int K) const {
    const int jc = J >> d.rys, kc = K >> d.rs;
    const int ic = I >> d.rs;
    const size_t b = ((size_t)kc * d.ny + jc) * d.nx;
    if ((I & (d.r - 1)) == 0) return us(b + ic);
    return (T)0.5 * (us(b + ic) + us(b + wrap(ic + 1, d.nx)));
  }
  __device__ __forceinline__ T vface(const Dims& d, int I, int J, int K) const {
    const int ic = I >> d.rs, kc = K >> d.rs;
    const int jc = J >> d.rys;
    const size_t b = (size_t)kc * d.ny * d.nx + ic;
    if ((J & (d.ry - 1)) == 0) return vs(b + (size_t)jc * d.nx);
    return (T)0.5 * (vs(b + (size_t)jc * d.nx) + vs(b + (size_t)wrap(jc + 1, d.ny) * d.nx));
  }
  // fine z-face K (0..fnz), K = 0 and fnz are walls
  __device__ __forceinline__ T wface(const Dims& d, int I, int J, int K) const {
    const int ic = I >> d.rs, jc = J >> d.rys;
    const size_t col = (size_t)jc * d.nx + ic;
    const size_t plane = (size_t)d.ny * d.nx;
    const int kc = K >> d.rs;
    if ((K & (d.r - 1)) == 0) return ws(kc * plane + col);
    return (T)0.5 * (ws(kc * plane + col) + ws((kc + 1) * plane + col));
  }
};

// Producer of the increment-form right side R for the x-transform kernel.
template <class T>
struct ChRhs {
  static constexpr const char* name = "ch_rhs_fftx";
  FineView<T> f;
  const T* mu;
  CoarseVel<T> vel;
  Dims d;
  T inv_mldt, inv_ml, ih, ih2;
  __device__ __forceinline__ T operator()(int line, int i) const {
    const int j = line % d.fny, k = line / d.fny;
    const size_t id = fidx(d, i, j, k);
    const int ip = wrap(i + 1, d.fnx), im = wrap(i - 1, d.fnx);
    const T c0 = f.star(id);
    // advection div(u* phi*), central conservative face fluxes
    const T cxm = f.star(fidx(d, im, j, k)), cxp = f.star(fidx(d, ip, j, k));
    T adv = vel.uface(d, ip, j, k) * (c0 + cxp) - vel.uface(d, i, j, k) * (cxm + c0);
    if (d.dim == 3) {
      const int jp = wrap(j + 1, d.fny), jm = wrap(j - 1, d.fny);
      const T cyp = f.star(fidx(d, i, jp, k)), cym = f.star(fidx(d, i, jm, k));
      adv += vel.vface(d, i, jp, k) * (c0 + cyp) - vel.vface(d, i, j, k) * (cym + c0);
    }
    if (k + 1 < d.fnz) adv += vel.wface(d, i, j, k + 1) * (c0 + f.star(fidx(d, i, j, k + 1)));
    if (k > 0) adv -= vel.wface(d, i, j, k) * (f.star(fidx(d, i, j, k - 1)) + c0);
    adv *= (T)0.5 * ih;
    // L_N mu*
    const T m0 = mu[id];
    T lap = mu[fidx(d, ip, j, k)] + mu[fidx(d, im, j, k)] - 2 * m0;
    if (d.dim == 3) lap += mu[fidx(d, i, wrap(j + 1, d.fny), k)] + mu[fidx(d, i, wrap(j - 1, d.fny), k)] - 2 * m0;
    const T zp = (k + 1 < d.fnz) ? mu[fidx(d, i, j, k + 1)] : m0;
    const T zm = (k > 0) ? mu[fidx(d, i, j, k - 1)] : m0;
    lap = (lap + zp + zm - 2 * m0) * ih2;
    return (f.po[id] - f.pn[id]) * inv_mldt - adv * inv_ml + lap;
  }
};

// phi^{n+1} = phi* + delta, written over phi^{n-1} (same index, no hazard).
template <class T>
struct ChFinish {
  static constexpr const char* name = "ch_ifftx_finish";
  const T* pn;
  T* po_new;  // holds phi^{n-1} on entry, phi^{n+1} on exit
  int fnx;
  __device__ __forceinline__ void operator()(int line, int i, T delta) const {
    const size_t id = (size_t)line * fnx + i;
    po_new[id] = (T)2 * pn[id] - po_new[id] + delta;
  }
};

// G = lambda (-(L_N phi + B(g)) + f(phi))  (Eq. NS5 with the wetting ghost)
template <class T>
__global__ void k_ch_G(const T* __restrict__ phi, const double* __restrict__ gwall, T* __restrict__ G, Dims d,
                       PhysT<T> q) {
  RowIdx x;
  if (!row_index(d.fnx, d.fny, x)) return;
  const int i = x.i, j = x.j, k = x.k;
  const size_t id = (size_t)x.row * d.fnx + i;
  const size_t plane = (size_t)d.fnx * d.fny;
  const T c0 = phi[id];
  T lap = phi[id - i + wrap(i + 1, d.fnx)] + phi[id - i + wrap(i - 1, d.fnx)] - 2 * c0;
  if (d.dim == 3) lap += phi[fidx(d, i, wrap(j + 1, d.fny), k)] + phi[fidx(d, i, wrap(j - 1, d.fny), k)] - 2 * c0;
  const T zp = (k + 1 < d.fnz) ? phi[id + plane] : c0;
  const T zm = (k > 0) ? phi[id - plane] : c0;
  lap = (lap + zp + zm - 2 * c0) * q.ih2;
  T B = 0;
  const size_t col = (size_t)j * d.fnx + i;
  if (k == 0) B += (T)gwall[col] * q.ih;
  if (k == d.fnz - 1) B += (T)gwall[plane + col] * q.ih;
  G[id] = q.lam * (-(lap + B) + c0 * (c0 * c0 - 1) * q.ie2);
}

// Coarse samples of the restricted phi and G (Eq. dual2).
template <class T>
struct Restricted {
  T *phic, *Gc;           // centres                      nz*ny*nx
  T *phifx, *Gfx;         // x-faces                      nz*ny*nx
  T *phify, *Gfy;         // y-faces (3D)                 nz*ny*nx
  T *phifz, *Gfz;         // z-faces k = 0..nz            (nz+1)*ny*nx
  T *phiexz, *phiexy, *phieyz;  // edges                  (nz+1)/nz/(nz+1) * ny*nx
};

// Mean of a fine field over x in [x0, x0+nx_), y in [y0, ..), z in [z0, ..);
// periodic wrap in x, y; mirror ghost (cell -1 -> 0, fnz -> fnz-1) in z.
template <class T>
__device__ __forceinline__ T box_mean(const T* a, const Dims& d, int x0, int nxr, int y0, int nyr, int z0, int nzr,
                                      T inv) {
  T s = 0;
  for (int kk = 0; kk < nzr; ++kk) {
    int z = z0 + kk;
    z = z < 0 ? 0 : (z >= d.fnz ? d.fnz - 1 : z);
    for (int jj = 0; jj < nyr; ++jj) {
      const int y = wrap(y0 + jj, d.fny);
      const T* rowp = a + ((size_t)z * d.fny + y) * d.fnx;
      for (int ii = 0; ii < nxr; ++ii) s += rowp[wrap(x0 + ii, d.fnx)];
    }
  }
  return s * inv;
}

// one thread per coarse (i, j, k), k = 0..nz (the last layer only for z-faces/edges)
template <class T>
__global__ void k_restrict(const T* __restrict__ phi, const T* __restrict__ G, Restricted<T> out, Dims d) {
  RowIdx x;
  if (!row_index(d.nx, d.ny, x)) return;
  const int i = x.i, j = x.j, k = x.k;
  const size_t id = (size_t)x.row * d.nx + i;
  const int r = d.r, ry = d.ry;
  const T i2 = (T)0.5, i4 = (T)0.25;
  const T irr = (T)1 / (T)(r * ry), irrr = (T)1 / (T)(r * ry * r), i2rr = (T)1 / (T)(2 * r * ry);
  const T i4r = (T)1 / (T)(4 * (d.dim == 3 ? r : 1));
  (void)i2; (void)i4;
  // z-faces and z-edges exist for k = 0..nz
  out.phifz[id] = box_mean(phi, d, r * i, r, ry * j, ry, r * k - 1, 2, i2rr);
  out.Gfz[id] = box_mean(G, d, r * i, r, ry * j, ry, r * k - 1, 2, i2rr);
  out.phiexz[id] = box_mean(phi, d, r * i - 1, 2, ry * j, ry, r * k - 1, 2, (T)1 / (T)(4 * ry));
  if (d.dim == 3) out.phieyz[id] = box_mean(phi, d, r * i, r, ry * j - 1, 2, r * k - 1, 2, (T)1 / (T)(4 * r));
  if (k == d.nz) return;
  out.phic[id] = box_mean(phi, d, r * i, r, ry * j, ry, r * k, r, irrr);
  out.Gc[id] = box_mean(G, d, r * i, r, ry * j, ry, r * k, r, irrr);
  out.phifx[id] = box_mean(phi, d, r * i - 1, 2, ry * j, ry, r * k, r, i2rr);
  out.Gfx[id] = box_mean(G, d, r * i - 1, 2, ry * j, ry, r * k, r, i2rr);
  if (d.dim == 3) {
    out.phify[id] = box_mean(phi, d, r * i, r, ry * j - 1, 2, r * k, r, (T)1 / (T)(2 * r * r));
    out.Gfy[id] = box_mean(G, d, r * i, r, ry * j - 1, 2, r * k, r, (T)1 / (T)(2 * r * r));
    out.phiexy[id] = box_mean(phi, d, r * i - 1, 2, ry * j - 1, 2, r * k, r, i4r);
  }
  (void)irr;
}

}  // namespace pf
