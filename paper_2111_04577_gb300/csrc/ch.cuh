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
#include <type_traits>
#include "common.cuh"

namespace pf {

template <class T>
struct FineView {
  const T* pn;   // phi^n
  const T* po;   // phi^{n-1}
  // Compensated storage (FP32 contexts): the rounding remainders of phi^n and
  // phi^{n-1} (phi = value + remainder to about 2^-48 relative), or null.  Only
  // the BDF2 difference phi^{n-1} - phi^n, of the size of one step's change,
  // needs them; phi* and every stencil take the stored values.
  const T* ln = nullptr;
  const T* lo = nullptr;
  // div(u* phi*) precomputed with the WENO5-Z fluxes (csrc/weno.cuh), or null
  // for the central second-order flux formed in the right-side kernels
  const T* aw = nullptr;
  __device__ __forceinline__ T star(size_t i) const { return (T)2 * pn[i] - po[i]; }
  // phi^{n-1} - phi^n at i, given the stored values a = phi^n[i], b = phi^{n-1}[i]
  __device__ __forceinline__ T back(size_t i, T a, T b) const {
    T r = b - a;
    if (ln) r += lo[i] - ln[i];
    return r;
  }
};

// Contact-angle flux (Eqs. NS15-NS16, NS34 with D_w = 0), in W = Wide<T>
// (FP64, or Dual when derivatives are carried).  cg = cos(theta_s)/(sqrt(2) eta)
// is formed once on the host, so that the FP64 pipe (a small fraction of the FP32
// rate on this GPU) takes three operations per wall cell and no division.
template <class W>
__device__ __forceinline__ W wall_g(W cg, W p0, W p1) {
  const W w = 1.5 * p0 - 0.5 * p1;
  return cg * (1.0 - w * w);
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

// phi^{n+1} = phi* + delta, written over phi^{n-1} (same index, no hazard).
template <class T>
struct ChFinish {
  static constexpr const char* name = "ch_ifftx_finish";
  // phi^n, phi^{n-1} -- and in FP32 contexts their remainders (compensated
  // storage, see FineView) -- are staged into shared memory before the transform
  static constexpr int kNPre = std::is_same<T, float>::value ? 4 : 2;
  const T* pn;
  T* po_new;  // holds phi^{n-1} on entry, phi^{n+1} on exit
  int fnx;
  const T* ln = nullptr;  // remainder of phi^n (FP32: required)
  T* lo_new = nullptr;    // remainder of phi^{n-1} on entry, of phi^{n+1} on exit
  __device__ __forceinline__ const T* pre(int j) const { return j == 0 ? pn : (j == 1 ? po_new : (j == 2 ? ln : lo_new)); }
  __device__ __forceinline__ int pre_n() const { return fnx; }
  // pv[j * stride]: the staged value of array j at (line, i)
  __device__ __forceinline__ void apply(int line, int i, T delta, const T* pv, int stride) const {
    const size_t id = (size_t)line * fnx + i;
    const T vn = pv[0], vo = pv[stride];
    if constexpr (kNPre == 2) {
      po_new[id] = (T)2 * vn - vo + delta;
    } else {
      // phi^{n+1} = 2 phi^n - phi^{n-1} + delta with the remainders carried: the
      // exact sum 2 vn - vo is split by TwoSum, the small terms are added to its
      // error, and the total is split again into value and remainder
      T s, e, hi, lo;
      two_sum((T)2 * vn, -vo, s, e);
      const T t = e + ((T)2 * pv[2 * stride] - pv[3 * stride]) + delta;
      two_sum(s, t, hi, lo);
      po_new[id] = hi;
      lo_new[id] = lo;
    }
  }
};

// G = lambda (-(L_N phi + B(g)) + f(phi))  (Eq. NS5 with the wetting ghost)
template <class T>
__global__ void k_ch_G(const T* __restrict__ phi, const Wide<T>* __restrict__ gwall, T* __restrict__ G, Dims d,
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

}  // namespace pf
