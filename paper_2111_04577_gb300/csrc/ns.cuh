// Navier-Stokes kernels on the coarse MAC mesh (Section 3.2.2, Eqs. NS35-NS39).
//
// Step 1 (Eq. NS36 with the -u_hat/dt of Eq. NS35 on the right side):
//   nu_m lap(u~) - (gamma0/dt) u~ = -u_hat/dt + div(u* u*) + (1/rho) J.grad(u*)
//       + (1/rho0) grad p^n + (1/rho - 1/rho0) grad p* + nu_m lap(u*)
//       - (1/rho) div(tau*) - (1/rho) div(mu (grad u* + grad u*^T))
//       - (1/rho) G grad(phi) - g,
// with J = -(rho1 - rho2)/2 M grad(G) (Eq. NS10) evaluated at u*, rho and mu
// from the restricted phi^{n+1} (Eqs. dual2, dual3), second-order central
// differences on the staggered mesh, 4-point averages for quantities needed
// off their home location, no-slip ghosts 2 u_w - u, mirror ghosts for tau.
// k_ns_rhs writes the right side divided by nu_m (minus the wall-velocity
// ghost term), ready for (L - gamma0/(dt nu_m)) u~ = rhs.
// Step 2 (Eq. NS37 with coefficient gamma0 rho0/dt): k_div feeds the Neumann
// Poisson solve; step 3 (Eqs. NS38-NS39): k_correct.
#pragma once
#include "ch.cuh"

namespace pf {

template <class T>
struct NsIn {
  const T *un, *uo, *vn, *vo, *wn, *wo;   // velocities at n, n-1
  const T *pn, *po;                       // pressure at n, n-1
  const T *tn[6], *to[6];                 // weighted stress comps at n, n-1 (may be null)
  Restricted<T> rs;                       // restricted phi^{n+1}, G^{n+1}
};

template <class T>
struct NsAcc {
  NsIn<T> a;
  Dims d;
  Phys p;
  __device__ __forceinline__ size_t c(int i, int j, int k) const {
    return ((size_t)k * d.ny + wrap(j, d.ny)) * d.nx + wrap(i, d.nx);
  }
  __device__ __forceinline__ T US(int i, int j, int k) const {
    if (k < 0) return (T)(2 * p.uw_bot) - US(i, j, 0);
    if (k >= d.nz) return (T)(2 * p.uw_top) - US(i, j, d.nz - 1);
    const size_t q = c(i, j, k);
    return (T)2 * a.un[q] - a.uo[q];
  }
  __device__ __forceinline__ T UH(int i, int j, int k) const {
    const size_t q = c(i, j, k);
    return (T)2 * a.un[q] - (T)0.5 * a.uo[q];
  }
  __device__ __forceinline__ T VS(int i, int j, int k) const {
    if (k < 0) return -VS(i, j, 0);
    if (k >= d.nz) return -VS(i, j, d.nz - 1);
    const size_t q = c(i, j, k);
    return (T)2 * a.vn[q] - a.vo[q];
  }
  __device__ __forceinline__ T VH(int i, int j, int k) const {
    const size_t q = c(i, j, k);
    return (T)2 * a.vn[q] - (T)0.5 * a.vo[q];
  }
  // w at z-faces 0..nz (walls stored as 0)
  __device__ __forceinline__ T WS(int i, int j, int k) const {
    const size_t q = c(i, j, k);
    return (T)2 * a.wn[q] - a.wo[q];
  }
  __device__ __forceinline__ T WH(int i, int j, int k) const {
    const size_t q = c(i, j, k);
    return (T)2 * a.wn[q] - (T)0.5 * a.wo[q];
  }
  __device__ __forceinline__ T Pn(int i, int j, int k) const { return a.pn[c(i, j, k)]; }
  __device__ __forceinline__ T Ps(int i, int j, int k) const {
    const size_t q = c(i, j, k);
    return (T)2 * a.pn[q] - a.po[q];
  }
  __device__ __forceinline__ T Gc(int i, int j, int k) const { return a.rs.Gc[c(i, j, k)]; }
  __device__ __forceinline__ T phic(int i, int j, int k) const { return a.rs.phic[c(i, j, k)]; }
  __device__ __forceinline__ T mu_of(T phi) const {
    return (T)0.5 * ((T)1 + phi) * (T)p.mu_s1 + (T)0.5 * ((T)1 - phi) * (T)p.mu_s2;
  }
  __device__ __forceinline__ T rho_of(T phi) const {
    return (T)0.5 * ((T)1 + phi) * (T)p.rho1 + (T)0.5 * ((T)1 - phi) * (T)p.rho2;
  }
  __device__ __forceinline__ T muc(int i, int j, int k) const { return mu_of(phic(i, j, k)); }
  __device__ __forceinline__ T muexz(int i, int j, int k) const { return mu_of(a.rs.phiexz[c(i, j, k)]); }
  __device__ __forceinline__ T muexy(int i, int j, int k) const { return mu_of(a.rs.phiexy[c(i, j, k)]); }
  __device__ __forceinline__ T mueyz(int i, int j, int k) const { return mu_of(a.rs.phieyz[c(i, j, k)]); }
  // J components at their faces
  __device__ __forceinline__ T Jx(int i, int j, int k) const {
    return (T)(-0.5 * (p.rho1 - p.rho2) * p.mob) * (Gc(i, j, k) - Gc(i - 1, j, k)) / (T)d.dx;
  }
  __device__ __forceinline__ T Jy(int i, int j, int k) const {
    return (T)(-0.5 * (p.rho1 - p.rho2) * p.mob) * (Gc(i, j, k) - Gc(i, j - 1, k)) / (T)d.dx;
  }
  __device__ __forceinline__ T Jz(int i, int j, int k) const {  // w-face k
    if (k <= 0 || k >= d.nz) return (T)0;
    return (T)(-0.5 * (p.rho1 - p.rho2) * p.mob) * (Gc(i, j, k) - Gc(i, j, k - 1)) / (T)d.dx;
  }
  // extrapolated weighted stress at centres, mirror ghost in z
  __device__ __forceinline__ T tau(int comp, int i, int j, int k) const {
    k = k < 0 ? 0 : (k >= d.nz ? d.nz - 1 : k);
    const size_t q = c(i, j, k);
    return (T)2 * a.tn[comp][q] - a.to[comp][q];
  }
  // centre -> edge averages
  __device__ __forceinline__ T Txz(int comp, int i, int j, int k) const {  // edge x = i dx, z = k dx
    return (T)0.25 * (tau(comp, i - 1, j, k - 1) + tau(comp, i, j, k - 1) + tau(comp, i - 1, j, k) + tau(comp, i, j, k));
  }
  __device__ __forceinline__ T Txy(int comp, int i, int j, int k) const {
    return (T)0.25 * (tau(comp, i - 1, j - 1, k) + tau(comp, i, j - 1, k) + tau(comp, i - 1, j, k) + tau(comp, i, j, k));
  }
  __device__ __forceinline__ T Tyz(int comp, int i, int j, int k) const {
    return (T)0.25 * (tau(comp, i, j - 1, k - 1) + tau(comp, i, j, k - 1) + tau(comp, i, j - 1, k) + tau(comp, i, j, k));
  }
  // advective edge products and viscous edge stresses
  __device__ __forceinline__ T Exz(int i, int j, int k) const {  // u w at (i dx, k dx)
    return (T)0.25 * (US(i, j, k - 1) + US(i, j, k)) * (WS(i - 1, j, k) + WS(i, j, k));
  }
  __device__ __forceinline__ T Exy(int i, int j, int k) const {
    return (T)0.25 * (US(i, j - 1, k) + US(i, j, k)) * (VS(i - 1, j, k) + VS(i, j, k));
  }
  __device__ __forceinline__ T Eyz(int i, int j, int k) const {
    return (T)0.25 * (VS(i, j, k - 1) + VS(i, j, k)) * (WS(i, j - 1, k) + WS(i, j, k));
  }
  __device__ __forceinline__ T Sxz(int i, int j, int k) const {
    const T D = (T)d.dx;
    return muexz(i, j, k) * ((US(i, j, k) - US(i, j, k - 1)) / D + (WS(i, j, k) - WS(i - 1, j, k)) / D);
  }
  __device__ __forceinline__ T Sxy(int i, int j, int k) const {
    const T D = (T)d.dx;
    return muexy(i, j, k) * ((US(i, j, k) - US(i, j - 1, k)) / D + (VS(i, j, k) - VS(i - 1, j, k)) / D);
  }
  __device__ __forceinline__ T Syz(int i, int j, int k) const {
    const T D = (T)d.dx;
    return mueyz(i, j, k) * ((VS(i, j, k) - VS(i, j, k - 1)) / D + (WS(i, j, k) - WS(i, j - 1, k)) / D);
  }
};

// comps: 3D xx,yy,zz,xy,xz,yz = 0..5 ; 2D xx,xz,zz = 0,1,2
template <class T>
__global__ void k_ns_rhs(NsAcc<T> A, T* __restrict__ ru, T* __restrict__ rv, T* __restrict__ rw, int have_tau) {
  const Dims& d = A.d;
  const Phys& p = A.p;
  const size_t n = (size_t)d.nx * d.ny * d.nz;
  const T D = (T)d.dx, iD = (T)(1.0 / d.dx), iD2 = (T)(1.0 / (d.dx * d.dx));
  const T idt = (T)(1.0 / p.dt), irho0 = (T)(1.0 / p.rho0), inum = (T)(1.0 / p.nu_m), num = (T)p.nu_m;
  const bool three = d.dim == 3;
  const int XX = 0, YY = 1, ZZ = three ? 2 : 2, XY = 3, XZ = three ? 4 : 1, YZ = 5;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(id % d.nx);
    const int j = (int)((id / d.nx) % d.ny);
    const int k = (int)(id / ((size_t)d.nx * d.ny));
    // ---------------- x momentum, u-face (i, j, k) ----------------
    {
      const T rho = A.rho_of(A.a.rs.phifx[id]);
      const T u0 = A.US(i, j, k);
      const T cxx0 = (T)0.25 * (u0 + A.US(i + 1, j, k)) * (u0 + A.US(i + 1, j, k));
      const T cxx1 = (T)0.25 * (A.US(i - 1, j, k) + u0) * (A.US(i - 1, j, k) + u0);
      T adv = (cxx0 - cxx1) * iD + (A.Exz(i, j, k + 1) - A.Exz(i, j, k)) * iD;
      const T Jzu = (T)0.25 * (A.Jz(i - 1, j, k) + A.Jz(i, j, k) + A.Jz(i - 1, j, k + 1) + A.Jz(i, j, k + 1));
      T jg = A.Jx(i, j, k) * (A.US(i + 1, j, k) - A.US(i - 1, j, k)) * (T)0.5 * iD +
             Jzu * (A.US(i, j, k + 1) - A.US(i, j, k - 1)) * (T)0.5 * iD;
      T lap = (A.US(i + 1, j, k) + A.US(i - 1, j, k) - 2 * u0 + A.US(i, j, k + 1) + A.US(i, j, k - 1) - 2 * u0) * iD2;
      const T sxx0 = 2 * A.muc(i, j, k) * (A.US(i + 1, j, k) - u0) * iD;
      const T sxx1 = 2 * A.muc(i - 1, j, k) * (u0 - A.US(i - 1, j, k)) * iD;
      T visc = (sxx0 - sxx1) * iD + (A.Sxz(i, j, k + 1) - A.Sxz(i, j, k)) * iD;
      T divt = 0;
      if (have_tau)
        divt = (A.tau(XX, i, j, k) - A.tau(XX, i - 1, j, k)) * iD + (A.Txz(XZ, i, j, k + 1) - A.Txz(XZ, i, j, k)) * iD;
      if (three) {
        adv += (A.Exy(i, j + 1, k) - A.Exy(i, j, k)) * iD;
        const T Jyu = (T)0.25 * (A.Jy(i - 1, j, k) + A.Jy(i, j, k) + A.Jy(i - 1, j + 1, k) + A.Jy(i, j + 1, k));
        jg += Jyu * (A.US(i, j + 1, k) - A.US(i, j - 1, k)) * (T)0.5 * iD;
        lap += (A.US(i, j + 1, k) + A.US(i, j - 1, k) - 2 * u0) * iD2;
        visc += (A.Sxy(i, j + 1, k) - A.Sxy(i, j, k)) * iD;
        if (have_tau) divt += (A.Txy(XY, i, j + 1, k) - A.Txy(XY, i, j, k)) * iD;
      }
      const T st = A.a.rs.Gfx[id] * (A.phic(i, j, k) - A.phic(i - 1, j, k)) * iD;
      const T gp = (A.Pn(i, j, k) - A.Pn(i - 1, j, k)) * iD * irho0 +
                   ((T)1 / rho - irho0) * (A.Ps(i, j, k) - A.Ps(i - 1, j, k)) * iD;
      const T R = -A.UH(i, j, k) * idt + adv + jg / rho + gp + num * lap - divt / rho - visc / rho - st / rho - (T)p.gx;
      T out = R * inum;
      if (k == 0) out -= (T)(2 * p.uw_bot) * iD2;
      if (k == d.nz - 1) out -= (T)(2 * p.uw_top) * iD2;
      ru[id] = out;
    }
    // ---------------- y momentum, v-face (i, j, k) (3D) ----------------
    if (three) {
      const T rho = A.rho_of(A.a.rs.phify[id]);
      const T v0 = A.VS(i, j, k);
      const T cyy0 = (T)0.25 * (v0 + A.VS(i, j + 1, k)) * (v0 + A.VS(i, j + 1, k));
      const T cyy1 = (T)0.25 * (A.VS(i, j - 1, k) + v0) * (A.VS(i, j - 1, k) + v0);
      const T adv = (cyy0 - cyy1) * iD + (A.Exy(i + 1, j, k) - A.Exy(i, j, k)) * iD +
                    (A.Eyz(i, j, k + 1) - A.Eyz(i, j, k)) * iD;
      const T Jxv = (T)0.25 * (A.Jx(i, j - 1, k) + A.Jx(i + 1, j - 1, k) + A.Jx(i, j, k) + A.Jx(i + 1, j, k));
      const T Jzv = (T)0.25 * (A.Jz(i, j - 1, k) + A.Jz(i, j, k) + A.Jz(i, j - 1, k + 1) + A.Jz(i, j, k + 1));
      const T jg = Jxv * (A.VS(i + 1, j, k) - A.VS(i - 1, j, k)) * (T)0.5 * iD +
                   A.Jy(i, j, k) * (A.VS(i, j + 1, k) - A.VS(i, j - 1, k)) * (T)0.5 * iD +
                   Jzv * (A.VS(i, j, k + 1) - A.VS(i, j, k - 1)) * (T)0.5 * iD;
      const T lap = (A.VS(i + 1, j, k) + A.VS(i - 1, j, k) + A.VS(i, j + 1, k) + A.VS(i, j - 1, k) +
                     A.VS(i, j, k + 1) + A.VS(i, j, k - 1) - 6 * v0) * iD2;
      const T syy0 = 2 * A.muc(i, j, k) * (A.VS(i, j + 1, k) - v0) * iD;
      const T syy1 = 2 * A.muc(i, j - 1, k) * (v0 - A.VS(i, j - 1, k)) * iD;
      const T visc = (syy0 - syy1) * iD + (A.Sxy(i + 1, j, k) - A.Sxy(i, j, k)) * iD +
                     (A.Syz(i, j, k + 1) - A.Syz(i, j, k)) * iD;
      T divt = 0;
      if (have_tau)
        divt = (A.tau(YY, i, j, k) - A.tau(YY, i, j - 1, k)) * iD + (A.Txy(XY, i + 1, j, k) - A.Txy(XY, i, j, k)) * iD +
               (A.Tyz(YZ, i, j, k + 1) - A.Tyz(YZ, i, j, k)) * iD;
      const T st = A.a.rs.Gfy[id] * (A.phic(i, j, k) - A.phic(i, j - 1, k)) * iD;
      const T gp = (A.Pn(i, j, k) - A.Pn(i, j - 1, k)) * iD * irho0 +
                   ((T)1 / rho - irho0) * (A.Ps(i, j, k) - A.Ps(i, j - 1, k)) * iD;
      const T R = -A.VH(i, j, k) * idt + adv + jg / rho + gp + num * lap - divt / rho - visc / rho - st / rho - (T)p.gy;
      rv[id] = R * inum;
    }
    // ---------------- z momentum, w-face k (interior k = 1..nz-1) ----------------
    if (k >= 1) {
      const T rho = A.rho_of(A.a.rs.phifz[id]);
      const T w0 = A.WS(i, j, k);
      const T czz0 = (T)0.25 * (w0 + A.WS(i, j, k + 1)) * (w0 + A.WS(i, j, k + 1));
      const T czz1 = (T)0.25 * (A.WS(i, j, k - 1) + w0) * (A.WS(i, j, k - 1) + w0);
      T adv = (A.Exz(i + 1, j, k) - A.Exz(i, j, k)) * iD + (czz0 - czz1) * iD;
      const T Jxw = (T)0.25 * (A.Jx(i, j, k - 1) + A.Jx(i + 1, j, k - 1) + A.Jx(i, j, k) + A.Jx(i + 1, j, k));
      T jg = Jxw * (A.WS(i + 1, j, k) - A.WS(i - 1, j, k)) * (T)0.5 * iD +
             A.Jz(i, j, k) * (A.WS(i, j, k + 1) - A.WS(i, j, k - 1)) * (T)0.5 * iD;
      T lap = (A.WS(i + 1, j, k) + A.WS(i - 1, j, k) - 2 * w0 + A.WS(i, j, k + 1) + A.WS(i, j, k - 1) - 2 * w0) * iD2;
      const T szz0 = 2 * A.muc(i, j, k) * (A.WS(i, j, k + 1) - w0) * iD;
      const T szz1 = 2 * A.muc(i, j, k - 1) * (w0 - A.WS(i, j, k - 1)) * iD;
      T visc = (A.Sxz(i + 1, j, k) - A.Sxz(i, j, k)) * iD + (szz0 - szz1) * iD;
      T divt = 0;
      if (have_tau)
        divt = (A.Txz(XZ, i + 1, j, k) - A.Txz(XZ, i, j, k)) * iD + (A.tau(ZZ, i, j, k) - A.tau(ZZ, i, j, k - 1)) * iD;
      if (three) {
        adv += (A.Eyz(i, j + 1, k) - A.Eyz(i, j, k)) * iD;
        const T Jyw = (T)0.25 * (A.Jy(i, j, k - 1) + A.Jy(i, j + 1, k - 1) + A.Jy(i, j, k) + A.Jy(i, j + 1, k));
        jg += Jyw * (A.WS(i, j + 1, k) - A.WS(i, j - 1, k)) * (T)0.5 * iD;
        lap += (A.WS(i, j + 1, k) + A.WS(i, j - 1, k) - 2 * w0) * iD2;
        visc += (A.Syz(i, j + 1, k) - A.Syz(i, j, k)) * iD;
        if (have_tau) divt += (A.Tyz(YZ, i, j + 1, k) - A.Tyz(YZ, i, j, k)) * iD;
      }
      const T st = A.a.rs.Gfz[id] * (A.phic(i, j, k) - A.phic(i, j, k - 1)) * iD;
      const T gp = (A.Pn(i, j, k) - A.Pn(i, j, k - 1)) * iD * irho0 +
                   ((T)1 / rho - irho0) * (A.Ps(i, j, k) - A.Ps(i, j, k - 1)) * iD;
      const T R = -A.WH(i, j, k) * idt + adv + jg / rho + gp + num * lap - divt / rho - visc / rho - st / rho - (T)p.gz;
      rw[id - (size_t)d.nx * d.ny] = R * inum;  // face rows 0..nz-2 hold faces 1..nz-1
    }
    (void)D;
  }
}

// (gamma0 rho0/dt) div(u~) at centres; wt holds faces 1..nz-1 as rows 0..nz-2
template <class T>
__global__ void k_div(const T* __restrict__ ut, const T* __restrict__ vt, const T* __restrict__ wt, T* __restrict__ out,
                      Dims d, T coef) {
  const size_t n = (size_t)d.nx * d.ny * d.nz;
  const size_t plane = (size_t)d.nx * d.ny;
  const T iD = (T)(1.0 / d.dx);
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(id % d.nx);
    const int j = (int)((id / d.nx) % d.ny);
    const int k = (int)(id / plane);
    const size_t rowb = id - i;
    T dv = (ut[rowb + wrap(i + 1, d.nx)] - ut[id]) * iD;
    if (d.dim == 3) dv += (vt[((size_t)k * d.ny + wrap(j + 1, d.ny)) * d.nx + i] - vt[id]) * iD;
    const T wtop = (k < d.nz - 1) ? wt[id] : (T)0;              // face k+1 -> row k
    const T wbot = (k > 0) ? wt[id - plane] : (T)0;             // face k   -> row k-1
    dv += (wtop - wbot) * iD;
    out[id] = coef * dv;
  }
}

// u = u~ - cf grad p', p^{n+1} = p^n + p'.  u, v corrected in place (they hold
// u~ on entry); w written with both walls zero from the face rows wt.
template <class T>
__global__ void k_correct(T* __restrict__ u, T* __restrict__ v, const T* __restrict__ wt, T* __restrict__ w,
                          const T* __restrict__ pp, const T* __restrict__ pn, T* __restrict__ pnew, Dims d, T cf) {
  const size_t plane = (size_t)d.nx * d.ny;
  const size_t n = plane * (d.nz + 1);
  const T iD = (T)(1.0 / d.dx);
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(id % d.nx);
    const int j = (int)((id / d.nx) % d.ny);
    const int k = (int)(id / plane);
    if (k == 0 || k == d.nz) {
      w[id] = (T)0;
    } else {
      w[id] = wt[id - plane] - cf * (pp[id] - pp[id - plane]) * iD;
    }
    if (k == d.nz) continue;
    const size_t rowb = id - i;
    u[id] = u[id] - cf * (pp[id] - pp[rowb + wrap(i - 1, d.nx)]) * iD;
    if (d.dim == 3) v[id] = v[id] - cf * (pp[id] - pp[((size_t)k * d.ny + wrap(j - 1, d.ny)) * d.nx + i]) * iD;
    pnew[id] = pn[id] + pp[id];
  }
}

}  // namespace pf
