// Right-hand side of Eq. NS36 (Section 3.2.2) on the 3D coarse MAC mesh as a
// z-march through shared memory.
//
// A CTA owns a TX x TY tile of (i, j) columns and walks a chunk of z layers.
// Every field the stencil reads is staged plane by plane into shared memory
// with a one-cell halo in x and y, so each value crosses from L2 to the SM once
// per CTA instead of once per reading thread:
//  - rings of three planes (k-1, k, k+1) for the fields read off the layer:
//    u*, v*, G at centres, the tau*_xz and tau*_yz stress components, and w*
//    at faces k-1, k, k+1;
//  - one plane for the fields read only within the layer: tau*_xx, tau*_yy,
//    tau*_xy, p^{n-1} - p^n, p*, phi_c, and phi at the x-z (face k), x-y and y-z (face k)
//    edges;
//  - values of the thread's own column one layer down (p^{n-1} - p^n, p*, phi_c,
//    tau*_zz) stay in registers from the previous layer.
// Extrapolations (2 a^n - a^{n-1}) are formed once, when a value is staged.
// Planes beyond the walls are staged as the wall-adjacent plane (the mirror
// ghost the stress terms use; the other fields are not read there), so the
// arithmetic per cell is exactly that of k_ns_rhs_v2_b in ns_rhs.cuh, term by
// term (conservative central advection with edge products, J.grad(u*) with
// 4-point averages, the rho0 pressure split in its cancellation-free form
// (1/rho0) grad(p^{n-1} - p^n) + (1/rho) grad p*, div(tau*) with
// 4-point edge averages, div(mu (grad u* + grad u*^T)) with mu at centres and
// edges, G_face grad(phi_c), body acceleration), written for the increment
// u~ - u* as described in ns.cuh.
#pragma once
#include "ns.cuh"

namespace pf {

struct NsMarch {
  static constexpr int TX = 32, TY = 8, NT = TX * TY;
  static constexpr int SX = TX + 2, SY = TY + 2, PL = SX * SY;  // staged plane with halo
  static constexpr int NSLOT = (PL + NT - 1) / NT;              // staging slots per thread
  // plane indices in shared memory
  enum { U0 = 0, V0 = 3, G0 = 6, XZ0 = 9, YZ0 = 12, W0 = 15,   // rings of 3
         TXX = 18, TYY, TXY, DP, PS, PHC, EXZ, EXY, EYZ, NPL };
  static constexpr size_t smem_elems() { return (size_t)NPL * PL; }
};

// Neighbour access for one cell from the staged planes.  dx, dy in {-1, 0, 1};
// dz in {-1, 0, 1} relative to the cell's layer (faces: relative to face k).
template <class T>
struct NsSmemAcc {
  const T* s;           // shared base + the cell's index in a staged plane
  int z[3];             // offsets of the ring slots holding layers k-1, k, k+1
  T dp_zm, ps_zm, phc_zm, tzz_c, tzz_zm, exz_zp, eyz_zp;
  T du, dv, dw, phifx, phify, phifz, gfx, gfy, gfz;  // du = u^n - u^{n-1} at the face
  static constexpr int PL = NsMarch::PL, SX = NsMarch::SX;
  __device__ __forceinline__ T r(int f, int dx, int dy, int dz) const { return s[f * PL + z[dz + 1] + dy * SX + dx]; }
  __device__ __forceinline__ T p(int f, int dx, int dy) const { return s[f * PL + dy * SX + dx]; }
  __device__ __forceinline__ T U(int dx, int dy, int dz) const { return r(NsMarch::U0, dx, dy, dz); }
  __device__ __forceinline__ T V(int dx, int dy, int dz) const { return r(NsMarch::V0, dx, dy, dz); }
  __device__ __forceinline__ T G(int dx, int dy, int dz) const { return r(NsMarch::G0, dx, dy, dz); }
  __device__ __forceinline__ T TXZ(int dx, int dy, int dz) const { return r(NsMarch::XZ0, dx, dy, dz); }
  __device__ __forceinline__ T TYZ(int dx, int dy, int dz) const { return r(NsMarch::YZ0, dx, dy, dz); }
  __device__ __forceinline__ T W(int dx, int dy, int dz) const { return r(NsMarch::W0, dx, dy, dz); }
  __device__ __forceinline__ T TXX(int dx, int dy) const { return p(NsMarch::TXX, dx, dy); }
  __device__ __forceinline__ T TYY(int dx, int dy) const { return p(NsMarch::TYY, dx, dy); }
  __device__ __forceinline__ T TXY(int dx, int dy) const { return p(NsMarch::TXY, dx, dy); }
  __device__ __forceinline__ T DP(int dx, int dy) const { return p(NsMarch::DP, dx, dy); }
  __device__ __forceinline__ T PS(int dx, int dy) const { return p(NsMarch::PS, dx, dy); }
  __device__ __forceinline__ T PHC(int dx, int dy) const { return p(NsMarch::PHC, dx, dy); }
  __device__ __forceinline__ T EXZ(int dx) const { return p(NsMarch::EXZ, dx, 0); }
  __device__ __forceinline__ T EXY(int dx, int dy) const { return p(NsMarch::EXY, dx, dy); }
  __device__ __forceinline__ T EYZ(int dy) const { return p(NsMarch::EYZ, 0, dy); }
};

// The three momentum rows of cell (i, j, k): x at the u-face, y at the v-face,
// z at the w-face k (k >= 1).  Terms and their order as in k_ns_rhs_v2_b.
template <class T, class Acc>
__device__ __forceinline__ void ns_rhs_cell3(const Acc& A, const PhysT<T>& q, const int k, const int nz,
                                             const int have_tau, T& ru, T& rv, T& rw) {
  const bool hasb = k > 0, hast = k < nz - 1;
  const T iD = q.iD, iD2 = q.iD2, h = (T)0.5;
  auto mu_of = [&](T ph) { return h * ((T)1 + ph) * q.mu_s1 + h * ((T)1 - ph) * q.mu_s2; };
  auto rho_of = [&](T ph) { return h * ((T)1 + ph) * q.rho1 + h * ((T)1 - ph) * q.rho2; };
  const T Uc = A.U(0, 0, 0), Uxp = A.U(1, 0, 0), Uxm = A.U(-1, 0, 0);
  const T Uzp = hast ? A.U(0, 0, 1) : q.uw2_top - Uc;
  const T Uzm = hasb ? A.U(0, 0, -1) : q.uw2_bot - Uc;
  const T Uxp_zm = hasb ? A.U(1, 0, -1) : (T)0;
  const T Wc = A.W(0, 0, 0), Wzp = A.W(0, 0, 1), Wxm = A.W(-1, 0, 0), Wxp = A.W(1, 0, 0);
  const T Wxm_zp = A.W(-1, 0, 1);
  const T Wzm = hasb ? A.W(0, 0, -1) : (T)0;
  const T Dp_c = A.DP(0, 0), Ps_c = A.PS(0, 0);
  const T phc = A.PHC(0, 0), phc_xm = A.PHC(-1, 0);
  const T Gc_c = A.G(0, 0, 0), Gc_xm = A.G(-1, 0, 0), Gc_xp = A.G(1, 0, 0);
  const T muc = mu_of(phc), muc_xm = mu_of(phc_xm);
  const T muexz = mu_of(A.EXZ(0)), muexz_zp = mu_of(A.exz_zp), muexz_xp = mu_of(A.EXZ(1));
  const T cj = q.cj_dx;
  const T Jx_c = cj * (Gc_c - Gc_xm);
  const T Gc_zp = hast ? A.G(0, 0, 1) : (T)0, Gc_xm_zp = hast ? A.G(-1, 0, 1) : (T)0;
  const T Gc_zm = hasb ? A.G(0, 0, -1) : (T)0, Gc_xm_zm = hasb ? A.G(-1, 0, -1) : (T)0;
  const T Jz_c = hasb ? cj * (Gc_c - Gc_zm) : (T)0;
  const T Jz_xm = hasb ? cj * (Gc_xm - Gc_xm_zm) : (T)0;
  const T Jz_zp = hast ? cj * (Gc_zp - Gc_c) : (T)0;
  const T Jz_xm_zp = hast ? cj * (Gc_xm_zp - Gc_xm) : (T)0;
  const T Uyp = A.U(0, 1, 0), Uym = A.U(0, -1, 0);
  const T Vc = A.V(0, 0, 0), Vxm = A.V(-1, 0, 0), Vyp = A.V(0, 1, 0);
  const T Gc_yp = A.G(0, 1, 0), Gc_ym = A.G(0, -1, 0);
  // ================= x momentum at the u-face =================
  {
    const T rho = rho_of(A.phifx);
    const T cxx0 = (T)0.25 * (Uc + Uxp) * (Uc + Uxp), cxx1 = (T)0.25 * (Uxm + Uc) * (Uxm + Uc);
    const T Exz_p = (T)0.25 * (Uc + Uzp) * (Wxm_zp + Wzp);
    const T Exz_0 = (T)0.25 * (Uzm + Uc) * (Wxm + Wc);
    T adv = (cxx0 - cxx1 + Exz_p - Exz_0) * iD;
    const T Jzu = (T)0.25 * (Jz_xm + Jz_c + Jz_xm_zp + Jz_zp);
    T jg = (Jx_c * (Uxp - Uxm) + Jzu * (Uzp - Uzm)) * h * iD;
    const T sxx0 = 2 * muc * (Uxp - Uc), sxx1 = 2 * muc_xm * (Uc - Uxm);
    const T sxz_p = muexz_zp * ((Uzp - Uc) + (Wzp - Wxm_zp));
    const T sxz_0 = muexz * ((Uc - Uzm) + (Wc - Wxm));
    T visc = (sxx0 - sxx1 + sxz_p - sxz_0) * iD2;
    T divt = 0;
    if (have_tau) {
      const T tzc = A.TXZ(0, 0, 0), tzxm = A.TXZ(-1, 0, 0);
      const T tzzp = A.TXZ(0, 0, 1), tzxmzp = A.TXZ(-1, 0, 1);
      const T tzzm = A.TXZ(0, 0, -1), tzxmzm = A.TXZ(-1, 0, -1);
      const T Txz_p = (T)0.25 * (tzxm + tzc + tzxmzp + tzzp);
      const T Txz_0 = (T)0.25 * (tzxmzm + tzzm + tzxm + tzc);
      divt = (A.TXX(0, 0) - A.TXX(-1, 0) + Txz_p - Txz_0) * iD;
      const T t00 = A.TXY(0, 0), t0m = A.TXY(-1, 0), tp0 = A.TXY(0, 1), tpm = A.TXY(-1, 1), tm0 = A.TXY(0, -1),
              tmm = A.TXY(-1, -1);
      divt += ((T)0.25 * (t0m + t00 + tpm + tp0) - (T)0.25 * (tmm + tm0 + t0m + t00)) * iD;
    }
    {
      const T Vxm_yp = A.V(-1, 1, 0);
      const T Exy_p = (T)0.25 * (Uc + Uyp) * (Vxm_yp + Vyp);
      const T Exy_0 = (T)0.25 * (Uym + Uc) * (Vxm + Vc);
      adv += (Exy_p - Exy_0) * iD;
      const T Gc_xm_yp = A.G(-1, 1, 0), Gc_xm_ym = A.G(-1, -1, 0);
      const T Jy_c = cj * (Gc_c - Gc_ym), Jy_xm = cj * (Gc_xm - Gc_xm_ym);
      const T Jy_yp = cj * (Gc_yp - Gc_c), Jy_xm_yp = cj * (Gc_xm_yp - Gc_xm);
      const T Jyu = (T)0.25 * (Jy_xm + Jy_c + Jy_xm_yp + Jy_yp);
      jg += Jyu * (Uyp - Uym) * h * iD;
      const T muexy = mu_of(A.EXY(0, 0)), muexy_yp = mu_of(A.EXY(0, 1));
      const T sxy_p = muexy_yp * ((Uyp - Uc) + (Vyp - Vxm_yp));
      const T sxy_0 = muexy * ((Uc - Uym) + (Vc - Vxm));
      visc += (sxy_p - sxy_0) * iD2;
    }
    const T st = A.gfx * (phc - phc_xm) * iD;
    const T gdp = (Dp_c - A.DP(-1, 0)) * iD, gps = (Ps_c - A.PS(-1, 0)) * iD;
    const T R = A.du * q.idt + adv + (jg - divt - visc - st + gps) / rho + gdp * q.irho0 - q.gx;
    ru = R * q.inum;
  }
  // ================= y momentum at the v-face =================
  {
    const T Vxp = A.V(1, 0, 0), Vym = A.V(0, -1, 0);
    const T Vzp = hast ? A.V(0, 0, 1) : -Vc;
    const T Vzm = hasb ? A.V(0, 0, -1) : -Vc;
    const T Uxp_ym = A.U(1, -1, 0);
    const T Wym = A.W(0, -1, 0), Wym_zp = A.W(0, -1, 1);
    const T rho = rho_of(A.phify);
    const T cyy0 = (T)0.25 * (Vc + Vyp) * (Vc + Vyp), cyy1 = (T)0.25 * (Vym + Vc) * (Vym + Vc);
    const T Exy_xp = (T)0.25 * (Uxp_ym + Uxp) * (Vc + Vxp);
    const T Exy_0 = (T)0.25 * (Uym + Uc) * (Vxm + Vc);
    const T Eyz_p = (T)0.25 * (Vc + Vzp) * (Wym_zp + Wzp);
    const T Eyz_0 = (T)0.25 * (Vzm + Vc) * (Wym + Wc);
    const T adv = (cyy0 - cyy1 + Exy_xp - Exy_0 + Eyz_p - Eyz_0) * iD;
    const T Gc_xp_ym = A.G(1, -1, 0), Gc_xm_ym = A.G(-1, -1, 0);
    const T Jx_ym = cj * (Gc_ym - Gc_xm_ym), Jx_xp_ym = cj * (Gc_xp_ym - Gc_ym), Jx_xp = cj * (Gc_xp - Gc_c);
    const T Jxv = (T)0.25 * (Jx_ym + Jx_xp_ym + Jx_c + Jx_xp);
    const T Jy_c = cj * (Gc_c - Gc_ym);
    const T Gc_ym_zm = hasb ? A.G(0, -1, -1) : (T)0, Gc_ym_zp = hast ? A.G(0, -1, 1) : (T)0;
    const T Jz_ym = hasb ? cj * (Gc_ym - Gc_ym_zm) : (T)0;
    const T Jz_ym_zp = hast ? cj * (Gc_ym_zp - Gc_ym) : (T)0;
    const T Jzv = (T)0.25 * (Jz_ym + Jz_c + Jz_ym_zp + Jz_zp);
    const T jg = (Jxv * (Vxp - Vxm) + Jy_c * (Vyp - Vym) + Jzv * (Vzp - Vzm)) * h * iD;
    const T muc_ym = mu_of(A.PHC(0, -1));
    const T syy0 = 2 * muc * (Vyp - Vc), syy1 = 2 * muc_ym * (Vc - Vym);
    const T muexy = mu_of(A.EXY(0, 0)), muexy_xp = mu_of(A.EXY(1, 0));
    const T sxy_xp = muexy_xp * ((Uxp - Uxp_ym) + (Vxp - Vc));
    const T sxy_0 = muexy * ((Uc - Uym) + (Vc - Vxm));
    const T mueyz = mu_of(A.EYZ(0)), mueyz_zp = mu_of(A.eyz_zp);
    const T syz_p = mueyz_zp * ((Vzp - Vc) + (Wzp - Wym_zp));
    const T syz_0 = mueyz * ((Vc - Vzm) + (Wc - Wym));
    const T visc = (syy0 - syy1 + sxy_xp - sxy_0 + syz_p - syz_0) * iD2;
    T divt = 0;
    if (have_tau) {
      const T a00 = A.TXY(0, 0), a0m = A.TXY(0, -1), ap0 = A.TXY(1, 0), apm = A.TXY(1, -1), am0 = A.TXY(-1, 0),
              amm = A.TXY(-1, -1);
      const T Txy_xp = (T)0.25 * (a0m + apm + a00 + ap0), Txy_0 = (T)0.25 * (amm + a0m + am0 + a00);
      const T b00 = A.TYZ(0, 0, 0), bm0 = A.TYZ(0, -1, 0), b0p = A.TYZ(0, 0, 1), bmp = A.TYZ(0, -1, 1),
              b0m = A.TYZ(0, 0, -1), bmm = A.TYZ(0, -1, -1);
      const T Tyz_p = (T)0.25 * (bm0 + b00 + bmp + b0p), Tyz_0 = (T)0.25 * (bmm + b0m + bm0 + b00);
      divt = (A.TYY(0, 0) - A.TYY(0, -1) + Txy_xp - Txy_0 + Tyz_p - Tyz_0) * iD;
    }
    const T st = A.gfy * (phc - A.PHC(0, -1)) * iD;
    const T gdp = (Dp_c - A.DP(0, -1)) * iD, gps = (Ps_c - A.PS(0, -1)) * iD;
    const T R = A.dv * q.idt + adv + (jg - divt - visc - st + gps) / rho + gdp * q.irho0 - q.gy;
    rv = R * q.inum;
  }
  // ================= z momentum at the w-face k (interior faces 1..nz-1) =================
  if (hasb) {
    const T rho = rho_of(A.phifz);
    const T Exz_xp = (T)0.25 * (Uxp_zm + Uxp) * (Wc + Wxp);
    const T Exz_0 = (T)0.25 * (Uzm + Uc) * (Wxm + Wc);
    const T czz0 = (T)0.25 * (Wc + Wzp) * (Wc + Wzp), czz1 = (T)0.25 * (Wzm + Wc) * (Wzm + Wc);
    T adv = (Exz_xp - Exz_0 + czz0 - czz1) * iD;
    const T Gc_xp_zm = A.G(1, 0, -1);
    const T Jx_zm = cj * (Gc_zm - Gc_xm_zm), Jx_xp_zm = cj * (Gc_xp_zm - Gc_zm), Jx_xp = cj * (Gc_xp - Gc_c);
    const T Jxw = (T)0.25 * (Jx_zm + Jx_xp_zm + Jx_c + Jx_xp);
    T jg = (Jxw * (Wxp - Wxm) + Jz_c * (Wzp - Wzm)) * h * iD;
    const T muc_zm = mu_of(A.phc_zm);
    const T szz0 = 2 * muc * (Wzp - Wc), szz1 = 2 * muc_zm * (Wc - Wzm);
    const T sxz_xp = muexz_xp * ((Uxp - Uxp_zm) + (Wxp - Wc));
    const T sxz_0 = muexz * ((Uc - Uzm) + (Wc - Wxm));
    T visc = (sxz_xp - sxz_0 + szz0 - szz1) * iD2;
    T divt = 0;
    if (have_tau) {
      const T e00 = A.TXZ(0, 0, 0), e0m = A.TXZ(0, 0, -1), ep0 = A.TXZ(1, 0, 0), epm = A.TXZ(1, 0, -1),
              em0 = A.TXZ(-1, 0, 0), emm = A.TXZ(-1, 0, -1);
      const T Txz_xp = (T)0.25 * (e0m + epm + e00 + ep0), Txz_0 = (T)0.25 * (emm + e0m + em0 + e00);
      divt = (Txz_xp - Txz_0 + A.tzz_c - A.tzz_zm) * iD;
      const T f00 = A.TYZ(0, 0, 0), f0m = A.TYZ(0, 0, -1), fp0 = A.TYZ(0, 1, 0), fpm = A.TYZ(0, 1, -1),
              fm0 = A.TYZ(0, -1, 0), fmm = A.TYZ(0, -1, -1);
      divt += ((T)0.25 * (f0m + fpm + f00 + fp0) - (T)0.25 * (fmm + f0m + fm0 + f00)) * iD;
    }
    {
      const T Vzm_r = A.V(0, 0, -1), Vyp_zm = A.V(0, 1, -1);
      const T Wyp = A.W(0, 1, 0), Wym = A.W(0, -1, 0);
      const T Eyz_yp = (T)0.25 * (Vyp_zm + Vyp) * (Wc + Wyp);
      const T Eyz_0 = (T)0.25 * (Vzm_r + Vc) * (Wym + Wc);
      adv += (Eyz_yp - Eyz_0) * iD;
      const T Gc_ym_zm = A.G(0, -1, -1), Gc_yp_zm = A.G(0, 1, -1);
      const T Jy_zm = cj * (Gc_zm - Gc_ym_zm), Jy_yp_zm = cj * (Gc_yp_zm - Gc_zm);
      const T Jy_c = cj * (Gc_c - Gc_ym), Jy_yp = cj * (Gc_yp - Gc_c);
      const T Jyw = (T)0.25 * (Jy_zm + Jy_yp_zm + Jy_c + Jy_yp);
      jg += Jyw * (Wyp - Wym) * h * iD;
      const T mueyz = mu_of(A.EYZ(0)), mueyz_yp = mu_of(A.EYZ(1));
      const T syz_yp = mueyz_yp * ((Vyp - Vyp_zm) + (Wyp - Wc));
      const T syz_0 = mueyz * ((Vc - Vzm_r) + (Wc - Wym));
      visc += (syz_yp - syz_0) * iD2;
    }
    const T st = A.gfz * (phc - A.phc_zm) * iD;
    const T gdp = (Dp_c - A.dp_zm) * iD, gps = (Ps_c - A.ps_zm) * iD;
    const T R = A.dw * q.idt + adv + (jg - divt - visc - st + gps) / rho + gdp * q.irho0 - q.gz;
    rw = R * q.inum;
  }
}

// grid: (ceil(nx/TX), ceil(ny/TY), ceil(nz/kz)); needs nx >= TX, ny >= TY (one
// wrap of a halo index suffices).  Dynamic shared memory: smem_elems() * sizeof(T).
template <class T, int MINB>
__global__ void __launch_bounds__(NsMarch::NT, MINB)
    k_ns_rhs_march3(const __grid_constant__ NsIn<T> a, const Dims d, const PhysT<T> q, T* __restrict__ ru,
                    T* __restrict__ rv, T* __restrict__ rw, const int have_tau, const int kz) {
  using M = NsMarch;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int nx = d.nx, ny = d.ny, nz = d.nz;
  const int P = nx * ny;
  const int tid = threadIdx.x;
  const int tx = tid % M::TX, ty = tid / M::TX;
  const int i0 = blockIdx.x * M::TX, j0 = blockIdx.y * M::TY;
  const int k0 = blockIdx.z * kz, k1 = min(k0 + kz, nz);
  // staging slots: the in-plane offset of each staged element
  int soff[M::NSLOT];
  bool sval[M::NSLOT];
#pragma unroll
  for (int s = 0; s < M::NSLOT; ++s) {
    const int e = tid + s * M::NT;
    sval[s] = e < M::PL;
    const int sx = e % M::SX, sy = e / M::SX;
    const int gi = wrap(i0 + sx - 1, nx), gj = wrap(j0 + sy - 1, ny);
    soff[s] = sval[s] ? gj * nx + gi : 0;
  }
  auto plane = [&](int p) { return sm + (size_t)p * M::PL; };
  auto ex = [](const T* n, const T* o, int idx) { return (T)2 * n[idx] - o[idx]; };
  const T* tn[6];
  const T* to[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    tn[c] = a.tn[c];
    to[c] = a.to[c];
  }
  // stage ring plane `slot` of the cell fields with layer kk (clamped to the
  // walls: the mirror plane), and of w with face kf (0..nz)
  auto stage_ring = [&](int slot, int kk, int kf) {
    kk = kk < 0 ? 0 : (kk > nz - 1 ? nz - 1 : kk);
    kf = kf < 0 ? 0 : kf;
    const int b = kk * P, bf = kf * P;
#pragma unroll
    for (int s = 0; s < M::NSLOT; ++s) {
      if (!sval[s]) continue;
      const int e = tid + s * M::NT;
      const int g = b + soff[s], gf = bf + soff[s];
      plane(M::U0 + slot)[e] = ex(a.un, a.uo, g);
      plane(M::V0 + slot)[e] = ex(a.vn, a.vo, g);
      plane(M::G0 + slot)[e] = a.rs.Gc[g];
      plane(M::W0 + slot)[e] = ex(a.wn, a.wo, gf);
      if (have_tau) {
        plane(M::XZ0 + slot)[e] = ex(tn[4], to[4], g);
        plane(M::YZ0 + slot)[e] = ex(tn[5], to[5], g);
      }
    }
  };
  auto stage_layer = [&](int kk) {
    const int b = kk * P;
#pragma unroll
    for (int s = 0; s < M::NSLOT; ++s) {
      if (!sval[s]) continue;
      const int e = tid + s * M::NT;
      const int g = b + soff[s];
      plane(M::DP)[e] = a.po[g] - a.pn[g];
      plane(M::PS)[e] = ex(a.pn, a.po, g);
      plane(M::PHC)[e] = a.rs.phic[g];
      plane(M::EXZ)[e] = a.rs.phiexz[g];
      plane(M::EXY)[e] = a.rs.phiexy[g];
      plane(M::EYZ)[e] = a.rs.phieyz[g];
      if (have_tau) {
        plane(M::TXX)[e] = ex(tn[0], to[0], g);
        plane(M::TYY)[e] = ex(tn[1], to[1], g);
        plane(M::TXY)[e] = ex(tn[3], to[3], g);
      }
    }
  };
  const int i = i0 + tx, j = j0 + ty;
  const bool own = i < nx && j < ny;
  const int col = own ? j * nx + i : 0;
  NsSmemAcc<T> A;
  A.s = sm + (ty + 1) * M::SX + tx + 1;
  // the thread's own column one layer below the chunk (unused at k = 0)
  {
    const int km = k0 > 0 ? k0 - 1 : 0;
    const int g = km * P + col;
    A.dp_zm = a.po[g] - a.pn[g];
    A.ps_zm = ex(a.pn, a.po, g);
    A.phc_zm = a.rs.phic[g];
    A.tzz_zm = have_tau ? ex(tn[2], to[2], g) : (T)0;
  }
  // ring slots: r0 holds layer k-1, r1 layer k, r2 layer k+1 (rotating)
  int r0 = 0, r1 = 1, r2 = 2;
  stage_ring(r0, k0 - 1, k0 - 1);
  stage_ring(r1, k0, k0);
  for (int k = k0; k < k1; ++k) {
    stage_ring(r2, k + 1, k + 1);
    stage_layer(k);
    __syncthreads();
    if (own) {
      const int c = k * P + col;
      A.z[0] = r0 * M::PL;
      A.z[1] = r1 * M::PL;
      A.z[2] = r2 * M::PL;
      A.du = a.un[c] - a.uo[c];
      A.dv = a.vn[c] - a.vo[c];
      A.dw = a.wn[c] - a.wo[c];
      A.phifx = a.rs.phifx[c];
      A.phify = a.rs.phify[c];
      A.phifz = a.rs.phifz[c];
      A.gfx = a.rs.Gfx[c];
      A.gfy = a.rs.Gfy[c];
      A.gfz = a.rs.Gfz[c];
      A.exz_zp = a.rs.phiexz[c + P];
      A.eyz_zp = a.rs.phieyz[c + P];
      A.tzz_c = have_tau ? ex(tn[2], to[2], c) : (T)0;
      T oru = 0, orv = 0, orw = 0;
      ns_rhs_cell3<T>(A, q, k, nz, have_tau, oru, orv, orw);
      ru[c] = oru;
      rv[c] = orv;
      if (k > 0) rw[c - P] = orw;  // face rows 0..nz-2 hold faces 1..nz-1
      // own column of this layer becomes the layer below of the next
      A.dp_zm = A.DP(0, 0);
      A.ps_zm = A.PS(0, 0);
      A.phc_zm = A.PHC(0, 0);
      A.tzz_zm = A.tzz_c;
    }
    __syncthreads();
    const int t = r0;
    r0 = r1;
    r1 = r2;
    r2 = t;
  }
}

}  // namespace pf
