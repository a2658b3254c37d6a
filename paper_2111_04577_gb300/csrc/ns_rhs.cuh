// Right-hand side of Eq. NS36 (Section 3.2.2) on the coarse MAC mesh, one
// thread per cell (i, j, k) computing the x-, y- (3D) and z-momentum rows of
// its own u-, v- and (bottom) w-face.  Every neighbour value is loaded once
// through 32-bit offsets; the terms follow the discretisation documented in
// ns.cuh: conservative central advection with edge products, J.grad(u*) with
// 4-point face averages of J = -(rho1 - rho2)/2 M grad(G), pressure split with
// rho0, nu_m lap(u*), div(tau*) with 4-point edge averages of the centre stress
// (mirror ghost at the walls), div(mu (grad u* + grad u*^T)) with mu at centres
// and edges, surface force G_face grad(phi_c), body acceleration g.  It is the
// right side of the increment delta = u~ - u* (ns.cuh), so u_hat/dt and
// nu_m lap(u*) do not appear: (u^n - u^{n-1})/dt stands in their place.
#pragma once
#include "ns.cuh"

namespace pf {

// The two momentum rows of 2D cell (i, k): x at its u-face, z at its w-face k
// (k >= 1).  T is the arithmetic type (float, double, or Dual for the
// derivatives the adjoint takes of it); the accessor A supplies the inputs by
// offset from the cell: U, W (extrapolated u*, w*; W's dz is relative to face
// k), DP = p^{n-1} - p^n, PS = p*, PHC, G (centres), EXZ (x-z edges, dz relative
// to face k), TXX, TXZ, TZZ (extrapolated tau*; layers beyond a wall read as the
// wall layer, the mirror ghost), and at the cell's own faces phifx, phifz, gfx,
// gfz, du = u^n - u^{n-1}, dw = w^n - w^{n-1}.  Terms as in k_ns_rhs_v2_b.
template <class T, class Acc>
__device__ __forceinline__ void ns_rhs_cell2(const Acc& A, const PhysT<T>& q, const int k, const int nz,
                                             const int have_tau, T& ru, T& rw) {
  const bool hasb = k > 0, hast = k < nz - 1;
  const T iD = q.iD, iD2 = q.iD2, h = (T)0.5;
  auto mu_of = [&](T ph) { return h * ((T)1 + ph) * q.mu_s1 + h * ((T)1 - ph) * q.mu_s2; };
  auto rho_of = [&](T ph) { return h * ((T)1 + ph) * q.rho1 + h * ((T)1 - ph) * q.rho2; };
  const T Uc = A.U(0, 0), Uxp = A.U(1, 0), Uxm = A.U(-1, 0);
  const T Uzp = hast ? A.U(0, 1) : q.uw2_top - Uc;
  const T Uzm = hasb ? A.U(0, -1) : q.uw2_bot - Uc;
  const T Uxp_zm = hasb ? A.U(1, -1) : (T)0;
  const T Wc = A.W(0, 0), Wzp = A.W(0, 1), Wxm = A.W(-1, 0), Wxp = A.W(1, 0), Wxm_zp = A.W(-1, 1);
  const T Wzm = hasb ? A.W(0, -1) : (T)0;
  const T Dp_c = A.DP(0, 0), Ps_c = A.PS(0, 0);
  const T phc = A.PHC(0, 0), phc_xm = A.PHC(-1, 0);
  const T Gc_c = A.G(0, 0), Gc_xm = A.G(-1, 0), Gc_xp = A.G(1, 0);
  const T muc = mu_of(phc), muc_xm = mu_of(phc_xm);
  const T muexz = mu_of(A.EXZ(0, 0)), muexz_zp = mu_of(A.EXZ(0, 1)), muexz_xp = mu_of(A.EXZ(1, 0));
  const T cj = q.cj_dx;
  const T Jx_c = cj * (Gc_c - Gc_xm);
  const T Gc_zp = hast ? A.G(0, 1) : (T)0, Gc_xm_zp = hast ? A.G(-1, 1) : (T)0;
  const T Gc_zm = hasb ? A.G(0, -1) : (T)0, Gc_xm_zm = hasb ? A.G(-1, -1) : (T)0;
  const T Jz_c = hasb ? cj * (Gc_c - Gc_zm) : (T)0;
  const T Jz_xm = hasb ? cj * (Gc_xm - Gc_xm_zm) : (T)0;
  const T Jz_zp = hast ? cj * (Gc_zp - Gc_c) : (T)0;
  const T Jz_xm_zp = hast ? cj * (Gc_xm_zp - Gc_xm) : (T)0;
  {  // x momentum at the u-face
    const T rho = rho_of(A.phifx());
    const T cxx0 = (T)0.25 * (Uc + Uxp) * (Uc + Uxp), cxx1 = (T)0.25 * (Uxm + Uc) * (Uxm + Uc);
    const T Exz_p = (T)0.25 * (Uc + Uzp) * (Wxm_zp + Wzp);
    const T Exz_0 = (T)0.25 * (Uzm + Uc) * (Wxm + Wc);
    const T adv = (cxx0 - cxx1 + Exz_p - Exz_0) * iD;
    const T Jzu = (T)0.25 * (Jz_xm + Jz_c + Jz_xm_zp + Jz_zp);
    const T jg = (Jx_c * (Uxp - Uxm) + Jzu * (Uzp - Uzm)) * h * iD;
    const T sxx0 = 2 * muc * (Uxp - Uc), sxx1 = 2 * muc_xm * (Uc - Uxm);
    const T sxz_p = muexz_zp * ((Uzp - Uc) + (Wzp - Wxm_zp));
    const T sxz_0 = muexz * ((Uc - Uzm) + (Wc - Wxm));
    const T visc = (sxx0 - sxx1 + sxz_p - sxz_0) * iD2;
    T divt = 0;
    if (have_tau) {
      const T tzc = A.TXZ(0, 0), tzxm = A.TXZ(-1, 0);
      const T tzzp = A.TXZ(0, 1), tzxmzp = A.TXZ(-1, 1);
      const T tzzm = A.TXZ(0, -1), tzxmzm = A.TXZ(-1, -1);
      const T Txz_p = (T)0.25 * (tzxm + tzc + tzxmzp + tzzp);
      const T Txz_0 = (T)0.25 * (tzxmzm + tzzm + tzxm + tzc);
      divt = (A.TXX(0, 0) - A.TXX(-1, 0) + Txz_p - Txz_0) * iD;
    }
    const T st = A.gfx() * (phc - phc_xm) * iD;
    const T gdp = (Dp_c - A.DP(-1, 0)) * iD, gps = (Ps_c - A.PS(-1, 0)) * iD;
    const T R = A.du() * q.idt + adv + (jg - divt - visc - st + gps) / rho + gdp * q.irho0 - q.gx;
    ru = R * q.inum;
  }
  if (hasb) {  // z momentum at the w-face k
    const T rho = rho_of(A.phifz());
    const T Exz_xp = (T)0.25 * (Uxp_zm + Uxp) * (Wc + Wxp);
    const T Exz_0 = (T)0.25 * (Uzm + Uc) * (Wxm + Wc);
    const T czz0 = (T)0.25 * (Wc + Wzp) * (Wc + Wzp), czz1 = (T)0.25 * (Wzm + Wc) * (Wzm + Wc);
    const T adv = (Exz_xp - Exz_0 + czz0 - czz1) * iD;
    const T Gc_xp_zm = A.G(1, -1);
    const T Jx_zm = cj * (Gc_zm - Gc_xm_zm), Jx_xp_zm = cj * (Gc_xp_zm - Gc_zm), Jx_xp = cj * (Gc_xp - Gc_c);
    const T Jxw = (T)0.25 * (Jx_zm + Jx_xp_zm + Jx_c + Jx_xp);
    const T jg = (Jxw * (Wxp - Wxm) + Jz_c * (Wzp - Wzm)) * h * iD;
    const T muc_zm = mu_of(A.PHC(0, -1));
    const T szz0 = 2 * muc * (Wzp - Wc), szz1 = 2 * muc_zm * (Wc - Wzm);
    const T sxz_xp = muexz_xp * ((Uxp - Uxp_zm) + (Wxp - Wc));
    const T sxz_0 = muexz * ((Uc - Uzm) + (Wc - Wxm));
    const T visc = (sxz_xp - sxz_0 + szz0 - szz1) * iD2;
    T divt = 0;
    if (have_tau) {
      const T e00 = A.TXZ(0, 0), e0m = A.TXZ(0, -1), ep0 = A.TXZ(1, 0), epm = A.TXZ(1, -1), em0 = A.TXZ(-1, 0),
              emm = A.TXZ(-1, -1);
      const T Txz_xp = (T)0.25 * (e0m + epm + e00 + ep0), Txz_0 = (T)0.25 * (emm + e0m + em0 + e00);
      divt = (Txz_xp - Txz_0 + A.TZZ(0, 0) - A.TZZ(0, -1)) * iD;
    }
    const T st = A.gfz() * (phc - A.PHC(0, -1)) * iD;
    const T gdp = (Dp_c - A.DP(0, -1)) * iD, gps = (Ps_c - A.PS(0, -1)) * iD;
    const T R = A.dw() * q.idt + adv + (jg - divt - visc - st + gps) / rho + gdp * q.irho0 - q.gz;
    rw = R * q.inum;
  }
}

// The inputs of ns_rhs_cell2 read from the fields of step n (arithmetic type
// R; storage type T).
template <class T, class R = T>
struct NsGlobalAcc2 {
  const NsIn<T>* a;
  int nx, nz, i, k;
  __device__ __forceinline__ int x(int dx) const { return wrap(i + dx, nx); }
  __device__ __forceinline__ int zc(int dz) const { return min(max(k + dz, 0), nz - 1) * nx; }
  __device__ __forceinline__ int zf(int dz) const { return (k + dz) * nx; }
  __device__ __forceinline__ R ex(const T* n, const T* o, int o_) const { return (R)((T)2 * n[o_] - o[o_]); }
  __device__ __forceinline__ R U(int dx, int dz) const { return ex(a->un, a->uo, zc(dz) + x(dx)); }
  __device__ __forceinline__ R W(int dx, int dz) const { return ex(a->wn, a->wo, zf(dz) + x(dx)); }
  __device__ __forceinline__ R DP(int dx, int dz) const {
    const int o = zc(dz) + x(dx);
    return (R)(a->po[o] - a->pn[o]);
  }
  __device__ __forceinline__ R PS(int dx, int dz) const { return ex(a->pn, a->po, zc(dz) + x(dx)); }
  __device__ __forceinline__ R PHC(int dx, int dz) const { return (R)a->rs.phic[zc(dz) + x(dx)]; }
  __device__ __forceinline__ R G(int dx, int dz) const { return (R)a->rs.Gc[zc(dz) + x(dx)]; }
  __device__ __forceinline__ R EXZ(int dx, int dz) const { return (R)a->rs.phiexz[zf(dz) + x(dx)]; }
  __device__ __forceinline__ R phifx() const { return (R)a->rs.phifx[k * nx + i]; }
  __device__ __forceinline__ R phifz() const { return (R)a->rs.phifz[k * nx + i]; }
  __device__ __forceinline__ R gfx() const { return (R)a->rs.Gfx[k * nx + i]; }
  __device__ __forceinline__ R gfz() const { return (R)a->rs.Gfz[k * nx + i]; }
  __device__ __forceinline__ R TXX(int dx, int dz) const { return ex(a->tn[0], a->to[0], zc(dz) + x(dx)); }
  __device__ __forceinline__ R TXZ(int dx, int dz) const { return ex(a->tn[1], a->to[1], zc(dz) + x(dx)); }
  __device__ __forceinline__ R TZZ(int dx, int dz) const { return ex(a->tn[2], a->to[2], zc(dz) + x(dx)); }
  __device__ __forceinline__ R du() const { return (R)(a->un[k * nx + i] - a->uo[k * nx + i]); }
  __device__ __forceinline__ R dw() const { return (R)(a->wn[k * nx + i] - a->wo[k * nx + i]); }
};

template <class T, int DIM>
__device__ __forceinline__ void k_ns_rhs_v2_b(const NsIn<T>& a, const Dims d, const PhysT<T> q, T* __restrict__ ru, T* __restrict__ rv, T* __restrict__ rw, const int have_tau, const int3 bid) {
  constexpr bool D3 = DIM == 3;
  RowIdx ix;
  if (!row_index_b(bid, d.nx, d.ny, ix)) return;
  const int i = ix.i, j = ix.j, k = ix.k;
  const int nx = d.nx, ny = d.ny, nz = d.nz;
  const int P = nx * ny;
  if constexpr (!D3) {
    const NsGlobalAcc2<T> acc{&a, nx, nz, i, k};
    T oru = 0, orw = 0;
    ns_rhs_cell2<T>(acc, q, k, nz, have_tau, oru, orw);
    ru[k * nx + i] = oru;
    if (k > 0) rw[(k - 1) * nx + i] = orw;  // face rows 0..nz-2 hold faces 1..nz-1
    return;
  }
  // 32-bit neighbour offsets (fields are smaller than 2^31 elements)
  const int x0 = i, xm = i == 0 ? nx - 1 : i - 1, xp = i == nx - 1 ? 0 : i + 1;
  const int r0 = j * nx;
  const int rm = D3 ? (j == 0 ? ny - 1 : j - 1) * nx : r0;
  const int rp = D3 ? (j == ny - 1 ? 0 : j + 1) * nx : r0;
  const int z0 = k * P;
  const bool hasb = k > 0, hast = k < nz - 1;
  const int zm = hasb ? z0 - P : z0, zp = hast ? z0 + P : z0;
  const int zpw = z0 + P;  // face k+1 of a face field (always exists, k+1 <= nz)
  const int c = z0 + r0 + x0;
  const T iD = q.iD, iD2 = q.iD2, h = (T)0.5;
  // extrapolations u* = 2u^n - u^{n-1}
  auto S = [](const T* n, const T* o, int off) { return (T)2 * n[off] - o[off]; };
  // ---- u* ----
  const T Uc = S(a.un, a.uo, c), Uxp = S(a.un, a.uo, z0 + r0 + xp), Uxm = S(a.un, a.uo, z0 + r0 + xm);
  const T Uzp = hast ? S(a.un, a.uo, zp + r0 + x0) : q.uw2_top - Uc;
  const T Uzm = hasb ? S(a.un, a.uo, zm + r0 + x0) : q.uw2_bot - Uc;
  const T Uxp_zm = hasb ? S(a.un, a.uo, zm + r0 + xp) : (T)0;
  // ---- w* (faces) ----
  const T Wc = S(a.wn, a.wo, c), Wzp = S(a.wn, a.wo, zpw + r0 + x0);
  const T Wxm = S(a.wn, a.wo, z0 + r0 + xm), Wxp = S(a.wn, a.wo, z0 + r0 + xp);
  const T Wxm_zp = S(a.wn, a.wo, zpw + r0 + xm);
  const T Wzm = hasb ? S(a.wn, a.wo, zm + r0 + x0) : (T)0;
  // ---- pressure ----
  // The pressure split (1/rho0) grad p^n + (1/rho - 1/rho0) grad p* is formed
  // as (1/rho0) grad(p^{n-1} - p^n) + (1/rho) grad p* (p^n - p* = p^{n-1} - p^n):
  // the same value, without cancelling two terms of size 1/rho0 (1000x the
  // result at density ratio 1000) in the working precision.
  const T Dp_c = a.po[c] - a.pn[c], Ps_c = S(a.pn, a.po, c);
  // ---- restricted fields ----
  const T phc = a.rs.phic[c], phc_xm = a.rs.phic[z0 + r0 + xm];
  const T Gc_c = a.rs.Gc[c], Gc_xm = a.rs.Gc[z0 + r0 + xm], Gc_xp = a.rs.Gc[z0 + r0 + xp];
  auto mu_of = [&](T ph) { return h * ((T)1 + ph) * q.mu_s1 + h * ((T)1 - ph) * q.mu_s2; };
  auto rho_of = [&](T ph) { return h * ((T)1 + ph) * q.rho1 + h * ((T)1 - ph) * q.rho2; };
  const T muc = mu_of(phc), muc_xm = mu_of(phc_xm);
  const T muexz = mu_of(a.rs.phiexz[c]), muexz_zp = mu_of(a.rs.phiexz[zpw + r0 + x0]);
  const T muexz_xp = mu_of(a.rs.phiexz[z0 + r0 + xp]);
  const T cj = q.cj_dx;
  // J at faces
  const T Jx_c = cj * (Gc_c - Gc_xm);
  const T Gc_zp = hast ? a.rs.Gc[zp + r0 + x0] : (T)0, Gc_xm_zp = hast ? a.rs.Gc[zp + r0 + xm] : (T)0;
  const T Gc_zm = hasb ? a.rs.Gc[zm + r0 + x0] : (T)0, Gc_xm_zm = hasb ? a.rs.Gc[zm + r0 + xm] : (T)0;
  const T Jz_c = hasb ? cj * (Gc_c - Gc_zm) : (T)0;
  const T Jz_xm = hasb ? cj * (Gc_xm - Gc_xm_zm) : (T)0;
  const T Jz_zp = hast ? cj * (Gc_zp - Gc_c) : (T)0;
  const T Jz_xm_zp = hast ? cj * (Gc_xm_zp - Gc_xm) : (T)0;
  // ================= x momentum at the u-face (i, j, k) =================
  {
    const T rho = rho_of(a.rs.phifx[c]);
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
      constexpr int XX = 0, XZ = D3 ? 4 : 1;
      auto tau = [&](int comp, int off) { return S(a.tn[comp], a.to[comp], off); };
      const T tzc = tau(XZ, c), tzxm = tau(XZ, z0 + r0 + xm);
      const T tzzp = tau(XZ, zp + r0 + x0), tzxmzp = tau(XZ, zp + r0 + xm);  // mirror: zp == z0 at top
      const T tzzm = tau(XZ, zm + r0 + x0), tzxmzm = tau(XZ, zm + r0 + xm);  // mirror: zm == z0 at bottom
      const T Txz_p = (T)0.25 * (tzxm + tzc + tzxmzp + tzzp);
      const T Txz_0 = (T)0.25 * (tzxmzm + tzzm + tzxm + tzc);
      divt = (tau(XX, c) - tau(XX, z0 + r0 + xm) + Txz_p - Txz_0) * iD;
      if constexpr (D3) {
        constexpr int XY = 3;
        const T t00 = tau(XY, c), t0m = tau(XY, z0 + r0 + xm), tp0 = tau(XY, z0 + rp + x0),
                tpm = tau(XY, z0 + rp + xm), tm0 = tau(XY, z0 + rm + x0), tmm = tau(XY, z0 + rm + xm);
        divt += ((T)0.25 * (t0m + t00 + tpm + tp0) - (T)0.25 * (tmm + tm0 + t0m + t00)) * iD;
      }
    }
    if constexpr (D3) {
      const T Uyp = S(a.un, a.uo, z0 + rp + x0), Uym = S(a.un, a.uo, z0 + rm + x0);
      const T Vc = S(a.vn, a.vo, c), Vxm = S(a.vn, a.vo, z0 + r0 + xm);
      const T Vyp = S(a.vn, a.vo, z0 + rp + x0), Vxm_yp = S(a.vn, a.vo, z0 + rp + xm);
      const T Exy_p = (T)0.25 * (Uc + Uyp) * (Vxm_yp + Vyp);
      const T Exy_0 = (T)0.25 * (Uym + Uc) * (Vxm + Vc);
      adv += (Exy_p - Exy_0) * iD;
      const T Gc_yp = a.rs.Gc[z0 + rp + x0], Gc_ym = a.rs.Gc[z0 + rm + x0];
      const T Gc_xm_yp = a.rs.Gc[z0 + rp + xm], Gc_xm_ym = a.rs.Gc[z0 + rm + xm];
      const T Jy_c = cj * (Gc_c - Gc_ym), Jy_xm = cj * (Gc_xm - Gc_xm_ym);
      const T Jy_yp = cj * (Gc_yp - Gc_c), Jy_xm_yp = cj * (Gc_xm_yp - Gc_xm);
      const T Jyu = (T)0.25 * (Jy_xm + Jy_c + Jy_xm_yp + Jy_yp);
      jg += Jyu * (Uyp - Uym) * h * iD;
      const T muexy = mu_of(a.rs.phiexy[c]), muexy_yp = mu_of(a.rs.phiexy[z0 + rp + x0]);
      const T sxy_p = muexy_yp * ((Uyp - Uc) + (Vyp - Vxm_yp));
      const T sxy_0 = muexy * ((Uc - Uym) + (Vc - Vxm));
      visc += (sxy_p - sxy_0) * iD2;
    }
    const T st = a.rs.Gfx[c] * (phc - phc_xm) * iD;
    const T gdp = (Dp_c - (a.po[z0 + r0 + xm] - a.pn[z0 + r0 + xm])) * iD, gps = (Ps_c - S(a.pn, a.po, z0 + r0 + xm)) * iD;
    const T R = (a.un[c] - a.uo[c]) * q.idt + adv + (jg - divt - visc - st + gps) / rho + gdp * q.irho0 - q.gx;
    ru[c] = R * q.inum;
  }
  // ================= y momentum at the v-face (i, j, k), 3D =================
  if constexpr (D3) {
    const T Vc = S(a.vn, a.vo, c), Vxp = S(a.vn, a.vo, z0 + r0 + xp), Vxm = S(a.vn, a.vo, z0 + r0 + xm);
    const T Vyp = S(a.vn, a.vo, z0 + rp + x0), Vym = S(a.vn, a.vo, z0 + rm + x0);
    const T Vzp = hast ? S(a.vn, a.vo, zp + r0 + x0) : -Vc;
    const T Vzm = hasb ? S(a.vn, a.vo, zm + r0 + x0) : -Vc;
    const T Uym = S(a.un, a.uo, z0 + rm + x0), Uxp_ym = S(a.un, a.uo, z0 + rm + xp);
    const T Wym = S(a.wn, a.wo, z0 + rm + x0), Wym_zp = S(a.wn, a.wo, zpw + rm + x0);
    const T rho = rho_of(a.rs.phify[c]);
    const T cyy0 = (T)0.25 * (Vc + Vyp) * (Vc + Vyp), cyy1 = (T)0.25 * (Vym + Vc) * (Vym + Vc);
    const T Exy_xp = (T)0.25 * (Uxp_ym + Uxp) * (Vc + Vxp);
    const T Exy_0 = (T)0.25 * (Uym + Uc) * (Vxm + Vc);
    const T Eyz_p = (T)0.25 * (Vc + Vzp) * (Wym_zp + Wzp);
    const T Eyz_0 = (T)0.25 * (Vzm + Vc) * (Wym + Wc);
    const T adv = (cyy0 - cyy1 + Exy_xp - Exy_0 + Eyz_p - Eyz_0) * iD;
    const T Gc_ym = a.rs.Gc[z0 + rm + x0], Gc_xp_ym = a.rs.Gc[z0 + rm + xp], Gc_xm_ym = a.rs.Gc[z0 + rm + xm];
    const T Jx_ym = cj * (Gc_ym - Gc_xm_ym), Jx_xp_ym = cj * (Gc_xp_ym - Gc_ym), Jx_xp = cj * (Gc_xp - Gc_c);
    const T Jxv = (T)0.25 * (Jx_ym + Jx_xp_ym + Jx_c + Jx_xp);
    const T Jy_c = cj * (Gc_c - Gc_ym);
    const T Gc_ym_zm = hasb ? a.rs.Gc[zm + rm + x0] : (T)0, Gc_ym_zp = hast ? a.rs.Gc[zp + rm + x0] : (T)0;
    const T Jz_ym = hasb ? cj * (Gc_ym - Gc_ym_zm) : (T)0;
    const T Jz_ym_zp = hast ? cj * (Gc_ym_zp - Gc_ym) : (T)0;
    const T Jzv = (T)0.25 * (Jz_ym + Jz_c + Jz_ym_zp + Jz_zp);
    const T jg = (Jxv * (Vxp - Vxm) + Jy_c * (Vyp - Vym) + Jzv * (Vzp - Vzm)) * h * iD;
    const T muc_ym = mu_of(a.rs.phic[z0 + rm + x0]);
    const T syy0 = 2 * muc * (Vyp - Vc), syy1 = 2 * muc_ym * (Vc - Vym);
    const T muexy = mu_of(a.rs.phiexy[c]), muexy_xp = mu_of(a.rs.phiexy[z0 + r0 + xp]);
    const T sxy_xp = muexy_xp * ((Uxp - Uxp_ym) + (Vxp - Vc));
    const T sxy_0 = muexy * ((Uc - Uym) + (Vc - Vxm));
    const T mueyz = mu_of(a.rs.phieyz[c]), mueyz_zp = mu_of(a.rs.phieyz[zpw + r0 + x0]);
    const T syz_p = mueyz_zp * ((Vzp - Vc) + (Wzp - Wym_zp));
    const T syz_0 = mueyz * ((Vc - Vzm) + (Wc - Wym));
    const T visc = (syy0 - syy1 + sxy_xp - sxy_0 + syz_p - syz_0) * iD2;
    T divt = 0;
    if (have_tau) {
      constexpr int YY = 1, XY = 3, YZ = 5;
      auto tau = [&](int comp, int off) { return S(a.tn[comp], a.to[comp], off); };
      const T a00 = tau(XY, c), a0m = tau(XY, z0 + rm + x0), ap0 = tau(XY, z0 + r0 + xp), apm = tau(XY, z0 + rm + xp),
              am0 = tau(XY, z0 + r0 + xm), amm = tau(XY, z0 + rm + xm);
      const T Txy_xp = (T)0.25 * (a0m + apm + a00 + ap0), Txy_0 = (T)0.25 * (amm + a0m + am0 + a00);
      const T b00 = tau(YZ, c), bm0 = tau(YZ, z0 + rm + x0), b0p = tau(YZ, zp + r0 + x0), bmp = tau(YZ, zp + rm + x0),
              b0m = tau(YZ, zm + r0 + x0), bmm = tau(YZ, zm + rm + x0);
      const T Tyz_p = (T)0.25 * (bm0 + b00 + bmp + b0p), Tyz_0 = (T)0.25 * (bmm + b0m + bm0 + b00);
      divt = (tau(YY, c) - tau(YY, z0 + rm + x0) + Txy_xp - Txy_0 + Tyz_p - Tyz_0) * iD;
    }
    const T st = a.rs.Gfy[c] * (phc - a.rs.phic[z0 + rm + x0]) * iD;
    const T gdp = (Dp_c - (a.po[z0 + rm + x0] - a.pn[z0 + rm + x0])) * iD, gps = (Ps_c - S(a.pn, a.po, z0 + rm + x0)) * iD;
    const T R = (a.vn[c] - a.vo[c]) * q.idt + adv + (jg - divt - visc - st + gps) / rho + gdp * q.irho0 - q.gy;
    rv[c] = R * q.inum;
  }
  // ================= z momentum at the w-face k (interior faces 1..nz-1) =================
  if (hasb) {
    const T rho = rho_of(a.rs.phifz[c]);
    const T Uzm_r = Uzm;  // real neighbour (k >= 1)
    const T Exz_xp = (T)0.25 * (Uxp_zm + Uxp) * (Wc + Wxp);
    const T Exz_0 = (T)0.25 * (Uzm_r + Uc) * (Wxm + Wc);
    const T czz0 = (T)0.25 * (Wc + Wzp) * (Wc + Wzp), czz1 = (T)0.25 * (Wzm + Wc) * (Wzm + Wc);
    T adv = (Exz_xp - Exz_0 + czz0 - czz1) * iD;
    const T Gc_xp_zm = a.rs.Gc[zm + r0 + xp];
    const T Jx_zm = cj * (Gc_zm - Gc_xm_zm), Jx_xp_zm = cj * (Gc_xp_zm - Gc_zm), Jx_xp = cj * (Gc_xp - Gc_c);
    const T Jxw = (T)0.25 * (Jx_zm + Jx_xp_zm + Jx_c + Jx_xp);
    T jg = (Jxw * (Wxp - Wxm) + Jz_c * (Wzp - Wzm)) * h * iD;
    const T muc_zm = mu_of(a.rs.phic[zm + r0 + x0]);
    const T szz0 = 2 * muc * (Wzp - Wc), szz1 = 2 * muc_zm * (Wc - Wzm);
    const T sxz_xp = muexz_xp * ((Uxp - Uxp_zm) + (Wxp - Wc));
    const T sxz_0 = muexz * ((Uc - Uzm_r) + (Wc - Wxm));
    T visc = (sxz_xp - sxz_0 + szz0 - szz1) * iD2;
    T divt = 0;
    if (have_tau) {
      constexpr int ZZ = 2, XZ = D3 ? 4 : 1;
      auto tau = [&](int comp, int off) { return S(a.tn[comp], a.to[comp], off); };
      const T e00 = tau(XZ, c), e0m = tau(XZ, zm + r0 + x0), ep0 = tau(XZ, z0 + r0 + xp), epm = tau(XZ, zm + r0 + xp),
              em0 = tau(XZ, z0 + r0 + xm), emm = tau(XZ, zm + r0 + xm);
      const T Txz_xp = (T)0.25 * (e0m + epm + e00 + ep0), Txz_0 = (T)0.25 * (emm + e0m + em0 + e00);
      divt = (Txz_xp - Txz_0 + tau(ZZ, c) - tau(ZZ, zm + r0 + x0)) * iD;
      if constexpr (D3) {
        constexpr int YZ = 5;
        const T f00 = tau(YZ, c), f0m = tau(YZ, zm + r0 + x0), fp0 = tau(YZ, z0 + rp + x0), fpm = tau(YZ, zm + rp + x0),
                fm0 = tau(YZ, z0 + rm + x0), fmm = tau(YZ, zm + rm + x0);
        divt += ((T)0.25 * (f0m + fpm + f00 + fp0) - (T)0.25 * (fmm + f0m + fm0 + f00)) * iD;
      }
    }
    if constexpr (D3) {
      const T Vc = S(a.vn, a.vo, c), Vyp = S(a.vn, a.vo, z0 + rp + x0);
      const T Vzm = S(a.vn, a.vo, zm + r0 + x0), Vyp_zm = S(a.vn, a.vo, zm + rp + x0);
      const T Wyp = S(a.wn, a.wo, z0 + rp + x0), Wym = S(a.wn, a.wo, z0 + rm + x0);
      const T Eyz_yp = (T)0.25 * (Vyp_zm + Vyp) * (Wc + Wyp);
      const T Eyz_0 = (T)0.25 * (Vzm + Vc) * (Wym + Wc);
      adv += (Eyz_yp - Eyz_0) * iD;
      const T Gc_ym = a.rs.Gc[z0 + rm + x0], Gc_yp = a.rs.Gc[z0 + rp + x0];
      const T Gc_ym_zm = a.rs.Gc[zm + rm + x0], Gc_yp_zm = a.rs.Gc[zm + rp + x0];
      const T Jy_zm = cj * (Gc_zm - Gc_ym_zm), Jy_yp_zm = cj * (Gc_yp_zm - Gc_zm);
      const T Jy_c = cj * (Gc_c - Gc_ym), Jy_yp = cj * (Gc_yp - Gc_c);
      const T Jyw = (T)0.25 * (Jy_zm + Jy_yp_zm + Jy_c + Jy_yp);
      jg += Jyw * (Wyp - Wym) * h * iD;
      const T mueyz = mu_of(a.rs.phieyz[c]), mueyz_yp = mu_of(a.rs.phieyz[z0 + rp + x0]);
      const T syz_yp = mueyz_yp * ((Vyp - Vyp_zm) + (Wyp - Wc));
      const T syz_0 = mueyz * ((Vc - Vzm) + (Wc - Wym));
      visc += (syz_yp - syz_0) * iD2;
    }
    const T st = a.rs.Gfz[c] * (phc - a.rs.phic[zm + r0 + x0]) * iD;
    const T gdp = (Dp_c - (a.po[zm + r0 + x0] - a.pn[zm + r0 + x0])) * iD, gps = (Ps_c - S(a.pn, a.po, zm + r0 + x0)) * iD;
    const T R = (a.wn[c] - a.wo[c]) * q.idt + adv + (jg - divt - visc - st + gps) / rho + gdp * q.irho0 - q.gz;
    rw[c - P] = R * q.inum;  // face rows 0..nz-2 hold faces 1..nz-1
  }
}


// Each CTA walks kz consecutive z rows at one (j) (kz = 1: one row per CTA):
// the rows it has just read are the z neighbours of the next, so they come
// from L1.  Every kz runs the same compiled loop body, so the result does not
// depend on kz.  MINB: CTAs of 256 threads per SM the register budget is sized for.
template <class T, int DIM, int MINB>
__global__ void __launch_bounds__(256, MINB) k_ns_rhs_v2z(const __grid_constant__ NsIn<T> a, const Dims d,
                                                          const PhysT<T> q, T* __restrict__ ru, T* __restrict__ rv,
                                                          T* __restrict__ rw, const int have_tau, const int kz) {
  const int j = blockIdx.x % d.ny, kc = blockIdx.x / d.ny;
  for (int kk = 0; kk < kz; ++kk) {
    const int k = kc * kz + kk;
    if (k >= d.nz) break;
    k_ns_rhs_v2_b<T, DIM>(a, d, q, ru, rv, rw, have_tau, make_int3(k * d.ny + j, blockIdx.y, 0));
  }
}

}  // namespace pf
