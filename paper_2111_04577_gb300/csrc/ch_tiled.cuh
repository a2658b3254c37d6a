// Shared-memory tiled Cahn-Hilliard stencils (fine mesh).
//
// k_ch_rhs: one pass from (phi^n, phi^{n-1}, coarse u^n, u^{n-1}) to the
//   increment-form right side R of the Psi solve (see ch.cuh):
//     phi* = 2 phi^n - phi^{n-1}                       (Eq. NS32)
//     mu*  = f(phi*) - (L_N phi* + B(g))               (Eqs. NS6, NS34)
//     R    = (phi^{n-1} - phi^n)/(M lambda dt) - div(u* phi*)/(M lambda) + L_N mu*
//   A CTA owns a TX x TY x TZ block of fine cells: phi* is staged with a halo of
//   2 cells, mu* is formed in shared memory on the block plus one cell, and R
//   on the block, so mu* never goes to HBM.  g, the contact-angle flux of the
//   wall columns, is evaluated in FP64 and stored for the chemical potential.
// k_ch_G_restrict: from phi^{n+1} (and g) to the chemical potential
//   G = lambda(-(L_N phi + B(g)) + f(phi)) (Eq. NS5) on a fine block with a
//   one-cell halo in shared memory, then every coarse sample of phi and G that
//   Eqs. dual2/dual3 need (centres, faces, edges), without writing fine G.
#pragma once
#include <type_traits>

#include "ch.cuh"

namespace pf {

__device__ __forceinline__ int pmod(int x, int n) {
  x %= n;
  return x < 0 ? x + n : x;
}
__device__ __forceinline__ int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

// wrap into [0, n) for -n <= x < 2n
__device__ __forceinline__ int wrap1(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

template <int DIM, int ES>
struct RhsTile {
  // ES: element size; FP64 tiles are half as deep to stay within shared memory
  static constexpr int TX = 64, TY = DIM == 3 ? 8 : 1, TZ = DIM == 3 ? (ES == 8 ? 4 : 8) : 16;
  static constexpr int HY = DIM == 3 ? 2 : 0;
  static constexpr int SX = TX + 4, SY = TY + 2 * HY, SZ = TZ + 4;
  static constexpr int MX = TX + 2, MY = TY + (DIM == 3 ? 2 : 0), MZ = TZ + 2;
  static constexpr int NS = SX * SY * SZ, NM = MX * MY * MZ;
  // coarse velocity box: x, y with one cell of halo on each side, z with one extra face
  __host__ __device__ static constexpr int VX(int rs) { return (TX >> rs) + 2; }
  __host__ __device__ static constexpr int VY(int rys) { return DIM == 3 ? (TY >> rys) + 2 : 1; }
  __host__ __device__ static constexpr int VZ(int rs) { return (TZ >> rs) + 1; }
  __host__ __device__ static constexpr int NV(int rs, int rys) { return VX(rs) * VY(rys) * VZ(rs); }
};

template <class T, int DIM>
__device__ __forceinline__ void k_ch_rhs_b(const FineView<T> f, const CoarseVel<T> vel, T* __restrict__ R, Wide<T>* __restrict__ gwall, const Dims d, const Phys p, const PhysT<T> q, const T inv_mldt, const T inv_ml, const int3 bid, unsigned char* smraw) {
  using TL = RhsTile<DIM, sizeof(T)>;
  T* ps = reinterpret_cast<T*>(smraw);  // phi*, [SZ][SY][SX]
  T* ms = ps + TL::NS;                  // mu*,  [MZ][MY][MX]
  const int VX = TL::VX(d.rs), VY = TL::VY(d.rys), VZ = TL::VZ(d.rs), NV = VX * VY * VZ;
  T* us = ms + TL::NM;                  // u*, v*, w* on the coarse box [VZ][VY][VX]
  T* vs = us + NV;
  T* wsm = vs + NV;
  const int x0 = bid.x * TL::TX, y0 = bid.y * TL::TY, z0 = bid.z * TL::TZ;
  const int fnx = d.fnx, fny = d.fny, fnz = d.fnz;
  const size_t plane = (size_t)fnx * fny;
  const bool smallx = fnx < TL::SX, smally = fny < TL::SY;  // tile wider than the domain
  // ---- stage phi* with a 2-cell halo (x, y periodic; z clamped, never read past a wall) ----
  {
    const float isx = 1.0f / TL::SX, isy = 1.0f / TL::SY;
    for (int e = threadIdx.x; e < TL::NS; e += blockDim.x) {
      const int zz = qdiv(e, TL::SX * TL::SY, isx * isy);
      const int rem = e - zz * TL::SX * TL::SY;
      const int yy = qdiv(rem, TL::SX, isx), xx = rem - yy * TL::SX;
      const int gx = smallx ? pmod(x0 - 2 + xx, fnx) : wrap1(x0 - 2 + xx, fnx);
      const int gy = DIM == 3 ? (smally ? pmod(y0 - TL::HY + yy, fny) : wrap1(y0 - TL::HY + yy, fny)) : 0;
      const int gz = clampi(z0 - 2 + zz, 0, fnz - 1);
      const size_t o = (size_t)gz * plane + (size_t)gy * fnx + gx;
      ps[e] = (T)2 * f.pn[o] - f.po[o];
    }
  }
  // ---- stage the extrapolated coarse velocities of the block (Eq. dual1 reads them) ----
  const int cx0 = (x0 >> d.rs) - 1, cy0 = DIM == 3 ? (y0 >> d.rys) - 1 : 0, cz0 = z0 >> d.rs;
  {
    const float ivx = 1.0f / VX, ivy = 1.0f / VY;
    const int cplane = d.nx * d.ny;
    for (int e = threadIdx.x; e < NV; e += blockDim.x) {
      const int zz = qdiv(e, VX * VY, ivx * ivy);
      const int rem = e - zz * VX * VY;
      const int yy = qdiv(rem, VX, ivx), xx = rem - yy * VX;
      const int cx = pmod(cx0 + xx, d.nx);
      const int cy = DIM == 3 ? pmod(cy0 + yy, d.ny) : 0;
      const int cz = cz0 + zz;
      const int czc = cz < d.nz ? cz : d.nz - 1;  // u, v live on cells (the extra layer is unused)
      const int czw = cz <= d.nz ? cz : d.nz;     // w on faces 0..nz
      const int oc = czc * cplane + cy * d.nx + cx, ow = czw * cplane + cy * d.nx + cx;
      us[e] = vel.us(oc);
      vs[e] = DIM == 3 ? vel.vs(oc) : (T)0;
      wsm[e] = vel.ws(ow);
    }
  }
  __syncthreads();
  // prolonged face velocities (Eq. dual1) from the staged coarse box
  auto V = [&](const T* a, int cx, int cy, int cz) -> T { return a[((cz - cz0) * VY + (cy - cy0)) * VX + (cx - cx0)]; };
  auto uface = [&](int I, int J, int K) -> T {  // fine x-face I (may be fnx: periodic image)
    const int ic = I >> d.rs, jc = DIM == 3 ? J >> d.rys : 0, kc = K >> d.rs;
    const T a = V(us, ic, jc, kc);
    return (I & (d.r - 1)) == 0 ? a : (T)0.5 * (a + V(us, ic + 1, jc, kc));
  };
  auto vface = [&](int I, int J, int K) -> T {
    const int ic = I >> d.rs, jc = J >> d.rys, kc = K >> d.rs;
    const T a = V(vs, ic, jc, kc);
    return (J & (d.ry - 1)) == 0 ? a : (T)0.5 * (a + V(vs, ic, jc + 1, kc));
  };
  auto wface = [&](int I, int J, int K) -> T {
    const int ic = I >> d.rs, jc = DIM == 3 ? J >> d.rys : 0, kc = K >> d.rs;
    const T a = V(wsm, ic, jc, kc);
    return (K & (d.r - 1)) == 0 ? a : (T)0.5 * (a + V(wsm, ic, jc, kc + 1));
  };
  auto P = [&](int sz, int sy, int sx) -> T { return ps[(sz * TL::SY + sy) * TL::SX + sx]; };
  // ---- mu* on the block plus one cell ----
  {
    const float imx = 1.0f / TL::MX, imy = 1.0f / TL::MY;
    for (int e = threadIdx.x; e < TL::NM; e += blockDim.x) {
      const int mz = qdiv(e, TL::MX * TL::MY, imx * imy);
      const int rem = e - mz * TL::MX * TL::MY;
      const int my = qdiv(rem, TL::MX, imx), mx = rem - my * TL::MX;
      const int gz = z0 - 1 + mz;
      if (gz < 0 || gz >= fnz) {
        ms[e] = (T)0;
        continue;
      }
      const int sx = mx + 1, sy = my + (DIM == 3 ? 1 : 0), sz = mz + 1;
      const T c0 = P(sz, sy, sx);
      T lap = P(sz, sy, sx + 1) + P(sz, sy, sx - 1) - 2 * c0;
      if (DIM == 3) lap += P(sz, sy + 1, sx) + P(sz, sy - 1, sx) - 2 * c0;
      const T czp = gz + 1 < fnz ? P(sz + 1, sy, sx) : c0;
      const T czm = gz > 0 ? P(sz - 1, sy, sx) : c0;
      lap = (lap + czp + czm - 2 * c0) * q.ih2;
      T B = 0;
      const bool own = mx >= 1 && mx <= TL::TX && (DIM == 2 || (my >= 1 && my <= TL::TY));
      const int gx = x0 - 1 + mx, gy = DIM == 3 ? y0 - 1 + my : 0;
      if (gz == 0) {
        const Wide<T> g = wall_g(q.gbot, (Wide<T>)c0, (Wide<T>)czp);
        if (own && gx < fnx && gy < fny) gwall[(size_t)gy * fnx + gx] = g;
        B += (T)(g * q.ihw);
      }
      if (gz == fnz - 1) {
        const Wide<T> g = wall_g(q.gtop, (Wide<T>)c0, (Wide<T>)czm);
        if (own && gx < fnx && gy < fny) gwall[plane + (size_t)gy * fnx + gx] = g;
        B += (T)(g * q.ihw);
      }
      ms[e] = c0 * (c0 * c0 - 1) * q.ie2 - (lap + B);
    }
  }
  __syncthreads();
  auto M = [&](int mz, int my, int mx) -> T { return ms[(mz * TL::MY + my) * TL::MX + mx]; };
  // ---- R on the block ----
  const float itx = 1.0f / TL::TX, ity = 1.0f / TL::TY;
  for (int e = threadIdx.x; e < TL::TX * TL::TY * TL::TZ; e += blockDim.x) {
    const int tz = qdiv(e, TL::TX * TL::TY, itx * ity);
    const int rem = e - tz * TL::TX * TL::TY;
    const int ty = qdiv(rem, TL::TX, itx), tx = rem - ty * TL::TX;
    const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
    if (gx >= fnx || gy >= fny || gz >= fnz) continue;
    const int sx = tx + 2, sy = ty + TL::HY, sz = tz + 2;
    const T c0 = P(sz, sy, sx);
    // faces are addressed by unwrapped fine indices: the staged box holds the periodic images
    T adv = uface(gx + 1, gy, gz) * (c0 + P(sz, sy, sx + 1)) - uface(gx, gy, gz) * (P(sz, sy, sx - 1) + c0);
    if (DIM == 3) adv += vface(gx, gy + 1, gz) * (c0 + P(sz, sy + 1, sx)) - vface(gx, gy, gz) * (P(sz, sy - 1, sx) + c0);
    if (gz + 1 < fnz) adv += wface(gx, gy, gz + 1) * (c0 + P(sz + 1, sy, sx));
    if (gz > 0) adv -= wface(gx, gy, gz) * (P(sz - 1, sy, sx) + c0);
    adv *= (T)0.5 * q.ih;
    const size_t o = (size_t)gz * plane + (size_t)gy * fnx + gx;
    if (f.aw) adv = f.aw[o];
    const int mx = tx + 1, my = ty + (DIM == 3 ? 1 : 0), mz = tz + 1;
    const T m0 = M(mz, my, mx);
    T lap = M(mz, my, mx + 1) + M(mz, my, mx - 1) - 2 * m0;
    if (DIM == 3) lap += M(mz, my + 1, mx) + M(mz, my - 1, mx) - 2 * m0;
    const T mzp = gz + 1 < fnz ? M(mz + 1, my, mx) : m0;
    const T mzm = gz > 0 ? M(mz - 1, my, mx) : m0;
    lap = (lap + mzp + mzm - 2 * m0) * q.ih2;
    R[o] = f.back(o, f.pn[o], f.po[o]) * inv_mldt - adv * inv_ml + lap;
  }
}

template <class T, int DIM>
__global__ void __launch_bounds__(256) k_ch_rhs(const FineView<T> f, const CoarseVel<T> vel, T* __restrict__ R, Wide<T>* __restrict__ gwall, const Dims d, const Phys p, const PhysT<T> q, const T inv_mldt, const T inv_ml) {
  extern __shared__ __align__(16) unsigned char smraw[];
  k_ch_rhs_b<T, DIM>(f, vel, R, gwall, d, p, q, inv_mldt, inv_ml, make_int3(blockIdx.x, blockIdx.y, blockIdx.z), smraw);
}

// ---------------------------------------------------------------------------
template <int DIM>
struct GrTile {
  // coarse block; the fine block is r times larger plus a halo
  static constexpr int CX = DIM == 3 ? 16 : 64, CY = DIM == 3 ? 4 : 1, CZ = 4;
  // fine G block [GZ][GY][GX] starting one fine cell before the coarse block
  // (the extra top layer serves the z-face at the top wall), phi block one
  // more cell each side
  __host__ __device__ static constexpr int GX(int r) { return r * CX + 1; }
  __host__ __device__ static constexpr int GY(int ry) { return DIM == 3 ? ry * CY + 1 : 1; }
  __host__ __device__ static constexpr int GZ(int r) { return r * CZ + 2; }
  __host__ __device__ static constexpr int PX(int r) { return GX(r) + 2; }
  __host__ __device__ static constexpr int PY(int ry) { return DIM == 3 ? GY(ry) + 2 : 1; }
  __host__ __device__ static constexpr int PZ(int r) { return GZ(r) + 2; }
  __host__ __device__ static constexpr int smem_elems(int r, int ry) {
    return PX(r) * PY(ry) * PZ(r) + GX(r) * GY(ry) * GZ(r);
  }
};

template <class T, int DIM, int R>
__device__ __forceinline__ void k_ch_G_restrict_b(const T* __restrict__ phi, const Wide<T>* __restrict__ gwall, Restricted<T> out, const Dims d, const PhysT<T> q, const int3 bid, unsigned char* smraw) {
  using TL = GrTile<DIM>;
  constexpr int RY = DIM == 3 ? R : 1;
  constexpr int GX = TL::GX(R), GY = TL::GY(RY), GZ = TL::GZ(R);
  constexpr int PX = TL::PX(R), PY = TL::PY(RY), PZ = TL::PZ(R);
  constexpr int HY = DIM == 3 ? 1 : 0;
  T* ph = reinterpret_cast<T*>(smraw);  // [PZ][PY][PX], z clamped at the walls (mirror ghosts)
  T* gs = ph + PX * PY * PZ;            // [GZ][GY][GX], G of the (mirrored) sample
  const int cx0 = bid.x * TL::CX, cy0 = bid.y * TL::CY, cz0 = bid.z * TL::CZ;
  const int fnx = d.fnx, fny = d.fny, fnz = d.fnz;
  const size_t plane = (size_t)fnx * fny;
  const int fx0 = R * cx0 - 1, fy0 = DIM == 3 ? RY * cy0 - 1 : 0, fz0 = R * cz0 - 1;  // G-block origin
  const bool smallx = fnx < PX, smally = fny < PY;
  {
    const float ipx = 1.0f / PX, ipy = 1.0f / PY;
    for (int e = threadIdx.x; e < PX * PY * PZ; e += blockDim.x) {
      const int zz = qdiv(e, PX * PY, ipx * ipy);
      const int rem = e - zz * PX * PY;
      const int yy = qdiv(rem, PX, ipx), xx = rem - yy * PX;
      const int gx = smallx ? pmod(fx0 - 1 + xx, fnx) : wrap1(fx0 - 1 + xx, fnx);
      const int gy = DIM == 3 ? (smally ? pmod(fy0 - 1 + yy, fny) : wrap1(fy0 - 1 + yy, fny)) : 0;
      const int gz = clampi(fz0 - 1 + zz, 0, fnz - 1);
      ph[e] = phi[(size_t)gz * plane + (size_t)gy * fnx + gx];
    }
  }
  __syncthreads();
  auto PH = [&](int z, int y, int x) -> T { return ph[(z * PY + y) * PX + x]; };
  {
    const float igx = 1.0f / GX, igy = 1.0f / GY;
    for (int e = threadIdx.x; e < GX * GY * GZ; e += blockDim.x) {
      const int gzl = qdiv(e, GX * GY, igx * igy);
      const int rem = e - gzl * GX * GY;
      const int gyl = qdiv(rem, GX, igx), gxl = rem - gyl * GX;
      const int gz = clampi(fz0 + gzl, 0, fnz - 1);  // the real cell this sample stands for
      const int pz = gz - (fz0 - 1), py = gyl + HY, px = gxl + 1;
      const T c0 = PH(pz, py, px);
      T lap = PH(pz, py, px + 1) + PH(pz, py, px - 1) - 2 * c0;
      if (DIM == 3) lap += PH(pz, py + 1, px) + PH(pz, py - 1, px) - 2 * c0;
      const T czp = gz + 1 < fnz ? PH(pz + 1, py, px) : c0;
      const T czm = gz > 0 ? PH(pz - 1, py, px) : c0;
      lap = (lap + czp + czm - 2 * c0) * q.ih2;
      T B = 0;
      if (gz == 0 || gz == fnz - 1) {
        const int gx = pmod(fx0 + gxl, fnx), gy = DIM == 3 ? pmod(fy0 + gyl, fny) : 0;
        const size_t col = (size_t)gy * fnx + gx;
        if (gz == 0) B += (T)gwall[col] * q.ih;
        if (gz == fnz - 1) B += (T)gwall[plane + col] * q.ih;
      }
      gs[e] = q.lam * (-(lap + B) + c0 * (c0 * c0 - 1) * q.ie2);
    }
  }
  __syncthreads();
  // phi and G at G-block coordinates (z mirrored through the clamped loads)
  auto PHs = [&](int z, int y, int x) -> T { return ph[((z + 1) * PY + (y + HY)) * PX + (x + 1)]; };
  auto GS = [&](int z, int y, int x) -> T { return gs[(z * GY + y) * GX + x]; };
  const int ncell = TL::CX * TL::CY * (TL::CZ + 1);
  const float icx = 1.0f / TL::CX, icy = 1.0f / TL::CY;
  for (int e = threadIdx.x; e < ncell; e += blockDim.x) {
    const int lz = qdiv(e, TL::CX * TL::CY, icx * icy);
    const int rem = e - lz * TL::CX * TL::CY;
    const int ly = qdiv(rem, TL::CX, icx), lx = rem - ly * TL::CX;
    const int i = cx0 + lx, j = cy0 + ly, k = cz0 + lz;
    if (i >= d.nx || j >= d.ny || k > d.nz) continue;
    if (lz == TL::CZ && k != d.nz) continue;  // the extra layer only for the top wall face
    const size_t id = ((size_t)k * d.ny + j) * d.nx + i;
    // G-block coordinates of this coarse cell's first fine cell
    const int bx = R * lx + 1, by = DIM == 3 ? RY * ly + 1 : 0, bz = R * lz + 1;
    auto mean = [&](auto&& F, int xa, auto nxr, int ya, auto nyr, int za, auto nzr) -> T {
      constexpr int NX = decltype(nxr)::value, NY = decltype(nyr)::value, NZ = decltype(nzr)::value;
      T s = 0;
#pragma unroll
      for (int zz = 0; zz < NZ; ++zz)
#pragma unroll
        for (int yy = 0; yy < NY; ++yy)
#pragma unroll
          for (int xx = 0; xx < NX; ++xx) s += F(za + zz, ya + yy, xa + xx);
      return s * ((T)1 / (T)(NX * NY * NZ));
    };
    using C1 = std::integral_constant<int, 1>;
    using C2 = std::integral_constant<int, 2>;
    using CR = std::integral_constant<int, R>;
    using CRY = std::integral_constant<int, RY>;
    (void)C1{};
    out.phifz[id] = mean(PHs, bx, CR{}, by, CRY{}, bz - 1, C2{});
    out.Gfz[id] = mean(GS, bx, CR{}, by, CRY{}, bz - 1, C2{});
    out.phiexz[id] = mean(PHs, bx - 1, C2{}, by, CRY{}, bz - 1, C2{});
    if (DIM == 3) out.phieyz[id] = mean(PHs, bx, CR{}, by - 1, C2{}, bz - 1, C2{});
    if (k == d.nz) continue;
    out.phic[id] = mean(PHs, bx, CR{}, by, CRY{}, bz, CR{});
    out.Gc[id] = mean(GS, bx, CR{}, by, CRY{}, bz, CR{});
    out.phifx[id] = mean(PHs, bx - 1, C2{}, by, CRY{}, bz, CR{});
    out.Gfx[id] = mean(GS, bx - 1, C2{}, by, CRY{}, bz, CR{});
    if (DIM == 3) {
      out.phify[id] = mean(PHs, bx, CR{}, by - 1, C2{}, bz, CR{});
      out.Gfy[id] = mean(GS, bx, CR{}, by - 1, C2{}, bz, CR{});
      out.phiexy[id] = mean(PHs, bx - 1, C2{}, by - 1, C2{}, bz, CR{});
    }
  }
}

template <class T, int DIM, int R>
__global__ void __launch_bounds__(256) k_ch_G_restrict(const T* __restrict__ phi, const Wide<T>* __restrict__ gwall, Restricted<T> out, const Dims d, const PhysT<T> q) {
  extern __shared__ __align__(16) unsigned char smraw[];
  k_ch_G_restrict_b<T, DIM, R>(phi, gwall, out, d, q, make_int3(blockIdx.x, blockIdx.y, blockIdx.z), smraw);
}

}  // namespace pf
