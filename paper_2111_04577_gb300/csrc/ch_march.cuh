// Cahn-Hilliard right side on the 3D fine mesh, marching along z.
//
// Computes the same R as k_ch_rhs (ch_tiled.cuh; Eqs. NS25-NS34 in increment
// form, velocity prolonged by Eq. dual1, wall flux g of Eqs. NS15-NS16/NS34 in
// FP64):
//     phi* = 2 phi^n - phi^{n-1}
//     mu*  = f(phi*) - (L_N phi* + B(g))
//     R    = (phi^{n-1} - phi^n)/(M lambda dt) - div(u* phi*)/(M lambda) + L_N mu*
// A CTA owns a TX x TY column of fine cells and walks a chunk of z planes.
// Shared memory holds rings of planes: phi* with a 2-cell x/y halo (five
// planes: the one being loaded and z-1..z+2), mu* with a 1-cell halo (three
// planes), phi^{n-1} - phi^n of the owned cells (four planes), and the
// extrapolated coarse velocities of the current coarse plane (two slots).
// Every thread keeps the same x/y positions for the whole march, so index
// arithmetic is done once; the next phi plane is prefetched into registers
// while the current planes are computed.
//
// Per plane: store the prefetched plane; sync; prefetch the next one; mu* of
// plane z+1; sync; R of plane z.  The ring depths make every slot that is
// written after a barrier one that no thread can still be reading.
#pragma once
#include "ch.cuh"
#include "spectral.cuh"

namespace pf {

struct MarchTile {
  static constexpr int TX = 64, TY = 8, NT = 256;
  static constexpr int SX = TX + 4, SY = TY + 4, SP = SX * SY;  // phi* plane with 2-cell halo
  static constexpr int MX = TX + 2, MY = TY + 2, MP = MX * MY;  // mu* plane with 1-cell halo
  static constexpr int OP = TX * TY;                            // owned cells per plane
  static constexpr int NPS = 5, NMS = 3, NDS = 4;               // ring depths
  static constexpr int KS = (SP + NT - 1) / NT;                 // staged phi* elements per thread
  static constexpr int KM = (MP + NT - 1) / NT;                 // mu* elements per thread
  static constexpr int KO = OP / NT;                            // owned cells per thread
  // coarse velocity box of one coarse plane: x, y from one cell before the tile
  __host__ __device__ static constexpr int VX(int rs) { return (TX >> rs) + 2; }
  __host__ __device__ static constexpr int VY(int rs) { return (TY >> rs) + 2; }
  // elements of T in shared memory
  __host__ __device__ static constexpr int smem_elems(int rs) {
    return NPS * SP + NMS * MP + NDS * OP + 2 * 4 * VX(rs) * VY(rs);
  }
};

__device__ __forceinline__ int pmod_m(int x, int n) {
  x %= n;
  return x < 0 ? x + n : x;
}

// MINB: CTAs per SM the register budget is sized for (a launch variant; the
// arithmetic is the same)
template <class T, int MINB>
__global__ void __launch_bounds__(MarchTile::NT, MINB) k_ch_rhs_march(const FineView<T> f, const CoarseVel<T> vel,
                                                                T* __restrict__ R, Wide<T>* __restrict__ gwall,
                                                                const Dims d, const Phys p, const PhysT<T> q,
                                                                const T inv_mldt, const T inv_ml, const int nzc) {
  using TL = MarchTile;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int VX = TL::VX(d.rs), VY = TL::VY(d.rs), NV = VX * VY;
  T* ps = reinterpret_cast<T*>(smraw);  // [NPS][SY][SX]
  T* ms = ps + TL::NPS * TL::SP;        // [NMS][MY][MX]
  T* ds = ms + TL::NMS * TL::MP;        // [NDS][TY][TX]
  T* vb = ds + TL::NDS * TL::OP;        // [2 slots][u, v, w_lo, w_hi][VY][VX]
  const int t = threadIdx.x;
  const int x0 = blockIdx.x * TL::TX, y0 = blockIdx.y * TL::TY;
  const int fnx = d.fnx, fny = d.fny, fnz = d.fnz;
  const size_t plane = (size_t)fnx * fny;
  const int zb = blockIdx.z * nzc, ze = min(zb + nzc, fnz);

  // ---- per-thread positions, fixed for the whole march ----
  int sxy[TL::KS];  // global x/y offset of each staged phi* element (-1: none)
  int sown[TL::KS]; // owned-cell index of a staged element, or -1
#pragma unroll
  for (int k = 0; k < TL::KS; ++k) {
    const int e = t + k * TL::NT;
    sxy[k] = -1;
    sown[k] = -1;
    if (e < TL::SP) {
      const int yy = e / TL::SX, xx = e - yy * TL::SX;
      sxy[k] = pmod_m(y0 - 2 + yy, fny) * fnx + pmod_m(x0 - 2 + xx, fnx);
      if (xx >= 2 && xx < TL::TX + 2 && yy >= 2 && yy < TL::TY + 2) sown[k] = (yy - 2) * TL::TX + (xx - 2);
    }
  }
  // mu* positions: offset in the phi* plane, owner flag for the wall flux
  int mso[TL::KM];
  int mcol[TL::KM];  // wall column (y * fnx + x) when owned, else -1
#pragma unroll
  for (int k = 0; k < TL::KM; ++k) {
    const int e = t + k * TL::NT;
    mso[k] = -1;
    mcol[k] = -1;
    if (e < TL::MP) {
      const int my = e / TL::MX, mx = e - my * TL::MX;
      mso[k] = (my + 1) * TL::SX + (mx + 1);
      const int gx = x0 - 1 + mx, gy = y0 - 1 + my;
      if (mx >= 1 && mx <= TL::TX && my >= 1 && my <= TL::TY && gx < fnx && gy < fny) mcol[k] = gy * fnx + gx;
    }
  }
  // coarse velocity box origin and loader positions
  const int cx0 = (x0 >> d.rs) - 1, cy0 = (y0 >> d.rs) - 1;
  const int cplane = d.nx * d.ny;

  auto star_load = [&](int gz, T (&reg)[TL::KS], T (&dreg)[TL::KS]) {
    const size_t zo = (size_t)min(max(gz, 0), fnz - 1) * plane;
#pragma unroll
    for (int k = 0; k < TL::KS; ++k) {
      if (sxy[k] >= 0) {
        const size_t o = zo + sxy[k];
        const T a = f.pn[o], b = f.po[o];
        reg[k] = (T)2 * a - b;
        dreg[k] = f.back(o, a, b);
      }
    }
  };
  auto star_store = [&](int slot, int dslot, const T (&reg)[TL::KS], const T (&dreg)[TL::KS]) {
    T* pp = ps + slot * TL::SP;
    T* dd = ds + dslot * TL::OP;
#pragma unroll
    for (int k = 0; k < TL::KS; ++k) {
      const int e = t + k * TL::NT;
      if (e < TL::SP) {
        pp[e] = reg[k];
        if (sown[k] >= 0) dd[sown[k]] = dreg[k];
      }
    }
  };
  auto vel_load = [&](int kc, int slot) {
    T* vu = vb + slot * 4 * NV;
    const int czw = kc + 1;  // w faces kc and kc + 1 (kc + 1 <= nz)
    for (int e = t; e < NV; e += TL::NT) {
      const int yy = e / VX, xx = e - yy * VX;
      const int cx = pmod_m(cx0 + xx, d.nx), cy = pmod_m(cy0 + yy, d.ny);
      const size_t oc = (size_t)kc * cplane + cy * d.nx + cx;
      const size_t colw = (size_t)cy * d.nx + cx;
      vu[e] = vel.us(oc);
      vu[NV + e] = vel.vs(oc);
      vu[2 * NV + e] = vel.ws((size_t)kc * cplane + colw);
      vu[3 * NV + e] = vel.ws((size_t)czw * cplane + colw);
    }
  };
  // mu* of plane gz into ring slot mslot, from phi* slots (gz-1, gz, gz+1)
  auto mu_plane = [&](int gz, int sm1, int s0, int sp1, int mslot) {
    T* mm = ms + mslot * TL::MP;
    const T* pm = ps + sm1 * TL::SP;
    const T* pc = ps + s0 * TL::SP;
    const T* pq = ps + sp1 * TL::SP;
#pragma unroll
    for (int k = 0; k < TL::KM; ++k) {
      const int e = t + k * TL::NT;
      if (mso[k] < 0) continue;
      if (gz < 0 || gz >= fnz) {
        mm[e] = (T)0;
        continue;
      }
      const int o = mso[k];
      const T c0 = pc[o];
      T lap = pc[o + 1] + pc[o - 1] - 2 * c0;
      lap += pc[o + TL::SX] + pc[o - TL::SX] - 2 * c0;
      const T czp = gz + 1 < fnz ? pq[o] : c0;
      const T czm = gz > 0 ? pm[o] : c0;
      lap = (lap + czp + czm - 2 * c0) * q.ih2;
      T B = 0;
      if (gz == 0) {
        const Wide<T> g = wall_g(q.gbot, (Wide<T>)c0, (Wide<T>)czp);
        if (mcol[k] >= 0) gwall[mcol[k]] = g;
        B += (T)(g * q.ihw);
      }
      if (gz == fnz - 1) {
        const Wide<T> g = wall_g(q.gtop, (Wide<T>)c0, (Wide<T>)czm);
        if (mcol[k] >= 0) gwall[plane + mcol[k]] = g;
        B += (T)(g * q.ihw);
      }
      mm[e] = c0 * (c0 * c0 - 1) * q.ie2 - (lap + B);
    }
  };

  // ---- owned cells: fixed offsets of the face velocities in the box ----
  // thread t owns (tx, ty) and (tx, ty + TY/2)
  const int tx = t % TL::TX, tyb = t / TL::TX;
  const int gx = x0 + tx;
  const bool xin = gx < fnx;
  // x faces gx and gx + 1; y faces gy and gy + 1 (unwrapped: the box holds the periodic images)
  const int iu0 = (gx >> d.rs) - cx0, iu1 = ((gx + 1) >> d.rs) - cx0;
  const bool hu0 = (gx & (d.r - 1)) != 0, hu1 = ((gx + 1) & (d.r - 1)) != 0;
  const int iwx = (gx >> d.rs) - cx0;

  // ---- prologue: phi* planes zb-2 .. zb+1, mu* planes zb-1, zb ----
  {
    T reg[TL::KS], dreg[TL::KS];
#pragma unroll
    for (int k = 0; k < TL::KS; ++k) reg[k] = dreg[k] = (T)0;
    for (int j = 0; j < 4; ++j) {
      star_load(zb - 2 + j, reg, dreg);
      star_store(j, j >= 2 ? j - 2 : 3, reg, dreg);  // d slots: plane zb + m at m & 3
    }
  }
  __syncthreads();
  mu_plane(zb - 1, 0, 1, 2, 0);
  mu_plane(zb, 1, 2, 3, 1);
  T reg[TL::KS], dreg[TL::KS];
#pragma unroll
  for (int k = 0; k < TL::KS; ++k) reg[k] = dreg[k] = (T)0;
  star_load(zb + 2, reg, dreg);
  int kc_loaded = -1;

  for (int z = zb; z < ze; ++z) {
    const int m = z - zb;
    // ring slots: phi* plane zb + j at (j + 2) % 5; mu* plane zb + j at (j + 1) % 3; d plane zb + j at j & 3
    const int sP = (m + 4) % 5;  // plane z + 2
    star_store(sP, (m + 2) & 3, reg, dreg);
    const int kc = z >> d.rs;
    if (kc != kc_loaded) {
      vel_load(kc, kc & 1);
      kc_loaded = kc;
    }
    __syncthreads();
    if (z + 1 < ze) star_load(z + 3, reg, dreg);
    mu_plane(z + 1, (m + 2) % 5, (m + 3) % 5, (m + 4) % 5, (m + 2) % 3);
    __syncthreads();
    // ---- R of plane z ----
    const T* pm = ps + ((m + 1) % 5) * TL::SP;
    const T* pc = ps + ((m + 2) % 5) * TL::SP;
    const T* pq = ps + ((m + 3) % 5) * TL::SP;
    const T* mmm = ms + (m % 3) * TL::MP;
    const T* mmc = ms + ((m + 1) % 3) * TL::MP;
    const T* mmp = ms + ((m + 2) % 3) * TL::MP;
    const T* dd = ds + (m & 3) * TL::OP;
    const T* vu = vb + (kc & 1) * 4 * NV;
    const T* vv = vu + NV;
    const T* vw = vu + 2 * NV;
    // fine z faces z (bottom) and z + 1 (top) of this plane, in layers of the box
    const int kf0 = (z >> d.rs) - kc, kf1 = ((z + 1) >> d.rs) - kc;
    const bool hw0 = (z & (d.r - 1)) != 0, hw1 = ((z + 1) & (d.r - 1)) != 0;
#pragma unroll
    for (int k = 0; k < TL::KO; ++k) {
      const int ty = tyb + k * (TL::TY / TL::KO);
      const int gy = y0 + ty;
      if (!xin || gy >= fny) continue;
      const int iv0 = (gy >> d.rs) - cy0, iv1 = ((gy + 1) >> d.rs) - cy0;
      const bool hv0 = (gy & (d.r - 1)) != 0, hv1 = ((gy + 1) & (d.r - 1)) != 0;
      const int jr = ((gy >> d.rs) - cy0) * VX;  // box row of this fine row
      // prolonged face velocities (Eq. dual1)
      const T ua = vu[jr + iu0], ub = vu[jr + iu1];
      const T u0 = hu0 ? (T)0.5 * (ua + vu[jr + iu0 + 1]) : ua;
      const T u1 = hu1 ? (T)0.5 * (ub + vu[jr + iu1 + 1]) : ub;
      const T va = vv[iv0 * VX + iwx], vb1 = vv[iv1 * VX + iwx];
      const T v0 = hv0 ? (T)0.5 * (va + vv[(iv0 + 1) * VX + iwx]) : va;
      const T v1 = hv1 ? (T)0.5 * (vb1 + vv[(iv1 + 1) * VX + iwx]) : vb1;
      const T wa = vw[kf0 * NV + jr + iwx], wb = vw[kf1 * NV + jr + iwx];
      const T w0 = hw0 ? (T)0.5 * (wa + vw[(kf0 + 1) * NV + jr + iwx]) : wa;
      const T w1 = hw1 ? (T)0.5 * (wb + vw[(kf1 + 1) * NV + jr + iwx]) : wb;
      const int so = (ty + 2) * TL::SX + (tx + 2);
      const T c0 = pc[so];
      T adv = u1 * (c0 + pc[so + 1]) - u0 * (pc[so - 1] + c0);
      adv += v1 * (c0 + pc[so + TL::SX]) - v0 * (pc[so - TL::SX] + c0);
      if (z + 1 < fnz) adv += w1 * (c0 + pq[so]);
      if (z > 0) adv -= w0 * (pm[so] + c0);
      adv *= (T)0.5 * q.ih;
      const size_t o = (size_t)z * plane + (size_t)gy * fnx + gx;
      if (f.aw) adv = f.aw[o];
      const int mo = (ty + 1) * TL::MX + (tx + 1);
      const T m0 = mmc[mo];
      T lap = mmc[mo + 1] + mmc[mo - 1] - 2 * m0;
      lap += mmc[mo + TL::MX] + mmc[mo - TL::MX] - 2 * m0;
      const T mzp = z + 1 < fnz ? mmp[mo] : m0;
      const T mzm = z > 0 ? mmm[mo] : m0;
      lap = (lap + mzp + mzm - 2 * m0) * q.ih2;
      R[o] = dd[ty * TL::TX + tx] * inv_mldt - adv * inv_ml + lap;
    }
  }
}

}  // namespace pf

namespace pf {

// ---------------------------------------------------------------------------
// Chemical potential and restriction on the 3D dual mesh (r = 2), marching
// along z.  Same outputs as k_ch_G_restrict (ch_tiled.cuh; Eqs. NS5, dual2,
// dual3): G = lambda(-(L_N phi + B(g)) + f(phi)) on the fine mesh, then the
// 2 x 2 x 2 means of phi and G at coarse centres, faces and edges.
// A CTA owns CX x CY coarse columns and walks coarse layers k; layer k needs
// fine planes 2k-1, 2k, 2k+1 (z mirrored at the walls).  phi is staged with a
// one-cell x/y halo in a ring of four planes, G of the two new planes is formed
// in shared memory, and each thread turns the 3 x 3 fine neighbourhood of its
// coarse cell into the seven means through 2 x 2 plane sums; the sums of plane
// 2k+1 serve as plane 2k-1 of the next layer.
// ---------------------------------------------------------------------------
struct GrMarch {
  static constexpr int CX = 32, CY = 8, NT = CX * CY;
  static constexpr int FX = 2 * CX + 1, FY = 2 * CY + 1, FN = FX * FY;  // G region (fine)
  static constexpr int PX = FX + 2, PY = FY + 2, PN = PX * PY;          // phi with halo
  // row strides even (G rows one wider: they are stored one column to the
  // right) so that every pair starting at an even index is one aligned
  // two-element load; slot sizes even for the same reason
  static constexpr int SGX = FX + 1, FP = SGX * FY;
  static constexpr int SPX = PX + 1, PP = SPX * PY;
  static_assert(SPX == FX + 3 && SGX % 2 == 0 && SPX % 2 == 0 && FP % 2 == 0 && PP % 2 == 0, "G tile layout");
  static constexpr int NPS = 4;
  static constexpr int KP = (PN + NT - 1) / NT;
  static constexpr int KG = (FN + NT - 1) / NT;
  static constexpr int smem_elems() { return NPS * PP + 2 * FP; }
};

// 2 x 2 sums of a 3 x 3 neighbourhood: hh = offsets {0,1}x{0,1}, lh = {-1,0}x{0,1},
// hl = {0,1}x{-1,0}, ll = {-1,0}x{-1,0} (x first)
template <class T>
struct Quad {
  T hh, lh, hl, ll;
};

template <class T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};
struct DualPair {
  Dual x, y;
};
template <>
struct Pair<Dual> {
  using type = DualPair;
};

template <class T>
__device__ __forceinline__ Quad<T> quad_sums(const T* p, int o, int sx) {
  // p[o + b * sx + a], a, b in {-1, 0, 1}; o and sx even, p two-element aligned:
  // each row is read as the pairs (-2, -1) and (0, 1)
  using P2 = typename Pair<T>::type;
  T rlo[3], rhi[3];
#pragma unroll
  for (int b = -1; b <= 1; ++b) {
    const P2 lo = *reinterpret_cast<const P2*>(p + o + b * sx - 2);
    const P2 hi = *reinterpret_cast<const P2*>(p + o + b * sx);
    const T m = lo.y, c = hi.x, q = hi.y;
    rlo[b + 1] = m + c;
    rhi[b + 1] = c + q;
  }
  Quad<T> r;
  r.hh = rhi[1] + rhi[2];
  r.lh = rlo[1] + rlo[2];
  r.hl = rhi[0] + rhi[1];
  r.ll = rlo[0] + rlo[1];
  return r;
}

template <class T>
__global__ void __launch_bounds__(GrMarch::NT, 3) k_ch_G_restrict_march(const T* __restrict__ phi,
                                                                        const Wide<T>* __restrict__ gwall,
                                                                        Restricted<T> out, const Dims d,
                                                                        const PhysT<T> q, const int nkc) {
  using TL = GrMarch;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* ps = reinterpret_cast<T*>(smraw);  // [NPS][PY][PX], fine plane zf at slot (zf + 1) & 3
  T* gs = ps + TL::NPS * TL::PP;        // [2][FY][SGX], fine plane zf at slot zf & 1
  const int t = threadIdx.x;
  const int cx0 = blockIdx.x * TL::CX, cy0 = blockIdx.y * TL::CY;
  const int kb = blockIdx.z * nkc, ke = min(kb + nkc, d.nz + 1);  // coarse layers kb..ke-1 (nz: top face)
  const int fnx = d.fnx, fny = d.fny, fnz = d.fnz;
  const size_t plane = (size_t)fnx * fny;
  const int fx0 = 2 * cx0 - 2, fy0 = 2 * cy0 - 2;  // fine origin of the phi tile
  // per-thread staging offsets (x/y part), fixed for the march
  // staged element e = yy * PX + xx sits at yy * SPX + xx = e + yy in a slot
  int sxy[TL::KP], sso[TL::KP];
#pragma unroll
  for (int kq = 0; kq < TL::KP; ++kq) {
    const int e = t + kq * TL::NT;
    sxy[kq] = -1;
    sso[kq] = 0;
    if (e < TL::PN) {
      const int yy = e / TL::PX, xx = e - yy * TL::PX;
      sxy[kq] = pmod_m(fy0 + yy, fny) * fnx + pmod_m(fx0 + xx, fnx);
      sso[kq] = e + yy;
    }
  }
  // per-thread G positions: offset in the phi tile, and the wall column
  // G element e = yy * FX + xx: its row yy (-1: none); it reads phi at
  // (yy + 1) * SPX + xx + 1 = e + 3 yy + FX + 4 (SPX = FX + 3) and is stored at
  // yy * SGX + xx + 1 = e + yy + 1 (SGX = FX + 1; one column to the right, so
  // that fine x even lands on an even index)
  int gy[TL::KG];
#pragma unroll
  for (int kq = 0; kq < TL::KG; ++kq) {
    const int e = t + kq * TL::NT;
    gy[kq] = e < TL::FN ? e / TL::FX : -1;
  }
  auto load_plane = [&](int zf, T (&reg)[TL::KP]) {
    const size_t zo = (size_t)min(max(zf, 0), fnz - 1) * plane;
#pragma unroll
    for (int kq = 0; kq < TL::KP; ++kq)
      if (sxy[kq] >= 0) reg[kq] = phi[zo + sxy[kq]];
  };
  auto store_plane = [&](int zf, const T (&reg)[TL::KP]) {
    T* p = ps + ((zf + 1) & 3) * TL::PP;
#pragma unroll
    for (int kq = 0; kq < TL::KP; ++kq)
      if (sxy[kq] >= 0) p[sso[kq]] = reg[kq];
  };
  // G of fine plane zf (0 <= zf < fnz) into slot zf & 1, from phi planes zf-1..zf+1
  auto g_plane = [&](int zf) {
    const T* pm = ps + ((zf) & 3) * TL::PP;  // plane zf - 1
    const T* pc = ps + ((zf + 1) & 3) * TL::PP;
    const T* pq = ps + ((zf + 2) & 3) * TL::PP;
    T* g = gs + (zf & 1) * TL::FP;
#pragma unroll
    for (int kq = 0; kq < TL::KG; ++kq) {
      if (gy[kq] < 0) continue;
      const int e = t + kq * TL::NT;
      const int o = e + 3 * gy[kq] + TL::FX + 4;
      const T c0 = pc[o];
      T lap = pc[o + 1] + pc[o - 1] - 2 * c0;
      lap += pc[o + TL::SPX] + pc[o - TL::SPX] - 2 * c0;
      const T czp = zf + 1 < fnz ? pq[o] : c0;
      const T czm = zf > 0 ? pm[o] : c0;
      lap = (lap + czp + czm - 2 * c0) * q.ih2;
      T B = 0;
      if (zf == 0 || zf == fnz - 1) {
        const int yy = gy[kq], xx = e - yy * TL::FX;
        const size_t gcol = (size_t)pmod_m(fy0 + 1 + yy, fny) * fnx + pmod_m(fx0 + 1 + xx, fnx);
        if (zf == 0) B += (T)gwall[gcol] * q.ih;
        if (zf == fnz - 1) B += (T)gwall[plane + gcol] * q.ih;
      }
      g[e + gy[kq] + 1] = q.lam * (-(lap + B) + c0 * (c0 * c0 - 1) * q.ie2);
    }
  };
  // this thread's coarse cell and its fine centre (2i, 2j) in the tiles
  const int lx = t % TL::CX, ly = t / TL::CX;
  const int i = cx0 + lx, j = cy0 + ly;
  const bool own = i < d.nx && j < d.ny;
  const int po = (2 * ly + 2) * TL::SPX + (2 * lx + 2);  // phi tile: fine (2i, 2j), even
  const int gq = (2 * ly + 1) * TL::SGX + (2 * lx + 2);  // G region: fine (2i, 2j), even
  const T eighth = (T)0.125;
  Quad<T> qpm{}, qgm{};  // sums of fine plane 2k-1
  T reg[TL::KP];
#pragma unroll
  for (int kq = 0; kq < TL::KP; ++kq) reg[kq] = (T)0;
  // ---- prologue: phi planes 2kb-2 .. 2kb (and G of 2kb-1 when kb > 0) ----
  for (int zf = 2 * kb - 2; zf <= 2 * kb; ++zf) {
    load_plane(zf, reg);
    store_plane(zf, reg);
  }
  __syncthreads();
  if (kb > 0) {
    g_plane(2 * kb - 1);
    __syncthreads();
    qpm = quad_sums(ps + ((2 * kb) & 3) * TL::PP, po, TL::SPX);
    qgm = quad_sums(gs + ((2 * kb - 1) & 1) * TL::FP, gq, TL::SGX);
  }
  // phi planes 2k+1, 2k+2 of the next layer are prefetched into registers
  T ra[TL::KP], rb[TL::KP];
#pragma unroll
  for (int kq = 0; kq < TL::KP; ++kq) ra[kq] = rb[kq] = (T)0;
  if (kb < d.nz) {
    load_plane(2 * kb + 1, ra);
    load_plane(2 * kb + 2, rb);
  }
  for (int k = kb; k < ke; ++k) {
    if (k < d.nz) {
      // into the slots of planes 2k-3, 2k-2: free after the previous layer's barrier
      store_plane(2 * k + 1, ra);
      store_plane(2 * k + 2, rb);
      __syncthreads();
      if (k + 1 < min(ke, d.nz)) {
        load_plane(2 * k + 3, ra);
        load_plane(2 * k + 4, rb);
      }
      g_plane(2 * k);
      g_plane(2 * k + 1);
      __syncthreads();
      const Quad<T> p0 = quad_sums(ps + ((2 * k + 1) & 3) * TL::PP, po, TL::SPX);
      const Quad<T> p1 = quad_sums(ps + ((2 * k + 2) & 3) * TL::PP, po, TL::SPX);
      const Quad<T> g0 = quad_sums(gs + ((2 * k) & 1) * TL::FP, gq, TL::SGX);
      const Quad<T> g1 = quad_sums(gs + ((2 * k + 1) & 1) * TL::FP, gq, TL::SGX);
      if (k == 0) {  // fine plane -1 mirrors plane 0
        qpm = p0;
        qgm = g0;
      }
      if (own) {
        const size_t id = ((size_t)k * d.ny + j) * d.nx + i;
        out.phic[id] = (p0.hh + p1.hh) * eighth;
        out.Gc[id] = (g0.hh + g1.hh) * eighth;
        out.phifx[id] = (p0.lh + p1.lh) * eighth;
        out.Gfx[id] = (g0.lh + g1.lh) * eighth;
        out.phify[id] = (p0.hl + p1.hl) * eighth;
        out.Gfy[id] = (g0.hl + g1.hl) * eighth;
        out.phiexy[id] = (p0.ll + p1.ll) * eighth;
        out.phifz[id] = (qpm.hh + p0.hh) * eighth;
        out.Gfz[id] = (qgm.hh + g0.hh) * eighth;
        out.phiexz[id] = (qpm.lh + p0.lh) * eighth;
        out.phieyz[id] = (qpm.hl + p0.hl) * eighth;
      }
      qpm = p1;
      qgm = g1;
      __syncthreads();
    } else if (own) {  // top wall face k = nz: fine plane 2nz mirrors 2nz-1
      const size_t id = ((size_t)k * d.ny + j) * d.nx + i;
      out.phifz[id] = (qpm.hh + qpm.hh) * eighth;
      out.Gfz[id] = (qgm.hh + qgm.hh) * eighth;
      out.phiexz[id] = (qpm.lh + qpm.lh) * eighth;
      out.phieyz[id] = (qpm.hl + qpm.hl) * eighth;
    }
  }
}

}  // namespace pf

namespace pf {

// ---------------------------------------------------------------------------
// k_ch_rhs_march4: the z-marching CH right side of k_ch_rhs_march (same R,
// same arithmetic per cell), FP32, with each thread owning four consecutive x
// cells of one row so that every shared-memory access moves a float4 and the
// offsets are shared by four cells.  Needs fnx % 4 == 0 (float4 rows never
// straddle the periodic seam).  RS = log2 of the refinement ratio (fine/coarse).
// Planes carry 4 floats of padding on both ends: the halo chunks read one
// float beyond their row, and only lanes that are never used depend on it.
// ---------------------------------------------------------------------------
// TY_ rows per CTA: 16 (256 threads, three CTAs per SM), or 14 (224 threads, 55.3 KB
// of shared memory in 3D dual resolution: four CTAs per SM at up to 72 registers)
template <int TY_>
struct March4T {
  static constexpr int TX = 64, TY = TY_, CH = TX / 4, NT = CH * TY;  // 16 chunks per row
  static constexpr int SXC = CH + 2, SXF = 4 * SXC;               // phi* chunks (x0-4 .. x0+68)
  static constexpr int SY = TY + 4, SPF = SY * SXF + 8;            // phi* rows y0-2 .. y0+TY+1, padded plane
  static constexpr int MY = TY + 2, MPF = MY * SXF + 8;            // mu* rows y0-1 .. y0+TY
  static constexpr int NPS = 5, NMS = 3;
  static constexpr int NSC = SY * SXC, NMC = MY * SXC;             // staged / mu chunks per plane
  static constexpr int KS = (NSC + NT - 1) / NT, KM = (NMC + NT - 1) / NT;
  __host__ __device__ static constexpr int VX(int rs) { return (TX >> rs) + 2; }
  __host__ __device__ static constexpr int VY(int rs) { return (TY >> rs) + 2; }
  __host__ __device__ static constexpr int smem_floats(int rs) {
    return NPS * SPF + NMS * MPF + 4 * VX(rs) * VY(rs) + 8 * NSC;
  }
};
using March4 = March4T<16>;

// AW: take div(u* phi*) from f.aw (WENO5-Z) instead of the central flux; a
// template flag, so that the default form carries no trace of it
template <int RS, int MINB, bool AW = false, int TYV = 16>
__global__ void __launch_bounds__(March4T<TYV>::NT, MINB) k_ch_rhs_march4(const FineView<float> f, const CoarseVel<float> vel,
                                                                     float* __restrict__ R, double* __restrict__ gwall,
                                                                     const Dims d, const Phys p, const PhysT<float> q,
                                                                     const float inv_mldt, const float inv_ml,
                                                                     const int nzc) {
  using TL = March4T<TYV>;
  static_assert(TL::TY % 2 == 0, "tile rows start on even fine rows (the velocity box rows)");
  extern __shared__ __align__(16) unsigned char smraw[];
  float* ps = reinterpret_cast<float*>(smraw);  // [NPS][4 + SY*SXF + 4]
  float* ms = ps + TL::NPS * TL::SPF;           // [NMS][4 + MY*SXF + 4]
  float* vb = ms + TL::NMS * TL::MPF;           // [u, v, w_lo, w_hi][VY][VX]
  float4* raw = reinterpret_cast<float4*>(vb + 4 * TL::VX(RS) * TL::VY(RS));  // [phi^n, phi^{n-1}][NSC] in flight
  constexpr int VX = TL::VX(RS), VY = TL::VY(RS), NV = VX * VY;
  const int t = threadIdx.x;
  const int x0 = blockIdx.x * TL::TX, y0 = blockIdx.y * TL::TY;
  const int fnx = d.fnx, fny = d.fny, fnz = d.fnz;
  const size_t plane = (size_t)fnx * fny;
  const int zb = blockIdx.z * nzc, ze = min(zb + nzc, fnz);
  // ---- staging chunks: global x/y offset (multiple of 4) ----
  int sxy[TL::KS];
#pragma unroll
  for (int k = 0; k < TL::KS; ++k) {
    const int e = t + k * TL::NT;
    sxy[k] = -1;
    if (e < TL::NSC) {
      const int yy = e / TL::SXC, xc = e - yy * TL::SXC;
      sxy[k] = pmod_m(y0 - 2 + yy, fny) * fnx + pmod_m(x0 - 4 + 4 * xc, fnx);
    }
  }
  // the next plane's phi^n and phi^{n-1} chunks go straight to shared memory
  // (cp.async, no register staging); each thread later combines the chunks it
  // copied itself into phi* = 2 phi^n - phi^{n-1}
  auto star_load = [&](int gz) {
    const size_t zo = (size_t)min(max(gz, 0), fnz - 1) * plane;
#pragma unroll
    for (int k = 0; k < TL::KS; ++k)
      if (sxy[k] >= 0) {
        const int e = t + k * TL::NT;
        cp_async16(raw + e, f.pn + zo + sxy[k]);
        cp_async16(raw + TL::NSC + e, f.po + zo + sxy[k]);
      }
    cp_async_commit();
  };
  auto star_store = [&](int slot) {
    cp_async_wait_all();  // this thread's own copies
    float* pp = ps + slot * TL::SPF + 4;
#pragma unroll
    for (int k = 0; k < TL::KS; ++k) {
      const int e = t + k * TL::NT;
      if (e < TL::NSC) {
        const float4 a = raw[e], b = raw[TL::NSC + e];
        reinterpret_cast<float4*>(pp)[e] = make_float4(2.f * a.x - b.x, 2.f * a.y - b.y, 2.f * a.z - b.z, 2.f * a.w - b.w);
      }
    }
  };
  const int cx0 = (x0 >> RS) - 1, cy0 = (y0 >> RS) - 1;
  const int cplane = d.nx * d.ny;
  auto vel_load = [&](int kc) {
    float* vu = vb;
    for (int e = t; e < NV; e += TL::NT) {
      const int yy = e / VX, xx = e - yy * VX;
      const int cx = pmod_m(cx0 + xx, d.nx), cy = pmod_m(cy0 + yy, d.ny);
      const size_t colw = (size_t)cy * d.nx + cx;
      const size_t oc = (size_t)kc * cplane + colw;
      vu[e] = vel.us(oc);
      vu[NV + e] = vel.vs(oc);
      vu[2 * NV + e] = vel.ws(oc);
      vu[3 * NV + e] = vel.ws((size_t)(kc + 1) * cplane + colw);
    }
  };
  // ---- mu* of one plane, four x cells per chunk ----
  auto mu_plane = [&](int gz, int sm1, int s0, int sp1, int mslot) {
    float* mm = ms + mslot * TL::MPF + 4;
    const float* pm = ps + sm1 * TL::SPF + 4;
    const float* pc = ps + s0 * TL::SPF + 4;
    const float* pq = ps + sp1 * TL::SPF + 4;
    static_assert(TL::KM == 2, "one full pass of the threads and one partial pass");
#pragma unroll
    for (int k = 0; k < TL::KM; ++k) {
      // whole warps take part (the x neighbours come by shuffle).  The partial
      // second pass runs on the highest warps (the chunks NMC - NT + t), so that
      // it does not fall on the warps that hold a second velocity-box element;
      // its lanes below chunk NT repeat chunks of the first pass and store nothing
      const int e0 = k == 0 ? t : t + (TL::NMC - TL::NT);
      if (k > 0 && (t | 31) + (TL::NMC - TL::NT) < TL::NT) continue;  // warp-uniform
      const bool valid = k == 0 || e0 >= TL::NT;
      const int e = e0;
      float4* mo = reinterpret_cast<float4*>(mm) + e;
      if (gz < 0 || gz >= fnz) {
        if (valid) *mo = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
      const int my = e / TL::SXC, mc = e - my * TL::SXC;
      const int o = (my + 1) * TL::SXF + 4 * mc;  // phi* row my+1
      const float4 c = *reinterpret_cast<const float4*>(pc + o);
      // x neighbours from the adjacent lanes (consecutive chunks of a row);
      // shared memory only at a row end or a warp edge
      float l = __shfl_up_sync(0xffffffffu, c.w, 1), r = __shfl_down_sync(0xffffffffu, c.x, 1);
      if (mc == 0 || (t & 31) == 0) l = pc[o - 1];
      if (mc == TL::SXC - 1 || (t & 31) == 31) r = pc[o + 4];
      const float4 up = *reinterpret_cast<const float4*>(pc + o + TL::SXF);
      const float4 dn = *reinterpret_cast<const float4*>(pc + o - TL::SXF);
      const float4 zp = gz + 1 < fnz ? *reinterpret_cast<const float4*>(pq + o) : c;
      const float4 zm = gz > 0 ? *reinterpret_cast<const float4*>(pm + o) : c;
      const float cv[6] = {l, c.x, c.y, c.z, c.w, r};
      const float uv[4] = {up.x, up.y, up.z, up.w}, dv[4] = {dn.x, dn.y, dn.z, dn.w};
      const float zpv[4] = {zp.x, zp.y, zp.z, zp.w}, zmv[4] = {zm.x, zm.y, zm.z, zm.w};
      float outv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float c0 = cv[i + 1];
        float lap = cv[i + 2] + cv[i] - 2 * c0;
        lap += uv[i] + dv[i] - 2 * c0;
        lap = (lap + zpv[i] + zmv[i] - 2 * c0) * q.ih2;
        outv[i] = c0 * (c0 * c0 - 1) * q.ie2 - lap;
      }
      if (gz == 0 || gz == fnz - 1) {
        const int gy = y0 - 1 + my;
        const bool rown = my >= 1 && my <= TL::TY && gy < fny;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int gx = x0 - 4 + 4 * mc + i;
          const bool own = valid && rown && gx >= x0 && gx < x0 + TL::TX && gx < fnx;
          const size_t col = (size_t)gy * fnx + gx;
          if (gz == 0) {
            const double g = wall_g(q.gbot, (double)cv[i + 1], (double)zpv[i]);
            if (own) gwall[col] = g;
            outv[i] -= (float)(g * q.ihw);
          }
          if (gz == fnz - 1) {
            const double g = wall_g(q.gtop, (double)cv[i + 1], (double)zmv[i]);
            if (own) gwall[plane + col] = g;
            outv[i] -= (float)(g * q.ihw);
          }
        }
      }
      if (valid) *mo = make_float4(outv[0], outv[1], outv[2], outv[3]);
    }
  };
  // ---- owned chunk of this thread ----
  const int cx = t % TL::CH, ty = t / TL::CH;
  const int gx = x0 + 4 * cx, gy = y0 + ty;
  const bool act = gx < fnx && gy < fny;
  const int so = (ty + 2) * TL::SXF + 4 * (cx + 1);  // phi* center chunk
  const int mo = (ty + 1) * TL::SXF + 4 * (cx + 1);  // mu* center chunk
  const size_t gof = (size_t)gy * fnx + gx;  // owned chunk within a plane
  // velocity box rows/columns (Eq. dual1)
  const int urow = ((ty >> RS) + 1) * VX;
  const int cb = ((4 * cx) >> RS) + 1;  // box column of the chunk's first coarse cell
  const bool yodd = RS == 1 && (gy & 1);
  const int vr0 = ((ty >> RS) + 1) * VX, vr1 = (((ty + 1) >> RS) + 1) * VX;

  // ---- prologue ----
  for (int j = 0; j < 4; ++j) {
    star_load(zb - 2 + j);
    star_store(j);
  }
  __syncthreads();
  mu_plane(zb - 1, 0, 1, 2, 0);
  mu_plane(zb, 1, 2, 3, 1);
  star_load(zb + 2);
  // owned phi^n and phi^{n-1} of the plane being formed, read one plane ahead
  // (an L2 hit: the plane was staged three planes earlier)
  // (with compensated storage also the remainders' difference dl = lo - ln)
  // (the remainders are kept as loaded and differenced where R uses them, so that
  // no warp waits for these loads at the end of the plane that issues them)
  float4 an = make_float4(0.f, 0.f, 0.f, 0.f), bo = an, la = an, lb = an;
  auto own_load = [&](int zz) {
    const size_t o = (size_t)zz * plane + gof;
    an = *reinterpret_cast<const float4*>(f.pn + o);
    bo = *reinterpret_cast<const float4*>(f.po + o);
    if (f.ln) {
      la = *reinterpret_cast<const float4*>(f.ln + o);
      lb = *reinterpret_cast<const float4*>(f.lo + o);
    }
  };
  if (act) own_load(zb);
  int kc_loaded = -1;
  // ring positions m % 5 and m % 3, advanced per plane (no integer division in the loop)
  int m5 = 0, m3 = 0;
  auto r5 = [](int a) { return a >= 5 ? a - 5 : a; };
  auto r3 = [](int a) { return a >= 3 ? a - 3 : a; };
  for (int z = zb; z < ze; ++z, m5 = r5(m5 + 1), m3 = r3(m3 + 1)) {
    star_store(r5(m5 + 4));
    const int kc = z >> RS;
    __syncthreads();
    // one velocity box: every reader of the previous layer has passed the barrier above
    if (kc != kc_loaded) {
      vel_load(kc);
      kc_loaded = kc;
    }
    if (z + 1 < ze) star_load(z + 3);
    mu_plane(z + 1, r5(m5 + 2), r5(m5 + 3), r5(m5 + 4), r3(m3 + 2));
    __syncthreads();
    // every lane forms its chunk (the shuffles below need whole warps); lanes
    // outside the mesh read only inside the tiles and store nothing
    const float* pm = ps + r5(m5 + 1) * TL::SPF + 4;
    const float* pc = ps + r5(m5 + 2) * TL::SPF + 4;
    const float* pq = ps + r5(m5 + 3) * TL::SPF + 4;
    const float* mmm = ms + m3 * TL::MPF + 4;
    const float* mmc = ms + r3(m3 + 1) * TL::MPF + 4;
    const float* mmp = ms + r3(m3 + 2) * TL::MPF + 4;
    const float* vu = vb;
    const float* vv = vu + NV;
    const float* vw = vu + 2 * NV;
    // face velocities of the four cells
    float uf[5];
#pragma unroll
    for (int fq = 0; fq < 5; ++fq) {
      const int cc = cb + ((4 * cx + fq) >> RS) - ((4 * cx) >> RS);
      const float a = vu[urow + cc];
      uf[fq] = (RS == 1 && (fq & 1)) ? 0.5f * (a + vu[urow + cc + 1]) : a;
    }
    float vlo[4], vhi[4], wlo[4], whi[4];
    const int kf0 = (z >> RS) - kc, kf1 = ((z + 1) >> RS) - kc;
    const bool hw0 = RS == 1 && (z & 1), hw1 = RS == 1 && ((z + 1) & 1);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int cc = cb + ((4 * cx + i) >> RS) - ((4 * cx) >> RS);
      // y faces gy (lo) and gy + 1 (hi)
      const float a0 = vv[vr0 + cc];
      vlo[i] = yodd ? 0.5f * (a0 + vv[vr0 + VX + cc]) : a0;
      const float a1 = vv[vr1 + cc];
      vhi[i] = (RS == 1 && !yodd) ? 0.5f * (a1 + vv[vr1 + VX + cc]) : a1;
      // z faces z (lo) and z + 1 (hi)
      const float w0 = vw[kf0 * NV + urow + cc];
      wlo[i] = hw0 ? 0.5f * (w0 + vw[(kf0 + 1) * NV + urow + cc]) : w0;
      const float w1 = vw[kf1 * NV + urow + cc];
      whi[i] = hw1 ? 0.5f * (w1 + vw[(kf1 + 1) * NV + urow + cc]) : w1;
    }
    const float4 c4 = *reinterpret_cast<const float4*>(pc + so);
    float pl = __shfl_up_sync(0xffffffffu, c4.w, 1), pr = __shfl_down_sync(0xffffffffu, c4.x, 1);
    if (cx == 0) pl = pc[so - 1];
    if (cx == TL::CH - 1) pr = pc[so + 4];
    const float pv[6] = {pl, c4.x, c4.y, c4.z, c4.w, pr};
    const float4 up = *reinterpret_cast<const float4*>(pc + so + TL::SXF);
    const float4 dn = *reinterpret_cast<const float4*>(pc + so - TL::SXF);
    const float4 zp = *reinterpret_cast<const float4*>(pq + so);
    const float4 zm = *reinterpret_cast<const float4*>(pm + so);
    const float uvp[4] = {up.x, up.y, up.z, up.w}, dvp[4] = {dn.x, dn.y, dn.z, dn.w};
    const float zpp[4] = {zp.x, zp.y, zp.z, zp.w}, zmp[4] = {zm.x, zm.y, zm.z, zm.w};
    const float4 m4 = *reinterpret_cast<const float4*>(mmc + mo);
    float ml = __shfl_up_sync(0xffffffffu, m4.w, 1), mr = __shfl_down_sync(0xffffffffu, m4.x, 1);
    if (cx == 0) ml = mmc[mo - 1];
    if (cx == TL::CH - 1) mr = mmc[mo + 4];
    const float mv[6] = {ml, m4.x, m4.y, m4.z, m4.w, mr};
    const float4 mu4 = *reinterpret_cast<const float4*>(mmc + mo + TL::SXF);
    const float4 md4 = *reinterpret_cast<const float4*>(mmc + mo - TL::SXF);
    const float4 mzp4 = *reinterpret_cast<const float4*>(mmp + mo);
    const float4 mzm4 = *reinterpret_cast<const float4*>(mmm + mo);
    const float muv[4] = {mu4.x, mu4.y, mu4.z, mu4.w}, mdv[4] = {md4.x, md4.y, md4.z, md4.w};
    const float mzpv[4] = {mzp4.x, mzp4.y, mzp4.z, mzp4.w}, mzmv[4] = {mzm4.x, mzm4.y, mzm4.z, mzm4.w};
    // phi^{n-1} - phi^n: the stored values' difference first (exact when they are
    // close), then the remainders' (zero without compensated storage)
    const float dv[4] = {(bo.x - an.x) + (lb.x - la.x), (bo.y - an.y) + (lb.y - la.y), (bo.z - an.z) + (lb.z - la.z),
                         (bo.w - an.w) + (lb.w - la.w)};
    float awv[4] = {0.f, 0.f, 0.f, 0.f};
    if constexpr (AW) {
      if (act) {
        const float4 a = *reinterpret_cast<const float4*>(f.aw + (size_t)z * plane + gof);
        awv[0] = a.x, awv[1] = a.y, awv[2] = a.z, awv[3] = a.w;
      }
    }
    float out[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float c0 = pv[i + 1];
      float adv = uf[i + 1] * (c0 + pv[i + 2]) - uf[i] * (pv[i] + c0);
      adv += vhi[i] * (c0 + uvp[i]) - vlo[i] * (dvp[i] + c0);
      if (z + 1 < fnz) adv += whi[i] * (c0 + zpp[i]);
      if (z > 0) adv -= wlo[i] * (zmp[i] + c0);
      adv *= 0.5f * q.ih;
      if constexpr (AW) adv = awv[i];
      const float m0 = mv[i + 1];
      float lap = mv[i + 2] + mv[i] - 2 * m0;
      lap += muv[i] + mdv[i] - 2 * m0;
      const float mzp = z + 1 < fnz ? mzpv[i] : m0;
      const float mzm = z > 0 ? mzmv[i] : m0;
      lap = (lap + mzp + mzm - 2 * m0) * q.ih2;
      out[i] = dv[i] * inv_mldt - adv * inv_ml + lap;
    }
    if (!act) continue;
    *reinterpret_cast<float4*>(R + (size_t)z * plane + gof) = make_float4(out[0], out[1], out[2], out[3]);
    if (z + 1 < ze) own_load(z + 1);
  }
}

}  // namespace pf
