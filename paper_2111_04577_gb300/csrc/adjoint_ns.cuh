// Reverse sweep of the coupled 2D step: the adjoints of the Navier-Stokes
// projection (Section 3.2.2, Eqs. NS35-NS39), the restriction and chemical
// potential (Eqs. dual2, dual3, NS5), the velocity's part in the CH step
// (Eq. dual1 and the advection of Eq. NS25) and the log-conformation update
// (Section 3.2.3, Eqs. NS40-NS46).
//
// Linear pieces are transposed by hand: the correction and divergence of the
// projection, the restriction, the prolongation, the advection stencils and
// the velocity gradient; the constant-coefficient solves are symmetric and are
// reused as they are.  The nonlinear per-cell pieces -- the momentum right
// side, the LCR right side's local part and tau(Theta) -- are differentiated
// exactly by evaluating the forward arithmetic (ns_rhs_cell2, lcr_rhs_local,
// lcr_tau) in dual numbers, seeding one input at a time: the derivative that
// comes out is the Jacobian column of that input, and the adjoint is its
// product with the incoming adjoint, scattered (atomically) to the input.
#pragma once
#include "ns_rhs.cuh"
#include "polymer.cuh"

namespace pf {

// ---------------------------------------------------------------------------
// momentum right side (ns_rhs_cell2)
// ---------------------------------------------------------------------------
enum NsSlot : signed char { S_U, S_W, S_DP, S_PS, S_PHC, S_G, S_EXZ, S_PHIFX, S_PHIFZ, S_GFX, S_GFZ, S_TXX, S_TXZ, S_TZZ,
                            S_DU, S_DW };
struct SlotDef {
  signed char f, dx, dz;
};
// every (field, offset) ns_rhs_cell2 reads
constexpr int kNsSlots = 50;
__constant__ SlotDef c_ns_slots[kNsSlots] = {
    {S_U, 0, 0},    {S_U, 1, 0},    {S_U, -1, 0},   {S_U, 0, 1},    {S_U, 0, -1},   {S_U, 1, -1},   {S_W, 0, 0},
    {S_W, 0, 1},    {S_W, -1, 0},   {S_W, 1, 0},    {S_W, -1, 1},   {S_W, 0, -1},   {S_DP, 0, 0},   {S_DP, -1, 0},
    {S_DP, 0, -1},  {S_PS, 0, 0},   {S_PS, -1, 0},  {S_PS, 0, -1},  {S_PHC, 0, 0},  {S_PHC, -1, 0}, {S_PHC, 0, -1},
    {S_G, 0, 0},    {S_G, -1, 0},   {S_G, 1, 0},    {S_G, 0, 1},    {S_G, -1, 1},   {S_G, 0, -1},   {S_G, -1, -1},
    {S_G, 1, -1},   {S_EXZ, 0, 0},  {S_EXZ, 0, 1},  {S_EXZ, 1, 0},  {S_PHIFX, 0, 0}, {S_PHIFZ, 0, 0}, {S_GFX, 0, 0},
    {S_GFZ, 0, 0},  {S_TXX, 0, 0},  {S_TXX, -1, 0}, {S_TXZ, 0, 0},  {S_TXZ, -1, 0}, {S_TXZ, 0, 1},  {S_TXZ, -1, 1},
    {S_TXZ, 0, -1}, {S_TXZ, -1, -1}, {S_TXZ, 1, 0}, {S_TXZ, 1, -1}, {S_TZZ, 0, 0},  {S_TZZ, 0, -1}, {S_DU, 0, 0},
    {S_DW, 0, 0}};

// The inputs of ns_rhs_cell2 in dual numbers, the one seeded slot carrying
// derivative 1.
template <class T>
struct NsSeedAcc2 {
  NsGlobalAcc2<T, double> g;
  int sf, sdx, sdz;
  __device__ __forceinline__ Dual m(int f, int dx, int dz, double v) const {
    return Dual(v, (f == sf && dx == sdx && dz == sdz) ? 1.0 : 0.0);
  }
  __device__ __forceinline__ Dual U(int dx, int dz) const { return m(S_U, dx, dz, g.U(dx, dz)); }
  __device__ __forceinline__ Dual W(int dx, int dz) const { return m(S_W, dx, dz, g.W(dx, dz)); }
  __device__ __forceinline__ Dual DP(int dx, int dz) const { return m(S_DP, dx, dz, g.DP(dx, dz)); }
  __device__ __forceinline__ Dual PS(int dx, int dz) const { return m(S_PS, dx, dz, g.PS(dx, dz)); }
  __device__ __forceinline__ Dual PHC(int dx, int dz) const { return m(S_PHC, dx, dz, g.PHC(dx, dz)); }
  __device__ __forceinline__ Dual G(int dx, int dz) const { return m(S_G, dx, dz, g.G(dx, dz)); }
  __device__ __forceinline__ Dual EXZ(int dx, int dz) const { return m(S_EXZ, dx, dz, g.EXZ(dx, dz)); }
  __device__ __forceinline__ Dual phifx() const { return m(S_PHIFX, 0, 0, g.phifx()); }
  __device__ __forceinline__ Dual phifz() const { return m(S_PHIFZ, 0, 0, g.phifz()); }
  __device__ __forceinline__ Dual gfx() const { return m(S_GFX, 0, 0, g.gfx()); }
  __device__ __forceinline__ Dual gfz() const { return m(S_GFZ, 0, 0, g.gfz()); }
  __device__ __forceinline__ Dual TXX(int dx, int dz) const { return m(S_TXX, dx, dz, g.TXX(dx, dz)); }
  __device__ __forceinline__ Dual TXZ(int dx, int dz) const { return m(S_TXZ, dx, dz, g.TXZ(dx, dz)); }
  __device__ __forceinline__ Dual TZZ(int dx, int dz) const { return m(S_TZZ, dx, dz, g.TZZ(dx, dz)); }
  __device__ __forceinline__ Dual du() const { return m(S_DU, 0, 0, g.du()); }
  __device__ __forceinline__ Dual dw() const { return m(S_DW, 0, 0, g.dw()); }
};

// adjoint accumulators of the step-n inputs of the momentum right side
template <class T>
struct NsBar {
  T *un, *uo, *wn, *wo, *pn, *po;  // u^n, u^{n-1}, ... (w at faces 0..nz)
  T *tn[3], *to[3];                // tau^n, tau^{n-1} (2D components xx, xz, zz)
  T *phic, *phifx, *phifz, *phiexz, *Gc, *Gfx, *Gfz;  // restricted phi^{n+1}, G^{n+1}
};

template <class T>
__device__ __forceinline__ void aadd(T* p, double v) {
  atomicAdd(p, (T)v);
}

// rbar_u: adjoint of the x rows (nz x nx); rbar_w: of the z rows (faces
// 1..nz-1 as rows 0..nz-2).  qd: the constants in dual numbers, derivatives
// zero; qm: the same with d(cj_dx)/dM in cj_dx.  mpart[block] accumulates the
// partial sums of M_bar from the J.grad(u) term.
template <class T>
__global__ void __launch_bounds__(128) k_adj_ns_rhs2(const __grid_constant__ NsIn<T> a, const Dims d,
                                                     const PhysT<Dual> qd, const PhysT<Dual> qm,
                                                     const T* __restrict__ rbar_u, const T* __restrict__ rbar_w,
                                                     const NsBar<T> bar, const int have_tau,
                                                     double* __restrict__ mpart) {
  __shared__ double sm[128];
  const int nx = d.nx, nz = d.nz;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double mb = 0.0;
  if (c < nx * nz) {
    const int k = c / nx, i = c - k * nx;
    const double ab_u = (double)rbar_u[c];
    const double ab_w = k > 0 ? (double)rbar_w[c - nx] : 0.0;
    NsSeedAcc2<T> A{{&a, nx, nz, i, k}, -1, 0, 0};
    {  // M through J = -(rho1 - rho2)/2 M grad(G)
      Dual ru = 0, rw = 0;
      ns_rhs_cell2<Dual>(A, qm, k, nz, have_tau, ru, rw);
      mb = ab_u * ru.d + ab_w * rw.d;
    }
    for (int s = 0; s < kNsSlots; ++s) {
      const SlotDef sd = c_ns_slots[s];
      const bool tau_slot = sd.f == S_TXX || sd.f == S_TXZ || sd.f == S_TZZ;
      if (tau_slot && !have_tau) continue;
      const int xi = wrap(i + sd.dx, nx);
      int z = k + sd.dz;
      const bool face = sd.f == S_W || sd.f == S_EXZ || sd.f == S_PHIFZ || sd.f == S_GFZ || sd.f == S_DW;
      if (face) {
        if (z < 0 || z > nz) continue;
      } else if (z < 0 || z >= nz) {
        if (!tau_slot) continue;  // not read there
        z = z < 0 ? 0 : nz - 1;   // the stresses' mirror ghost
      }
      A.sf = sd.f;
      A.sdx = sd.dx;
      A.sdz = sd.dz;
      Dual ru = 0, rw = 0;
      ns_rhs_cell2<Dual>(A, qd, k, nz, have_tau, ru, rw);
      const double g = ab_u * ru.d + ab_w * rw.d;
      if (g == 0.0) continue;
      const int o = z * nx + xi;
      switch (sd.f) {
        case S_U: aadd(bar.un + o, 2 * g); aadd(bar.uo + o, -g); break;
        case S_W: aadd(bar.wn + o, 2 * g); aadd(bar.wo + o, -g); break;
        case S_DP: aadd(bar.po + o, g); aadd(bar.pn + o, -g); break;
        case S_PS: aadd(bar.pn + o, 2 * g); aadd(bar.po + o, -g); break;
        case S_PHC: aadd(bar.phic + o, g); break;
        case S_G: aadd(bar.Gc + o, g); break;
        case S_EXZ: aadd(bar.phiexz + o, g); break;
        case S_PHIFX: aadd(bar.phifx + o, g); break;
        case S_PHIFZ: aadd(bar.phifz + o, g); break;
        case S_GFX: aadd(bar.Gfx + o, g); break;
        case S_GFZ: aadd(bar.Gfz + o, g); break;
        case S_TXX: aadd(bar.tn[0] + o, 2 * g); aadd(bar.to[0] + o, -g); break;
        case S_TXZ: aadd(bar.tn[1] + o, 2 * g); aadd(bar.to[1] + o, -g); break;
        case S_TZZ: aadd(bar.tn[2] + o, 2 * g); aadd(bar.to[2] + o, -g); break;
        case S_DU: aadd(bar.un + o, g); aadd(bar.uo + o, -g); break;
        case S_DW: aadd(bar.wn + o, g); aadd(bar.wo + o, -g); break;
        default: break;
      }
    }
  }
  sm[threadIdx.x] = mb;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) mpart[blockIdx.x] += sm[0];
}

// ---------------------------------------------------------------------------
// projection (Eqs. NS37-NS39): u = u~ - cf d_x p', w = w~ - cf d_z p' on the
// interior faces, p^{n+1} = p^n + p'.  Given the adjoints ub, wb of u^{n+1},
// w^{n+1} and pb of p^{n+1}, the adjoint of p' (before the Poisson solve).
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_adj_correct2(const T* __restrict__ ub, const T* __restrict__ wb, const T* __restrict__ pb,
                               T* __restrict__ ppb, Dims d, T cfD) {
  const int nx = d.nx, nz = d.nz;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nx * nz) return;
  const int k = c / nx, i = c - k * nx;
  T v = pb[c] - cfD * ub[c] + cfD * ub[k * nx + wrap(i + 1, nx)];
  if (k >= 1) v -= cfD * wb[c];                // face k
  if (k + 1 <= nz - 1) v += cfD * wb[c + nx];  // face k + 1
  ppb[c] = v;
}

// div = (u~_{i+1} - u~_i + w~_{k+1} - w~_k)/D (walls zero): the adjoint of
// u~, w~ from that of div (scaled by coef, the Poisson right side's factor),
// added to ut_b, wt_b (w on faces 0..nz; walls untouched).
template <class T>
__global__ void k_adj_div2(const T* __restrict__ divb, T* __restrict__ utb, T* __restrict__ wtb, Dims d, T coefD) {
  const int nx = d.nx, nz = d.nz;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nx * nz) return;
  const int k = c / nx, i = c - k * nx;
  utb[c] += coefD * (divb[k * nx + wrap(i - 1, nx)] - divb[c]);
  if (k >= 1) wtb[c] += coefD * (divb[c - nx] - divb[c]);  // face k between cells k-1 and k
}

// u~ = u* + delta (the increment-form solve): the adjoints of u^n and u^{n-1}
// from that of u~ (faces: rows 1..nz-1 of w only)
template <class T>
__global__ void k_adj_ustar(const T* __restrict__ ub, T* __restrict__ un, T* __restrict__ uo, size_t n0, size_t n1) {
  const size_t e = n0 + blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= n1) return;
  const T v = ub[e];
  un[e] += 2 * v;
  uo[e] -= v;
}

// ---------------------------------------------------------------------------
// restriction (Eq. dual2) and chemical potential (Eq. NS5), transposed
// ---------------------------------------------------------------------------
// For fine cell (fi, fk): the coarse samples that average it and its weight in
// each (r = 2: quarters, with the wall mirror counted twice; r = 1: halves).
// gather form: phib_f += sum weight * (sample adjoint); Gf = the same for G.
template <class T>
__global__ void k_adj_restrict2(const NsBar<T> bar, T* __restrict__ phib, T* __restrict__ Gb, Dims d) {
  const int fnx = d.fnx, fnz = d.fnz, nx = d.nx, nz = d.nz, r = d.r;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= fnx * fnz) return;
  const int fk = e / fnx, fi = e - fk * fnx;
  double sp = 0, sg = 0;
  // x-face pairs straddling column fi: faces at coarse column xa (as the right cell) and xb (as the left)
  // r = 2: fine 2i-1, 2i straddle face i; r = 1: fine i-1, i straddle face i.
  const double wz = r == 2 ? 0.5 : 1.0;  // weight of one fine row within a coarse row (r = 2: mean of 2)
  if (r == 2) {
    const int ci = fi >> 1, ck = fk >> 1;
    sp += 0.25 * (double)bar.phic[ck * nx + ci];
    sg += 0.25 * (double)bar.Gc[ck * nx + ci];
    // x-face: column fi is 2i (face i) or 2i - 1 with i = (fi + 1)/2
    const int fx = (fi & 1) ? wrap((fi + 1) >> 1, nx) : (fi >> 1);
    sp += 0.25 * (double)bar.phifx[ck * nx + fx];
    sg += 0.25 * (double)bar.Gfx[ck * nx + fx];
    // z-face: row fk is 2k (face k) or 2k - 1 with k = (fk + 1)/2; mirrors at the walls
    const int fz = (fk & 1) ? ((fk + 1) >> 1) : (fk >> 1);
    int mult = 1;
    if (fk == 0 || fk == fnz - 1) mult = 2;  // the wall face's pair is this row and its mirror
    sp += 0.25 * mult * (double)bar.phifz[fz * nx + ci];
    sg += 0.25 * mult * (double)bar.Gfz[fz * nx + ci];
    sp += 0.25 * mult * (double)bar.phiexz[fz * nx + fx];
  } else {
    sp += (double)bar.phic[fk * nx + fi];
    sg += (double)bar.Gc[fk * nx + fi];
    const int fxp = wrap(fi + 1, nx);
    sp += 0.5 * ((double)bar.phifx[fk * nx + fi] + (double)bar.phifx[fk * nx + fxp]);
    sg += 0.5 * ((double)bar.Gfx[fk * nx + fi] + (double)bar.Gfx[fk * nx + fxp]);
    const double mb = fk == 0 ? 1.0 : 0.5, mt = fk == nz - 1 ? 1.0 : 0.5;  // faces fk, fk + 1 (mirror at walls)
    sp += mb * (double)bar.phifz[fk * nx + fi] + mt * (double)bar.phifz[(fk + 1) * nx + fi];
    sg += mb * (double)bar.Gfz[fk * nx + fi] + mt * (double)bar.Gfz[(fk + 1) * nx + fi];
    // edge (i, k): pairs in x (i-1, i) and z (k-1, k)
    sp += 0.5 * mb * ((double)bar.phiexz[fk * nx + fi] + (double)bar.phiexz[fk * nx + fxp]) +
          0.5 * mt * ((double)bar.phiexz[(fk + 1) * nx + fi] + (double)bar.phiexz[(fk + 1) * nx + fxp]);
  }
  (void)wz;
  phib[e] += (T)sp;
  Gb[e] = (T)sg;
}

// G = lambda (-(L_N phi + B(g)) + f(phi)), f(x) = x (x^2 - 1)/eta^2: adds
// lambda (-L_N Gb + f'(phi) Gb) to phib (L_N symmetric), and writes the wall
// flux adjoints gbx[col] = -lambda Gb_0/h (bottom), gbx[plane + col] (top).
template <class T>
__global__ void k_adj_G2(const T* __restrict__ phi, const T* __restrict__ Gb, T* __restrict__ phib,
                         double* __restrict__ gbx, Dims d, PhysT<T> q) {
  const int fnx = d.fnx, fnz = d.fnz;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= fnx * fnz) return;
  const int k = e / fnx, i = e - k * fnx;
  const T g0 = Gb[e];
  T lap = Gb[k * fnx + wrap(i + 1, fnx)] + Gb[k * fnx + wrap(i - 1, fnx)] - 2 * g0;
  lap += (k + 1 < fnz ? Gb[e + fnx] : g0) + (k > 0 ? Gb[e - fnx] : g0) - 2 * g0;
  const T c0 = phi[e];
  phib[e] += q.lam * (-lap * q.ih2 + (3 * c0 * c0 - 1) * q.ie2 * g0);
  if (k == 0) gbx[i] = -(double)q.lam * (double)g0 / d.h;
  if (k == fnz - 1) gbx[fnx + i] = -(double)q.lam * (double)g0 / d.h;
}

// The CH advection's velocity adjoint, brought back to the coarse faces
// (Eq. dual1 transposed) and to u^n, u^{n-1} (u* = 2u^n - u^{n-1}).  On a fine
// face f between cells L and R: ub_f = -a2 (phi*_L + phi*_R)/(2h) (Rb_L - Rb_R).
template <class T>
__device__ __forceinline__ double ch_ub_x(const T* phis, const T* rbar, int fnx, int fk, int fi) {
  const int l = fk * fnx + wrap(fi - 1, fnx), r = fk * fnx + fi;
  return ((double)phis[l] + (double)phis[r]) * ((double)rbar[l] - (double)rbar[r]);
}
template <class T>
__device__ __forceinline__ double ch_ub_z(const T* phis, const T* rbar, int fnx, int fnz, int ff, int fi) {
  if (ff <= 0 || ff >= fnz) return 0.0;  // wall faces carry no flux
  const int l = (ff - 1) * fnx + fi, r = ff * fnx + fi;
  return ((double)phis[l] + (double)phis[r]) * ((double)rbar[l] - (double)rbar[r]);
}
template <class T>
__global__ void k_adj_ch_vel2(const T* __restrict__ phis, const T* __restrict__ rbar, T* __restrict__ un,
                              T* __restrict__ uo, T* __restrict__ wn, T* __restrict__ wo, Dims d, double s) {
  // s = -a2/(2h); one thread per coarse cell: its u-face (i, k) and w-face k
  const int nx = d.nx, nz = d.nz, fnx = d.fnx, fnz = d.fnz;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nx * nz) return;
  const int k = c / nx, i = c - k * nx;
  double gu = 0, gw = 0;
  if (d.r == 2) {
    for (int fk = 2 * k; fk <= 2 * k + 1; ++fk)
      gu += ch_ub_x(phis, rbar, fnx, fk, 2 * i) +
            0.5 * (ch_ub_x(phis, rbar, fnx, fk, 2 * i + 1) + ch_ub_x(phis, rbar, fnx, fk, wrap(2 * i - 1, fnx)));
    if (k >= 1)
      for (int fi = 2 * i; fi <= 2 * i + 1; ++fi)
        gw += ch_ub_z(phis, rbar, fnx, fnz, 2 * k, fi) +
              0.5 * (ch_ub_z(phis, rbar, fnx, fnz, 2 * k + 1, fi) + ch_ub_z(phis, rbar, fnx, fnz, 2 * k - 1, fi));
  } else {
    gu = ch_ub_x(phis, rbar, fnx, k, i);
    if (k >= 1) gw = ch_ub_z(phis, rbar, fnx, fnz, k, i);
  }
  un[c] += (T)(2 * s * gu);
  uo[c] -= (T)(s * gu);
  if (k >= 1) {
    wn[c] += (T)(2 * s * gw);
    wo[c] -= (T)(s * gw);
  }
}

// ---------------------------------------------------------------------------
// LCR update (2D), Theta as components (xx, xz, zz)
// ---------------------------------------------------------------------------
struct PolyFaces {  // u^{n+1} at x-faces, w^{n+1} at z-faces 0..nz
  const void* u;
  const void* w;
};

// velocity gradient at cell (i, k) (as polymer_cell: face differences along the
// normal, central differences of centre averages across, no-slip ghosts)
template <class T, class R>
__device__ __forceinline__ void grad_u2(const T* U, const T* W, const Dims& d, const PhysT<R>& q, int i, int k,
                                        R (&L)[2][2]) {
  const int nx = d.nx, ip = wrap(i + 1, nx), im = wrap(i - 1, nx);
  const bool top = k + 1 == d.nz, bot = k == 0;
  auto uc = [&](int kk) { return (R)0.5 * ((R)U[kk * nx + i] + (R)U[kk * nx + ip]); };
  auto wc = [&](int ii) { return (R)0.5 * ((R)W[k * nx + ii] + (R)W[(k + 1) * nx + ii]); };
  const R uc0 = uc(k);
  const R ucp = top ? q.uw2_top - uc0 : uc(k + 1);
  const R ucm = bot ? q.uw2_bot - uc0 : uc(k - 1);
  L[0][0] = ((R)U[k * nx + ip] - (R)U[k * nx + i]) * q.iD;
  L[0][1] = (ucp - ucm) * (R)0.5 * q.iD;
  L[1][0] = (wc(ip) - wc(im)) * (R)0.5 * q.iD;
  L[1][1] = ((R)W[(k + 1) * nx + i] - (R)W[k * nx + i]) * q.iD;
}

// scatter Lb (the adjoint of the gradient at cell (i, k)) to the face adjoints
template <class T>
__device__ __forceinline__ void grad_u2_T(T* ub, T* wb, const Dims& d, double iD, int i, int k, const double (&Lb)[2][2]) {
  const int nx = d.nx, ip = wrap(i + 1, nx), im = wrap(i - 1, nx);
  const bool top = k + 1 == d.nz, bot = k == 0;
  // dudx
  aadd(ub + k * nx + ip, Lb[0][0] * iD);
  aadd(ub + k * nx + i, -Lb[0][0] * iD);
  // dudz = (ucp - ucm)/(2D): uc(kk) = (u_i + u_ip)/2 at row kk
  const double h = 0.5 * iD * Lb[0][1];
  auto add_uc = [&](int kk, double v) {
    aadd(ub + kk * nx + i, 0.5 * v);
    aadd(ub + kk * nx + ip, 0.5 * v);
  };
  double c0 = 0;
  if (top) c0 -= h;
  else add_uc(k + 1, h);
  if (bot) c0 += h;
  else add_uc(k - 1, -h);
  if (c0 != 0) add_uc(k, c0);
  // dwdx = (wc(ip) - wc(im))/(2D): wc(ii) = (w_k + w_{k+1})/2 at column ii (walls fixed)
  const double g = 0.5 * iD * Lb[1][0];
  auto add_wc = [&](int ii, double v) {
    if (k > 0) aadd(wb + k * nx + ii, 0.5 * v);
    if (k + 1 < d.nz) aadd(wb + (k + 1) * nx + ii, 0.5 * v);
  };
  add_wc(ip, g);
  add_wc(im, -g);
  // dwdz
  if (k + 1 < d.nz) aadd(wb + (k + 1) * nx + i, Lb[1][1] * iD);
  if (k > 0) aadd(wb + k * nx + i, -Lb[1][1] * iD);
}

// advection div(u Theta) of one component at cell (i, k) (central, no wall flux)
template <class T, class R>
__device__ __forceinline__ R adv2(const T* th, const T* U, const T* W, const Dims& d, R iD, int i, int k) {
  const int nx = d.nx, ip = wrap(i + 1, nx), im = wrap(i - 1, nx), c = k * nx + i;
  const R t0 = (R)th[c];
  R a = (R)U[k * nx + ip] * (t0 + (R)th[k * nx + ip]) - (R)U[c] * ((R)th[k * nx + im] + t0);
  if (k + 1 < d.nz) a += (R)W[(k + 1) * nx + i] * (t0 + (R)th[c + nx]);
  if (k > 0) a -= (R)W[c] * ((R)th[c - nx] + t0);
  return (R)0.5 * iD * a;
}

// (A^T ab)_J of one component: the adjoint of Theta at cell J from the
// adjoint ab of the advection (gather over the cells whose flux reads J)
template <class T>
__device__ __forceinline__ double adv2_T(const T* ab, const T* U, const T* W, const Dims& d, double iD, int i, int k) {
  const int nx = d.nx, ip = wrap(i + 1, nx), im = wrap(i - 1, nx), c = k * nx + i;
  const double u0 = (double)U[c], u1 = (double)U[k * nx + ip];
  double s = (double)ab[c] * (u1 - u0);
  s += (double)ab[k * nx + im] * u0 - (double)ab[k * nx + ip] * u1;
  if (k + 1 < d.nz) {
    const double w1 = (double)W[(k + 1) * nx + i];
    s += (double)ab[c] * w1 - (double)ab[c + nx] * w1;
  }
  if (k > 0) {
    const double w0 = (double)W[c];
    s += -(double)ab[c] * w0 + (double)ab[c - nx] * w0;
  }
  return 0.5 * iD * s;
}

// velocity adjoint of the advection of Theta (all components) with adjoint ab:
// on the u-face i of row k and the w-face k, as k_adj_ch_vel2's fine faces
template <class T>
__device__ __forceinline__ void adv2_vel_T(const T* const (&th)[3], const T* const (&ab)[3], const Dims& d, double iD,
                                           int i, int k, double& gu, double& gw) {
  const int nx = d.nx, im = wrap(i - 1, nx), c = k * nx + i;
  gu = 0;
  gw = 0;
  for (int q = 0; q < 3; ++q) {
    gu += ((double)th[q][k * nx + im] + (double)th[q][c]) * ((double)ab[q][k * nx + im] - (double)ab[q][c]);
    if (k >= 1) gw += ((double)th[q][c - nx] + (double)th[q][c]) * ((double)ab[q][c - nx] - (double)ab[q][c]);
  }
  gu *= 0.5 * iD;
  gw *= 0.5 * iD;
}

// Jacobian-transpose product of the local RH (lcr_rhs_local) at one cell:
// given v[3], adds J_theta^T v to thb, J_L^T v to Lb, and returns dRH/dlambda_H . v
// (qd: constants in dual numbers with derivative zero; qw: with d(1/lambda_H)
// and d(mu_p/lambda_H) per unit lambda_H)
__device__ __forceinline__ double lcr_local_T(const double (&th)[3], const double (&L)[2][2], const PhysT<Dual>& qd,
                                              const PhysT<Dual>& qw, const double (&v)[3], double (&thb)[3],
                                              double (&Lb)[2][2]) {
  for (int s = 0; s < 7; ++s) {
    Dual t[3], Ld[2][2], out[3], R[2][2], dg[2];
    for (int q = 0; q < 3; ++q) t[q] = Dual(th[q], s == q ? 1.0 : 0.0);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) Ld[a][b] = Dual(L[a][b], s == 3 + 2 * a + b ? 1.0 : 0.0);
    lcr_rhs_local<Dual, 2>(t, Ld, qd, out, R, dg);
    const double g = out[0].d * v[0] + out[1].d * v[1] + out[2].d * v[2];
    if (s < 3) thb[s] += g;
    else Lb[(s - 3) >> 1][(s - 3) & 1] += g;
  }
  Dual t[3], Ld[2][2], out[3], R[2][2], dg[2];
  for (int q = 0; q < 3; ++q) t[q] = Dual(th[q]);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) Ld[a][b] = Dual(L[a][b]);
  lcr_rhs_local<Dual, 2>(t, Ld, qw, out, R, dg);
  return out[0].d * v[0] + out[1].d * v[1] + out[2].d * v[2];
}

// Inputs of the polymer's reverse passes (2D).
template <class T>
struct PolyAdj {
  const T *th0[3], *th1[3];  // Theta^n, Theta1 (stage 1 of the step)
  const T *U, *W;            // u^{n+1}, w^{n+1}
  const T* phic;             // restricted phi^{n+1} at centres
  const T *thb_in[3], *taub[3];  // adjoints of Theta^{n+1} and tau^{n+1}
  T *thb_out[3];             // adjoint of Theta^n (complete after pass C)
  T *th1b[3], *ab1[3], *ab0[3];  // work: Theta1 adjoint (local part), advection adjoints of stages 2 and 1
  T *ub, *wb;                // adjoints of u^{n+1}, w^{n+1} (accumulated)
  T* phicb;                  // adjoint of the restricted phi at centres (accumulated)
  double* wipart;            // per-block partial sums of dJ/d lambda_H
};

// pass A: tau and stage 2.  Theta2 = Theta^n/2 + (Theta1 + dt RH(Theta1))/2,
// tau = tau(Theta2, phic).
template <class T>
__global__ void __launch_bounds__(128) k_adj_poly2_a(const PolyAdj<T> P, const Dims d, const PhysT<T> q,
                                                     const PhysT<Dual> qd, const PhysT<Dual> qw) {
  __shared__ double sm[128];
  const int nx = d.nx, nz = d.nz;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double wb = 0;
  if (c < nx * nz) {
    const int k = c / nx, i = c - k * nx;
    const double dt = (double)q.dt, iD = (double)q.iD;
    double L[2][2];
    {
      PhysT<double> qq;
      qq.iD = iD;
      qq.uw2_top = (double)q.uw2_top;
      qq.uw2_bot = (double)q.uw2_bot;
      grad_u2<T, double>(P.U, P.W, d, qq, i, k, L);
    }
    double t1[3], t0[3];
    for (int cq = 0; cq < 3; ++cq) {
      t1[cq] = (double)P.th1[cq][c];
      t0[cq] = (double)P.th0[cq][c];
    }
    // Theta2 (forward, in FP64 arithmetic)
    double th2[3];
    {
      Dual t[3], Ld[2][2], out[3], R[2][2], dg[2];
      for (int cq = 0; cq < 3; ++cq) t[cq] = Dual(t1[cq]);
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) Ld[a][b] = Dual(L[a][b]);
      lcr_rhs_local<Dual, 2>(t, Ld, qd, out, R, dg);
      for (int cq = 0; cq < 3; ++cq) {
        const double a1 = adv2<T, double>(P.th1[cq], P.U, P.W, d, iD, i, k);
        th2[cq] = 0.5 * t0[cq] + 0.5 * (t1[cq] + dt * (out[cq].v - a1));
      }
    }
    // tau(Theta2, phic): Theta2_bar = Theta^{n+1}_bar + J^T tau_bar; phic_bar; lambda_H
    double th2b[3], tb[3];
    for (int cq = 0; cq < 3; ++cq) {
      th2b[cq] = (double)P.thb_in[cq][c];
      tb[cq] = (double)P.taub[cq][c];
    }
    const double ph = (double)P.phic[c];
    for (int s = 0; s < 5; ++s) {
      Dual t[3], out[3];
      for (int cq = 0; cq < 3; ++cq) t[cq] = Dual(th2[cq], s == cq ? 1.0 : 0.0);
      const Dual pc(ph, s == 3 ? 1.0 : 0.0);
      lcr_tau<Dual, 2>(t, pc, s == 4 ? qw : qd, out);
      const double g = out[0].d * tb[0] + out[1].d * tb[1] + out[2].d * tb[2];
      if (s < 3) th2b[s] += g;
      else if (s == 3) aadd(P.phicb + c, g);
      else wb += g;
    }
    // stage 2: v = dt/2 Theta2_bar through the local RH at Theta1
    double v[3], t1b[3] = {0, 0, 0}, Lb[2][2] = {{0, 0}, {0, 0}};
    for (int cq = 0; cq < 3; ++cq) v[cq] = 0.5 * dt * th2b[cq];
    wb += lcr_local_T(t1, L, qd, qw, v, t1b, Lb);
    for (int cq = 0; cq < 3; ++cq) {
      P.thb_out[cq][c] = (T)(0.5 * th2b[cq]);
      P.th1b[cq][c] = (T)(0.5 * th2b[cq] + t1b[cq]);
      P.ab1[cq][c] = (T)(-v[cq]);
    }
    grad_u2_T(P.ub, P.wb, d, iD, i, k, Lb);
  }
  sm[threadIdx.x] = wb;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) P.wipart[blockIdx.x] += sm[0];
}

// pass B: stage 1.  Theta1 = Theta^n + dt RH(Theta^n); Theta1_bar = local part
// + A^T ab1 (the stage-2 advection); then through the local RH at Theta^n.
template <class T>
__global__ void __launch_bounds__(128) k_adj_poly2_b(const PolyAdj<T> P, const Dims d, const PhysT<T> q,
                                                     const PhysT<Dual> qd, const PhysT<Dual> qw) {
  __shared__ double sm[128];
  const int nx = d.nx, nz = d.nz;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double wb = 0;
  if (c < nx * nz) {
    const int k = c / nx, i = c - k * nx;
    const double dt = (double)q.dt, iD = (double)q.iD;
    double L[2][2];
    {
      PhysT<double> qq;
      qq.iD = iD;
      qq.uw2_top = (double)q.uw2_top;
      qq.uw2_bot = (double)q.uw2_bot;
      grad_u2<T, double>(P.U, P.W, d, qq, i, k, L);
    }
    double t0[3], t1b[3], v[3], t0b[3] = {0, 0, 0}, Lb[2][2] = {{0, 0}, {0, 0}};
    for (int cq = 0; cq < 3; ++cq) {
      t0[cq] = (double)P.th0[cq][c];
      t1b[cq] = (double)P.th1b[cq][c] + adv2_T<T>(P.ab1[cq], P.U, P.W, d, iD, i, k);
      v[cq] = dt * t1b[cq];
    }
    wb += lcr_local_T(t0, L, qd, qw, v, t0b, Lb);
    for (int cq = 0; cq < 3; ++cq) {
      P.thb_out[cq][c] += (T)(t1b[cq] + t0b[cq]);
      P.ab0[cq][c] = (T)(-v[cq]);
    }
    grad_u2_T(P.ub, P.wb, d, iD, i, k, Lb);
  }
  sm[threadIdx.x] = wb;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) P.wipart[blockIdx.x] += sm[0];
}

// pass C: Theta^n_bar += A^T ab0 (the stage-1 advection); the velocity adjoint
// of both advections (Theta1 with ab1, Theta^n with ab0) on the u-face and the
// w-face k of the cell
template <class T>
__global__ void k_adj_poly2_c(const PolyAdj<T> P, const Dims d, const PhysT<T> q) {
  const int nx = d.nx, nz = d.nz;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nx * nz) return;
  const int k = c / nx, i = c - k * nx;
  const double iD = (double)q.iD;
  for (int cq = 0; cq < 3; ++cq) P.thb_out[cq][c] += (T)adv2_T<T>(P.ab0[cq], P.U, P.W, d, iD, i, k);
  double gu1, gw1, gu0, gw0;
  const T* const th1[3] = {P.th1[0], P.th1[1], P.th1[2]};
  const T* const th0[3] = {P.th0[0], P.th0[1], P.th0[2]};
  const T* const ab1[3] = {P.ab1[0], P.ab1[1], P.ab1[2]};
  const T* const ab0[3] = {P.ab0[0], P.ab0[1], P.ab0[2]};
  adv2_vel_T<T>(th1, ab1, d, iD, i, k, gu1, gw1);
  adv2_vel_T<T>(th0, ab0, d, iD, i, k, gu0, gw0);
  P.ub[c] += (T)(gu1 + gu0);
  if (k >= 1) P.wb[c] += (T)(gw1 + gw0);
}

}  // namespace pf
