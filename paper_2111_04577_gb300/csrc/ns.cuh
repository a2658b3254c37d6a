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
// The solve is taken for the increment delta = u~ - u*: with L the discrete
// Laplacian with the walls' homogeneous ghosts and k = gamma0/(dt nu_m),
// (L - k) delta = R/nu_m - (L - k) u* (R and its wall-velocity ghost term as
// above), where nu_m lap(u*) cancels against L u* and -u_hat/dt + gamma0 u*/dt
// = (u^n - u^{n-1})/dt.  k_ns_rhs therefore writes
//   [(u^n - u^{n-1})/dt + div(u* u*) + (1/rho) J.grad(u*) + ... - g]/nu_m
// (the terms above less the two), and the inverse transform of the solve adds
// u* back (IncEpi).  The discrete u~ is the same; the working-precision right
// side no longer carries u/dt-sized terms that cancel to the increment.
// Step 2 (Eq. NS37 with coefficient gamma0 rho0/dt): k_div feeds the Neumann
// Poisson solve; step 3 (Eqs. NS38-NS39): k_correct.
#pragma once
#include "ch.cuh"

namespace pf {

// Epilogue of the velocity solves' inverse x transform: out = delta + u*,
// u* = 2 u^n - u^{n-1} read at offset `off` (one plane for the w faces, whose
// solve rows 0..nz-2 hold faces 1..nz-1).  `o` may be `a` itself (u~ lands in
// the u^{n-1} buffer): each element is read before it is written, by one thread.
template <class T>
struct IncEpi {
  static constexpr const char* name = "irfft_x_coarse";
  static constexpr int kNPre = 0;
  T* a;
  const T* n;
  const T* o;
  int nx;
  size_t off;
  __device__ __forceinline__ void operator()(int line, int x, T v) const {
    const size_t i = (size_t)line * nx + x;
    a[i] = v + ((T)2 * n[i + off] - o[i + off]);
  }
};

template <class T>
struct NsIn {
  const T *un, *uo, *vn, *vo, *wn, *wo;   // velocities at n, n-1
  const T *pn, *po;                       // pressure at n, n-1
  const T *tn[6], *to[6];                 // weighted stress comps at n, n-1 (may be null)
  Restricted<T> rs;                       // restricted phi^{n+1}, G^{n+1}
};

// (gamma0 rho0/dt) div(u~) at centres; wt holds faces 1..nz-1 as rows 0..nz-2
template <class T>
__device__ __forceinline__ void k_div_b(const T* __restrict__ ut, const T* __restrict__ vt, const T* __restrict__ wt, T* __restrict__ out, Dims d, T coef, T iD, const int3 bid, unsigned char* smraw) {
  const size_t plane = (size_t)d.nx * d.ny;
  RowIdx x;
  if (!row_index_b(bid, d.nx, d.ny, x)) return;
  {
    const int i = x.i, j = x.j, k = x.k;
    const size_t id = (size_t)x.row * d.nx + i;
    const size_t rowb = id - i;
    T dv = (ut[rowb + wrap(i + 1, d.nx)] - ut[id]) * iD;
    if (d.dim == 3) dv += (vt[((size_t)k * d.ny + wrap(j + 1, d.ny)) * d.nx + i] - vt[id]) * iD;
    const T wtop = (k < d.nz - 1) ? wt[id] : (T)0;              // face k+1 -> row k
    const T wbot = (k > 0) ? wt[id - plane] : (T)0;             // face k   -> row k-1
    dv += (wtop - wbot) * iD;
    out[id] = coef * dv;
  }
}

template <class T>
__global__ void k_div(const T* __restrict__ ut, const T* __restrict__ vt, const T* __restrict__ wt, T* __restrict__ out, Dims d, T coef, T iD) {
  extern __shared__ __align__(16) unsigned char smraw[];
  k_div_b(ut, vt, wt, out, d, coef, iD, make_int3(blockIdx.x, blockIdx.y, blockIdx.z), smraw);
}

// u = u~ - cf grad p', p^{n+1} = p^n + p'.  u, v corrected in place (they hold
// u~ on entry); w written with both walls zero from the face rows wt.
template <class T>
__device__ __forceinline__ void k_correct_b(T* __restrict__ u, T* __restrict__ v, const T* __restrict__ wt, T* __restrict__ w, const T* __restrict__ pp, const T* __restrict__ pn, T* __restrict__ pnew, Dims d, T cf, T iD, const int3 bid, unsigned char* smraw) {
  const size_t plane = (size_t)d.nx * d.ny;
  RowIdx x;
  if (!row_index_b(bid, d.nx, d.ny, x)) return;
  {
    const int i = x.i, j = x.j, k = x.k;
    const size_t id = (size_t)x.row * d.nx + i;
    if (k == 0 || k == d.nz) {
      w[id] = (T)0;
    } else {
      w[id] = wt[id - plane] - cf * (pp[id] - pp[id - plane]) * iD;
    }
    if (k == d.nz) return;
    const size_t rowb = id - i;
    u[id] = u[id] - cf * (pp[id] - pp[rowb + wrap(i - 1, d.nx)]) * iD;
    if (d.dim == 3) v[id] = v[id] - cf * (pp[id] - pp[((size_t)k * d.ny + wrap(j - 1, d.ny)) * d.nx + i]) * iD;
    pnew[id] = pn[id] + pp[id];
  }
}

template <class T>
__global__ void k_correct(T* __restrict__ u, T* __restrict__ v, const T* __restrict__ wt, T* __restrict__ w, const T* __restrict__ pp, const T* __restrict__ pn, T* __restrict__ pnew, Dims d, T cf, T iD) {
  extern __shared__ __align__(16) unsigned char smraw[];
  k_correct_b(u, v, wt, w, pp, pn, pnew, d, cf, iD, make_int3(blockIdx.x, blockIdx.y, blockIdx.z), smraw);
}

// The same update, each thread walking kz layers of its (i, j) column: p' of
// the layer below stays in a register for the w correction.  blockIdx.x =
// (z chunk, j), blockIdx.y = x block.  Same arithmetic per face as k_correct_b.
template <class T>
__global__ void k_correct_z(T* __restrict__ u, T* __restrict__ v, const T* __restrict__ wt, T* __restrict__ w,
                            const T* __restrict__ pp, const T* __restrict__ pn, T* __restrict__ pnew, Dims d, T cf,
                            T iD, int kz) {
  const int i = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= d.nx) return;
  const int j = blockIdx.x % d.ny, k0 = (blockIdx.x / d.ny) * kz;
  const size_t plane = (size_t)d.nx * d.ny;
  const int im = wrap(i - 1, d.nx);
  const size_t col = (size_t)j * d.nx, colm = (size_t)wrap(j - 1, d.ny) * d.nx;
  T pbelow = k0 > 0 ? pp[(size_t)(k0 - 1) * plane + col + i] : (T)0;
  const int k1 = min(k0 + kz, d.nz + 1);
  for (int k = k0; k < k1; ++k) {
    const size_t id = (size_t)k * plane + col + i;
    if (k == d.nz) {
      w[id] = (T)0;
      break;
    }
    const T pc = pp[id];
    w[id] = k == 0 ? (T)0 : wt[id - plane] - cf * (pc - pbelow) * iD;
    u[id] = u[id] - cf * (pc - pp[(size_t)k * plane + col + im]) * iD;
    if (d.dim == 3) v[id] = v[id] - cf * (pc - pp[(size_t)k * plane + colm + i]) * iD;
    pnew[id] = pn[id] + pc;
    pbelow = pc;
  }
}

}  // namespace pf
