// Batched sweep of independent two-dimensional problems of uneven size in one
// persistent launch per time step.
//
// Every problem advances by the step of Section 3.2 (CH on the fine mesh,
// chemical potential and restriction, NS projection, polymer), split into the
// same passes the single-problem path launches as separate kernels.  The host
// lists (problem, pass, tile) work items pass-major; the persistent kernel's
// CTAs take items in list order from a global counter.  Before running a tile
// of pass s of problem b, a CTA waits until every tile of pass s-1 of problem b
// has been counted done.  Items are taken in list order, so the tiles waited
// for were taken earlier by CTAs that are running: the waits end without any
// co-residency assumption.  Each wait is bounded (a spin budget); when it runs
// out the kernel records PF_ERR_TIMEOUT in a status word and every CTA stops
// taking work, so the launch always returns.
#pragma once
#include "ch_tiled.cuh"
#include "ns_rhs.cuh"
#include "polymer.cuh"
#include "spectral.cuh"

namespace pf {

enum BatchPass {
  BP_CH_RHS = 0, BP_RFFT_F, BP_ZPAIR, BP_IFFT_F, BP_GRES, BP_NSRHS,
  BP_U_RFFT, BP_U_Z, BP_U_IFFT, BP_W_RFFT, BP_W_Z, BP_W_IFFT, BP_DIV,
  BP_P_RFFT, BP_P_Z, BP_P_ZERO, BP_P_IFFT, BP_CORR, BP_POLY1, BP_POLY2, BP_N
};

template <class T>
struct FinePro {
  static constexpr const char* name = "rfft_x_fine";
  const T* a;
  int n;
  __device__ __forceinline__ T operator()(int line, int x) const { return a[(size_t)line * n + x]; }
};
template <class T>
struct PlainEpi {
  static constexpr const char* name = "irfft_x";
  static constexpr int kNPre = 0;
  T* a;
  int n;
  __device__ __forceinline__ void operator()(int line, int x, T v) const { a[(size_t)line * n + x] = v; }
};

// Everything one problem's passes need, resident in device memory.
template <class T>
struct BatchProb {
  Dims d;
  Phys p;
  PhysT<T> q;
  T inv_mldt, inv_ml, div_coef, corr_coef;
  T* phi[2];
  T* philo[2];  // remainders of phi (compensated FP32 storage) or null
  T *u[2], *v[2], *w[2], *pr[2];
  T *R, *ru, *rw, *wt, *pp, *dv;
  double *gwall, *zwork;
  Restricted<T> rs;
  cpx<T> *spF, *spU, *spW, *spP;
  int pF, pC, npairF, npairC, tx;
  FftPlan plFx, plCx;
  const cpx<T> *twFx, *twCx;
  const double *eFx, *eFy, *eCx, *eCy;
  ZSolve zpair, zu, zw, zp;
  NsIn<T> ns[2];        // by flow parity fc
  PolyIn<T> poly[2][2]; // [fc][stage-1]
  int visco;
  int3 gdim[BP_N];
  int ntiles[BP_N];
};

struct BatchItem {
  int prob, pass, tile;
};

template <class T>
__device__ __forceinline__ void batch_run_item(const BatchProb<T>& B, int pass, int tile, unsigned char* sm, int pc,
                                               int fc) {
  const int3 g = B.gdim[pass];
  const int3 bid = make_int3(tile % g.x, (tile / g.x) % g.y, tile / (g.x * g.y));
  const Dims& d = B.d;
  const int po = pc ^ 1, fo = fc ^ 1;
  switch (pass) {
    case BP_CH_RHS: {
      const FineView<T> fv{B.phi[pc], B.phi[po], B.philo[pc], B.philo[po]};
      const CoarseVel<T> vel{B.u[fc], B.u[fo], B.v[fc], B.v[fo], B.w[fc], B.w[fo]};
      k_ch_rhs_b<T, 2>(fv, vel, B.R, B.gwall, d, B.p, B.q, B.inv_mldt, B.inv_ml, bid, sm);
      break;
    }
    case BP_RFFT_F:
      k_rfft_x_b<T, FinePro<T>>(FinePro<T>{B.R, d.fnx}, B.spF, d.fnx, d.fnz, B.pF, B.plFx, B.twFx, B.npairF, bid, sm);
      break;
    case BP_ZPAIR: k_zsolve_b<T, T>(B.spF, B.eFx, B.eFy, B.zpair, B.tx, bid, sm); break;
    case BP_IFFT_F:
      k_irfft_x_b<T, ChFinish<T>>(B.spF, ChFinish<T>{B.phi[pc], B.phi[po], d.fnx, B.philo[pc], B.philo[po]}, d.fnx,
                                  d.fnz, B.pF, B.plFx, B.twFx, B.npairF, (T)1, bid, sm);
      break;
    case BP_GRES:
      if (d.r == 2) k_ch_G_restrict_b<T, 2, 2>(B.phi[po], B.gwall, B.rs, d, B.q, bid, sm);
      else k_ch_G_restrict_b<T, 2, 1>(B.phi[po], B.gwall, B.rs, d, B.q, bid, sm);
      break;
    case BP_NSRHS: k_ns_rhs_v2_b<T, 2>(B.ns[fc], d, B.q, B.ru, B.ru, B.rw, B.visco, bid); break;
    case BP_U_RFFT:
      k_rfft_x_b<T, FinePro<T>>(FinePro<T>{B.ru, d.nx}, B.spU, d.nx, d.nz, B.pC, B.plCx, B.twCx, B.npairC, bid, sm);
      break;
    case BP_U_Z: k_zsolve_b<T, T>(B.spU, B.eCx, B.eCy, B.zu, B.tx, bid, sm); break;
    case BP_U_IFFT:
      k_irfft_x_b<T, IncEpi<T>>(B.spU, IncEpi<T>{B.u[fo], B.u[fc], B.u[fo], d.nx, 0}, d.nx, d.nz, B.pC, B.plCx,
                                B.twCx, B.npairC, (T)1, bid, sm);
      break;
    case BP_W_RFFT:
      k_rfft_x_b<T, FinePro<T>>(FinePro<T>{B.rw, d.nx}, B.spW, d.nx, d.nz - 1, B.pC, B.plCx, B.twCx, B.npairC, bid,
                                sm);
      break;
    case BP_W_Z: k_zsolve_b<T, T>(B.spW, B.eCx, B.eCy, B.zw, B.tx, bid, sm); break;
    case BP_W_IFFT:
      k_irfft_x_b<T, IncEpi<T>>(B.spW, IncEpi<T>{B.wt, B.w[fc], B.w[fo], d.nx, (size_t)d.nx * d.ny}, d.nx, d.nz - 1,
                                B.pC, B.plCx, B.twCx, B.npairC, (T)1, bid, sm);
      break;
    case BP_DIV: k_div_b<T>(B.u[fo], B.v[fo], B.wt, B.dv, d, B.div_coef, (T)(1.0 / d.dx), bid, sm); break;
    case BP_P_RFFT:
      k_rfft_x_b<T, FinePro<T>>(FinePro<T>{B.dv, d.nx}, B.spP, d.nx, d.nz, B.pC, B.plCx, B.twCx, B.npairC, bid, sm);
      break;
    case BP_P_Z: k_zsolve_b<T, T>(B.spP, B.eCx, B.eCy, B.zp, B.tx, bid, sm); break;
    case BP_P_ZERO: k_zero_mode_b<T>(B.spP, d.nz, 1, B.pC, B.zp.h2, B.zp.scale, B.zwork, bid, sm); break;
    case BP_P_IFFT:
      k_irfft_x_b<T, PlainEpi<T>>(B.spP, PlainEpi<T>{B.pp, d.nx}, d.nx, d.nz, B.pC, B.plCx, B.twCx, B.npairC, (T)1,
                                  bid, sm);
      break;
    case BP_CORR:
      k_correct_b<T>(B.u[fo], B.v[fo], B.wt, B.w[fo], B.pp, B.pr[fc], B.pr[fo], d, B.corr_coef, (T)(1.0 / d.dx), bid, sm);
      break;
    case BP_POLY1: k_polymer_b<T, 2>(B.poly[fc][0], d, B.q, 1, bid, sm); break;
    case BP_POLY2: k_polymer_b<T, 2>(B.poly[fc][1], d, B.q, 2, bid, sm); break;
    default: break;
  }
}

// done[prob * BP_N + pass] counts finished tiles; ctl[0] = work head, ctl[1] = status
template <class T>
__global__ void __launch_bounds__(256) k_batch_step(const BatchProb<T>* __restrict__ probs,
                                                    const BatchItem* __restrict__ items, int nitems,
                                                    int* __restrict__ done, int* __restrict__ ctl, int pc, int fc,
                                                    long long spin_limit) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_item, s_stop;
  for (;;) {
    if (threadIdx.x == 0) {
      const int st = *reinterpret_cast<volatile int*>(&ctl[1]);
      s_stop = st != 0;
      s_item = s_stop ? nitems : atomicAdd(&ctl[0], 1);
    }
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const BatchItem w = items[it];
    const BatchProb<T>& B = probs[w.prob];
    if (threadIdx.x == 0 && w.pass > 0) {
      const int need = B.ntiles[w.pass - 1];
      volatile int* cnt = &done[w.prob * BP_N + w.pass - 1];
      long long n = 0;
      while (*cnt < need) {
        if (++n > spin_limit || *reinterpret_cast<volatile int*>(&ctl[1]) != 0) {
          atomicCAS(&ctl[1], 0, PF_ERR_TIMEOUT);
          s_stop = 1;
          break;
        }
        __nanosleep(128);
      }
      __threadfence();
    }
    __syncthreads();
    if (s_stop) break;
    __threadfence();  // acquire side for every thread: see the producers' data, not stale L1 lines
    batch_run_item<T>(B, w.pass, w.tile, smraw, pc, fc);
    __threadfence();  // release side: this thread's results before the count
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&done[w.prob * BP_N + w.pass], 1);
  }
}

}  // namespace pf
