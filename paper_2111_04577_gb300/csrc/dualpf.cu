// Step orchestrator and C ABI of the dual-resolution phase-field library.
//
// A context owns every field of the coupled problem on one GPU, the spectral
// work arrays of the fine Cahn-Hilliard solves and of the coarse
// Navier-Stokes solves, the FFT twiddles and eigenvalues, and one CUDA graph
// per (phase parity, flow parity, flags) that replays a whole time step in the
// order of Section 3.2: CH on the fine mesh (Eqs. dual1, NS25-NS34), the
// chemical potential and restriction (Eqs. NS5, dual2, dual3), the NS
// projection step (Eqs. NS35-NS39) and the polymer (Eqs. NS40-NS46).  Time
// levels rotate by pointer parity, never by copies.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "../../include/dualpf.h"
#include "ch.cuh"
#include "ch_tiled.cuh"
#include "ch_march.cuh"
#include "zsolve_seg.cuh"
#include "fft_reg.cuh"
#include "ns.cuh"
#include "ns_rhs.cuh"
#include "ns_march.cuh"
#include "polymer.cuh"
#include "reduce.cuh"
#include "spectral.cuh"
#include "batch.cuh"
#include "adjoint.cuh"
#include "adjoint_ns.cuh"
#include "robin.cuh"

namespace pf {

struct ApiError : std::runtime_error {
  int code;
  ApiError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

static bool smooth(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

static FftPlan make_plan(int n) {
  FftPlan pl{};
  pl.n = n;
  int m = n;
  std::vector<int> r;
  while (m % 4 == 0) { r.push_back(4); m /= 4; }
  while (m % 2 == 0) { r.push_back(2); m /= 2; }
  for (int p : {3, 5, 7})
    while (m % p == 0) { r.push_back(p); m /= p; }
  if (m != 1 || r.size() > 21) throw ApiError(PF_ERR_UNSUPPORTED, "FFT length " + std::to_string(n) + " is not 2^a 3^b 5^c 7^d");
  pl.ns = (int)r.size();
  pl.code = 0;
  for (size_t i = 0; i < r.size(); ++i) pl.code |= (unsigned long long)r[i] << (3 * i);
  return pl;
}

// ---------------------------------------------------------------------------
// device memory registry
// ---------------------------------------------------------------------------
struct Arena {
  std::vector<void*> ptrs;
  size_t total = 0;
  template <class X>
  X* get(size_t count) {
    if (count == 0) count = 1;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(X));
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw ApiError(PF_ERR_NOMEM, "cudaMalloc of " + std::to_string(count * sizeof(X)) + " bytes failed");
    }
    PF_CUDA_TRY(cudaMemset(p, 0, count * sizeof(X)));
    ptrs.push_back(p);
    total += count * sizeof(X);
    return static_cast<X*>(p);
  }
  ~Arena() {
    for (void* p : ptrs) cudaFree(p);
  }
};

// producers / consumers for the x transforms of plain arrays
template <class T>
struct ArrPro {
  static constexpr const char* name = "rfft_x_coarse";
  const T* a;
  int n;
  __device__ __forceinline__ T operator()(int line, int x) const { return a[(size_t)line * n + x]; }
};
// The Poisson right side coef * div(u~) of Eq. NS37 produced on the fly for the
// pressure solve's x transform (same arithmetic as k_div, no stored array).
template <class T>
struct DivPro {
  static constexpr const char* name = "div_rfft_x_coarse";
  const T *ut, *vt, *wt;
  Dims d;
  T coef, iD;
  __device__ __forceinline__ T operator()(int line, int i) const {
    const int k = line / d.ny, j = line - k * d.ny;
    const size_t plane = (size_t)d.nx * d.ny;
    const size_t id = (size_t)line * d.nx + i;
    const size_t rowb = id - i;
    T dv = (ut[rowb + (i + 1 == d.nx ? 0 : i + 1)] - ut[id]) * iD;
    if (d.dim == 3) dv += (vt[((size_t)k * d.ny + (j + 1 == d.ny ? 0 : j + 1)) * d.nx + i] - vt[id]) * iD;
    const T wtop = (k < d.nz - 1) ? wt[id] : (T)0;   // face k+1 -> row k
    const T wbot = (k > 0) ? wt[id - plane] : (T)0;  // face k   -> row k-1
    dv += (wtop - wbot) * iD;
    return coef * dv;
  }
};

template <class T>
struct FineArrPro {
  static constexpr const char* name = "rfft_x_fine";
  const T* a;
  int n;
  __device__ __forceinline__ T operator()(int line, int x) const { return a[(size_t)line * n + x]; }
};
template <class T>
struct ArrEpi {
  static constexpr const char* name = "irfft_x_coarse";
  static constexpr int kNPre = 0;
  T* a;
  int n;
  __device__ __forceinline__ void operator()(int line, int x, T v) const { a[(size_t)line * n + x] = v; }
};

struct ImplBase {
  pf_params raw_prm{};  // the parameters as last given to pf_set_params
  virtual ~ImplBase() {}
  virtual const pf_grid_desc& grid_desc() const = 0;
  virtual bool params_ready() const = 0;
  virtual void set_params(const pf_params& prm) = 0;
  virtual void field_info(int f, size_t* count, size_t* eb) const = 0;
  virtual void set_field(int f, const void* src, size_t bytes, int on_dev) = 0;
  virtual void get_field(int f, void* dst, size_t bytes, int on_dev) = 0;
  virtual void step(int nsteps, int flags) = 0;
  virtual void diagnostics(double out[6]) = 0;
  virtual void profile(int nsteps, int flags, std::vector<std::string>& names, std::vector<double>& ms,
                       std::vector<int>& counts, int& per_step) = 0;
  virtual void set_tuning(int knob, int value) = 0;
  virtual void adjoint(int nsteps, int K, int which, double out[3], void* dphi0, int on_dev) = 0;
  virtual void adjoint_coupled(int nsteps, int K, int which, double out[4], void* dphi0, int on_dev) = 0;
  virtual int get_tuning(int knob) const = 0;
};

static Phys derive(const pf_params& q, const pf_grid_desc& g) {
  if (!(q.rho1 > 0 && q.rho2 > 0 && q.sigma > 0 && q.eta > 0 && q.mobility > 0 && q.dt > 0 && q.mu1 >= 0 &&
        q.mu2 >= 0))
    throw ApiError(PF_ERR_ARG, "rho1, rho2, sigma, eta, mobility, dt must be > 0 and mu1, mu2 >= 0");
  if (q.theta_bot_deg < 0 || q.theta_bot_deg > 180 || q.theta_top_deg < 0 || q.theta_top_deg > 180)
    throw ApiError(PF_ERR_ARG, "contact angles must lie in [0, 180] degrees");
  if (!(q.dw >= 0.0)) throw ApiError(PF_ERR_ARG, "the wall relaxation D_w must be >= 0");
  if (!(q.alpha_giesekus >= 0.0 && q.alpha_giesekus < 1.0))
    throw ApiError(PF_ERR_ARG, "the Giesekus mobility must lie in [0, 1)");
  Phys p{};
  p.dt = q.dt;
  p.gamma0 = 1.5;
  p.eta = q.eta;
  p.lam = 3.0 * q.sigma * q.eta / (2.0 * std::sqrt(2.0));            // Eq. NS7
  p.mob = q.mobility;
  p.Ml = p.mob * p.lam;
  const double smin = q.eta * q.eta * std::sqrt(4.0 * p.gamma0 / (p.Ml * q.dt));  // Eq. NS30
  const double S = q.S > 0 ? q.S : smin;
  if (S < smin * (1.0 - 1e-12)) throw ApiError(PF_ERR_DISCRIMINANT, "S is below the bound of Eq. NS30");
  double disc = 1.0 - 4.0 * p.gamma0 * std::pow(q.eta, 4) / (p.Ml * q.dt * S * S);
  if (disc < 0) disc = 0;
  p.S = S;
  p.alpha = -S / (2.0 * q.eta * q.eta) * (1.0 + std::sqrt(disc));     // Eq. NS29
  p.c = p.alpha + S / (q.eta * q.eta);
  p.cos_bot = std::cos(q.theta_bot_deg * M_PI / 180.0);
  p.cos_top = std::cos(q.theta_top_deg * M_PI / 180.0);
  if (q.advection != 0 && q.advection != 1)
    throw ApiError(PF_ERR_ARG, "advection must be 0 (central) or 1 (WENO5-Z)");
  if (q.advection == 1 && (g.nx < 4 || g.nz < 4 || (g.ny > 1 && g.ny < 4)))
    throw ApiError(PF_ERR_ARG, "WENO5-Z advection needs at least 4 coarse cells along every axis");
  if (q.polymer_approach != 0 && q.polymer_approach != 1)
    throw ApiError(PF_ERR_ARG, "polymer_approach must be 0 (Eq. NS12) or 1 (Eq. NS11)");
  p.approach1 = q.polymer_approach;
  p.weno = q.advection;
  p.dw = q.dw;
  p.kappa = q.dw * p.gamma0 / q.dt;  // implicit wall coefficient of Eq. NS34
  double beta;
  if (p.approach1) {
    if (!(q.beta > 0 && q.beta <= 1.0) || !(q.mu_p2 >= 0))
      throw ApiError(PF_ERR_ARG, "approach 1 needs beta in (0, 1] and mu_p2 >= 0");
    p.visco = ((q.beta < 1.0 && q.mu1 > 0) || q.mu_p2 > 0) ? 1 : 0;
    if (p.visco && !(q.wi > 0 && q.wi2 > 0))
      throw ApiError(PF_ERR_ARG, "approach 1 needs both relaxation times wi, wi2 > 0");
    if (!(q.alpha_giesekus2 >= 0.0 && q.alpha_giesekus2 < 1.0))
      throw ApiError(PF_ERR_ARG, "the Giesekus mobility must lie in [0, 1)");
    beta = q.beta;
    p.mu_p2 = q.mu_p2;
    p.lam_h2 = q.wi2;
    p.alpha_g2 = q.alpha_giesekus2;
  } else {
    p.visco = (q.wi > 0 && q.beta < 1.0) ? 1 : 0;
    beta = p.visco ? q.beta : 1.0;
  }
  p.rho1 = q.rho1;
  p.rho2 = q.rho2;
  p.rho0 = std::min(q.rho1, q.rho2);
  p.mu_s1 = beta * q.mu1;
  p.mu_p1 = (1.0 - beta) * q.mu1;
  p.mu_s2 = q.mu2;
  p.lam_h = q.wi;
  p.alpha_g = q.alpha_giesekus;
  p.nu_m = q.nu_m > 0 ? q.nu_m : 0.5 * std::max(p.mu_s1, p.mu_s2) / p.rho0;
  if (!(p.nu_m > 0)) throw ApiError(PF_ERR_ARG, "nu_m must be > 0 (give a viscosity)");
  p.uw_bot = q.uw_bot;
  p.uw_top = q.uw_top;
  p.gx = q.gx;
  p.gy = q.gy;
  p.gz = q.gz;
  return p;
}

template <class T, class TC>
struct Impl : ImplBase {
  pf_grid_desc g;
  Dims d{};
  Phys p{};
  PhysT<T> q{};
  // derivatives, with respect to one parameter, of constants the step forms on
  // the host (nonzero only in a derivative-carrying step seeded with it)
  struct {
    double inv_mldt = 0, inv_ml = 0, c = 0, alpha = 0;
  } dseed;
  double sigma = 1.0;
  double prm_S = 0.0;  // S as given (0: the Eq. NS30 minimum, which moves with M)
  bool have_params = false;
  cudaStream_t st;
  Arena ar;
  int ncomp;
  // fields
  T *phi[2], *u[2], *v[2], *w[2], *pr[2];
  // FP32 contexts: the rounding remainders of phi at both parities (compensated
  // storage, phi = phi + philo to about 2^-48 relative); null otherwise
  T* philo[2] = {nullptr, nullptr};
  T *theta[6], *theta1[6], *tau[2][6];
  T *mu, *G;
  Wide<T>* gwall;  // contact-line flux g of both walls (FP64; Dual when derivatives are carried)
  Restricted<T> rs{};
  T *ru, *rv, *rw, *wt, *pp, *dv;
  cpx<T> *spF, *spU, *spV, *spW, *spP;
  int pF, pC;
  FftPlan plFx, plFy, plCx, plCy;
  cpx<T> *twFx, *twFy, *twCx, *twCy;
  double *eFx, *eFy, *eCx, *eCy;
  float *k2F = nullptr, *k2C = nullptr;  // FP32 eliminations: -(lambda_x + lambda_y) per mode
  Wide<T>* zwork;
  double* partial;
  Wide<T>* wpartial;  // diagnostics partial sums
  int nred_blocks = 0;
  int pc = 0, fc = 0;  // parities: phi^n = phi[pc]; u^n = u[fc], ...
  std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;
  long long steps_done = 0;
  // tuning knobs (pf_set_tuning); 0 = built-in default
  int tune[PF_TUNE_COUNT] = {0};
  // per-kernel timing (pf_profile): one event before every launch of a step
  bool prof = false;
  int nlaunch = 0;
  std::vector<const char*> mark_names;
  std::vector<cudaEvent_t> mark_ev;
  void mark(const char* name) {
    ++nlaunch;
    if (!prof) return;
    const size_t i = mark_names.size();
    if (i >= mark_ev.size()) {
      cudaEvent_t e;
      PF_CUDA_TRY(cudaEventCreate(&e));
      mark_ev.push_back(e);
    }
    PF_CUDA_TRY(cudaEventRecord(mark_ev[i], st));
    mark_names.push_back(name);
  }

  Impl(const pf_grid_desc& gd, cudaStream_t s) : g(gd), st(s) {
    d.nx = g.nx;
    d.ny = g.ny;
    d.nz = g.nz;
    d.dim = g.ny == 1 ? 2 : 3;
    d.r = g.dual ? 2 : 1;
    d.ry = d.dim == 3 ? d.r : 1;
    d.rs = d.r == 2 ? 1 : 0;
    d.rys = d.ry == 2 ? 1 : 0;
    d.fnx = d.r * g.nx;
    d.fny = d.ry * g.ny;
    d.fnz = d.r * g.nz;
    d.dx = g.lx / g.nx;
    d.h = d.dx / d.r;
    ncomp = d.dim == 2 ? 3 : 6;
    if (zsolve_cols(std::max(d.fnz, d.nz + 1), true) == 0)
      throw ApiError(PF_ERR_UNSUPPORTED, "z lines too long for the segmented z solve (at most 4096 rows)");
    const size_t nf = (size_t)d.fnx * d.fny * d.fnz;
    const size_t nc = (size_t)d.nx * d.ny * d.nz;
    const size_t ncw = (size_t)d.nx * d.ny * (d.nz + 1);
    for (int q = 0; q < 2; ++q) {
      phi[q] = ar.get<T>(nf);
      if constexpr (std::is_same<T, float>::value) philo[q] = ar.get<T>(nf);
      u[q] = ar.get<T>(nc);
      v[q] = d.dim == 3 ? ar.get<T>(nc) : ar.get<T>(1);
      w[q] = ar.get<T>(ncw);
      pr[q] = ar.get<T>(nc);
      for (int c = 0; c < 6; ++c) tau[q][c] = c < ncomp ? ar.get<T>(nc) : nullptr;
    }
    for (int c = 0; c < 6; ++c) {
      theta[c] = c < ncomp ? ar.get<T>(nc) : nullptr;
      theta1[c] = c < ncomp ? ar.get<T>(nc) : nullptr;
    }
    mu = ar.get<T>(nf);
    G = ar.get<T>(nf);
    gwall = ar.get<Wide<T>>(2 * (size_t)d.fnx * d.fny);
    rs.phic = ar.get<T>(nc);
    rs.Gc = ar.get<T>(nc);
    rs.phifx = ar.get<T>(nc);
    rs.Gfx = ar.get<T>(nc);
    rs.phify = d.dim == 3 ? ar.get<T>(nc) : rs.phifx;
    rs.Gfy = d.dim == 3 ? ar.get<T>(nc) : rs.Gfx;
    rs.phifz = ar.get<T>(ncw);
    rs.Gfz = ar.get<T>(ncw);
    rs.phiexz = ar.get<T>(ncw);
    rs.phiexy = d.dim == 3 ? ar.get<T>(nc) : rs.phic;
    rs.phieyz = d.dim == 3 ? ar.get<T>(ncw) : rs.phifz;
    ru = ar.get<T>(nc);
    rv = ar.get<T>(nc);
    rw = ar.get<T>(nc);
    wt = ar.get<T>(nc);
    pp = ar.get<T>(nc);
    dv = ar.get<T>(nc);
    pF = ((d.fnx / 2 + 1) + 1) & ~1;
    pC = ((d.nx / 2 + 1) + 1) & ~1;
    spF = ar.get<cpx<T>>((size_t)pF * d.fny * d.fnz);
    spU = ar.get<cpx<T>>((size_t)pC * d.ny * d.nz);
    spV = d.dim == 3 ? ar.get<cpx<T>>((size_t)pC * d.ny * d.nz) : spU;
    spW = ar.get<cpx<T>>((size_t)pC * d.ny * d.nz);
    spP = ar.get<cpx<T>>((size_t)pC * d.ny * d.nz);
    plFx = make_plan(d.fnx);
    plCx = make_plan(d.nx);
    plFy = make_plan(d.fny);
    plCy = make_plan(d.ny);
    twFx = twiddles(d.fnx);
    twFy = twiddles(d.fny);
    twCx = twiddles(d.nx);
    twCy = twiddles(d.ny);
    {
      const auto hFx = eig_host(d.fnx, d.h, d.fnx / 2 + 1);
      const auto hFy = d.dim == 3 ? eig_host(d.fny, d.h, d.fny) : eig_host(1, d.h, 1);
      const auto hCx = eig_host(d.nx, d.dx, d.nx / 2 + 1);
      const auto hCy = d.dim == 3 ? eig_host(d.ny, d.dx, d.ny) : eig_host(1, d.dx, 1);
      eFx = upload(hFx);
      eFy = upload(hFy);
      eCx = upload(hCx);
      eCy = upload(hCy);
      if (std::is_same<TC, float>::value) {
        k2F = k2_table(hFx, hFy);
        k2C = k2_table(hCx, hCy);
      }
    }
    zwork = ar.get<Wide<T>>(4 * (size_t)(d.nz + 2));
    nred_blocks = 2 * 152;
    partial = ar.get<double>((size_t)nred_blocks * RED_N);
    wpartial = std::is_same<Wide<T>, double>::value ? reinterpret_cast<Wide<T>*>(partial)
                                                    : ar.get<Wide<T>>((size_t)nred_blocks * RED_N);
    set_smem_limits();
  }

  ~Impl() override {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    for (auto e : mark_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : {ev_fork, ev_join, ev_ns, ev_v, ev_w, ev_z0, ev_z1})
      if (e) cudaEventDestroy(e);
    for (cudaStream_t x : {st2, st3, st4})
      if (x) cudaStreamDestroy(x);
  }

  // The polymer update of step n needs u^{n+1}, Theta and the restricted phi
  // only, so pf_step runs it during step n+1's CH transform chain on a second
  // stream (joined before the restriction overwrites the restricted phi); the
  // last one of a call is run at the end of the call.  Every update sees the
  // same inputs as in the sequential order.
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool poly_pending = false;  // the update for the velocity in parity fc is owed
  // the coarse velocity solves (u, v, w: independent chains) also run on three
  // streams; st3 and the events below serve that fork/join
  cudaStream_t st3 = nullptr;
  cudaEvent_t ev_ns = nullptr, ev_v = nullptr, ev_w = nullptr;
  // the pressure's mean mode is solved on st3 beside the other columns
  cudaEvent_t ev_z0 = nullptr, ev_z1 = nullptr;
  cudaStream_t st4 = nullptr;  // the w velocity solve
  void ensure_side_stream() {
    if (st2) return;
    PF_CUDA_TRY(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
    PF_CUDA_TRY(cudaStreamCreateWithFlags(&st3, cudaStreamNonBlocking));
    PF_CUDA_TRY(cudaStreamCreateWithFlags(&st4, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&ev_fork, &ev_join, &ev_ns, &ev_v, &ev_w, &ev_z0, &ev_z1})
      PF_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  // launches issued while alive go to stream s (the launchers use the member st)
  struct OnStream {
    cudaStream_t& ref;
    cudaStream_t saved;
    OnStream(cudaStream_t& r, cudaStream_t s) : ref(r), saved(r) { ref = s; }
    ~OnStream() { ref = saved; }
  };
  // both LCR stages for the velocity in parity fv (tau written to parity fv)
  void launch_polymer(int fv, cudaStream_t s) {
    PolyIn<T> P{};
    P.u = u[fv];
    P.v = v[fv];
    P.w = w[fv];
    P.phic = rs.phic;
    for (int c = 0; c < ncomp; ++c) {
      P.th[c] = theta[c];
      P.out[c] = theta1[c];
    }
    mark("polymer_stage1");
    const RowLaunch lp = rows(d.ny * d.nz, d.nx, 128);
    if (d.dim == 2) k_polymer<T, 2, 1><<<lp.grid, lp.block, 0, s>>>(P, d, q);
    else k_polymer<T, 3, 1><<<lp.grid, lp.block, 0, s>>>(P, d, q);
    for (int c = 0; c < ncomp; ++c) {
      P.th[c] = theta1[c];
      P.base[c] = theta[c];
      P.out[c] = theta[c];
      P.tau[c] = tau[fv][c];
    }
    mark("polymer_stage2");
    if (d.dim == 2) k_polymer<T, 2, 2><<<lp.grid, lp.block, 0, s>>>(P, d, q);
    else k_polymer<T, 3, 2><<<lp.grid, lp.block, 0, s>>>(P, d, q);
  }
  void flush_polymer() {
    if (!poly_pending) return;
    poly_pending = false;
    launch_polymer(fc, st);
    check_launch();
  }

  cpx<T>* twiddles(int n) {
    std::vector<cpx<T>> h(n);
    for (int m = 0; m < n; ++m) {
      const double a = 2.0 * M_PI * (double)m / (double)n;
      h[m] = mk<T>((T)std::cos(a), (T)-std::sin(a));
    }
    cpx<T>* dptr = ar.get<cpx<T>>(n);
    PF_CUDA_TRY(cudaMemcpy(dptr, h.data(), n * sizeof(cpx<T>), cudaMemcpyHostToDevice));
    return dptr;
  }
  std::vector<double> eig_host(int n, double hh, int count) {
    std::vector<double> h(count);
    for (int k = 0; k < count; ++k) {
      const double s = std::sin(M_PI * (double)k / (double)n);
      h[k] = -4.0 / (hh * hh) * s * s;
    }
    return h;
  }
  double* upload(const std::vector<double>& h) {
    double* dptr = ar.get<double>(h.size());
    PF_CUDA_TRY(cudaMemcpy(dptr, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
    return dptr;
  }
  // [ny][ncol] floats -(lambda_x + lambda_y), the rounding the FP32 elimination applied to
  // the same FP64 sum on the device
  float* k2_table(const std::vector<double>& hx, const std::vector<double>& hy) {
    std::vector<float> t(hx.size() * hy.size());
    for (size_t j = 0; j < hy.size(); ++j)
      for (size_t c = 0; c < hx.size(); ++c) t[j * hx.size() + c] = (float)(-(hx[c] + hy[j]));
    float* dptr = ar.get<float>(t.size());
    PF_CUDA_TRY(cudaMemcpy(dptr, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice));
    return dptr;
  }

  static constexpr int kMaxSmem = 200 * 1024;
  void set_smem_limits() {
    PF_CUDA_TRY(cudaFuncSetAttribute(k_fft_y<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_zsolve_seg<T, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_rfft_x<T, ArrPro<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_rfft_x<T, DivPro<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_rfft_x<T, FineArrPro<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_rhs<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_rhs<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_rhs_march<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_rhs_march<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    if constexpr (std::is_same<T, float>::value) {
      PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_rhs_march4<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
      PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_rhs_march4<1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
      PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_rhs_march4<1, 4, false, 14>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
      // four 55.3 KB CTAs per SM need the whole shared-memory carveout
      PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_rhs_march4<1, 4, false, 14>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared));
      PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_rhs_march4<0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
      PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_rhs_march4<1, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
      PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_rhs_march4<0, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    }
    PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_G_restrict_march<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_ns_rhs_march3<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_ns_rhs_march3<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_zero_mode_smem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    for (int n : {64, 128, 256, 512, 1024})
      reg_fft_dispatch(n, [&](auto NN) {
        constexpr int N = decltype(NN)::value;
        PF_CUDA_TRY(cudaFuncSetAttribute(k_rfft_x_reg<T, N, FineArrPro<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
        PF_CUDA_TRY(cudaFuncSetAttribute(k_rfft_x_reg<T, N, ArrPro<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
        PF_CUDA_TRY(cudaFuncSetAttribute(k_rfft_x_reg<T, N, DivPro<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
        PF_CUDA_TRY(cudaFuncSetAttribute(k_irfft_x_reg<T, N, ChFinish<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
        PF_CUDA_TRY(cudaFuncSetAttribute(k_irfft_x_reg<T, N, ArrEpi<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
        PF_CUDA_TRY(cudaFuncSetAttribute(k_irfft_x_reg<T, N, IncEpi<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
        PF_CUDA_TRY(cudaFuncSetAttribute(k_fft_y_reg<T, N, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
      });
    PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_G_restrict<T, 2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_G_restrict<T, 2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_G_restrict<T, 3, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_ch_G_restrict<T, 3, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_irfft_x<T, ChFinish<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_irfft_x<T, ArrEpi<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PF_CUDA_TRY(cudaFuncSetAttribute(k_irfft_x<T, IncEpi<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
  }

  // ------------------------------------------------------------------ launches
  // row grids: blockIdx.x = row, (blockIdx.y, threadIdx.x) = x
  struct RowLaunch {
    dim3 grid, block;
  };
  RowLaunch rows(int nrows, int nxrow, int maxbs = 256) const {
    if (tune[PF_TUNE_ROW_BLOCK] > 0) maxbs = std::min(maxbs, tune[PF_TUNE_ROW_BLOCK]);
    int bs = ((nxrow + 31) / 32) * 32;
    if (bs > maxbs) bs = maxbs;
    RowLaunch r;
    r.block = dim3(bs);
    r.grid = dim3(nrows, (nxrow + bs - 1) / bs);
    return r;
  }
  // line pairs per CTA of the register-resident x transforms (NT = n/8 threads a line)
  int reg_lpc(int n) const {
    const int nt = n / 8;
    const int want = tune[PF_TUNE_XFFT_PAIRS] > 0 ? tune[PF_TUNE_XFFT_PAIRS] : std::max(1, 256 / nt);
    return std::max(1, std::min(want, 1024 / nt));
  }
  template <class Pro>
  void rfft_x(Pro pro, cpx<T>* out, int n, int nlines, int pitch, const FftPlan& pl, const cpx<T>* tw) {
    if (reg_fft_size(n)) {
      int lpc = reg_lpc(n);
      const int pairs = (nlines + 1) / 2;
      while (lpc > 1 && (size_t)lpc * fft_pad_len(n) * sizeof(cpx<T>) > (size_t)kMaxSmem) lpc /= 2;
      const size_t sm = (size_t)lpc * fft_pad_len(n) * sizeof(cpx<T>);
      mark(Pro::name);
      reg_fft_dispatch(n, [&](auto NN) {
        constexpr int N = decltype(NN)::value;
        k_rfft_x_reg<T, N, Pro><<<(pairs + lpc - 1) / lpc, lpc * (N / 8), sm, st>>>(pro, out, nlines, pitch, tw);
      });
      return;
    }
    const int npair = tune[PF_TUNE_XFFT_PAIRS] > 0 ? tune[PF_TUNE_XFFT_PAIRS] : std::max(1, 1024 / n);
    const int pairs = (nlines + 1) / 2;
    const int grid = (pairs + npair - 1) / npair;
    const size_t sm = 2 * (size_t)npair * n * sizeof(cpx<T>);
    mark(Pro::name);
    k_rfft_x<T, Pro><<<grid, 256, sm, st>>>(pro, out, n, nlines, pitch, pl, tw, npair);
  }
  template <class Epi>
  void irfft_x(const cpx<T>* in, Epi epi, int n, int nlines, int pitch, const FftPlan& pl, const cpx<T>* tw, T scale) {
    if (reg_fft_size(n)) {
      int lpc = reg_lpc(n);
      const int pairs = (nlines + 1) / 2;
      const size_t per_line = (size_t)n * (sizeof(cpx<T>) + 2 * Epi::kNPre * sizeof(T));
      while (lpc > 1 && (size_t)lpc * per_line > (size_t)kMaxSmem) lpc /= 2;
      const size_t sm = (size_t)lpc * per_line;
      mark(Epi::name);
      reg_fft_dispatch(n, [&](auto NN) {
        constexpr int N = decltype(NN)::value;
        k_irfft_x_reg<T, N, Epi><<<(pairs + lpc - 1) / lpc, lpc * (N / 8), sm, st>>>(in, epi, nlines, pitch, tw, scale);
      });
      return;
    }
    const int npair = tune[PF_TUNE_XFFT_PAIRS] > 0 ? tune[PF_TUNE_XFFT_PAIRS] : std::max(1, 1024 / n);
    const int pairs = (nlines + 1) / 2;
    const int grid = (pairs + npair - 1) / npair;
    const size_t sm = irfft_x_smem<T, Epi>(n, npair);
    mark(Epi::name);
    k_irfft_x<T, Epi><<<grid, 256, sm, st>>>(in, epi, n, nlines, pitch, pl, tw, npair, scale);
  }
  void fft_y(cpx<T>* data, int ny, int pitch, int ncol, int levels, const FftPlan& pl, const cpx<T>* tw, int sign) {
    if (reg_fft_size(ny)) {
      constexpr int E = 16;  // elements a thread: 16-column tiles read 128-byte rows
      const int nt = ny / E;
      const int want = tune[PF_TUNE_YFFT_COLS] > 0 ? tune[PF_TUNE_YFFT_COLS] : 16;
      int txc = std::max(1, std::min(want, 512 / nt));
      const size_t line = (size_t)fft_pad_len(ny) * sizeof(cpx<T>);
      while (txc > 1 && (size_t)txc * line > (size_t)kMaxSmem) txc /= 2;  // wide elements (Dual)
      const size_t sm = (size_t)txc * line;
      mark(ny == d.fny && levels == d.fnz && d.r > 1 ? "fft_y_fine" : "fft_y_coarse");
      reg_fft_dispatch(ny, [&](auto NN) {
        constexpr int N = decltype(NN)::value;
        k_fft_y_reg<T, N, E><<<dim3((ncol + txc - 1) / txc, levels), txc * (N / E), sm, st>>>(data, pitch, ncol, tw, sign);
      });
      return;
    }
    const int tx = tune[PF_TUNE_YFFT_COLS] > 0 ? tune[PF_TUNE_YFFT_COLS] : (sizeof(T) == 4 ? 8 : 4);
    dim3 grid((ncol + tx - 1) / tx, levels);
    const size_t sm = 2 * (size_t)ny * tx * sizeof(cpx<T>);
    mark(ny == d.fny && levels == d.fnz && d.r > 1 ? "fft_y_fine" : "fft_y_coarse");
    k_fft_y<T><<<grid, 256, sm, st>>>(data, ny, pitch, ncol, pl, tw, sign, tx);
  }
  // kx columns per CTA of a z solve over `rows` rows: the tuned (else 16)
  // count, halved until the CTA's threads (two per column and segment, at most
  // 512) and its shared memory fit; 0 if not even one column fits
  int zsolve_cols(int rows, bool dual) const {
    const int nseg = (rows + ZSEG - 1) / ZSEG;
    for (int t = tune[PF_TUNE_ZSOLVE_COLS] > 0 ? tune[PF_TUNE_ZSOLVE_COLS] : 16; t >= 1; t >>= 1)
      if (2 * t * nseg <= 512 && zsolve_seg_smem<TC>(rows, t, dual) <= (size_t)kMaxSmem) return t;
    return 0;
  }

  void zsolve(cpx<T>* data, int rows, int ny, int pitch, int ncol, const double* ex, const double* ey, int bc,
              double h2, double s1, double s2, bool two, double scale, bool poisson, double ds1 = 0.0,
              double ds2 = 0.0) {
    ZSolve zs{};
    zs.rows = rows;
    zs.ny = ny;
    zs.pitch = pitch;
    zs.ncol = ncol;
    zs.bc = bc;
    zs.two = two ? 1 : 0;
    zs.same = (!two || (std::fabs(s1 - s2) <= 1e-14 * std::fabs(s1) && ds1 == ds2)) ? 1 : 0;
    zs.skip_zero = poisson ? 1 : 0;
    zs.h2 = h2;
    zs.shift1 = s1;
    zs.shift2 = s2;
    zs.dshift1 = ds1;
    zs.dshift2 = ds2;
    zs.scale = scale;
    zs.k2f = ex == eFx ? k2F : (ex == eCx ? k2C : nullptr);  // null unless the elimination is FP32
    zs.h2f = (float)h2;
    zs.s1f = (float)s1;
    zs.s2f = (float)s2;
    zs.rsf = (float)(h2 * scale);
    // the mean mode (kx = ky = 0) of the pressure has its own solve, which the
    // column solve skips; outside pf_profile it runs on st3 at the same time
    auto zero_mode = [&]() {
      mark("zero_mode");
      if ((size_t)2 * rows * sizeof(Wide<T>) <= (size_t)kMaxSmem)
        k_zero_mode_smem<T><<<1, 256, 2 * rows * sizeof(Wide<T>), st>>>(data, rows, ny, pitch, h2, scale);
      else
        k_zero_mode<T><<<1, 32, 0, st>>>(data, rows, ny, pitch, h2, scale, zwork);
    };
    const bool zside = poisson && !prof && st3 != nullptr;
    if (zside) {
      PF_CUDA_TRY(cudaEventRecord(ev_z0, st));
      PF_CUDA_TRY(cudaStreamWaitEvent(st3, ev_z0, 0));
      {
        OnStream on(st, st3);
        zero_mode();
      }
      PF_CUDA_TRY(cudaEventRecord(ev_z1, st3));
    }
    mark(two ? "zsolve_pair" : "zsolve");
    const int txs = zsolve_cols(rows, two && !zs.same);
    const int nseg = (rows + ZSEG - 1) / ZSEG;
    dim3 grid((ncol + txs - 1) / txs, ny);
    k_zsolve_seg<T, TC><<<grid, 2 * txs * nseg, zsolve_seg_smem<TC>(rows, txs, two && !zs.same), st>>>(data, ex, ey, zs, txs);
    if (zside) PF_CUDA_TRY(cudaStreamWaitEvent(st, ev_z1, 0));
    else if (poisson) zero_mode();
  }

  // one transform solve on the coarse mesh: rhs (real, lines of nx) -> out
  void coarse_solve(const T* rhs, T* out, cpx<T>* sp, int rows, int bc, double shift, bool poisson) {
    coarse_solve_pro(ArrPro<T>{rhs, d.nx}, ArrEpi<T>{out, d.nx}, sp, rows, bc, shift, poisson);
  }
  // velocity solve for the increment u~ - u*; out = u~ (IncEpi adds u* back)
  void velocity_solve(const T* rhs, T* out, const T* un, const T* uo, size_t off, cpx<T>* sp, int rows, int bc,
                      double shift) {
    coarse_solve_pro(ArrPro<T>{rhs, d.nx}, IncEpi<T>{out, un, uo, d.nx, off}, sp, rows, bc, shift, false);
  }
  template <class Pro, class Epi>
  void coarse_solve_pro(Pro pro, Epi epi, cpx<T>* sp, int rows, int bc, double shift, bool poisson) {
    const int nlines = d.ny * rows;
    rfft_x(pro, sp, d.nx, nlines, pC, plCx, twCx);
    if (d.dim == 3) fft_y(sp, d.ny, pC, d.nx / 2 + 1, rows, plCy, twCy, -1);
    zsolve(sp, rows, d.ny, pC, d.nx / 2 + 1, eCx, eCy, bc, d.dx * d.dx, shift, shift, false,
           1.0 / ((double)d.nx * d.ny), poisson);
    if (d.dim == 3) fft_y(sp, d.ny, pC, d.nx / 2 + 1, rows, plCy, twCy, +1);
    irfft_x(sp, epi, d.nx, nlines, pC, plCx, twCx, (T)1);
  }

  // pend_in: first run the owed polymer update (parity fc) on the side stream,
  // joined before the restriction; defer: leave this step's update owed.
  void launch_step(int flags, bool pend_in = false, bool defer = false) {
    const int po = pc ^ 1, fo = fc ^ 1;
    // ---- Cahn-Hilliard on the fine mesh ----
    FineView<T> fv{phi[pc], phi[po], philo[pc], philo[po]};
    const CoarseVel<T> vel{u[fc], u[fo], v[fc], v[fo], w[fc], w[fo]};
    if (p.weno) {  // div(u* phi*) with WENO5-Z fluxes, read by the right side
      mark("weno_adv");
      const RowLaunch lw = rows(d.fny * d.fnz, d.fnx);
      k_weno_adv_fine<T><<<lw.grid, lw.block, 0, st>>>(fv, vel, wadv, d, q);
      fv.aw = wadv;
    }
    T inv_mldt = (T)(1.0 / (p.Ml * p.dt)), inv_ml = (T)(1.0 / p.Ml);
    if constexpr (IsDual<T>::value) {
      inv_mldt.d = dseed.inv_mldt;
      inv_ml.d = dseed.inv_ml;
    }
    mark("ch_rhs");
    if (d.dim == 2) {
      using TL = RhsTile<2, sizeof(T)>;
      dim3 grid((d.fnx + TL::TX - 1) / TL::TX, 1, (d.fnz + TL::TZ - 1) / TL::TZ);
      const size_t sm = (TL::NS + TL::NM + 3 * TL::NV(d.rs, d.rys)) * sizeof(T);
      k_ch_rhs<T, 2><<<grid, 256, sm, st>>>(fv, vel, mu, gwall, d, p, q, inv_mldt, inv_ml);
    } else {
      using TL = MarchTile;
      const int nzc = std::min(d.fnz, tune[PF_TUNE_CH_ZCHUNK] > 0 ? tune[PF_TUNE_CH_ZCHUNK] : 32);
      bool done = false;
      if constexpr (std::is_same<T, float>::value) {
        if (d.fnx % 4 == 0) {  // four x cells per thread, float4 rows
          using T4 = March4;
          dim3 g4((d.fnx + T4::TX - 1) / T4::TX, (d.fny + T4::TY - 1) / T4::TY, (d.fnz + nzc - 1) / nzc);
          const size_t s4 = (size_t)T4::smem_floats(d.rs) * sizeof(float);
          const int mb = tune[PF_TUNE_CH_MINB];
          if (fv.aw) {  // WENO5-Z advection: the precomputed divergence, default register budget
            if (d.rs == 1) k_ch_rhs_march4<1, 3, true><<<g4, T4::NT, s4, st>>>(fv, vel, mu, gwall, d, p, q, inv_mldt, inv_ml, nzc);
            else k_ch_rhs_march4<0, 2, true><<<g4, T4::NT, s4, st>>>(fv, vel, mu, gwall, d, p, q, inv_mldt, inv_ml, nzc);
          } else if (d.rs == 1) {
            if (mb == 2) k_ch_rhs_march4<1, 2><<<g4, T4::NT, s4, st>>>(fv, vel, mu, gwall, d, p, q, inv_mldt, inv_ml, nzc);
            else if (mb == 4) {  // 14-row tiles of 224 threads: four CTAs per SM by shared memory and registers
              using T14 = March4T<14>;
              const dim3 g14((d.fnx + T14::TX - 1) / T14::TX, (d.fny + T14::TY - 1) / T14::TY, (d.fnz + nzc - 1) / nzc);
              const size_t s14 = (size_t)T14::smem_floats(d.rs) * sizeof(float);
              k_ch_rhs_march4<1, 4, false, 14><<<g14, T14::NT, s14, st>>>(fv, vel, mu, gwall, d, p, q, inv_mldt, inv_ml, nzc);
            }
            else k_ch_rhs_march4<1, 3><<<g4, T4::NT, s4, st>>>(fv, vel, mu, gwall, d, p, q, inv_mldt, inv_ml, nzc);
          } else {
            k_ch_rhs_march4<0, 2><<<g4, T4::NT, s4, st>>>(fv, vel, mu, gwall, d, p, q, inv_mldt, inv_ml, nzc);
          }
          done = true;
        }
      }
      if (!done) {
      dim3 grid((d.fnx + TL::TX - 1) / TL::TX, (d.fny + TL::TY - 1) / TL::TY, (d.fnz + nzc - 1) / nzc);
      const size_t sm = (size_t)TL::smem_elems(d.rs) * sizeof(T);
      if (tune[PF_TUNE_CH_MINB] == 2) k_ch_rhs_march<T, 2><<<grid, TL::NT, sm, st>>>(fv, vel, mu, gwall, d, p, q, inv_mldt, inv_ml, nzc);
      else k_ch_rhs_march<T, 3><<<grid, TL::NT, sm, st>>>(fv, vel, mu, gwall, d, p, q, inv_mldt, inv_ml, nzc);
      }
    }
    const bool robin = !IsDual<T>::value && p.dw > 0;
    const dim3 rgrid((d.fnx + 127) / 128, d.fny);
    if constexpr (!IsDual<T>::value) {
      if (robin) {  // D_w > 0: the flux g* of phi* into the right side (csrc/robin.cuh)
        mark("robin_wall");
        k_robin_wall<T><<<rgrid, 128, 0, st>>>(fv, rgE, rdg, d, p, q, p.dw, p.kappa);
        mark("robin_rhs");
        k_robin_rhs<T><<<rgrid, 128, 0, st>>>(mu, rdg, d, q);
      }
    }
    // the owed polymer update runs beside the memory-bound transform chain (not
    // beside the CH right side, which fills the SMs' registers and shared memory)
    if (pend_in) {
      PF_CUDA_TRY(cudaEventRecord(ev_fork, st));
      PF_CUDA_TRY(cudaStreamWaitEvent(st2, ev_fork, 0));
      launch_polymer(fc, st2);
      PF_CUDA_TRY(cudaEventRecord(ev_join, st2));
    }
    const int nlf = d.fny * d.fnz;
    rfft_x(FineArrPro<T>{mu, d.fnx}, spF, d.fnx, nlf, pF, plFx, twFx);
    if (d.dim == 3) fft_y(spF, d.fny, pF, d.fnx / 2 + 1, d.fnz, plFy, twFy, -1);
    zsolve(spF, d.fnz, d.fny, pF, d.fnx / 2 + 1, eFx, eFy, Z_NEUMANN, d.h * d.h, p.c, -p.alpha, true,
           1.0 / ((double)d.fnx * d.fny), false, dseed.c, -dseed.alpha);
    if constexpr (!IsDual<T>::value) {
      if (robin) {  // the Robin walls: delta = delta0 + b_bot D + b_top D mirrored
        const int ncol = d.fnx / 2 + 1;
        mark("robin_correct");
        k_robin_correct<T, TC><<<dim3((2 * ncol + 127) / 128, d.fny), 128, 0, st>>>(spF, d.fnz, d.fny, pF, ncol, rD,
                                                                                   rsx, (TC)p.kappa);
      }
    }
    if (d.dim == 3) fft_y(spF, d.fny, pF, d.fnx / 2 + 1, d.fnz, plFy, twFy, +1);
    irfft_x(spF, ChFinish<T>{phi[pc], phi[po], d.fnx, philo[pc], philo[po]}, d.fnx, nlf, pF, plFx, twFx, (T)1);
    if constexpr (!IsDual<T>::value) {
      if (robin) {  // the flux of phi^{n+1}, for G (Eq. NS5)
        mark("robin_flux");
        k_robin_flux<T><<<rgrid, 128, 0, st>>>(phi[po], philo[po], rgE, gwall, d, p.kappa);
      }
    }
    if (flags & PF_STEP_CH_ONLY) return;
    if (pend_in) PF_CUDA_TRY(cudaStreamWaitEvent(st, ev_join, 0));  // the update read the restricted phi
    // ---- chemical potential and restriction to the coarse mesh ----
    mark("ch_G_restrict");
    if (d.dim == 2) {
      using TL = GrTile<2>;
      const size_t sm = TL::smem_elems(d.r, 1) * sizeof(T);
      dim3 grid((d.nx + TL::CX - 1) / TL::CX, 1, (d.nz + TL::CZ - 1) / TL::CZ);
      if (d.r == 2) k_ch_G_restrict<T, 2, 2><<<grid, 256, sm, st>>>(phi[po], gwall, rs, d, q);
      else k_ch_G_restrict<T, 2, 1><<<grid, 256, sm, st>>>(phi[po], gwall, rs, d, q);
    } else {
      using TL = GrTile<3>;
      const size_t sm = TL::smem_elems(d.r, d.ry) * sizeof(T);
      dim3 grid((d.nx + TL::CX - 1) / TL::CX, (d.ny + TL::CY - 1) / TL::CY, (d.nz + TL::CZ - 1) / TL::CZ);
      if (d.r == 2) {
        using TM = GrMarch;
        const int nkc = tune[PF_TUNE_G_ZCHUNK] > 0 ? tune[PF_TUNE_G_ZCHUNK] : 16;
        dim3 gm((d.nx + TM::CX - 1) / TM::CX, (d.ny + TM::CY - 1) / TM::CY, (d.nz + 1 + nkc - 1) / nkc);
        k_ch_G_restrict_march<T><<<gm, TM::NT, TM::smem_elems() * sizeof(T), st>>>(phi[po], gwall, rs, d, q, nkc);
      } else {
        k_ch_G_restrict<T, 3, 1><<<grid, 256, sm, st>>>(phi[po], gwall, rs, d, q);
      }
    }
    const RowLaunch lw = rows(d.ny * (d.nz + 1), d.nx);
    const RowLaunch lc = rows(d.ny * d.nz, d.nx);
    // ---- Navier-Stokes ----
    NsIn<T> A;
    A.un = u[fc];
    A.uo = u[fo];
    A.vn = v[fc];
    A.vo = v[fo];
    A.wn = w[fc];
    A.wo = w[fo];
    A.pn = pr[fc];
    A.po = pr[fo];
    for (int c = 0; c < 6; ++c) {
      A.tn[c] = tau[fc][c];
      A.to[c] = tau[fo][c];
    }
    A.rs = rs;
    mark("ns_rhs");
    const bool ns3 = tune[PF_TUNE_NS_MINB] == 3;
    const int kz = tune[PF_TUNE_NS_KZ] > 1 ? tune[PF_TUNE_NS_KZ] : 1;
    {
      const dim3 gz(d.ny * ((d.nz + kz - 1) / kz), lc.grid.y);
      if (d.dim == 2) {
        if (ns3) k_ns_rhs_v2z<T, 2, 3><<<gz, lc.block, 0, st>>>(A, d, q, ru, rv, rw, p.visco, kz);
        else k_ns_rhs_v2z<T, 2, 4><<<gz, lc.block, 0, st>>>(A, d, q, ru, rv, rw, p.visco, kz);
      } else if (d.nx >= NsMarch::TX && d.ny >= NsMarch::TY) {
        // z-march through shared memory; the chunk is the same knob (layers per CTA)
        const int kc = tune[PF_TUNE_NS_KZ] > 1 ? tune[PF_TUNE_NS_KZ] : 16;
        const dim3 gm((d.nx + NsMarch::TX - 1) / NsMarch::TX, (d.ny + NsMarch::TY - 1) / NsMarch::TY,
                      (d.nz + kc - 1) / kc);
        const size_t sm = NsMarch::smem_elems() * sizeof(T);
        if (ns3) k_ns_rhs_march3<T, 3><<<gm, NsMarch::NT, sm, st>>>(A, d, q, ru, rv, rw, p.visco, kc);
        else k_ns_rhs_march3<T, 4><<<gm, NsMarch::NT, sm, st>>>(A, d, q, ru, rv, rw, p.visco, kc);
      } else {
        if (ns3) k_ns_rhs_v2z<T, 3, 3><<<gz, lc.block, 0, st>>>(A, d, q, ru, rv, rw, p.visco, kz);
        else k_ns_rhs_v2z<T, 3, 4><<<gz, lc.block, 0, st>>>(A, d, q, ru, rv, rw, p.visco, kz);
      }
    }
    const double kk = p.gamma0 / (p.dt * p.nu_m);
    // u~, v~ land in the n-1 buffers (free once the right sides exist).  The
    // three solves share nothing but their inputs, so outside pf_profile (which
    // times kernels one after another) they run on three streams.
    const size_t P = (size_t)d.nx * d.ny;
    if (!prof) {
      ensure_side_stream();
      PF_CUDA_TRY(cudaEventRecord(ev_ns, st));
      PF_CUDA_TRY(cudaStreamWaitEvent(st4, ev_ns, 0));
      {
        OnStream on(st, st4);
        velocity_solve(rw, wt, w[fc], w[fo], P, spW, d.nz - 1, Z_FACES, kk);
        PF_CUDA_TRY(cudaEventRecord(ev_w, st));
      }
      if (d.dim == 3) {
        PF_CUDA_TRY(cudaStreamWaitEvent(st3, ev_ns, 0));
        OnStream on(st, st3);
        velocity_solve(rv, v[fo], v[fc], v[fo], 0, spV, d.nz, Z_DIRICH, kk);
        PF_CUDA_TRY(cudaEventRecord(ev_v, st));
      }
      velocity_solve(ru, u[fo], u[fc], u[fo], 0, spU, d.nz, Z_DIRICH, kk);
      PF_CUDA_TRY(cudaStreamWaitEvent(st, ev_w, 0));
      if (d.dim == 3) PF_CUDA_TRY(cudaStreamWaitEvent(st, ev_v, 0));
    } else {
      velocity_solve(ru, u[fo], u[fc], u[fo], 0, spU, d.nz, Z_DIRICH, kk);
      if (d.dim == 3) velocity_solve(rv, v[fo], v[fc], v[fo], 0, spV, d.nz, Z_DIRICH, kk);
      velocity_solve(rw, wt, w[fc], w[fo], P, spW, d.nz - 1, Z_FACES, kk);
    }
    // pressure Poisson (Eq. NS37), its right side formed inside the first transform
    coarse_solve_pro(DivPro<T>{u[fo], v[fo], wt, d, (T)(p.gamma0 * p.rho0 / p.dt), (T)(1.0 / d.dx)},
                     ArrEpi<T>{pp, d.nx}, spP, d.nz, Z_NEUMANN, 0.0, true);
    mark("correct");
    {
      constexpr int kzc = 8;
      const dim3 gc(d.ny * ((d.nz + 1 + kzc - 1) / kzc), lw.grid.y);
      // 1/dx formed here: an FP64 division in every thread would sit on GB300's slow FP64 pipe
      k_correct_z<T><<<gc, lw.block, 0, st>>>(u[fo], v[fo], wt, w[fo], pp, pr[fc], pr[fo], d,
                                               (T)(p.dt / (p.gamma0 * p.rho0)), (T)(1.0 / d.dx), kzc);
    }
    // ---- polymer ----
    if (p.visco && !defer) launch_polymer(fo, st);
  }

  // ------------------------------------------------------------------ API
  const pf_grid_desc& grid_desc() const override { return g; }
  bool params_ready() const override { return have_params; }
  // the scheme's constants in arithmetic type TT, from the FP64 derived ones
  template <class TT>
  PhysT<TT> phys_of() const {
    PhysT<TT> r{};
    r.idt = (TT)(1.0 / p.dt);
    r.irho0 = (TT)(1.0 / p.rho0);
    r.inum = (TT)(1.0 / p.nu_m);
    r.num = (TT)p.nu_m;
    r.rho1 = (TT)p.rho1;
    r.rho2 = (TT)p.rho2;
    r.mu_s1 = (TT)p.mu_s1;
    r.mu_s2 = (TT)p.mu_s2;
    r.uw2_bot = (TT)(2 * p.uw_bot);
    r.uw2_top = (TT)(2 * p.uw_top);
    r.cj_dx = (TT)(-0.5 * (p.rho1 - p.rho2) * p.mob / d.dx);
    r.gx = (TT)p.gx;
    r.gy = (TT)p.gy;
    r.gz = (TT)p.gz;
    r.ih = (TT)(1.0 / d.h);
    r.ih2 = (TT)(1.0 / (d.h * d.h));
    r.iD = (TT)(1.0 / d.dx);
    r.iD2 = (TT)(1.0 / (d.dx * d.dx));
    r.ie2 = (TT)(1.0 / (p.eta * p.eta));
    r.lam = (TT)p.lam;
    r.dt = (TT)p.dt;
    r.ilh = p.visco ? (TT)(1.0 / p.lam_h) : (TT)0;
    r.wtau = p.visco ? (TT)(p.mu_p1 / p.lam_h) : (TT)0;
    r.ag = (TT)p.alpha_g;
    r.ap1 = p.approach1;
    r.weno = p.weno;
    r.lh1 = (TT)p.lam_h;
    r.lh2 = (TT)p.lam_h2;
    r.mp1 = (TT)p.mu_p1;
    r.mp2 = (TT)p.mu_p2;
    r.ag2 = (TT)p.alpha_g2;
    r.gbot = p.cos_bot / (1.4142135623730951 * p.eta);
    r.gtop = p.cos_top / (1.4142135623730951 * p.eta);
    r.ihw = 1.0 / d.h;
    return r;
  }
  void set_params(const pf_params& prm) override {
    p = derive(prm, g);
    raw_prm = prm;
    sigma = prm.sigma;
    prm_S = prm.S;
    q = phys_of<T>();
    have_params = true;
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
    if (p.weno && !wadv) {  // the WENO5-Z advection of phi*: one fine array, made on first use
      weno_ar.reset(new Arena());
      wadv = weno_ar->get<T>((size_t)d.fnx * d.fny * d.fnz);
    }
    if constexpr (!IsDual<T>::value) {
      if (p.dw > 0) robin_tables();
    }
  }
  // ---- dynamic contact angle (D_w > 0): the pair's response to a unit wall flux ----
  std::unique_ptr<Arena> robin_ar;
  TC* rD = nullptr;       // [fnz][fny][ncol]: delta of the pair for a unit flux at the bottom wall
  TC* rsx = nullptr;      // [fny][ncol][2]: its wall values w_bot, w_top
  Wide<T>* rgE = nullptr; // [2][fny][fnx]: explicit part E of the wall flux
  Wide<T>* rdg = nullptr; // [2][fny][fnx]: g* - g0
  void robin_tables() {
    const int R = d.fnz, ny = d.fny, ncol = d.fnx / 2 + 1;
    if (!robin_ar) {
      robin_ar.reset(new Arena());
      rD = robin_ar->get<TC>((size_t)R * ny * ncol);
      rsx = robin_ar->get<TC>((size_t)2 * ny * ncol);
      rgE = robin_ar->get<Wide<T>>((size_t)2 * d.fnx * d.fny);
      rdg = robin_ar->get<Wide<T>>((size_t)2 * d.fnx * d.fny);
    }
    // per mode, with lam the x-y eigenvalue of the Laplacian and L_N the
    // Neumann tridiagonal along z (all FP64):
    //   (L_N + lam - c) eps = -(c/h) e_0,   (L_N + lam + alpha) D = eps - (1/h) e_0
    const double h = d.h, ih2 = 1.0 / (h * h);
    auto eig = [&](int k, int n) {
      if (n == 1) return 0.0;
      const double s = std::sin(M_PI * k / n);
      return -4.0 * ih2 * s * s;
    };
    std::vector<TC> hD((size_t)R * ny * ncol), hs((size_t)2 * ny * ncol);
    std::vector<double> cp(R), x(R), e(R);
    // Thomas algorithm for (L_N + sh) x = b (b overwritten with x)
    auto tri = [&](double sh, std::vector<double>& b) {
      for (int k = 0; k < R; ++k) {
        const double diag = -2.0 * ih2 + ((k == 0 || k == R - 1) ? ih2 : 0.0) + sh;
        const double den = diag - (k > 0 ? ih2 * cp[k - 1] : 0.0);
        cp[k] = ih2 / den;
        b[k] = (b[k] - (k > 0 ? ih2 * b[k - 1] : 0.0)) / den;
      }
      for (int k = R - 2; k >= 0; --k) b[k] -= cp[k] * b[k + 1];
    };
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < ncol; ++i) {
        const double lam = eig(i, d.fnx) + eig(j, ny);
        std::fill(e.begin(), e.end(), 0.0);
        e[0] = -p.c / h;
        tri(lam - p.c, e);
        x = e;
        x[0] -= 1.0 / h;
        tri(lam + p.alpha, x);
        const size_t m = (size_t)j * ncol + i;
        for (int k = 0; k < R; ++k) hD[(size_t)k * ny * ncol + m] = (TC)x[k];
        hs[2 * m] = (TC)(1.5 * x[0] - 0.5 * x[1]);
        hs[2 * m + 1] = (TC)(1.5 * x[R - 1] - 0.5 * x[R - 2]);
      }
    PF_CUDA_TRY(cudaMemcpy(rD, hD.data(), hD.size() * sizeof(TC), cudaMemcpyHostToDevice));
    PF_CUDA_TRY(cudaMemcpy(rsx, hs.data(), hs.size() * sizeof(TC), cudaMemcpyHostToDevice));
  }
  std::unique_ptr<Arena> weno_ar;
  T* wadv = nullptr;

  void field_info(int f, size_t* count, size_t* eb) const override {
    const size_t nf = (size_t)d.fnx * d.fny * d.fnz;
    const size_t nc = (size_t)d.nx * d.ny * d.nz;
    const size_t ncw = (size_t)d.nx * d.ny * (d.nz + 1);
    size_t c = 0;
    switch (f) {
      case PF_PHI: case PF_PHI_OLD: case PF_G: case PF_PHI_REM: c = nf; break;
      case PF_U: case PF_U_OLD: case PF_P: case PF_P_OLD: c = nc; break;
      case PF_V: case PF_V_OLD: c = d.dim == 3 ? nc : 0; break;
      case PF_W: case PF_W_OLD: c = ncw; break;
      case PF_THETA: case PF_TAU: case PF_TAU_OLD: c = nc * ncomp; break;
      default: throw ApiError(PF_ERR_ARG, "unknown field id " + std::to_string(f));
    }
    *count = c;
    *eb = sizeof(T);
  }

  // pointers of a field's storage (components contiguous in the caller's view)
  std::vector<T*> field_ptrs(int f) {
    const int po = pc ^ 1, fo = fc ^ 1;
    switch (f) {
      case PF_PHI: return {phi[pc]};
      case PF_PHI_OLD: return {phi[po]};
      case PF_U: return {u[fc]};
      case PF_U_OLD: return {u[fo]};
      case PF_V: return {v[fc]};
      case PF_V_OLD: return {v[fo]};
      case PF_W: return {w[fc]};
      case PF_W_OLD: return {w[fo]};
      case PF_P: return {pr[fc]};
      case PF_P_OLD: return {pr[fo]};
      case PF_G: return {G};
      case PF_PHI_REM: return {philo[pc]};  // null in FP64 contexts (read as zeros)
      case PF_THETA: return std::vector<T*>(theta, theta + ncomp);
      case PF_TAU: return std::vector<T*>(tau[fc], tau[fc] + ncomp);
      case PF_TAU_OLD: return std::vector<T*>(tau[fo], tau[fo] + ncomp);
    }
    throw ApiError(PF_ERR_ARG, "unknown field id");
  }

  void copy_field(int f, const void* src, size_t bytes, int on_dev) {
    size_t cnt, eb;
    field_info(f, &cnt, &eb);
    if (bytes != cnt * eb) throw ApiError(PF_ERR_ARG, "byte count does not match the field size");
    auto ptrs = field_ptrs(f);
    const size_t per = cnt / ptrs.size();
    for (size_t q = 0; q < ptrs.size(); ++q)
      PF_CUDA_TRY(cudaMemcpyAsync(ptrs[q], static_cast<const char*>(src) + q * per * eb, per * eb,
                                  on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  }

  void set_field(int f, const void* src, size_t bytes, int on_dev) override {
    flush_polymer();
    if (f == PF_G || f == PF_PHI_REM) throw ApiError(PF_ERR_ARG, "PF_G and PF_PHI_REM are read-only");
    copy_field(f, src, bytes, on_dev);
    // phi set from outside carries no remainder
    const size_t nfb = (size_t)d.fnx * d.fny * d.fnz * sizeof(T);
    if (philo[0] && (f == PF_PHI || f == PF_PHI_OLD)) {
      PF_CUDA_TRY(cudaMemsetAsync(philo[f == PF_PHI ? pc : pc ^ 1], 0, nfb, st));
      if (f == PF_PHI) PF_CUDA_TRY(cudaMemsetAsync(philo[pc ^ 1], 0, nfb, st));
    }
    int twin = -1;
    if (f == PF_PHI) twin = PF_PHI_OLD;
    if (f == PF_U) twin = PF_U_OLD;
    if (f == PF_V) twin = PF_V_OLD;
    if (f == PF_W) twin = PF_W_OLD;
    if (f == PF_P) twin = PF_P_OLD;
    if (f == PF_TAU) twin = PF_TAU_OLD;
    if (twin >= 0) copy_field(twin, src, bytes, on_dev);
    if (!on_dev) PF_CUDA_TRY(cudaStreamSynchronize(st));
  }

  void get_field(int f, void* dst, size_t bytes, int on_dev) override {
    flush_polymer();
    size_t cnt, eb;
    field_info(f, &cnt, &eb);
    if (f == PF_G) {  // chemical potential of phi^n, formed on request
      const RowLaunch lf = rows(d.fny * d.fnz, d.fnx);
      k_ch_G<T><<<lf.grid, lf.block, 0, st>>>(phi[pc], gwall, G, d, q);
      check_launch();
    }
    if (bytes != cnt * eb) throw ApiError(PF_ERR_ARG, "byte count does not match the field size");
    auto ptrs = field_ptrs(f);
    const size_t per = cnt / ptrs.size();
    for (size_t q = 0; q < ptrs.size(); ++q) {
      if (!ptrs[q]) {  // PF_PHI_REM of an FP64 context
        if (on_dev) PF_CUDA_TRY(cudaMemsetAsync(static_cast<char*>(dst) + q * per * eb, 0, per * eb, st));
        else std::memset(static_cast<char*>(dst) + q * per * eb, 0, per * eb);
        continue;
      }
      PF_CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(dst) + q * per * eb, ptrs[q], per * eb,
                                  on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    PF_CUDA_TRY(cudaStreamSynchronize(st));
  }

  void check_launch() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw CudaError(e, "kernel launch", __FILE__, __LINE__);
  }

  void run_one(int flags, bool pend_in, bool defer) {
    if (flags & PF_STEP_NO_GRAPH) {
      launch_step(flags, pend_in, defer);
      check_launch();
      return;
    }
    auto key = std::make_tuple(pc, fc, (flags & PF_STEP_CH_ONLY) | (pend_in ? 2 : 0) | (defer ? 4 : 0));
    auto it = graphs.find(key);
    if (it == graphs.end()) {
      cudaGraph_t gr;
      PF_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      launch_step(flags, pend_in, defer);
      cudaError_t le = cudaGetLastError();
      cudaError_t ce = cudaStreamEndCapture(st, &gr);
      if (le != cudaSuccess) throw CudaError(le, "kernel launch during capture", __FILE__, __LINE__);
      PF_CUDA_TRY(ce);
      cudaGraphExec_t ex;
      PF_CUDA_TRY(cudaGraphInstantiate(&ex, gr, 0));
      cudaGraphDestroy(gr);
      it = graphs.emplace(key, ex).first;
    }
    PF_CUDA_TRY(cudaGraphLaunch(it->second, st));
  }

  void set_tuning(int knob, int value) override {
    if (knob < 0 || knob >= PF_TUNE_COUNT) throw ApiError(PF_ERR_ARG, "unknown tuning knob");
    if (value < 0) throw ApiError(PF_ERR_ARG, "tuning value must be >= 0");
    auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    if (value > 0) {
      if (knob == PF_TUNE_XFFT_PAIRS && (value > 16 || irfft_x_smem<T, ChFinish<T>>(std::max(d.fnx, d.nx), value) > (size_t)kMaxSmem))
        throw ApiError(PF_ERR_ARG, "x-transform line pairs do not fit in shared memory");
      if (knob == PF_TUNE_YFFT_COLS && (!pow2(value) || value > 32 || 2 * (size_t)value * std::max(d.fny, d.ny) * sizeof(cpx<T>) > (size_t)kMaxSmem))
        throw ApiError(PF_ERR_ARG, "y-transform columns must be a power of two that fits in shared memory");
      if (knob == PF_TUNE_ZSOLVE_COLS && (value % 16 || value > 64))
        throw ApiError(PF_ERR_ARG, "z-solve columns must be a multiple of 16, at most 64");
      if (knob == PF_TUNE_ROW_BLOCK && (value % 32 || value > 1024)) throw ApiError(PF_ERR_ARG, "row block must be a multiple of 32");
      if (knob == PF_TUNE_CH_ZCHUNK && value < 2) throw ApiError(PF_ERR_ARG, "z chunk must be at least 2 planes");
      if (knob == PF_TUNE_G_ZCHUNK && value < 1) throw ApiError(PF_ERR_ARG, "z chunk must be at least 1 layer");
      if (knob == PF_TUNE_NS_KZ && value > 64) throw ApiError(PF_ERR_ARG, "NS z rows per CTA must be <= 64");
      if (knob == PF_TUNE_CH_MINB && (value < 2 || value > 4)) throw ApiError(PF_ERR_ARG, "CH register budget: 2, 3 or 4 CTAs per SM");
      if (knob == PF_TUNE_NS_MINB && value != 3 && value != 4) throw ApiError(PF_ERR_ARG, "NS register budget: 3 or 4 CTAs per SM");
    }
    tune[knob] = value;
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
  }
  int get_tuning(int knob) const override {
    if (knob < 0 || knob >= PF_TUNE_COUNT) throw ApiError(PF_ERR_ARG, "unknown tuning knob");
    return tune[knob];
  }


  // ------------------------------------------------------------------ adjoint
  std::unique_ptr<Arena> adj_ar;
  int adj_K = 0, adj_nseg = 0;
  std::vector<T*> ck_n, ck_o, st_buf;
  T *a_phis = nullptr, *a_adv = nullptr, *a_delta = nullptr, *a_eps = nullptr, *a_ebar = nullptr,
    *a_rbar = nullptr, *a_mubar = nullptr, *a_tmp = nullptr, *a_next = nullptr, *a_cur = nullptr,
    *a_next2 = nullptr, *a_cur2 = nullptr, *a_fin_n = nullptr, *a_fin_o = nullptr, *a_fin_nl = nullptr,
    *a_fin_ol = nullptr;
  double *a_thb = nullptr, *a_part = nullptr;

  void adj_alloc(int K, int nseg) {
    if (adj_ar && adj_K >= K && adj_nseg >= nseg) return;
    adj_ar.reset(new Arena());
    const size_t nf = (size_t)d.fnx * d.fny * d.fnz;
    ck_n.assign(nseg, nullptr);
    ck_o.assign(nseg, nullptr);
    const size_t per = philo[0] ? 2 * nf : nf;  // value, then remainder
    for (int s = 0; s < nseg; ++s) {
      ck_n[s] = adj_ar->get<T>(per);
      ck_o[s] = adj_ar->get<T>(per);
    }
    a_fin_nl = philo[0] ? adj_ar->get<T>(nf) : nullptr;
    a_fin_ol = philo[0] ? adj_ar->get<T>(nf) : nullptr;
    st_buf.assign(K + 2, nullptr);
    for (int m = 0; m < K + 2; ++m) st_buf[m] = adj_ar->get<T>(nf);
    T** ws[] = {&a_phis, &a_adv, &a_delta, &a_eps, &a_ebar, &a_rbar, &a_mubar, &a_tmp,
                &a_next, &a_cur, &a_next2, &a_cur2, &a_fin_n, &a_fin_o};
    for (T** w : ws) *w = adj_ar->get<T>(nf);
    a_thb = adj_ar->get<double>((size_t)d.fnx * d.fny);
    a_part = adj_ar->get<double>((size_t)nred_blocks * 5 * K);  // one slot per step of a segment
    adj_K = K;
    adj_nseg = nseg;
  }

  void dcopy(T* dst, const T* src) {
    const size_t nf = (size_t)d.fnx * d.fny * d.fnz;
    PF_CUDA_TRY(cudaMemcpyAsync(dst, src, nf * sizeof(T), cudaMemcpyDeviceToDevice, st));
  }
  // phi of parity q with its remainder (compensated storage) to or from a
  // checkpoint of 2 nf elements (nf without remainders)
  void save_phi(T* ck, int q) {
    dcopy(ck, phi[q]);
    if (philo[q]) dcopy(ck + (size_t)d.fnx * d.fny * d.fnz, philo[q]);
  }
  void load_phi(int q, const T* ck) {
    dcopy(phi[q], ck);
    if (philo[q]) dcopy(philo[q], ck + (size_t)d.fnx * d.fny * d.fnz);
  }

  // out = (L_N - c)^-1 (L_N + alpha)^-1 in: the forward step's paired transform solve
  void fine_solve_pair(const T* in, T* out) {
    const int nlf = d.fny * d.fnz;
    rfft_x(FineArrPro<T>{in, d.fnx}, spF, d.fnx, nlf, pF, plFx, twFx);
    if (d.dim == 3) fft_y(spF, d.fny, pF, d.fnx / 2 + 1, d.fnz, plFy, twFy, -1);
    zsolve(spF, d.fnz, d.fny, pF, d.fnx / 2 + 1, eFx, eFy, Z_NEUMANN, d.h * d.h, p.c, -p.alpha, true,
           1.0 / ((double)d.fnx * d.fny), false);
    if (d.dim == 3) fft_y(spF, d.fny, pF, d.fnx / 2 + 1, d.fnz, plFy, twFy, +1);
    irfft_x(spF, ArrEpi<T>{out, d.fnx}, d.fnx, nlf, pF, plFx, twFx, (T)1);
  }

  // d c/d M and d alpha/d M of Eq. NS29 (S at its minimum moves with M)
  void dshift_dM(double& dc, double& da) const {
    const double M = p.mob;
    if (prm_S <= 0.0) {
      dc = -p.c / (2.0 * M);
      da = p.c / (2.0 * M);
      return;
    }
    const double S = p.S, eta2 = p.eta * p.eta;
    const double kap = 4.0 * p.gamma0 * eta2 * eta2 / (p.lam * p.dt * S * S);
    const double disc = 1.0 - kap / M;
    if (disc <= 1e-300) throw ApiError(PF_ERR_DISCRIMINANT, "d alpha/dM is unbounded at the Eq. NS30 limit with a fixed S");
    da = -S / (2.0 * eta2) * (kap / (M * M)) / (2.0 * std::sqrt(disc));
    dc = da;
  }

  // one reverse step; its FP64 partial sums go to part[0 .. 5 nb) (read by adjoint_accumulate)
  void adjoint_step(const T* pn, const T* po, const T* pnew, double* part) {
    const int fo = fc ^ 1;
    adjoint_step_v(pn, po, pnew, part, CoarseVel<T>{u[fc], u[fo], v[fc], v[fo], w[fc], w[fo]}, nullptr);
  }
  // the same with the step's velocity given, and an extra wall-flux adjoint gbx
  // (per wall column, bottom then top; null for none)
  void adjoint_step_v(const T* pn, const T* po, const T* pnew, double* part, const CoarseVel<T> vel,
                      const double* gbx) {
    const size_t nf = (size_t)d.fnx * d.fny * d.fnz;
    const RowLaunch lf = rows(d.fny * d.fnz, d.fnx);
    const FineView<T> fv{pn, po};
    const T a1 = (T)(1.0 / (p.Ml * p.dt)), a2 = (T)(1.0 / p.Ml);
    const int nb = nred_blocks;
    k_adj_prep<T><<<lf.grid, lf.block, 0, st>>>(fv, vel, a_phis, a_adv, d, q);
    k_sub<T><<<nb, 256, 0, st>>>(pnew, a_phis, a_delta, nf);
    k_lapN_axpy<T><<<lf.grid, lf.block, 0, st>>>(a_delta, a_delta, (T)p.alpha, a_eps, d, q);
    // (L_N + alpha) eps_bar = phi_bar^{n+1}, (L_N - c) R_bar = eps_bar: the two operators
    // commute, so R_bar is the forward step's paired solve of phi_bar^{n+1}, and
    // eps_bar = (L_N - c) R_bar is one stencil pass instead of a second solve
    fine_solve_pair(a_next, a_rbar);
    k_lapN_two<T><<<lf.grid, lf.block, 0, st>>>(a_rbar, (T)(-p.c), a_mubar, a_ebar, d, q);  // mu_bar, eps_bar
    k_dots<T><<<nb, 256, 0, st>>>(a_ebar, a_delta, a_rbar, a_eps, a_rbar, po, a_rbar, a_adv, nf, part, pn);
    k_adj_phibar<T><<<lf.grid, lf.block, 0, st>>>(a_phis, a_rbar, a_mubar, a_next, a_cur, a_next2, a_cur2, a_thb, vel,
                                                  d, p, q, a1, a2, gbx);
    k_sum_d<<<nb, 256, 0, st>>>(a_thb, (size_t)d.fnx * d.fny, part + (size_t)4 * nb);
    check_launch();
    std::swap(a_next, a_next2);
    std::swap(a_cur, a_cur2);
  }
  // the parameter adjoints of one reverse step from its partial sums h[0 .. 5 nb)
  void adjoint_accumulate(const double* h, double& thb, double& mb) {
    const int nb = nred_blocks;
    const T a1 = (T)(1.0 / (p.Ml * p.dt)), a2 = (T)(1.0 / p.Ml);
    double dots[4] = {0, 0, 0, 0}, th = 0;
    for (int b = 0; b < nb; ++b) {
      for (int k = 0; k < 4; ++k) dots[k] += h[(size_t)b * 4 + k];
      th += h[(size_t)4 * nb + b];
    }
    const double alpha_bar = -dots[0], c_bar = dots[1], s1 = dots[2], s2 = dots[3];
    double dc = 0, da = 0;
    dshift_dM(dc, da);
    const double M = p.mob;
    mb += -(double)a1 / M * s1 + (double)a2 / M * s2 + c_bar * dc + alpha_bar * da;
    thb += th;
  }

  // Gradients of an objective of phi after nsteps CH steps (velocity fixed):
  // out[0] = J, out[1] = dJ/d theta_bot (per degree), out[2] = dJ/d mobility;
  // dphi0 (optional) receives dJ/d phi^0.  Checkpoints every K steps; each
  // segment is recomputed forward before its reverse sweep.
  void adjoint(int nsteps, int K, int which, double out[3], void* dphi0, int on_dev) override {
    if constexpr (IsDual<T>::value) {  // derivative-carrying steps have no reverse sweep
      (void)nsteps, (void)K, (void)which, (void)out, (void)dphi0, (void)on_dev;
      throw ApiError(PF_ERR_UNSUPPORTED, "the adjoint runs on PF_FP64 and the mixed contexts");
    } else {
      flush_polymer();
      if (!have_params) throw ApiError(PF_ERR_ARG, "pf_set_params must precede pf_adjoint");
      if (p.weno) throw ApiError(PF_ERR_UNSUPPORTED, "the reverse sweep transposes the central advection flux");
      if (p.dw > 0) throw ApiError(PF_ERR_UNSUPPORTED, "the reverse sweep is built for the static contact angle (D_w = 0)");
      if (nsteps < 1 || K < 1) throw ApiError(PF_ERR_ARG, "nsteps and ckpt_every must be >= 1");
      if (which != 0 && which != 1) throw ApiError(PF_ERR_ARG, "objective must be PF_OBJ_WETTED or PF_OBJ_CENTROID_Z");
      const int nseg = (nsteps + K - 1) / K;
      adj_alloc(K, nseg);
      const size_t nf = (size_t)d.fnx * d.fny * d.fnz;
      // forward sweep with checkpoints of the BDF2 state (phi^n, phi^{n-1})
      for (int s = 0; s < nseg; ++s) {
        save_phi(ck_n[s], pc);
        save_phi(ck_o[s], pc ^ 1);
        step(std::min(K, nsteps - s * K), PF_STEP_CH_ONLY);
      }
      double dg[6];
      diagnostics(dg);
      const double J = which == 0 ? dg[2] : dg[5];
      dcopy(a_fin_n, phi[pc]);
      dcopy(a_fin_o, phi[pc ^ 1]);
      if (philo[0]) {
        dcopy(a_fin_nl, philo[pc]);
        dcopy(a_fin_ol, philo[pc ^ 1]);
      }
      const RowLaunch lf = rows(d.fny * d.fnz, d.fnx);
      const double D = 0.5 * ((double)nf + dg[0] / std::pow(d.h, d.dim));
      k_obj_seed<T><<<lf.grid, lf.block, 0, st>>>(a_next, d, which, dg[5], D);
      PF_CUDA_TRY(cudaMemsetAsync(a_cur, 0, nf * sizeof(T), st));
      double thb = 0, mb = 0;
      for (int s = nseg - 1; s >= 0; --s) {
        const int len = std::min(K, nsteps - s * K);
        // recompute the segment: st_buf[0] = phi^{sK-1}, st_buf[m+1] = phi^{sK+m}
        load_phi(pc, ck_n[s]);
        load_phi(pc ^ 1, ck_o[s]);
        dcopy(st_buf[0], ck_o[s]);
        dcopy(st_buf[1], ck_n[s]);
        for (int m = 1; m <= len; ++m) {
          run_one(PF_STEP_CH_ONLY, false, false);
          pc ^= 1;
          ++steps_done;
          dcopy(st_buf[m + 1], phi[pc]);
        }
        const size_t slot = (size_t)5 * nred_blocks;
        for (int m = len; m >= 1; --m) adjoint_step(st_buf[m], st_buf[m - 1], st_buf[m + 1], a_part + (len - m) * slot);
        std::vector<double> h(len * slot);
        PF_CUDA_TRY(cudaMemcpyAsync(h.data(), a_part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        PF_CUDA_TRY(cudaStreamSynchronize(st));
        for (int m = len; m >= 1; --m) adjoint_accumulate(h.data() + (len - m) * slot, thb, mb);
      }
      // phi^{-1} = phi^0 at start-up: both adjoints land on phi^0
      if (dphi0) {  // a_tmp = a_next + a_cur, summed on the device
        k_add<T><<<nred_blocks, 256, 0, st>>>(a_next, a_cur, a_tmp, nf);
        check_launch();
        PF_CUDA_TRY(cudaMemcpyAsync(dphi0, a_tmp, nf * sizeof(T), on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
      }
      // leave the context at phi^N, as pf_step would
      dcopy(phi[pc], a_fin_n);
      dcopy(phi[pc ^ 1], a_fin_o);
      if (philo[0]) {
        dcopy(philo[pc], a_fin_nl);
        dcopy(philo[pc ^ 1], a_fin_ol);
      }
      PF_CUDA_TRY(cudaStreamSynchronize(st));
      out[0] = J;
      out[1] = thb * M_PI / 180.0;
      out[2] = mb;
    }
  }

  // ------------------------------------------------------------------
  // Reverse sweep of the coupled 2D step (CH, restriction, NS, LCR).
  // out[0] = J, out[1] = dJ/d theta_bot (per degree), out[2] = dJ/d M,
  // out[3] = dJ/d lambda_H (the Weissenberg number); dphi0 (optional)
  // receives dJ/d phi^0.  Checkpoints of the whole state every K steps; each
  // segment is recomputed forward, storing the state of every step, and each
  // reverse step re-runs its forward step for the intermediates (restricted
  // fields, Theta1, the wall flux).
  // ------------------------------------------------------------------
  std::unique_ptr<Arena> cadj_ar;
  int cadj_K = 0, cadj_nseg = 0;
  std::vector<T*> cck, csb;  // checkpoints and the segment's per-step states
  T *cb[32] = {nullptr};      // coarse adjoint buffers (see cadj_alloc)
  T *cGb = nullptr, *cwork[6] = {nullptr}, *cpoly[9] = {nullptr}, *crf[7] = {nullptr}, *cfin = nullptr;
  double *cgbx = nullptr, *cmpart = nullptr, *cwpart = nullptr;

  size_t state_elems() const {
    const size_t nf = (size_t)d.fnx * d.fny * d.fnz, nc = (size_t)d.nx * d.ny * d.nz,
                 ncw = (size_t)d.nx * d.ny * (d.nz + 1);
    return nf * (philo[0] ? 4 : 2) + nc * 4 + ncw * 2 + (size_t)nc * ncomp * 3;
  }
  // copy the state (current and old levels in that order) to or from b
  void state_io(T* b, bool save) {
    const size_t nf = (size_t)d.fnx * d.fny * d.fnz, nc = (size_t)d.nx * d.ny * d.nz,
                 ncw = (size_t)d.nx * d.ny * (d.nz + 1);
    size_t o = 0;
    auto io = [&](T* a, size_t n) {
      if (save) PF_CUDA_TRY(cudaMemcpyAsync(b + o, a, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
      else PF_CUDA_TRY(cudaMemcpyAsync(a, b + o, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
      o += n;
    };
    io(phi[pc], nf);
    io(phi[pc ^ 1], nf);
    if (philo[0]) {
      io(philo[pc], nf);
      io(philo[pc ^ 1], nf);
    }
    io(u[fc], nc);
    io(u[fc ^ 1], nc);
    io(w[fc], ncw);
    io(w[fc ^ 1], ncw);
    io(pr[fc], nc);
    io(pr[fc ^ 1], nc);
    for (int c = 0; c < ncomp; ++c) io(theta[c], nc);
    for (int c = 0; c < ncomp; ++c) io(tau[fc][c], nc);
    for (int c = 0; c < ncomp; ++c) io(tau[fc ^ 1][c], nc);
  }
  struct StateView {
    const T *phi_n, *phi_o, *u_n, *u_o, *w_n, *w_o, *p_n, *p_o, *th[3], *tau_n[3], *tau_o[3];
  };
  StateView state_view(const T* b) const {
    const size_t nf = (size_t)d.fnx * d.fny * d.fnz, nc = (size_t)d.nx * d.ny * d.nz,
                 ncw = (size_t)d.nx * d.ny * (d.nz + 1);
    StateView v{};
    size_t o = 0;
    v.phi_n = b + o, o += nf;
    v.phi_o = b + o, o += nf;
    if (philo[0]) o += 2 * nf;
    v.u_n = b + o, o += nc;
    v.u_o = b + o, o += nc;
    v.w_n = b + o, o += ncw;
    v.w_o = b + o, o += ncw;
    v.p_n = b + o, o += nc;
    v.p_o = b + o, o += nc;
    for (int c = 0; c < 3; ++c) v.th[c] = c < ncomp ? b + o + (size_t)c * nc : nullptr;
    o += (size_t)nc * ncomp;
    for (int c = 0; c < 3; ++c) v.tau_n[c] = c < ncomp ? b + o + (size_t)c * nc : nullptr;
    o += (size_t)nc * ncomp;
    for (int c = 0; c < 3; ++c) v.tau_o[c] = c < ncomp ? b + o + (size_t)c * nc : nullptr;
    return v;
  }

  // coarse adjoint buffers, by index:
  //  0 ub1  1 ub0p  2 wb1  3 wb0p  4 pb1  5 pb0p  6-8 thb1  9-11 taub1  12-14 taub0p
  // 15 ub0 16 ubm 17 wb0 18 wbm 19 pb0 20 pbm 21-23 thb0 24-26 taub0 27-29 taubm
  // work: ppb, divb, utb, wtb, rbu, rbw, rphib (c, fx, fz, exz), rGb (c, fx, fz)
  void cadj_alloc(int K, int nseg) {
    if (cadj_ar && cadj_K >= K && cadj_nseg >= nseg) return;
    cadj_ar.reset(new Arena());
    const size_t nf = (size_t)d.fnx * d.fny * d.fnz, nc = (size_t)d.nx * d.ny * d.nz,
                 ncw = (size_t)d.nx * d.ny * (d.nz + 1);
    const size_t se = state_elems();
    cck.assign(nseg, nullptr);
    for (int s = 0; s < nseg; ++s) cck[s] = cadj_ar->get<T>(se);
    csb.assign(K + 1, nullptr);
    for (int m = 0; m <= K; ++m) csb[m] = cadj_ar->get<T>(se);
    for (int b = 0; b < 30; ++b) cb[b] = cadj_ar->get<T>(ncw);  // ncw >= nc: one size for all
    for (int b = 0; b < 6; ++b) cwork[b] = cadj_ar->get<T>(ncw);
    for (int b = 0; b < 9; ++b) cpoly[b] = cadj_ar->get<T>(nc);
    for (int b = 0; b < 7; ++b) crf[b] = cadj_ar->get<T>(ncw);
    cfin = cadj_ar->get<T>(se);
    cGb = cadj_ar->get<T>(nf);
    cgbx = cadj_ar->get<double>(2 * (size_t)d.fnx * d.fny);
    const int nblk = (int)((nc + 127) / 128);
    cmpart = cadj_ar->get<double>(nblk);
    cwpart = cadj_ar->get<double>(nblk);
    for (int b = 0; b < 30; ++b) PF_CUDA_TRY(cudaMemsetAsync(cb[b], 0, ncw * sizeof(T), st));
    cadj_K = K;
    cadj_nseg = nseg;
  }

  void adjoint_coupled(int nsteps, int K, int which, double out[4], void* dphi0, int on_dev) override {
    if constexpr (IsDual<T>::value) {
      (void)nsteps, (void)K, (void)which, (void)out, (void)dphi0, (void)on_dev;
      throw ApiError(PF_ERR_UNSUPPORTED, "the adjoint runs on PF_FP64 and the mixed contexts");
    } else {
      flush_polymer();
      if (!have_params) throw ApiError(PF_ERR_ARG, "pf_set_params must precede pf_adjoint_ex");
      if (d.dim != 2) throw ApiError(PF_ERR_UNSUPPORTED, "the coupled reverse sweep is built for 2D meshes");
      if (p.approach1)
        throw ApiError(PF_ERR_UNSUPPORTED, "the coupled reverse sweep is built for polymer approach 2 (Eq. NS12)");
      if (p.weno) throw ApiError(PF_ERR_UNSUPPORTED, "the reverse sweep transposes the central advection flux");
      if (p.dw > 0) throw ApiError(PF_ERR_UNSUPPORTED, "the reverse sweep is built for the static contact angle (D_w = 0)");
      if (nsteps < 1 || K < 1) throw ApiError(PF_ERR_ARG, "nsteps and ckpt_every must be >= 1");
      if (which != 0 && which != 1) throw ApiError(PF_ERR_ARG, "objective must be PF_OBJ_WETTED or PF_OBJ_CENTROID_Z");
      const int nseg = (nsteps + K - 1) / K;
      adj_alloc(K, nseg);  // the CH adjoint's buffers
      cadj_alloc(K, nseg);
      const size_t nf = (size_t)d.fnx * d.fny * d.fnz, nc = (size_t)d.nx * d.ny * d.nz,
                   ncw = (size_t)d.nx * d.ny * (d.nz + 1);
      const int nblk = (int)((nc + 127) / 128);
      const int nbf = (int)((nf + 255) / 256);
      const int nbc = (int)((nc + 255) / 256);
      // forward sweep with checkpoints of the whole state
      for (int s = 0; s < nseg; ++s) {
        state_io(cck[s], true);
        step(std::min(K, nsteps - s * K), 0);
      }
      double dg[6];
      diagnostics(dg);
      const double J = which == 0 ? dg[2] : dg[5];
      state_io(cfin, true);  // the final state, put back at the end
      // adjoint seeds
      const RowLaunch lf = rows(d.fny * d.fnz, d.fnx);
      const double D = 0.5 * ((double)nf + dg[0] / std::pow(d.h, d.dim));
      k_obj_seed<T><<<lf.grid, lf.block, 0, st>>>(a_next, d, which, dg[5], D);
      PF_CUDA_TRY(cudaMemsetAsync(a_cur, 0, nf * sizeof(T), st));
      for (int b = 0; b < 30; ++b) PF_CUDA_TRY(cudaMemsetAsync(cb[b], 0, ncw * sizeof(T), st));
      PF_CUDA_TRY(cudaMemsetAsync(cmpart, 0, nblk * sizeof(double), st));
      PF_CUDA_TRY(cudaMemsetAsync(cwpart, 0, nblk * sizeof(double), st));
      const PhysT<Dual> qd = phys_of<Dual>();
      PhysT<Dual> qm = qd, qw = qd;
      qm.cj_dx.d = -0.5 * (p.rho1 - p.rho2) / d.dx;                       // d(cj_dx)/dM
      if (p.visco) {
        qw.ilh.d = -1.0 / (p.lam_h * p.lam_h);                          // d(1/lambda_H)/d lambda_H
        qw.wtau.d = -p.mu_p1 / (p.lam_h * p.lam_h);                     // d(mu_p/lambda_H)/d lambda_H
      }
      const double kk = p.gamma0 / (p.dt * p.nu_m);
      const T cfD = (T)(p.dt / (p.gamma0 * p.rho0) / d.dx);
      const T coefD = (T)(p.gamma0 * p.rho0 / p.dt / d.dx);
      double thb = 0, mb = 0;
      for (int s = nseg - 1; s >= 0; --s) {
        const int len = std::min(K, nsteps - s * K);
        state_io(cck[s], false);
        state_io(csb[0], true);
        for (int m = 1; m <= len; ++m) {
          fwd1();
          state_io(csb[m], true);
        }
        const size_t slot = (size_t)5 * nred_blocks;
        for (int m = len; m >= 1; --m) {
          // re-run step n (state csb[m-1]) for its intermediates; the context then holds state n+1
          state_io(csb[m - 1], false);
          fwd1();
          coupled_reverse_step(state_view(csb[m - 1]), a_part + (len - m) * slot, qd, qm, qw, kk, cfD, coefD, nbf,
                               nbc, nblk);
        }
        std::vector<double> h(len * slot);
        PF_CUDA_TRY(cudaMemcpyAsync(h.data(), a_part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        PF_CUDA_TRY(cudaStreamSynchronize(st));
        for (int m = len; m >= 1; --m) adjoint_accumulate(h.data() + (len - m) * slot, thb, mb);
      }
      if (dphi0) {  // phi^{-1} = phi^0: both adjoints land on phi^0
        k_add<T><<<nred_blocks, 256, 0, st>>>(a_next, a_cur, a_tmp, nf);
        check_launch();
        PF_CUDA_TRY(cudaMemcpyAsync(dphi0, a_tmp, nf * sizeof(T), on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
      }
      std::vector<double> hm(nblk), hw(nblk);
      PF_CUDA_TRY(cudaMemcpyAsync(hm.data(), cmpart, nblk * sizeof(double), cudaMemcpyDeviceToHost, st));
      PF_CUDA_TRY(cudaMemcpyAsync(hw.data(), cwpart, nblk * sizeof(double), cudaMemcpyDeviceToHost, st));
      state_io(cfin, false);  // leave the context at step N, as pf_step would
      PF_CUDA_TRY(cudaStreamSynchronize(st));
      double mns = 0, wi = 0;
      for (int b = 0; b < nblk; ++b) {
        mns += hm[b];
        wi += hw[b];
      }
      out[0] = J;
      out[1] = thb * M_PI / 180.0;
      out[2] = mb + mns;
      out[3] = wi;
    }
  }

  // One reverse step of the coupled step n.  sv: the state of step n; the
  // context holds state n+1 and the step's intermediates (rs, theta1, gwall).
  // one coupled step with the polymer update in place (no deferral, no
  // finiteness check): the adjoint's recomputation
  void fwd1() {
    run_one(0, false, false);
    pc ^= 1;
    fc ^= 1;
    ++steps_done;
  }

  void coupled_reverse_step(const StateView& sv, double* part, const PhysT<Dual>& qd, const PhysT<Dual>& qm,
                            const PhysT<Dual>& qw, double kk, T cfD, T coefD, int nbf, int nbc, int nblk) {
    const size_t nf = (size_t)d.fnx * d.fny * d.fnz, nc = (size_t)d.nx * d.ny * d.nz,
                 ncw = (size_t)d.nx * d.ny * (d.nz + 1);
    T *ub1 = cb[0], *ub0p = cb[1], *wb1 = cb[2], *wb0p = cb[3], *pb1 = cb[4], *pb0p = cb[5];
    T *ub0 = cb[15], *ubm = cb[16], *wb0 = cb[17], *wbm = cb[18], *pb0 = cb[19], *pbm = cb[20];
    T *ppb = cwork[0], *divb = cwork[1], *utb = cwork[2], *wtb = cwork[3], *rbu = cwork[4], *rbw = cwork[5];
    NsBar<T> bar{};
    // restricted-field adjoints: phic, phifx, phifz, phiexz, Gc, Gfx, Gfz
    T* const* rfield = crf;
    for (int f = 0; f < 7; ++f) PF_CUDA_TRY(cudaMemsetAsync(rfield[f], 0, ncw * sizeof(T), st));
    bar.phic = rfield[0];
    bar.phifx = rfield[1];
    bar.phifz = rfield[2];
    bar.phiexz = rfield[3];
    bar.Gc = rfield[4];
    bar.Gfx = rfield[5];
    bar.Gfz = rfield[6];
    // ---- 1. LCR update ----
    if (p.visco) {
      PolyAdj<T> P{};
      for (int c = 0; c < 3; ++c) {
        P.th0[c] = sv.th[c];
        P.th1[c] = theta1[c];
        P.thb_in[c] = cb[6 + c];
        P.taub[c] = cb[9 + c];
        P.thb_out[c] = cb[21 + c];
        P.th1b[c] = cpoly[c];
        P.ab1[c] = cpoly[3 + c];
        P.ab0[c] = cpoly[6 + c];
      }
      P.U = u[fc];
      P.W = w[fc];
      P.phic = rs.phic;
      P.ub = ub1;
      P.wb = wb1;
      P.phicb = bar.phic;
      P.wipart = cwpart;
      k_adj_poly2_a<T><<<nblk, 128, 0, st>>>(P, d, q, qd, qw);
      k_adj_poly2_b<T><<<nblk, 128, 0, st>>>(P, d, q, qd, qw);
      k_adj_poly2_c<T><<<nbc, 256, 0, st>>>(P, d, q);
      check_launch();
    }
    // ---- 2. projection ----
    k_adj_correct2<T><<<nbc, 256, 0, st>>>(ub1, wb1, pb1, ppb, d, cfD);
    coarse_solve(ppb, divb, spP, d.nz, Z_NEUMANN, 0.0, true);   // P+ is symmetric
    PF_CUDA_TRY(cudaMemcpyAsync(utb, ub1, nc * sizeof(T), cudaMemcpyDeviceToDevice, st));
    PF_CUDA_TRY(cudaMemcpyAsync(wtb, wb1, ncw * sizeof(T), cudaMemcpyDeviceToDevice, st));
    k_adj_div2<T><<<nbc, 256, 0, st>>>(divb, utb, wtb, d, coefD);
    coarse_solve(utb, rbu, spU, d.nz, Z_DIRICH, kk, false);     // H^{-1}, symmetric
    coarse_solve(wtb + d.nx, rbw, spW, d.nz - 1, Z_FACES, kk, false);
    PF_CUDA_TRY(cudaMemcpyAsync(ub0, ub0p, nc * sizeof(T), cudaMemcpyDeviceToDevice, st));
    PF_CUDA_TRY(cudaMemsetAsync(ubm, 0, nc * sizeof(T), st));
    PF_CUDA_TRY(cudaMemcpyAsync(wb0, wb0p, ncw * sizeof(T), cudaMemcpyDeviceToDevice, st));
    PF_CUDA_TRY(cudaMemsetAsync(wbm, 0, ncw * sizeof(T), st));
    k_adj_ustar<T><<<nbc, 256, 0, st>>>(utb, ub0, ubm, 0, nc);
    k_adj_ustar<T><<<nbc, 256, 0, st>>>(wtb, wb0, wbm, (size_t)d.nx, (size_t)d.nx * d.nz);
    k_add<T><<<nbc, 256, 0, st>>>(pb0p, pb1, pb0, nc);          // p^{n+1} = p^n + p'
    PF_CUDA_TRY(cudaMemsetAsync(pbm, 0, nc * sizeof(T), st));
    for (int c = 0; c < 3; ++c) {
      PF_CUDA_TRY(cudaMemcpyAsync(cb[24 + c], cb[12 + c], nc * sizeof(T), cudaMemcpyDeviceToDevice, st));
      PF_CUDA_TRY(cudaMemsetAsync(cb[27 + c], 0, nc * sizeof(T), st));
    }
    // ---- 3. momentum right side ----
    NsIn<T> A{};
    A.un = sv.u_n;
    A.uo = sv.u_o;
    A.vn = A.vo = sv.u_n;
    A.wn = sv.w_n;
    A.wo = sv.w_o;
    A.pn = sv.p_n;
    A.po = sv.p_o;
    for (int c = 0; c < 6; ++c) {
      A.tn[c] = c < 3 ? sv.tau_n[c] : nullptr;
      A.to[c] = c < 3 ? sv.tau_o[c] : nullptr;
    }
    A.rs = rs;
    bar.un = ub0;
    bar.uo = ubm;
    bar.wn = wb0;
    bar.wo = wbm;
    bar.pn = pb0;
    bar.po = pbm;
    for (int c = 0; c < 3; ++c) {
      bar.tn[c] = cb[24 + c];
      bar.to[c] = cb[27 + c];
    }
    k_adj_ns_rhs2<T><<<nblk, 128, 0, st>>>(A, d, qd, qm, rbu, rbw, bar, p.visco, cmpart);
    check_launch();
    // ---- 4. restriction and chemical potential ----
    k_adj_restrict2<T><<<nbf, 256, 0, st>>>(bar, a_next, cGb, d);
    k_adj_G2<T><<<nbf, 256, 0, st>>>(phi[pc], cGb, a_next, cgbx, d, q);
    check_launch();
    // ---- 5. CH step, velocity from step n ----
    const CoarseVel<T> vel{sv.u_n, sv.u_o, sv.u_n, sv.u_o, sv.w_n, sv.w_o};
    adjoint_step_v(sv.phi_n, sv.phi_o, phi[pc], part, vel, cgbx);
    k_adj_ch_vel2<T><<<nbc, 256, 0, st>>>(a_phis, a_rbar, ub0, ubm, wb0, wbm, d, -1.0 / (p.Ml * 2.0 * d.h));
    check_launch();
    // ---- 6. the adjoints of step n become the incoming ones ----
    std::swap(cb[0], cb[15]);   // ub1 <- ub0
    std::swap(cb[1], cb[16]);   // ub0p <- ubm
    std::swap(cb[2], cb[17]);
    std::swap(cb[3], cb[18]);
    std::swap(cb[4], cb[19]);
    std::swap(cb[5], cb[20]);
    for (int c = 0; c < 3; ++c) {
      std::swap(cb[6 + c], cb[21 + c]);   // thb1 <- thb0
      std::swap(cb[9 + c], cb[24 + c]);   // taub1 <- taub0
      std::swap(cb[12 + c], cb[27 + c]);  // taub0p <- taubm
    }
    (void)nf;
  }

  // per-kernel average device time over nsteps direct (non-graph) steps
  void profile(int nsteps, int flags, std::vector<std::string>& names, std::vector<double>& ms,
               std::vector<int>& counts, int& per_step) override {
    if (!have_params) throw ApiError(PF_ERR_ARG, "pf_set_params must precede pf_profile");
    flush_polymer();
    std::map<std::string, double> acc;
    std::map<std::string, int> cnt;
    std::vector<std::string> order;
    cudaEvent_t last;
    PF_CUDA_TRY(cudaEventCreate(&last));
    per_step = 0;
    for (int s = 0; s < nsteps; ++s) {
      prof = true;
      nlaunch = 0;
      mark_names.clear();
      launch_step(flags);
      check_launch();
      PF_CUDA_TRY(cudaEventRecord(last, st));
      prof = false;
      PF_CUDA_TRY(cudaEventSynchronize(last));
      per_step = nlaunch;
      for (size_t i = 0; i < mark_names.size(); ++i) {
        float t = 0;
        PF_CUDA_TRY(cudaEventElapsedTime(&t, mark_ev[i], i + 1 < mark_names.size() ? mark_ev[i + 1] : last));
        if (!acc.count(mark_names[i])) order.push_back(mark_names[i]);
        acc[mark_names[i]] += t;
        if (s == 0) cnt[mark_names[i]] += 1;
      }
      pc ^= 1;
      if (!(flags & PF_STEP_CH_ONLY)) fc ^= 1;
      ++steps_done;
    }
    cudaEventDestroy(last);
    names = order;
    ms.clear();
    counts.clear();
    for (auto& n : order) {
      ms.push_back(acc[n] / std::max(1, nsteps));
      counts.push_back(cnt[n]);
    }
  }

  int launches_per_step(int flags) {
    prof = false;
    nlaunch = 0;
    // count without launching: replay the launch sequence into a throwaway capture
    cudaGraph_t gr;
    PF_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    launch_step(flags);
    cudaGetLastError();
    PF_CUDA_TRY(cudaStreamEndCapture(st, &gr));
    cudaGraphDestroy(gr);
    return nlaunch;
  }

  // sum of phi after a run of steps: finite unless a NaN or Inf appeared
  double mass_check() {
    const size_t n = (size_t)d.fnx * d.fny * d.fnz;
    k_sum_phi<T><<<nred_blocks, 256, 0, st>>>(phi[pc], n, partial);
    check_launch();
    std::vector<double> h((size_t)nred_blocks);
    PF_CUDA_TRY(cudaMemcpyAsync(h.data(), partial, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    PF_CUDA_TRY(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : h) s += v;
    return s;
  }

  void step(int nsteps, int flags) override {
    if (!have_params) throw ApiError(PF_ERR_ARG, "pf_set_params must precede pf_step");
    if (nsteps < 0) throw ApiError(PF_ERR_ARG, "nsteps < 0");
    flush_polymer();  // owed by a call that stopped early
    const bool visco_steps = p.visco && !(flags & PF_STEP_CH_ONLY);
    if (!(flags & PF_STEP_CH_ONLY)) ensure_side_stream();  // before any capture
    for (int s = 0; s < nsteps; ++s) {
      const bool pend_in = visco_steps && poly_pending;
      run_one(flags, pend_in, visco_steps);
      poly_pending = visco_steps;
      pc ^= 1;
      if (!(flags & PF_STEP_CH_ONLY)) fc ^= 1;
      ++steps_done;
      if (s == nsteps - 1) flush_polymer();
      if (steps_done % 50 == 0 || s == nsteps - 1) {
        const double m = mass_check();
        if (!std::isfinite(m)) throw ApiError(PF_ERR_NONFINITE, "phi mass is not finite after step " + std::to_string(steps_done));
      }
    }
  }

  void diagnostics(double out[6]) override {
    Wide<T> w[6];
    diagnostics_wide(w);
    for (int q = 0; q < 6; ++q) out[q] = (double)w[q];
  }
  // the six diagnostics in Wide<T> (their derivatives too when T carries them)
  void diagnostics_wide(Wide<T> out[6]) {
    using W = Wide<T>;
    k_reduce<T><<<nred_blocks, 256, 0, st>>>(phi[pc], d, p, sigma, d.dim == 3 ? d.h : g.ly, wpartial, philo[pc]);
    check_launch();
    std::vector<W> h((size_t)nred_blocks * RED_N);
    PF_CUDA_TRY(cudaMemcpyAsync(h.data(), wpartial, h.size() * sizeof(W), cudaMemcpyDeviceToHost, st));
    PF_CUDA_TRY(cudaStreamSynchronize(st));
    W s[RED_N];
    for (int q = 0; q < RED_N; ++q) s[q] = 0.0;
    for (int b = 0; b < nred_blocks; ++b)
      for (int q = 0; q < RED_N; ++q) s[q] += h[(size_t)b * RED_N + q];
    const double hd = std::pow(d.h, d.dim), hw = std::pow(d.h, d.dim - 1);
    out[0] = s[0] * hd;
    out[1] = p.lam * s[1] * hd + s[2] * hw;
    out[2] = s[3] * hw;
    out[3] = s[4] / s[7];
    out[4] = s[5] / s[7];
    out[5] = s[6] / s[7];
  }
};


// ---------------------------------------------------------------------------
// batched sweep of independent 2D problems (one persistent launch per step)
// ---------------------------------------------------------------------------
struct BatchBase {
  virtual ~BatchBase() {}
  virtual ImplBase* problem(int i) = 0;
  virtual int count() const = 0;
  virtual void step(int nsteps) = 0;
};

template <class T>
struct Batch : BatchBase {
  std::vector<std::unique_ptr<Impl<T, T>>> probs;
  cudaStream_t st;
  Arena ar;
  BatchProb<T>* d_probs = nullptr;
  BatchItem* d_items = nullptr;
  int nitems = 0;
  int* d_done = nullptr;
  int* d_head = nullptr;
  size_t smem = 0;
  int grid = 0;
  int pc = 0, fc = 0;
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
  static constexpr long long kSpin = 1ll << 24;

  Batch(int n, const pf_grid_desc* g, const pf_params* prm, cudaStream_t s) : st(s) {
    if (n < 1) throw ApiError(PF_ERR_ARG, "a batch needs at least one problem");
    for (int i = 0; i < n; ++i) {
      if (g[i].ny != 1) throw ApiError(PF_ERR_UNSUPPORTED, "batched problems must be two-dimensional (ny = 1)");
      if (g[i].precision != g[0].precision) throw ApiError(PF_ERR_ARG, "all batched problems share one precision");
      if (prm[i].advection != 0) throw ApiError(PF_ERR_UNSUPPORTED, "batched problems use the central advection flux");
      if (prm[i].dw != 0) throw ApiError(PF_ERR_UNSUPPORTED, "batched problems use the static contact angle (D_w = 0)");
      probs.emplace_back(new Impl<T, T>(g[i], st));
      probs.back()->set_params(prm[i]);
    }
    build();
  }
  ~Batch() override {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
  }
  ImplBase* problem(int i) override { return probs.at(i).get(); }
  int count() const override { return (int)probs.size(); }

  void build() {
    const int n = (int)probs.size();
    std::vector<BatchProb<T>> hp(n);
    std::vector<BatchItem> items;
    size_t maxsm = 0;
    const int tx = sizeof(T) == 4 ? 32 : 16;
    for (int b = 0; b < n; ++b) {
      Impl<T, T>& I = *probs[b];
      BatchProb<T>& B = hp[b];
      const Dims& d = I.d;
      B.d = d;
      B.p = I.p;
      B.q = I.q;
      B.inv_mldt = (T)(1.0 / (I.p.Ml * I.p.dt));
      B.inv_ml = (T)(1.0 / I.p.Ml);
      B.div_coef = (T)(I.p.gamma0 * I.p.rho0 / I.p.dt);
      B.corr_coef = (T)(I.p.dt / (I.p.gamma0 * I.p.rho0));
      for (int k = 0; k < 2; ++k) {
        B.phi[k] = I.phi[k];
        B.philo[k] = I.philo[k];
        B.u[k] = I.u[k];
        B.v[k] = I.v[k];
        B.w[k] = I.w[k];
        B.pr[k] = I.pr[k];
      }
      B.R = I.mu;
      B.ru = I.ru;
      B.rw = I.rw;
      B.wt = I.wt;
      B.pp = I.pp;
      B.dv = I.dv;
      B.gwall = I.gwall;
      B.zwork = I.zwork;
      B.rs = I.rs;
      B.spF = I.spF;
      B.spU = I.spU;
      B.spW = I.spW;
      B.spP = I.spP;
      B.pF = I.pF;
      B.pC = I.pC;
      B.npairF = std::max(1, 1024 / d.fnx);
      B.npairC = std::max(1, 1024 / d.nx);
      B.tx = tx;
      B.plFx = I.plFx;
      B.plCx = I.plCx;
      B.twFx = I.twFx;
      B.twCx = I.twCx;
      B.eFx = I.eFx;
      B.eFy = I.eFy;
      B.eCx = I.eCx;
      B.eCy = I.eCy;
      B.visco = I.p.visco;
      auto zs = [&](int rows, int pitch, int ncol, int bc, double h2, double s1, double s2, bool two, double scale,
                    bool poisson) {
        ZSolve z{};
        z.rows = rows;
        z.ny = 1;
        z.pitch = pitch;
        z.ncol = ncol;
        z.bc = bc;
        z.two = two ? 1 : 0;
        z.same = (!two || std::fabs(s1 - s2) <= 1e-14 * std::fabs(s1)) ? 1 : 0;
        z.skip_zero = poisson ? 1 : 0;
        z.h2 = h2;
        z.shift1 = s1;
        z.shift2 = s2;
        z.scale = scale;
        return z;
      };
      const double kk = I.p.gamma0 / (I.p.dt * I.p.nu_m);
      B.zpair = zs(d.fnz, I.pF, d.fnx / 2 + 1, Z_NEUMANN, d.h * d.h, I.p.c, -I.p.alpha, true, 1.0 / d.fnx, false);
      B.zu = zs(d.nz, I.pC, d.nx / 2 + 1, Z_DIRICH, d.dx * d.dx, kk, kk, false, 1.0 / d.nx, false);
      B.zw = zs(d.nz - 1, I.pC, d.nx / 2 + 1, Z_FACES, d.dx * d.dx, kk, kk, false, 1.0 / d.nx, false);
      B.zp = zs(d.nz, I.pC, d.nx / 2 + 1, Z_NEUMANN, d.dx * d.dx, 0.0, 0.0, false, 1.0 / d.nx, true);
      for (int f = 0; f < 2; ++f) {
        const int fo = f ^ 1;
        NsIn<T>& A = B.ns[f];
        A.un = I.u[f];
        A.uo = I.u[fo];
        A.vn = I.v[f];
        A.vo = I.v[fo];
        A.wn = I.w[f];
        A.wo = I.w[fo];
        A.pn = I.pr[f];
        A.po = I.pr[fo];
        for (int c = 0; c < 6; ++c) {
          A.tn[c] = I.tau[f][c];
          A.to[c] = I.tau[fo][c];
        }
        A.rs = I.rs;
        for (int stg = 0; stg < 2; ++stg) {
          PolyIn<T>& P = B.poly[f][stg];
          P = PolyIn<T>{};
          P.u = I.u[fo];  // the corrected velocity u^{n+1} lives in the n-1 buffer
          P.v = I.v[fo];
          P.w = I.w[fo];
          P.phic = I.rs.phic;
          for (int c = 0; c < I.ncomp; ++c) {
            P.th[c] = stg == 0 ? I.theta[c] : I.theta1[c];
            P.out[c] = stg == 0 ? I.theta1[c] : I.theta[c];
            P.base[c] = I.theta[c];
            P.tau[c] = I.tau[fo][c];
          }
        }
      }
      // grids of every pass (the launch shapes of the single-problem path)
      using TR = RhsTile<2, sizeof(T)>;
      using TG = GrTile<2>;
      auto cdiv = [](int a, int b) { return (a + b - 1) / b; };
      const int rowsx = cdiv(d.nx, 256);
      B.gdim[BP_CH_RHS] = make_int3(cdiv(d.fnx, TR::TX), 1, cdiv(d.fnz, TR::TZ));
      B.gdim[BP_RFFT_F] = make_int3(cdiv(cdiv(d.fnz, 2), B.npairF), 1, 1);
      B.gdim[BP_ZPAIR] = make_int3(cdiv(d.fnx / 2 + 1, tx), 1, 1);
      B.gdim[BP_IFFT_F] = B.gdim[BP_RFFT_F];
      B.gdim[BP_GRES] = make_int3(cdiv(d.nx, TG::CX), 1, cdiv(d.nz, TG::CZ));
      B.gdim[BP_NSRHS] = make_int3(d.nz, rowsx, 1);
      B.gdim[BP_U_RFFT] = make_int3(cdiv(cdiv(d.nz, 2), B.npairC), 1, 1);
      B.gdim[BP_U_Z] = make_int3(cdiv(d.nx / 2 + 1, tx), 1, 1);
      B.gdim[BP_U_IFFT] = B.gdim[BP_U_RFFT];
      B.gdim[BP_W_RFFT] = make_int3(cdiv(cdiv(d.nz - 1, 2), B.npairC), 1, 1);
      B.gdim[BP_W_Z] = B.gdim[BP_U_Z];
      B.gdim[BP_W_IFFT] = B.gdim[BP_W_RFFT];
      B.gdim[BP_DIV] = make_int3(d.nz, rowsx, 1);
      B.gdim[BP_P_RFFT] = B.gdim[BP_U_RFFT];
      B.gdim[BP_P_Z] = B.gdim[BP_U_Z];
      B.gdim[BP_P_ZERO] = make_int3(1, 1, 1);
      B.gdim[BP_P_IFFT] = B.gdim[BP_U_RFFT];
      B.gdim[BP_CORR] = make_int3(d.nz + 1, rowsx, 1);
      B.gdim[BP_POLY1] = B.visco ? make_int3(d.nz, rowsx, 1) : make_int3(0, 1, 1);
      B.gdim[BP_POLY2] = B.gdim[BP_POLY1];
      for (int ps = 0; ps < BP_N; ++ps) B.ntiles[ps] = B.gdim[ps].x * B.gdim[ps].y * B.gdim[ps].z;
      // shared memory of the largest pass
      auto zsm = [&](const ZSolve& z) { return (size_t)z.rows * tx * (sizeof(cpx<T>) + sizeof(T) * (z.same ? 1 : 2)); };
      maxsm = std::max(maxsm, (size_t)(TR::NS + TR::NM + 3 * TR::NV(d.rs, 0)) * sizeof(T));
      maxsm = std::max(maxsm, irfft_x_smem<T, ChFinish<T>>(d.fnx, B.npairF));
      maxsm = std::max(maxsm, 2 * (size_t)B.npairC * d.nx * sizeof(cpx<T>));
      maxsm = std::max(maxsm, (size_t)TG::smem_elems(d.r, 1) * sizeof(T));
      maxsm = std::max({maxsm, zsm(B.zpair), zsm(B.zu), zsm(B.zw), zsm(B.zp)});
    }
    // pass-major work list
    for (int ps = 0; ps < BP_N; ++ps)
      for (int b = 0; b < n; ++b)
        for (int t = 0; t < hp[b].ntiles[ps]; ++t) items.push_back(BatchItem{b, ps, t});
    nitems = (int)items.size();
    d_probs = ar.get<BatchProb<T>>(n);
    d_items = ar.get<BatchItem>(items.size());
    d_done = ar.get<int>((size_t)n * BP_N);
    d_head = ar.get<int>(2);  // [0] work head (reset every step), [1] sticky status
    PF_CUDA_TRY(cudaMemcpy(d_probs, hp.data(), n * sizeof(BatchProb<T>), cudaMemcpyHostToDevice));
    PF_CUDA_TRY(cudaMemcpy(d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
    smem = maxsm;
    if (smem > 200 * 1024) throw ApiError(PF_ERR_UNSUPPORTED, "batched problem too large for one persistent CTA");
    PF_CUDA_TRY(cudaFuncSetAttribute(k_batch_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per = 0, dev = 0, nsm = 0;
    PF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_step<T>, 256, smem));
    PF_CUDA_TRY(cudaGetDevice(&dev));
    PF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    grid = std::max(1, per) * nsm;
  }

  void launch(int p_c, int f_c) {
    PF_CUDA_TRY(cudaMemsetAsync(d_done, 0, probs.size() * BP_N * sizeof(int), st));
    PF_CUDA_TRY(cudaMemsetAsync(d_head, 0, sizeof(int), st));
    // the kernel's ctl[0] is the work head, ctl[1] the sticky status: both in one array
    k_batch_step<T><<<grid, 256, smem, st>>>(d_probs, d_items, nitems, d_done, d_head, p_c, f_c, kSpin);
  }

  void step(int nsteps) override {
    for (int s = 0; s < nsteps; ++s) {
      auto key = std::make_pair(pc, fc);
      auto it = graphs.find(key);
      if (it == graphs.end()) {
        cudaGraph_t gr;
        PF_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        launch(pc, fc);
        cudaError_t le = cudaGetLastError();
        cudaError_t ce = cudaStreamEndCapture(st, &gr);
        if (le != cudaSuccess) throw CudaError(le, "batch launch during capture", __FILE__, __LINE__);
        PF_CUDA_TRY(ce);
        cudaGraphExec_t ex;
        PF_CUDA_TRY(cudaGraphInstantiate(&ex, gr, 0));
        cudaGraphDestroy(gr);
        it = graphs.emplace(key, ex).first;
      }
      PF_CUDA_TRY(cudaGraphLaunch(it->second, st));
      pc ^= 1;
      fc ^= 1;
      for (auto& I : probs) {
        I->pc ^= 1;
        I->fc ^= 1;
        I->steps_done++;
      }
    }
    int status = 0;
    PF_CUDA_TRY(cudaMemcpyAsync(&status, d_head + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    PF_CUDA_TRY(cudaStreamSynchronize(st));
    if (status != 0) throw ApiError(status, "a bounded wait of the batched step expired");
  }
};
}  // namespace pf

// ===========================================================================
// C ABI
// ===========================================================================
struct pf_ctx {
  std::unique_ptr<pf::ImplBase> impl;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
};

static std::string g_init_err;

template <class F>
static int guarded(pf_ctx* ctx, F&& f) {
  try {
    f();
    return PF_OK;
  } catch (const pf::ApiError& e) {
    if (ctx) ctx->err = e.what();
    return e.code;
  } catch (const pf::CudaError& e) {
    if (ctx)
      ctx->err = std::string("CUDA error ") + cudaGetErrorString(e.err) + " in " + e.expr + " (" + e.file + ":" +
                 std::to_string(e.line) + ")";
    return PF_ERR_CUDA;
  } catch (const std::exception& e) {
    if (ctx) ctx->err = e.what();
    return PF_ERR_ARG;
  }
}

// A translation unit that instantiates Impl for another element type
// (tangent.cu) defines PF_IMPL_ONLY and includes this file without its
// exported functions.
#ifndef PF_IMPL_ONLY
extern "C" {

int pf_init_grid(pf_ctx** out, const pf_grid_desc* g, void* stream) {
  if (!out || !g) {
    g_init_err = "null argument";
    return PF_ERR_ARG;
  }
  *out = nullptr;
  auto ctx = std::make_unique<pf_ctx>();
  int rc = guarded(ctx.get(), [&] {
    if (g->nx < 2 || g->ny < 1 || g->nz < 2) throw pf::ApiError(PF_ERR_ARG, "need nx >= 2, ny >= 1, nz >= 2");
    if (!(g->lx > 0 && g->lz > 0)) throw pf::ApiError(PF_ERR_ARG, "lx and lz must be > 0");
    const double dx = g->lx / g->nx;
    if (std::fabs(g->lz / g->nz - dx) > 1e-9 * dx || (g->ny > 1 && std::fabs(g->ly / g->ny - dx) > 1e-9 * dx))
      throw pf::ApiError(PF_ERR_ARG, "cells must be cubes: lx/nx = ly/ny = lz/nz");
    if (g->precision != PF_FP64 && g->precision != PF_MIXED && g->precision != PF_MIXED_Z64 &&
        g->precision != PF_MIXED_Z2F)
      throw pf::ApiError(PF_ERR_ARG, "precision must be PF_FP64, PF_MIXED, PF_MIXED_Z64 or PF_MIXED_Z2F");
    if (g->nx % 2 || (g->ny > 1 && g->ny % 2)) throw pf::ApiError(PF_ERR_UNSUPPORTED, "nx and ny (3D) must be even");
    for (int n : {g->nx, g->ny, g->nz})
      if (!pf::smooth(n)) throw pf::ApiError(PF_ERR_UNSUPPORTED, "sizes must be 2^a 3^b 5^c 7^d");
    if (stream) {
      ctx->stream = static_cast<cudaStream_t>(stream);
    } else {
      PF_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
      ctx->own_stream = true;
    }
    if (g->precision == PF_FP64) ctx->impl.reset(new pf::Impl<double, double>(*g, ctx->stream));
    else if (g->precision == PF_MIXED_Z64) ctx->impl.reset(new pf::Impl<float, double>(*g, ctx->stream));
    else if (g->precision == PF_MIXED_Z2F) ctx->impl.reset(new pf::Impl<float, pf::DF>(*g, ctx->stream));
    else ctx->impl.reset(new pf::Impl<float, float>(*g, ctx->stream));
  });
  if (rc != PF_OK) {
    g_init_err = ctx->err;
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    return rc;
  }
  *out = ctx.release();
  return PF_OK;
}

int pf_set_params(pf_ctx* ctx, const pf_params* prm) {
  if (!ctx || !prm) return PF_ERR_ARG;
  return guarded(ctx, [&] { ctx->impl->set_params(*prm); });
}

int pf_field_info(const pf_ctx* ctx, int field_id, size_t* count, size_t* elem_bytes) {
  if (!ctx || !count || !elem_bytes) return PF_ERR_ARG;
  return guarded(const_cast<pf_ctx*>(ctx), [&] { ctx->impl->field_info(field_id, count, elem_bytes); });
}

int pf_set_fields(pf_ctx* ctx, int field_id, const void* src, size_t bytes, int src_on_device) {
  if (!ctx || !src) return PF_ERR_ARG;
  return guarded(ctx, [&] { ctx->impl->set_field(field_id, src, bytes, src_on_device); });
}

int pf_step_ex(pf_ctx* ctx, int nsteps, int flags) {
  if (!ctx) return PF_ERR_ARG;
  return guarded(ctx, [&] { ctx->impl->step(nsteps, flags); });
}

int pf_step(pf_ctx* ctx, int nsteps) { return pf_step_ex(ctx, nsteps, 0); }

int pf_get_fields(pf_ctx* ctx, int field_id, void* dst, size_t bytes, int dst_on_device) {
  if (!ctx || !dst) return PF_ERR_ARG;
  return guarded(ctx, [&] { ctx->impl->get_field(field_id, dst, bytes, dst_on_device); });
}

int pf_diagnostics(pf_ctx* ctx, double out[6]) {
  if (!ctx || !out) return PF_ERR_ARG;
  return guarded(ctx, [&] { ctx->impl->diagnostics(out); });
}

int pf_profile(pf_ctx* ctx, int nsteps, int flags, int max_entries, char* names, double* avg_ms, int* counts,
               int* n_entries, int* launches_per_step) {
  if (!ctx || nsteps < 1 || max_entries < 1 || !names || !avg_ms || !counts || !n_entries || !launches_per_step)
    return PF_ERR_ARG;
  return guarded(ctx, [&] {
    std::vector<std::string> nm;
    std::vector<double> ms;
    std::vector<int> cn;
    int per = 0;
    ctx->impl->profile(nsteps, flags, nm, ms, cn, per);
    const int n = std::min<int>(max_entries, (int)nm.size());
    for (int i = 0; i < n; ++i) {
      std::strncpy(names + (size_t)i * PF_PROFILE_NAME, nm[i].c_str(), PF_PROFILE_NAME - 1);
      names[(size_t)i * PF_PROFILE_NAME + PF_PROFILE_NAME - 1] = 0;
      avg_ms[i] = ms[i];
      counts[i] = cn[i];
    }
    *n_entries = n;
    *launches_per_step = per;
  });
}

int pf_set_tuning(pf_ctx* ctx, int knob, int value) {
  if (!ctx) return PF_ERR_ARG;
  return guarded(ctx, [&] { ctx->impl->set_tuning(knob, value); });
}

int pf_get_tuning(const pf_ctx* ctx, int knob, int* value) {
  if (!ctx || !value) return PF_ERR_ARG;
  return guarded(const_cast<pf_ctx*>(ctx), [&] { *value = ctx->impl->get_tuning(knob); });
}

int pf_adjoint(pf_ctx* ctx, int nsteps, int ckpt_every, int objective, double out[3], void* dphi0, int dphi0_on_device) {
  if (!ctx || !out) return PF_ERR_ARG;
  return guarded(ctx, [&] { ctx->impl->adjoint(nsteps, ckpt_every, objective, out, dphi0, dphi0_on_device); });
}

int pf_adjoint_ex(pf_ctx* ctx, int nsteps, int ckpt_every, int objective, int flags, double out[4], void* dphi0,
                  int dphi0_on_device) {
  if (!ctx || !out) return PF_ERR_ARG;
  if (flags & ~PF_ADJ_COUPLED) return PF_ERR_ARG;
  return guarded(ctx, [&] {
    if (flags & PF_ADJ_COUPLED) {
      ctx->impl->adjoint_coupled(nsteps, ckpt_every, objective, out, dphi0, dphi0_on_device);
    } else {
      ctx->impl->adjoint(nsteps, ckpt_every, objective, out, dphi0, dphi0_on_device);
      out[3] = 0.0;
    }
  });
}

const char* pf_last_error(const pf_ctx* ctx) { return ctx ? ctx->err.c_str() : g_init_err.c_str(); }

}  // extern "C"
#endif

struct pf_batch {
  std::unique_ptr<pf::BatchBase> impl;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
};

template <class F>
static int bguarded(pf_batch* b, F&& f) {
  pf_ctx tmp;
  const int rc = guarded(&tmp, std::forward<F>(f));
  if (b && rc != PF_OK) b->err = tmp.err;
  return rc;
}

#ifndef PF_IMPL_ONLY
extern "C" {

int pf_batch_create(pf_batch** out, int nproblems, const pf_grid_desc* grids, const pf_params* params, void* stream) {
  if (!out || !grids || !params || nproblems < 1) {
    g_init_err = "bad arguments to pf_batch_create";
    return PF_ERR_ARG;
  }
  *out = nullptr;
  auto b = std::make_unique<pf_batch>();
  int rc = bguarded(b.get(), [&] {
    for (int i = 0; i < nproblems; ++i) {
      const pf_grid_desc& g = grids[i];
      if (g.precision != PF_FP64 && g.precision != PF_MIXED)
        throw pf::ApiError(PF_ERR_UNSUPPORTED, "batched problems run PF_FP64 or PF_MIXED");
      if (g.nx < 2 || g.nz < 2 || g.nx % 2) throw pf::ApiError(PF_ERR_ARG, "need even nx >= 2 and nz >= 2");
      const double dx = g.lx / g.nx;
      if (std::fabs(g.lz / g.nz - dx) > 1e-9 * dx) throw pf::ApiError(PF_ERR_ARG, "cells must be squares");
      for (int n : {g.nx, g.nz})
        if (!pf::smooth(n)) throw pf::ApiError(PF_ERR_UNSUPPORTED, "sizes must be 2^a 3^b 5^c 7^d");
    }
    if (stream) {
      b->stream = static_cast<cudaStream_t>(stream);
    } else {
      PF_CUDA_TRY(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
      b->own_stream = true;
    }
    if (grids[0].precision == PF_FP64) b->impl.reset(new pf::Batch<double>(nproblems, grids, params, b->stream));
    else b->impl.reset(new pf::Batch<float>(nproblems, grids, params, b->stream));
  });
  if (rc != PF_OK) {
    g_init_err = b->err;
    if (b->own_stream) cudaStreamDestroy(b->stream);
    return rc;
  }
  *out = b.release();
  return PF_OK;
}

int pf_batch_field_info(const pf_batch* b, int problem, int field_id, size_t* count, size_t* elem_bytes) {
  if (!b || !count || !elem_bytes) return PF_ERR_ARG;
  return bguarded(const_cast<pf_batch*>(b), [&] { b->impl->problem(problem)->field_info(field_id, count, elem_bytes); });
}

int pf_batch_set_fields(pf_batch* b, int problem, int field_id, const void* src, size_t bytes, int src_on_device) {
  if (!b || !src) return PF_ERR_ARG;
  return bguarded(b, [&] { b->impl->problem(problem)->set_field(field_id, src, bytes, src_on_device); });
}

int pf_batch_get_fields(pf_batch* b, int problem, int field_id, void* dst, size_t bytes, int dst_on_device) {
  if (!b || !dst) return PF_ERR_ARG;
  return bguarded(b, [&] { b->impl->problem(problem)->get_field(field_id, dst, bytes, dst_on_device); });
}

int pf_batch_step(pf_batch* b, int nsteps) {
  if (!b || nsteps < 0) return PF_ERR_ARG;
  return bguarded(b, [&] { b->impl->step(nsteps); });
}

int pf_batch_diagnostics(pf_batch* b, int problem, double out[6]) {
  if (!b || !out) return PF_ERR_ARG;
  return bguarded(b, [&] { b->impl->problem(problem)->diagnostics(out); });
}

int pf_batch_adjoint(pf_batch* b, int problem, int nsteps, int ckpt_every, int objective, double out[3], void* dphi0,
                     int dphi0_on_device) {
  if (!b || !out) return PF_ERR_ARG;
  return bguarded(b, [&] { b->impl->problem(problem)->adjoint(nsteps, ckpt_every, objective, out, dphi0, dphi0_on_device); });
}

int pf_batch_adjoint_ex(pf_batch* b, int problem, int nsteps, int ckpt_every, int objective, int flags, double out[4],
                        void* dphi0, int dphi0_on_device) {
  if (!b || !out) return PF_ERR_ARG;
  if (flags & ~PF_ADJ_COUPLED) return PF_ERR_ARG;
  return bguarded(b, [&] {
    auto* I = b->impl->problem(problem);
    if (flags & PF_ADJ_COUPLED) {
      I->adjoint_coupled(nsteps, ckpt_every, objective, out, dphi0, dphi0_on_device);
    } else {
      I->adjoint(nsteps, ckpt_every, objective, out, dphi0, dphi0_on_device);
      out[3] = 0.0;
    }
  });
}

const char* pf_batch_last_error(const pf_batch* b) { return b ? b->err.c_str() : g_init_err.c_str(); }

void pf_batch_destroy(pf_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  b->impl.reset();
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

void pf_destroy(pf_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  ctx->impl.reset();
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

}  // extern "C"
#endif
