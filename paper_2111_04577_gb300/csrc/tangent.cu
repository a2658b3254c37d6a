// Forward-mode (tangent) sensitivity of an objective to one scalar parameter
// through the whole coupled time step of Section 3.2: the Cahn-Hilliard step
// with its wetting condition (Eqs. NS25-NS34), the restriction (Eq. dual2),
// the projection of Eqs. NS35-NS39 and the log-conformation update of
// Eqs. NS40-NS46.  The same step runs with every value a Dual number (value
// and derivative, csrc/dual.cuh); the parameter's derivative is seeded where
// it enters the step:
//   Wi = lambda_H:   1/lambda_H and mu_p/lambda_H of the polymer update
//                    (Eqs. NS41, NS46), derivatives -1/lambda_H^2 and
//                    -mu_p/lambda_H^2;
//   theta_s (bottom): cos(theta_s) of the wall flux (Eq. NS34), derivative
//                    -sin(theta_s) per radian;
//   phi^0 along v:   the derivative parts of phi^n and phi^{n-1} set to v
//                    (start-up phi^{-1} = phi^0), giving <dJ/dphi^0, v>;
//   M (mobility):    1/(M lambda dt) and 1/(M lambda) of the CH right side,
//                    the two shifts c(M), -alpha(M) of the paired solve
//                    (Eqs. NS26-NS30, through S when S follows Eq. NS30) and
//                    the flux J = -(rho1 - rho2)/2 M grad G of Eq. NS36.
// The objective's derivative then follows by the chain rule through every
// kernel, exactly up to FP64 rounding of the value and derivative parts: the
// same result a reverse sweep gives for one parameter.
#define PF_IMPL_ONLY
#include "dualpf.cu"

namespace pf {

// A derivative-carrying copy of a context's state: the fields of the source
// context (any precision) with zero derivatives, and its grid and parameters.
struct TangentRun {
  std::unique_ptr<Impl<Dual, Dual>> impl;

  TangentRun(ImplBase& src, cudaStream_t st) {
    if (!src.params_ready()) throw ApiError(PF_ERR_ARG, "pf_set_params must precede pf_tangent");
    if (src.raw_prm.dw > 0)
      throw ApiError(PF_ERR_UNSUPPORTED, "forward mode is built for the static contact angle (D_w = 0)");
    impl.reset(new Impl<Dual, Dual>(src.grid_desc(), st));
    impl->set_params(src.raw_prm);
    // PHI before PHI_OLD (setting PHI also sets PHI_OLD), likewise U/V/W/P/TAU
    const int order[] = {PF_PHI, PF_PHI_OLD, PF_U, PF_U_OLD, PF_V, PF_V_OLD, PF_W,
                         PF_W_OLD, PF_P, PF_P_OLD, PF_THETA, PF_TAU, PF_TAU_OLD};
    for (int f : order) {
      size_t cnt = 0, eb = 0, dcnt = 0, deb = 0;
      src.field_info(f, &cnt, &eb);
      impl->field_info(f, &dcnt, &deb);
      if (cnt != dcnt) throw ApiError(PF_ERR_ARG, "field sizes of the source and the tangent copy differ");
      if (cnt == 0) continue;
      std::vector<unsigned char> raw(cnt * eb);
      src.get_field(f, raw.data(), raw.size(), 0);
      std::vector<Dual> dv(cnt);
      for (size_t i = 0; i < cnt; ++i) {
        double x;
        if (eb == sizeof(double)) std::memcpy(&x, raw.data() + i * eb, sizeof(double));
        else {
          float y;
          std::memcpy(&y, raw.data() + i * eb, sizeof(float));
          x = y;
        }
        dv[i] = Dual(x, 0.0);
      }
      impl->set_field(f, dv.data(), dv.size() * sizeof(Dual), 0);
    }
  }

  void seed(int param, const void* dir, int dir_on_device) {
    Impl<Dual, Dual>& I = *impl;
    if (param == PF_PARAM_PHI0) {
      if (!dir) throw ApiError(PF_ERR_ARG, "PF_PARAM_PHI0 needs a direction");
      size_t cnt = 0, eb = 0;
      I.field_info(PF_PHI, &cnt, &eb);
      std::vector<double> v(cnt);
      if (dir_on_device) PF_CUDA_TRY(cudaMemcpy(v.data(), dir, cnt * sizeof(double), cudaMemcpyDeviceToHost));
      else std::memcpy(v.data(), dir, cnt * sizeof(double));
      std::vector<Dual> hn(cnt), ho(cnt);
      I.get_field(PF_PHI, hn.data(), cnt * sizeof(Dual), 0);
      I.get_field(PF_PHI_OLD, ho.data(), cnt * sizeof(Dual), 0);
      for (size_t i = 0; i < cnt; ++i) hn[i].d = ho[i].d = v[i];
      I.set_field(PF_PHI, hn.data(), cnt * sizeof(Dual), 0);  // (sets PF_PHI_OLD too)
      I.set_field(PF_PHI_OLD, ho.data(), cnt * sizeof(Dual), 0);
      return;
    }
    if (param == PF_PARAM_WI) {
      if (!I.p.visco) throw ApiError(PF_ERR_ARG, "Wi has no effect: the context is not viscoelastic");
      const double lh = I.p.lam_h;
      I.q.ilh = Dual(1.0 / lh, -1.0 / (lh * lh));
      I.q.wtau = Dual(I.p.mu_p1 / lh, -I.p.mu_p1 / (lh * lh));
      I.q.lh1 = Dual(lh, 1.0);  // approach 1: the droplet's lambda_H, mixed per cell
    } else if (param == PF_PARAM_MOBILITY) {
      const double M = I.p.mob;
      double dc = 0, da = 0;
      I.dshift_dM(dc, da);
      I.dseed.inv_mldt = -(1.0 / (I.p.Ml * I.p.dt)) / M;
      I.dseed.inv_ml = -(1.0 / I.p.Ml) / M;
      I.dseed.c = dc;
      I.dseed.alpha = da;
      I.q.cj_dx.d = I.q.cj_dx.v / M;
    } else if (param == PF_PARAM_THETA_BOT) {
      const double th = I.raw_prm.theta_bot_deg * M_PI / 180.0;
      const double s2eta = 1.4142135623730951 * I.p.eta;
      I.q.gbot = Dual(std::cos(th) / s2eta, -std::sin(th) / s2eta);
    } else {
      throw ApiError(PF_ERR_ARG, "param must be PF_PARAM_WI, PF_PARAM_THETA_BOT, PF_PARAM_PHI0 or PF_PARAM_MOBILITY");
    }
  }
};

}  // namespace pf

namespace pf {

static void tangent_run(ImplBase& src, cudaStream_t stream, int nsteps, int param, int objective, int flags,
                        const void* dir, int dir_on_device, double out[2]) {
  if (nsteps < 1) throw ApiError(PF_ERR_ARG, "nsteps must be >= 1");
  if (objective != PF_OBJ_WETTED && objective != PF_OBJ_CENTROID_Z)
    throw ApiError(PF_ERR_ARG, "objective must be PF_OBJ_WETTED or PF_OBJ_CENTROID_Z");
  if (flags & ~PF_STEP_CH_ONLY) throw ApiError(PF_ERR_ARG, "flags: 0 or PF_STEP_CH_ONLY");
  if (param == PF_PARAM_WI && (flags & PF_STEP_CH_ONLY))
    throw ApiError(PF_ERR_ARG, "Wi has no effect on CH steps with the velocity fixed");
  TangentRun run(src, stream);
  run.seed(param, dir, dir_on_device);
  run.impl->step(nsteps, flags);
  Dual w[6];
  run.impl->diagnostics_wide(w);
  const Dual J = objective == PF_OBJ_WETTED ? w[2] : w[5];
  out[0] = J.v;
  out[1] = param == PF_PARAM_THETA_BOT ? J.d * M_PI / 180.0 : J.d;  // theta per degree, as pf_adjoint
}

}  // namespace pf

extern "C" {

int pf_tangent_ex(pf_ctx* ctx, int nsteps, int param, int objective, int flags, const void* dir, int dir_on_device,
                  double out[2]) {
  if (!ctx || !out) return PF_ERR_ARG;
  return guarded(ctx, [&] {
    pf::tangent_run(*ctx->impl, ctx->stream, nsteps, param, objective, flags, dir, dir_on_device, out);
  });
}

int pf_tangent(pf_ctx* ctx, int nsteps, int param, int objective, double out[2]) {
  return pf_tangent_ex(ctx, nsteps, param, objective, 0, nullptr, 0, out);
}

int pf_batch_tangent(pf_batch* b, int problem, int nsteps, int param, int objective, int flags, const void* dir,
                     int dir_on_device, double out[2]) {
  if (!b || !out) return PF_ERR_ARG;
  return bguarded(b, [&] {
    pf::tangent_run(*b->impl->problem(problem), b->stream, nsteps, param, objective, flags, dir, dir_on_device, out);
  });
}

}  // extern "C"
