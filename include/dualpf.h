/*
 * dualpf.h -- C ABI of the GB300 dual-resolution phase-field library.
 *
 * One time step of the coupled Cahn-Hilliard / Navier-Stokes / Oldroyd-B
 * problem of arXiv 2111.04577 (Section 2, Eqs. NS1-NS16 with the
 * log-conformation of Eqs. NS17-NS24), discretised as in Section 3:
 * phase field phi on a mesh twice as fine as the flow mesh (Section 3.1,
 * Fig. 1), Dong's split Cahn-Hilliard scheme (Section 3.2.1, Eqs. NS25-NS34),
 * the constant-coefficient Navier-Stokes split (Section 3.2.2, Eqs.
 * NS35-NS39) and the RK2-TVD log-conformation update (Section 3.2.3,
 * Eqs. NS40-NS46), coupled by the transfers of Eqs. dual1-dual3.
 *
 * Conventions shared by every entry point
 *  - Return value: 0 on success, a negative PF_ERR_* code otherwise; the
 *    message of the last failure is returned by pf_last_error().
 *  - Streams: all device work is enqueued on the cudaStream_t given to
 *    pf_init_grid; given NULL, the context creates and owns a non-blocking
 *    stream (the legacy default stream cannot be captured into a graph).
 *    pf_set_fields from host memory, pf_get_fields, pf_diagnostics and
 *    pf_profile synchronise that stream before returning.
 *  - Ownership: the library allocates and owns every field buffer of a
 *    context; callers own the src/dst buffers they pass in.  Nothing is
 *    retained after a call returns.
 *  - Layout: every field is a dense array, x fastest, then y, then z
 *    (C order [z][y][x]).  Coarse mesh nx x ny x nz cells of side dx
 *    (ny = 1: two-dimensional x-z problem), periodic in x and y, walls at
 *    z = 0 and z = lz.  u and v live on the x- and y-faces (nz*ny*nx values,
 *    u[k][j][i] on the face x = i*dx), w on the z-faces including both walls
 *    ((nz+1)*ny*nx values, w = 0 on the walls), p at centres.  The phase
 *    field lives on the fine mesh of r*nx x ry*ny x r*nz cells (r = 2 for
 *    dual resolution, 1 for single resolution; ry = r in 3D, 1 in 2D);
 *    coarse cell i holds fine cells r*i .. r*i+r-1.  Tensor fields (THETA,
 *    TAU, TAU_OLD) are component-major: 3 components (xx, xz, zz) in 2D,
 *    6 (xx, yy, zz, xy, xz, yz) in 3D, each a coarse centre array.
 *  - Element type: a context computes and stores in double (PF_FP64) or in
 *    float with FP64 kept in the named places (PF_MIXED: the contact-line
 *    flux, the pressure zero mode and the global reductions; PF_MIXED_Z64
 *    adds the wall-normal tridiagonal eliminations of every transform solve;
 *    PF_MIXED_Z2F runs those eliminations in double-float instead, two FP32
 *    words per value with error-free transformations: a 48-bit significand,
 *    relative rounding about 2^-47 against FP64's 2^-53, on the FP32 pipes).
 *    pf_set_fields and pf_get_fields move elements of the context's storage
 *    type: double for PF_FP64, float otherwise (see pf_field_info).
 */
#ifndef DUALPF_H
#define DUALPF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PF_OK = 0,
  PF_ERR_ARG = -1,          /* invalid argument or call order                 */
  PF_ERR_DISCRIMINANT = -2, /* S below the bound of Eq. NS30                  */
  PF_ERR_UNSUPPORTED = -3,  /* a size not 2^a3^b5^c7^d, an option a path lacks  */
  PF_ERR_NONFINITE = -4,    /* the phi-sum check (FP64 accumulator) saw NaN/Inf */
  PF_ERR_TIMEOUT = -5,      /* a bounded device-side wait expired             */
  PF_ERR_CUDA = -6,         /* a CUDA runtime call failed                     */
  PF_ERR_NOMEM = -7         /* device allocation failed                       */
};

enum { PF_FP64 = 0, PF_MIXED = 1, PF_MIXED_Z64 = 2, PF_MIXED_Z2F = 3 };

/* Field identifiers for pf_set_fields / pf_get_fields. */
enum {
  PF_PHI = 0,      /* fine, phi^n                                   */
  PF_PHI_OLD = 1,  /* fine, phi^{n-1}                               */
  PF_U = 2, PF_U_OLD = 3,
  PF_V = 4, PF_V_OLD = 5,
  PF_W = 6, PF_W_OLD = 7,
  PF_P = 8, PF_P_OLD = 9,
  PF_THETA = 10,   /* log-conformation Theta^n (Eq. NS20)           */
  PF_TAU = 11,     /* weighted polymer stress tau^n = (1+phi)/2 tau_p (Eq. NS12) */
  PF_TAU_OLD = 12,
  PF_G = 13,       /* fine chemical potential G^n (Eq. NS5), read-only */
  PF_PHI_REM = 14, /* fine, read-only: the rounding remainders of phi^n in FP32
                      contexts (phi = value + remainder), zeros in PF_FP64     */
  PF_NFIELDS = 15
};

/* Step flags for pf_step_ex. */
enum {
  PF_STEP_CH_ONLY = 1,  /* advance phi only (velocity held fixed); for tests */
  PF_STEP_NO_GRAPH = 2  /* launch kernels directly instead of replaying the CUDA graph */
};

typedef struct pf_ctx pf_ctx;

/* Grid of Section 3.1 (Fig. 1).  nx, ny, nz: COARSE cells, each of the form
 * 2^a 3^b 5^c 7^d, nz >= 2; cells must be cubes (lx/nx = ly/ny = lz/nz;
 * ly is ignored when ny = 1).  dual = 1: phi on the 2x finer mesh, 0: phi on
 * the coarse mesh (single resolution). */
typedef struct {
  int nx, ny, nz;
  double lx, ly, lz;
  int precision; /* PF_FP64 | PF_MIXED | PF_MIXED_Z64 | PF_MIXED_Z2F */
  int dual;
} pf_grid_desc;

/* Physical parameters (Section 2.1; the droplet phase phi = +1 is fluid 1).
 * mu1, mu2: total viscosities; the droplet is viscoelastic when wi > 0 and
 * beta < 1, with solvent mu_s1 = beta mu1 and polymer mu_p1 = (1-beta) mu1
 * (Eq. NS12, second approach).  polymer_approach = 1 selects the first
 * approach instead (Eq. NS11): mu_p, lambda_H and alpha are linear in phi
 * between the droplet's (mu_p1, wi, alpha_giesekus) and phase 2's (mu_p2,
 * wi2, alpha_giesekus2) at each coarse centre, tau = tau_p (no phase weight),
 * phase 2's solvent viscosity stays mu2; it needs wi, wi2 > 0 when either
 * phase has a polymer.  advection = 1 takes the paper's WENO5-Z face values
 * (Section 3.2.1; before Eq. NS40) for div(u phi) of the CH step and div(u Theta)
 * of the polymer update instead of the central flux; it needs at least 4
 * coarse cells along every axis, and the batch and the reverse sweeps reject
 * it.  mobility: M of Eq. NS1.  sigma, eta: Eq. NS7.
 * theta_*_deg: equilibrium angles of Eq. NS16 at z = 0 and z = lz, measured
 * through phase 1.  dw: the wall relaxation D_w >= 0 of Eq. NS15 (0: static
 * contact angle); with D_w > 0 the wall flux of Eq. NS34 holds the BDF2 time
 * derivative of the wall value (1.5 phi_0 - 0.5 phi_1), implicit, and the wall
 * advection u_w d_x phi*, and the two CH solves take it as a Robin condition
 * (the batch, forward mode and the reverse sweeps reject D_w > 0).  alpha_giesekus:
 * the Giesekus mobility alpha of Eqs. NS18/NS22 in [0, 1), constant in the
 * viscoelastic phase (0: Oldroyd-B).  S = 0 selects the smallest S of Eq. NS30; nu_m = 0
 * selects nu_m = max(mu_s)/(2 min(rho)) (text after Eq. NS39).  uw_*: x
 * velocity of the walls.  g*: body acceleration (f_ext = rho g). */
typedef struct {
  double rho1, rho2, mu1, mu2;
  double sigma, eta, mobility;
  double theta_bot_deg, theta_top_deg, dw;
  double wi, beta, alpha_giesekus;
  double dt, S, nu_m;
  double uw_bot, uw_top, gx, gy, gz;
  double mu_p2, wi2, alpha_giesekus2; /* phase 2's polymer (polymer_approach 1)      */
  int polymer_approach;               /* 0: Eq. NS12 (default), 1: Eq. NS11            */
  int advection;                      /* 0: central second order (default), 1: WENO5-Z */
} pf_params;

/* Create a context for grid *g and allocate all fields on the current CUDA
 * device (all zero).  stream: a cudaStream_t, or NULL for a private one.  On success *out owns
 * the context; release it with pf_destroy.  Errors: PF_ERR_ARG (bad sizes,
 * non-cubic cells), PF_ERR_UNSUPPORTED (a size with a prime factor > 7, or more than 4096
 * fine z rows),
 * PF_ERR_NOMEM, PF_ERR_CUDA. */
int pf_init_grid(pf_ctx** out, const pf_grid_desc* g, void* stream);

/* Set the physical parameters and derive the scheme's constants:
 * lambda (Eq. NS7), S (Eq. NS30), alpha (Eq. NS29), c = alpha + S/eta^2,
 * rho0 and nu_m (text after Eq. NS39).  May be called again between steps.
 * Errors: PF_ERR_ARG (non-positive rho, sigma, eta, mobility, dt, an angle
 * outside [0, 180], alpha_giesekus or alpha_giesekus2 outside [0, 1),
 * polymer_approach or advection not 0 or 1, approach 1 without wi, wi2 > 0,
 * WENO5-Z on fewer than 4 coarse cells along an axis,
 * dw < 0), PF_ERR_DISCRIMINANT (S below Eq. NS30). */
int pf_set_params(pf_ctx* ctx, const pf_params* prm);

/* Number of elements and element size (bytes) of a field. */
int pf_field_info(const pf_ctx* ctx, int field_id, size_t* count, size_t* elem_bytes);

/* Copy one field into the context from host (src_on_device = 0) or device
 * memory.  bytes must equal count*elem_bytes of pf_field_info.  Setting
 * PF_PHI also sets PF_PHI_OLD to the same values, and likewise U/V/W/P/TAU set
 * their *_OLD twin (the start-up reading phi^{-1} = phi^0; set the _OLD field
 * afterwards to resume from a full BDF2 state).  Errors: PF_ERR_ARG. */
int pf_set_fields(pf_ctx* ctx, int field_id, const void* src, size_t bytes, int src_on_device);

/* Advance nsteps time steps (Section 3.2 order: CH, restriction, NS,
 * polymer), replaying a captured CUDA graph per step.  Every 50 steps and
 * at the end, a sum of phi (float4 loads, FP64 accumulator) is checked for
 * NaN/Inf -> PF_ERR_NONFINITE.
 * Asynchronous otherwise. */
int pf_step(pf_ctx* ctx, int nsteps);
int pf_step_ex(pf_ctx* ctx, int nsteps, int flags);

/* Copy one field out (synchronises the stream).  bytes as for pf_set_fields. */
int pf_get_fields(pf_ctx* ctx, int field_id, void* dst, size_t bytes, int dst_on_device);

/* FP64 global reductions of phi^n (synchronises the stream):
 * out[0] mass = sum(phi) h^d;
 * out[1] free energy lambda sum(|grad phi|^2/2 + (phi^2-1)^2/(4 eta^2)) h^d
 *        + sum_walls f_w(phi_w) h^(d-1)  (Eqs. NS5-NS7, NS16);
 * out[2] wetted length (2D) / area (3D) sum_bottom (1+phi_w)/2 h^(d-1);
 * out[3..5] centroid of (1+phi)/2 in x, y, z.
 * phi_w = 1.5 phi_0 - 0.5 phi_1 is the wall value of the contact-angle law. */
int pf_diagnostics(pf_ctx* ctx, double out[6]);

/* Per-kernel profile: run nsteps steps launching kernels directly (no graph)
 * with a CUDA event before each launch, and report for each distinct kernel
 * its name (NUL-terminated, PF_PROFILE_NAME bytes per entry in `names`), its
 * summed device time per step in milliseconds (`avg_ms`, averaged over the
 * steps) and its number of launches per step (`counts`), in launch order.
 * *n_entries receives the number of entries written (<= max_entries) and
 * *launches_per_step the number of kernel launches one step makes.  The
 * state advances by nsteps steps exactly as pf_step_ex would.  Synchronises.
 * Errors: PF_ERR_ARG, PF_ERR_CUDA. */
#define PF_PROFILE_NAME 48
int pf_profile(pf_ctx* ctx, int nsteps, int flags, int max_entries, char* names, double* avg_ms,
               int* counts, int* n_entries, int* launches_per_step);

/* ------------------------------------------------------------------------
 * Batched sweep: many independent two-dimensional problems of uneven size
 * (each its own grid and parameters, one precision for all), advanced
 * together by ONE persistent kernel launch per time step, replayed from a
 * CUDA graph.  Each problem takes exactly the step of pf_step (same kernels'
 * device code, same order of Section 3.2); the persistent CTAs walk a
 * pass-major list of (problem, pass, tile) items and wait, with a bounded
 * spin, for the previous pass of the same problem.  A wait that runs out
 * makes pf_batch_step return PF_ERR_TIMEOUT (the status is sticky).
 * Field access and diagnostics take a problem index 0..nproblems-1 and
 * behave as pf_set_fields / pf_get_fields / pf_diagnostics on that problem.
 * Precision PF_FP64 or PF_MIXED (PF_MIXED_Z64: PF_ERR_UNSUPPORTED); the
 * central advection flux and the static contact angle only (advection = 1 or
 * dw > 0: PF_ERR_UNSUPPORTED).
 * ------------------------------------------------------------------------ */
typedef struct pf_batch pf_batch;
int pf_batch_create(pf_batch** out, int nproblems, const pf_grid_desc* grids, const pf_params* params,
                    void* stream);
int pf_batch_field_info(const pf_batch* b, int problem, int field_id, size_t* count, size_t* elem_bytes);
int pf_batch_set_fields(pf_batch* b, int problem, int field_id, const void* src, size_t bytes, int src_on_device);
int pf_batch_get_fields(pf_batch* b, int problem, int field_id, void* dst, size_t bytes, int dst_on_device);
int pf_batch_step(pf_batch* b, int nsteps);
int pf_batch_diagnostics(pf_batch* b, int problem, double out[6]);
/* pf_adjoint on one problem of the batch (its own buffers and parameters):
 * the same CH adjoint, run with the single-problem kernels; afterwards the
 * problem holds phi^N.  Errors as pf_adjoint, PF_ERR_ARG for a bad index. */
int pf_batch_adjoint(pf_batch* b, int problem, int nsteps, int ckpt_every, int objective, double out[3], void* dphi0,
                     int dphi0_on_device);
/* pf_adjoint_ex on one problem of the batch (its own buffers, parameters and
 * the single-problem kernels); afterwards the problem holds step N.  Errors as
 * pf_adjoint_ex, PF_ERR_ARG for a bad index. */
int pf_batch_adjoint_ex(pf_batch* b, int problem, int nsteps, int ckpt_every, int objective, int flags, double out[4],
                        void* dphi0, int dphi0_on_device);
const char* pf_batch_last_error(const pf_batch* b);
void pf_batch_destroy(pf_batch* b);

/* Allocation-free diagnostics.  The paper has no counterpart: this is a
 * service for callers that may not allocate device memory (an application
 * whose memory pool owns the whole GPU, an allocator that forbids
 * cudaMalloc/cudaFree, a real-time loop in which an allocation would stall).
 * It computes the six FP64 reductions of pf_diagnostics from a phase field
 * the caller already holds on the current device -- phi_device points to the
 * fine mesh of *g in the element type of g->precision (double for PF_FP64,
 * float for the mixed precisions), layout as above -- with no context and no allocation
 * of any kind.  Its scratch is one file-scope device array of 1 MiB that
 * every GPU which loads the library holds until the process exits; the
 * phase field may have at most 134,217,728 fine cells, larger fields are
 * rejected with PF_ERR_UNSUPPORTED.  Work is enqueued on `stream` (a
 * cudaStream_t, NULL for the legacy stream) and the call synchronises it.
 * Every call resolves the array's device address with cudaGetSymbolAddress
 * (cheap; no allocation); make the first call on a device before any stream
 * capture, since the runtime may load the module at that call.  All calls share the array: calls
 * that overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  Each call overwrites every slot it reads, so
 * the contents left by an earlier call never matter.  Errors: PF_ERR_ARG,
 * PF_ERR_UNSUPPORTED, PF_ERR_CUDA. */
int pf_diagnostics_noalloc(const pf_grid_desc* g, const pf_params* prm, const void* phi_device, double out[6],
                           void* stream);

/* Discrete adjoint of the Cahn-Hilliard step (Section 3.2.1) with the velocity
 * held fixed (the flow fields of the context are not advanced): gradients of
 * an objective of phi^N after nsteps steps from the context's current state,
 * taken as phi^0 with phi^{-1} = phi^0.
 *   objective PF_OBJ_WETTED:     wetted length/area sum_bottom (1 + phi_w)/2 h^(d-1)
 *   objective PF_OBJ_CENTROID_Z: z-centroid of (1 + phi)/2
 * out[0] = J, out[1] = dJ/d theta_bot (per degree), out[2] = dJ/d mobility.
 * dphi0 (may be NULL) receives dJ/d phi^0 (fine mesh, storage element type;
 * host memory, or device memory when dphi0_on_device).  The forward sweep
 * stores the BDF2 state every ckpt_every steps; the reverse sweep recomputes
 * each segment, then runs the transposed kernels and the same (symmetric)
 * transform solves.  The context is left at phi^N.  The mobility derivative
 * follows S when S = 0 selects the bound of Eq. NS30.
 * Errors: PF_ERR_ARG, PF_ERR_DISCRIMINANT, PF_ERR_UNSUPPORTED (WENO5-Z
 * advection, D_w > 0), PF_ERR_CUDA, PF_ERR_NOMEM. */
enum { PF_OBJ_WETTED = 0, PF_OBJ_CENTROID_Z = 1 };
int pf_adjoint(pf_ctx* ctx, int nsteps, int ckpt_every, int objective, double out[3], void* dphi0,
               int dphi0_on_device);

/* Discrete adjoint of the whole coupled step (Sections 3.2.1-3.2.3: the CH
 * update, the restriction of Eqs. dual2-dual3, the NS projection of Eqs.
 * NS35-NS39 and the log-conformation update of Eqs. NS40-NS46), on a 2D
 * context: gradients of an objective of phi^N after nsteps coupled steps from
 * the context's current state (phi^{-1} = phi^0, u^{-1} = u^0, p^{-1} = p^0,
 * tau^{-1} = tau^0), in one reverse sweep.
 *   flags: PF_ADJ_COUPLED (required; 0 is reserved for pf_adjoint's CH-only
 *   sweep, which this call then runs with out[3] = 0).
 * out[0] = J, out[1] = dJ/d theta_bot (per degree), out[2] = dJ/d mobility,
 * out[3] = dJ/d lambda_H (the Weissenberg number; 0 for a Newtonian droplet).
 * dphi0 (may be NULL) receives dJ/d phi^0 as for pf_adjoint.  The forward
 * sweep stores the whole state every ckpt_every steps; each segment is
 * recomputed, keeping the state of each of its steps (memory: ckpt_every + 1
 * states), and each reverse step re-runs its forward step for the restricted
 * fields, the polymer's first stage and the wall flux.  The linear parts
 * (projection, solves, restriction, prolongation, advection and velocity
 * gradient stencils) are transposed; the nonlinear per-cell parts (momentum
 * right side, the polymer's right side and stress) are differentiated exactly
 * with dual numbers.  The context is left at step N.
 * Errors: PF_ERR_ARG, PF_ERR_UNSUPPORTED (a 3D context, PF_ADJ_COUPLED on a
 * derivative-carrying context, polymer approach 1, WENO5-Z advection, D_w > 0),
 * PF_ERR_CUDA, PF_ERR_NOMEM. */
enum { PF_ADJ_COUPLED = 1 };
int pf_adjoint_ex(pf_ctx* ctx, int nsteps, int ckpt_every, int objective, int flags, double out[4], void* dphi0,
                  int dphi0_on_device);

/* Sensitivity of an objective to one scalar parameter through the whole
 * coupled step of Section 3.2 (forward mode): the Cahn-Hilliard step with its
 * wetting condition (Eqs. NS25-NS34), the restriction (Eq. dual2), the
 * projection (Eqs. NS35-NS39) and the log-conformation update (Eqs.
 * NS40-NS46), velocity and polymer stress included.  From the context's
 * current state, a derivative-carrying FP64 copy of the state (each value
 * paired with its derivative with respect to `param`) is advanced nsteps full
 * steps; the context itself is not advanced.  The derivative follows by the
 * chain rule through every kernel, so it is exact up to FP64 rounding: the
 * value a reverse sweep gives for this one parameter.
 *   param PF_PARAM_WI:        the Weissenberg number Wi = lambda_H (needs a
 *                             viscoelastic context, wi > 0 and beta < 1)
 *   param PF_PARAM_THETA_BOT: the bottom contact angle, per degree
 *   param PF_PARAM_MOBILITY:  the mobility M (with S following M when S = 0
 *                             selects the bound of Eq. NS30, as pf_adjoint)
 *   objective: PF_OBJ_WETTED or PF_OBJ_CENTROID_Z, as pf_adjoint
 * out[0] = J after nsteps steps, out[1] = dJ/d param.  The copy holds every
 * field in 16 bytes per value (value and derivative) besides the context's
 * own; its kernels are those of PF_FP64 run on that pair.
 * Errors: PF_ERR_ARG, PF_ERR_UNSUPPORTED (D_w > 0), PF_ERR_NONFINITE, PF_ERR_CUDA,
 * PF_ERR_NOMEM. */
enum { PF_PARAM_WI = 0, PF_PARAM_THETA_BOT = 1, PF_PARAM_PHI0 = 2, PF_PARAM_MOBILITY = 3 };
int pf_tangent(pf_ctx* ctx, int nsteps, int param, int objective, double out[2]);
/* pf_tangent with two more choices.
 *   flags PF_STEP_CH_ONLY: Cahn-Hilliard steps only, the velocity held fixed (the
 *     model pf_adjoint differentiates); PF_PARAM_WI is then an error.
 *   param PF_PARAM_PHI0: the directional derivative <dJ/dphi^0, dir> along the
 *     fine-mesh array dir (FP64, layout of PF_PHI, host or device memory as
 *     dir_on_device says, read only), with phi^{-1} = phi^0 as at start-up:
 *     the derivative parts of PF_PHI and PF_PHI_OLD are both set to dir.
 * dir is ignored for the other parameters. */
int pf_tangent_ex(pf_ctx* ctx, int nsteps, int param, int objective, int flags, const void* dir, int dir_on_device,
                  double out[2]);
/* pf_tangent_ex on one problem of a batch (its state, grid and parameters);
 * the problem is not advanced.  Errors as pf_tangent_ex, PF_ERR_ARG for a bad
 * index. */
int pf_batch_tangent(pf_batch* b, int problem, int nsteps, int param, int objective, int flags, const void* dir,
                     int dir_on_device, double out[2]);

/* Launch-shape knobs picked by the autotuner (paper_2111_04577_gb300/autotune.py);
 * 0 restores the built-in default.  They change only how the work is tiled,
 * never the arithmetic of a cell.
 *   PF_TUNE_XFFT_PAIRS   pairs of x-lines per CTA of the x transforms (1..16)
 *   PF_TUNE_YFFT_COLS    kx columns per CTA of the y transforms (power of two <= 32)
 *   PF_TUNE_ZSOLVE_COLS  kx columns per CTA of the z solves (multiple of 16, <= 64); halved
 *                        for a long z line until its CTA fits (two threads per column and
 *                        16-row segment, at most 512)
 *   PF_TUNE_ROW_BLOCK    threads per CTA of the row kernels (multiple of 32)
 *   PF_TUNE_CH_ZCHUNK    fine z planes one CTA of the 3D CH right side walks (>= 2)
 *   PF_TUNE_CH_MINB      CTAs per SM the 3D CH right side's registers are sized for (2, 3, 4;
 *                        4 takes 14-row tiles of 224 threads, whose shared memory lets four fit)
 *   PF_TUNE_NS_MINB      CTAs per SM the NS right side's registers are sized for (3, 4)
 *   PF_TUNE_G_ZCHUNK     coarse layers one CTA of the 3D restriction walks (>= 1)
 *   PF_TUNE_NS_KZ        z rows one CTA of the NS right side walks (1..64)
 * Errors: PF_ERR_ARG for an unknown knob or a value that does not fit. */
enum { PF_TUNE_XFFT_PAIRS = 0, PF_TUNE_YFFT_COLS = 1, PF_TUNE_ZSOLVE_COLS = 2, PF_TUNE_ROW_BLOCK = 3, PF_TUNE_CH_ZCHUNK = 4,
       PF_TUNE_CH_MINB = 5, PF_TUNE_NS_MINB = 6, PF_TUNE_G_ZCHUNK = 7,
       PF_TUNE_NS_KZ = 8, PF_TUNE_COUNT = 9 };
int pf_set_tuning(pf_ctx* ctx, int knob, int value);
int pf_get_tuning(const pf_ctx* ctx, int knob, int* value);

/* Message of the last failed call on ctx (or of the last failed
 * pf_init_grid when ctx is NULL).  Valid until the next call. */
const char* pf_last_error(const pf_ctx* ctx);

/* Free all device memory and graphs of ctx.  ctx may be NULL. */
void pf_destroy(pf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DUALPF_H */
