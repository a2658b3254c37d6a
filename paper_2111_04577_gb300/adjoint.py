"""torch.autograd.Functions around the library's gradients.

    J = CHObjective.apply(phi0, theta_bot_deg, mobility, solver, nsteps, ckpt_every, objective)
    J = CoupledObjective.apply(wi, theta_bot_deg, solver, params, nsteps, objective)
    J = CoupledAdjointObjective.apply(phi0, theta_bot_deg, mobility, wi, solver, params, nsteps, ckpt_every,
                                      objective)

CHObjective.forward loads phi0 (phi^{-1} = phi^0) into the solver and runs
nsteps CH steps on the GPU (velocity fixed) to evaluate the objective; its
backward reloads phi0 and calls pf_adjoint, which re-runs the forward with
checkpoints and returns dJ/dphi0, dJ/dtheta_bot (per degree) and
dJ/dmobility.  CoupledObjective takes the whole coupled step through
pf_tangent (forward-mode derivatives in Wi and theta_bot, 2D or 3D).
CoupledAdjointObjective takes the whole coupled 2D step through one reverse
sweep (pf_adjoint_ex): dJ/dphi0, dJ/dtheta_bot, dJ/dmobility and dJ/dWi at
once.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding


class CHObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, theta_bot_deg, mobility, solver, params, nsteps, ckpt_every, objective):
        p = params.__class__(**params.as_dict())
        p.theta_bot_deg = float(theta_bot_deg)
        p.mobility = float(mobility)
        solver.set_params(p)
        phi_np = phi0.detach().cpu().numpy().astype(solver.dtype)
        solver.set("phi", phi_np)
        solver.step(int(nsteps), binding.PF_STEP_CH_ONLY)
        dg = solver.diagnostics()
        J = dg["wetted"] if objective == binding.PF_OBJ_WETTED else dg["centroid"][2]
        ctx.state = (solver, phi_np, int(nsteps), int(ckpt_every), int(objective))
        ctx.dtypes = (phi0.dtype, phi0.device)
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        solver, phi_np, nsteps, ck, obj = ctx.state
        solver.set("phi", phi_np)
        _, dth, dm, dphi = solver.adjoint(nsteps, ck, obj)
        dt, dev = ctx.dtypes
        g = float(gJ)
        dphi_t = torch.from_numpy(np.asarray(dphi, dtype=np.float64) * g).to(dtype=dt, device=dev)
        return (dphi_t, torch.tensor(dth * g, dtype=torch.float64), torch.tensor(dm * g, dtype=torch.float64),
                None, None, None, None, None)


class CoupledObjective(torch.autograd.Function):
    """J after nsteps full coupled steps (CH, NS, LCR) from the solver's
    current state, as a function of Wi and theta_bot (degrees).  forward runs
    pf_tangent for each parameter that requires a gradient (one
    derivative-carrying run each, which also yields J), backward scales those
    derivatives.  The solver is not advanced."""

    @staticmethod
    def forward(ctx, wi, theta_bot_deg, solver, params, nsteps, objective):
        p = params.__class__(**params.as_dict())
        p.wi = float(wi)
        p.theta_bot_deg = float(theta_bot_deg)
        solver.set_params(p)
        need = (ctx.needs_input_grad[0], ctx.needs_input_grad[1])
        grads = [0.0, 0.0]
        J = None
        for k, param in enumerate((binding.PF_PARAM_WI, binding.PF_PARAM_THETA_BOT)):
            if need[k]:
                J, grads[k] = solver.tangent(int(nsteps), param, int(objective))
        if J is None:  # no gradient wanted: the value alone, from a run on a copy of the state
            J, _ = solver.tangent(int(nsteps), binding.PF_PARAM_THETA_BOT, int(objective))
        ctx.grads = grads
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        g = float(gJ)
        return (torch.tensor(ctx.grads[0] * g, dtype=torch.float64),
                torch.tensor(ctx.grads[1] * g, dtype=torch.float64), None, None, None, None)


class CoupledAdjointObjective(torch.autograd.Function):
    """J after nsteps coupled 2D steps (CH, restriction, NS, LCR) from phi0 and
    the solver's current flow and polymer state, as a function of phi0,
    theta_bot (degrees), the mobility and Wi.  forward loads phi0 and runs the
    reverse sweep once (it yields J and every gradient); backward scales the
    gradients.  The solver is left at step nsteps."""

    @staticmethod
    def forward(ctx, phi0, theta_bot_deg, mobility, wi, solver, params, nsteps, ckpt_every, objective):
        p = params.__class__(**params.as_dict())
        p.theta_bot_deg = float(theta_bot_deg)
        p.mobility = float(mobility)
        p.wi = float(wi)
        solver.set_params(p)
        solver.set("phi", phi0.detach().cpu().numpy().astype(solver.dtype))
        J, dth, dm, dwi, dphi = solver.adjoint_coupled(int(nsteps), int(ckpt_every), int(objective))
        ctx.grads = (dphi, dth, dm, dwi)
        ctx.dtypes = (phi0.dtype, phi0.device)
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        dphi, dth, dm, dwi = ctx.grads
        dt, dev = ctx.dtypes
        g = float(gJ)
        dphi_t = torch.from_numpy(np.asarray(dphi, dtype=np.float64) * g).to(dtype=dt, device=dev)
        return (dphi_t, torch.tensor(dth * g, dtype=torch.float64), torch.tensor(dm * g, dtype=torch.float64),
                torch.tensor(dwi * g, dtype=torch.float64), None, None, None, None, None)
