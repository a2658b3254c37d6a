"""torch.autograd.Function around the library's hand-written CH adjoint.

    J = CHObjective.apply(phi0, theta_bot_deg, mobility, solver, nsteps, ckpt_every, objective)

forward: loads phi0 (phi^{-1} = phi^0) into the solver and runs nsteps CH
steps on the GPU (velocity fixed) to evaluate the objective; backward: reloads
phi0 and calls pf_adjoint, which re-runs the forward with checkpoints and
returns dJ/dphi0, dJ/dtheta_bot (per degree) and dJ/dmobility.
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
