"""Differentiable FP64 restatement of the oracle's Cahn-Hilliard step (test
infrastructure only).

The same step as oracle.ch.ch_step (Section 3.2.1, Eqs. NS25-NS34, literal
R1 form) written with plain PyTorch CPU ops in float64 so that torch.autograd
yields the exact discrete adjoint: gradients of an objective after N steps
with respect to phi0, the bottom contact angle and the mobility.  The two
constant-coefficient solves use dense LU of the assembled operator, so it is
meant for tiny grids only.  The velocity is held fixed (u* = u).  S takes the
default of Eq. NS30 (its smallest admissible value), so it moves with M.
"""
import math

import numpy as np
import torch

from . import operators as op


def _lap_matrix(nz, ny, nx, h):
    """Dense L_N (periodic x, y; mirror ghosts at both z walls), row-major [k, j, i]."""
    n = nz * ny * nx
    A = np.zeros((n, n))
    idx = lambda k, j, i: (k * ny + j) * nx + i
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = idx(k, j, i)
                for di in (-1, 1):
                    A[r, idx(k, j, (i + di) % nx)] += 1
                    A[r, r] -= 1
                if ny > 1:
                    for dj in (-1, 1):
                        A[r, idx(k, (j + dj) % ny, i)] += 1
                        A[r, r] -= 1
                for dk in (-1, 1):
                    if 0 <= k + dk < nz:
                        A[r, idx(k + dk, j, i)] += 1
                        A[r, r] -= 1
    return torch.tensor(A / h ** 2)


class CHTorch:
    def __init__(self, grid, prm, vel):
        self.g = grid
        self.prm = dict(prm)
        nz, ny, nx = grid.fine_shape
        self.shape = (nz, ny, nx)
        self.L = _lap_matrix(nz, ny, nx, grid.h)
        self.I = torch.eye(nz * ny * nx, dtype=torch.float64)
        uf, vf, wf = op.prolong_velocity(vel[0], vel[1], vel[2], grid.r, grid.ry, grid.dim)
        self.uf = torch.tensor(uf)
        self.vf = torch.tensor(vf)
        self.wf = torch.tensor(wf)

    def lapN(self, a):
        return (self.L @ a.reshape(-1)).reshape(self.shape)

    def advection(self, ph):
        h = self.g.h
        xm = torch.roll(ph, 1, dims=2)
        Fx = self.uf * 0.5 * (xm + ph)
        A = (torch.roll(Fx, -1, dims=2) - Fx) / h
        if self.g.dim == 3:
            Fy = self.vf * 0.5 * (torch.roll(ph, 1, dims=1) + ph)
            A = A + (torch.roll(Fy, -1, dims=1) - Fy) / h
        inner = self.wf[1:-1] * 0.5 * (ph[:-1] + ph[1:])
        zero = torch.zeros((1,) + ph.shape[1:], dtype=ph.dtype)
        Fz = torch.cat([zero, inner, zero], 0)
        return A + (Fz[1:] - Fz[:-1]) / h

    def step(self, pn, po, theta_bot_deg, mobility):
        """One step.  `mobility` is a scalar tensor, or a triple (M_a, M_b, M_s) of
        copies of it entering the 1/(M lambda dt) term, the advection term 1/(M lambda)
        and S of Eq. NS30 respectively (their gradients add up to dJ/dM)."""
        p = self.prm
        h, eta, dt = self.g.h, p["eta"], p["dt"]
        g0 = 1.5
        lam = 3.0 * p["sigma"] * eta / (2.0 * math.sqrt(2.0))
        Ma, Mb, Ms = mobility if isinstance(mobility, tuple) else (mobility,) * 3
        S = eta ** 2 * torch.sqrt(4.0 * g0 / (Ms * lam * dt))      # Eq. NS30, equality
        alpha = -S / (2.0 * eta ** 2)                               # Eq. NS29 at zero discriminant
        c = alpha + S / eta ** 2
        phs = 2 * pn - po
        phh = 2 * pn - 0.5 * po
        A = self.advection(phs)
        hh = phs * (phs * phs - 1) / eta ** 2 - S / eta ** 2 * phs
        s2 = math.sqrt(2.0)
        cb = torch.cos(theta_bot_deg * math.pi / 180.0)
        ct = math.cos(math.radians(p["theta_top_deg"]))
        wb = 1.5 * phs[0] - 0.5 * phs[1]
        wt = 1.5 * phs[-1] - 0.5 * phs[-2]
        gb = cb * (1 - wb * wb) / (s2 * eta)
        gt = ct * (1 - wt * wt) / (s2 * eta)
        zero = torch.zeros_like(phs[1:-1])
        B = torch.cat([(gb / h)[None], zero, (gt / h)[None]], 0)
        R1 = phh / (dt * Ma * lam) - A / (Mb * lam) + self.lapN(hh) - c * B
        psi = torch.linalg.solve(self.L - c * self.I, R1.reshape(-1)).reshape(self.shape)
        phi = torch.linalg.solve(self.L + alpha * self.I, (psi - B).reshape(-1)).reshape(self.shape)
        return phi


def objective(phi, grid, which):
    """'wetted': sum over the bottom (1 + phi_w)/2 h^(d-1); 'centroid': z-centroid of (1+phi)/2."""
    h = grid.h
    if which == "wetted":
        wb = 1.5 * phi[0] - 0.5 * phi[1]
        return torch.sum(0.5 * (1 + wb)) * h ** (grid.dim - 1)
    nz = phi.shape[0]
    z = (torch.arange(nz, dtype=torch.float64) + 0.5) * h
    wgt = 0.5 * (1 + phi)
    return torch.sum(wgt * z[:, None, None]) / torch.sum(wgt)


def run(grid, prm, vel, phi0, steps, which, theta=None, mobility=None, split_mobility=False):
    """Objective after `steps` CH steps from phi^{-1} = phi^0; returns (J, tensors).

    With split_mobility the returned `mob` is the triple of copies described in
    CHTorch.step: dJ/dM is the sum of their gradients, and the size of each part
    shows how much cancellation dJ/dM carries."""
    m = CHTorch(grid, prm, vel)
    ph0 = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
    th = torch.tensor(float(prm["theta_bot_deg"] if theta is None else theta), dtype=torch.float64,
                      requires_grad=True)
    m0 = float(prm["mobility"] if mobility is None else mobility)
    if split_mobility:
        mob = tuple(torch.tensor(m0, dtype=torch.float64, requires_grad=True) for _ in range(3))
    else:
        mob = torch.tensor(m0, dtype=torch.float64, requires_grad=True)
    pn, po = ph0, ph0
    for _ in range(steps):
        pn, po = m.step(pn, po, th, mob), pn
    J = objective(pn, grid, which)
    return J, ph0, th, mob, pn
