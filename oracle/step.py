"""The coupled dual-resolution time step (oracle; test infrastructure only).

Order (Section 3.2): prolong u* and advance phi on the fine mesh (Eqs. dual1,
NS25-NS34); restrict phi^{n+1} and G^{n+1} to the coarse mesh (Eqs. dual2,
dual3); Navier-Stokes with rho, mu, G, phi known at n+1 (Eqs. NS35-NS39); then
the polymer with u^{n+1} and phi^{n+1} (Eqs. NS42-NS46).

Start-up (a reading: the paper is silent): phi^{-1} = phi^0, u^{-1} = u^0,
p^{-1} = p^0, tau^{-1} = tau^0, and BDF2 from the first step.
"""
import numpy as np

from . import ch, ns, polymer
from . import operators as op
from .params import Derived


class State:
    def __init__(self, grid, prm, phi0, vel0=None, p0=None, theta0=None):
        self.grid = grid
        self.d = Derived(prm)
        nz, ny, nx = grid.coarse_shape
        n = 2 if grid.dim == 2 else 3
        self.phi = np.array(phi0, dtype=np.float64)
        self.phi_old = self.phi.copy()
        if vel0 is None:
            vel0 = (np.zeros((nz, ny, nx)), np.zeros((nz, ny, nx)), np.zeros((nz + 1, ny, nx)))
        self.vel = tuple(np.array(a, dtype=np.float64) for a in vel0)
        self.vel_old = tuple(a.copy() for a in self.vel)
        self.p = np.zeros((nz, ny, nx)) if p0 is None else np.array(p0, dtype=np.float64)
        self.p_old = self.p.copy()
        self.theta = np.zeros((nz, ny, nx, n, n)) if theta0 is None else np.array(theta0)
        self.tau = np.zeros((nz, ny, nx, n, n))
        self.tau_old = self.tau.copy()
        self.G = None
        self.nsteps = 0

    def step(self, with_ns=True):
        g, d = self.grid, self.d
        out = ch.ch_step(self.phi, self.phi_old, self.vel, self.vel_old, d, g)
        phi_new, G = out["phi"], out["G"]
        self.G = G
        if with_ns:
            rphi = op.restrict(phi_new, g.r, g.ry, g.dim)
            rG = op.restrict(G, g.r, g.ry, g.dim)
            tau_s = None
            if d.visco:
                tau_s = polymer.tau_components(2 * self.tau - self.tau_old, g.dim)
            o = ns.ns_step(self.vel, self.vel_old, self.p, self.p_old, tau_s, rphi, rG, d, g)
            vel_new = (o["u"], o["v"], o["w"])
            self.vel_old, self.vel = self.vel, vel_new
            self.p_old, self.p = self.p, o["p"]
            if d.visco:
                th, tau = polymer.polymer_step(self.theta, *vel_new, rphi["c"], d, g)
                self.theta = th
                self.tau_old, self.tau = self.tau, tau
        self.phi_old, self.phi = self.phi, phi_new
        self.nsteps += 1
        return out


def run(grid, prm, phi0, steps, with_ns=True, **kw):
    st = State(grid, prm, phi0, **kw)
    for _ in range(steps):
        st.step(with_ns=with_ns)
    return st
