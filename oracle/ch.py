"""Cahn-Hilliard step on the phase-field mesh (oracle; test infrastructure only).

Follows Section 3.2.1 in the paper's order:
  Eq. NS31/NS32  phi* = 2 phi^n - phi^{n-1},  phi_hat = 2 phi^n - phi^{n-1}/2,
                 u* = 2 u^n - u^{n-1}, prolonged by Eq. dual1;
  Eq. NS25       the stabilised BDF2 scheme, advection by the central
                 (second-order) conservative face flux u_f (phi_L + phi_R)/2;
  Eq. NS28       Q = (phi_hat/dt - div(u* phi*))/(M lambda) + lap[f(phi*) - S/eta^2 phi*];
  Eq. NS26       (lap - (alpha + S/eta^2)) Psi = Q            with Eq. NS33 on the walls;
  Eq. NS27       (lap + alpha) phi^{n+1} = Psi                with Eq. NS34 on the walls;
  Eq. NS15/16/34 with D_w = 0: n.grad(phi^{n+1}) = -f_w'(phi*)/lambda
                 = cos(theta_s) (1 - phi*_w^2)/(sqrt(2) eta), n the outward normal;
                 with D_w > 0 the flux also holds -D_w (dphi/dt + u.grad phi*) at
                 the wall, implicit in phi^{n+1}: the two solves are then one
                 system per Fourier mode (spectral.solve_ch_robin, wall_explicit);
  Eq. NS5/NS6    G = lambda(-lap phi + f(phi)), f(phi) = phi (phi^2 - 1)/eta^2.

Readings (the paper is silent or ambiguous):
  * phi*_w, the wall value entering the contact-angle law, is the linear
    extrapolation 1.5 phi*_0 - 0.5 phi*_1 of the first two cells to the wall face.
  * The ghost of phi^{n+1} is phi_0 + h g, so the wall cell's Laplacian is the
    Neumann one plus g/h ("B(g)").
  * Eq. NS33 needs n.grad(f(phi*) - S/eta^2 phi*) on the wall; any discrete
    choice g_h cancels between Q and the Psi ghost (see ch_step_two_ghost), so
    the oracle uses g_h = 0, i.e. the homogeneous-Neumann L_N of that term.
  * G uses the same wetting ghost for lap phi^{n+1}.
"""
import math

import numpy as np

from . import operators as op, weno
from . import spectral


def f_bulk(phi, eta):
    """Eq. NS6."""
    return phi * (phi * phi - 1.0) / eta ** 2


def wall_flux(phis, d):
    """Eq. NS34 (D_w = 0) at the bottom and top walls: g = n.grad(phi) per column."""
    s2 = math.sqrt(2.0)
    wb = 1.5 * phis[0] - 0.5 * phis[1]
    wt = 1.5 * phis[-1] - 0.5 * phis[-2]
    gb = d.cos_bot * (1.0 - wb * wb) / (s2 * d.eta)
    gt = d.cos_top * (1.0 - wt * wt) / (s2 * d.eta)
    return gb, gt


def wall_explicit(phis, phih, d, grid):
    """The explicit part E of the dynamic contact-angle condition, Eq. NS34 with
    D_w > 0, at the bottom and top walls: the wall flux of phi^{n+1} is
    g = E - kappa phi_w^{n+1} with kappa = D_w gamma0/dt and
        E = -f_w'(phi*_w)/lambda - D_w (u_w . grad phi*)_w + (D_w/dt) phi_hat_w,
    the BDF2 time derivative of Eq. NS31 taken at the wall.  Readings: every
    wall value (phi*, phi_hat, phi^{n+1}) is the extrapolation 1.5 v_0 - 0.5 v_1;
    the wall velocity is the no-slip u_w along x (w = 0, v = 0 there), times the
    central x difference of phi*_w."""
    gb, gt = wall_flux(phis, d)
    h = grid.h
    out = []
    for g, a, uw in ((gb, (0, 1), d.uw_bot), (gt, (-1, -2), d.uw_top)):
        ws = 1.5 * phis[a[0]] - 0.5 * phis[a[1]]
        wh = 1.5 * phih[a[0]] - 0.5 * phih[a[1]]
        dx = (np.roll(ws, -1, axis=-1) - np.roll(ws, 1, axis=-1)) / (2.0 * h)
        out.append(g - d.dw * uw * dx + d.dw / d.dt * wh)
    return out


def wall_term(shape, gb, gt, h):
    """B(g): g/h on the first and last fine z-layer, zero elsewhere."""
    B = np.zeros(shape)
    B[0] += gb / h
    B[-1] += gt / h
    return B


def advection(phis, uf, vf, wf, h, dim):
    """div(u* phi*) with the central conservative flux; no flux through the walls."""
    Fx = uf * 0.5 * (op.xm(phis) + phis)
    A = (op.xp(Fx) - Fx) / h
    if dim == 3:
        Fy = vf * 0.5 * (op.ym(phis) + phis)
        A = A + (op.yp(Fy) - Fy) / h
    nz = phis.shape[0]
    Fz = np.zeros((nz + 1,) + phis.shape[1:])
    Fz[1:-1] = wf[1:-1] * 0.5 * (phis[:-1] + phis[1:])
    A = A + (Fz[1:] - Fz[:-1]) / h
    return A


def ch_step(phi_n, phi_nm1, vel_n, vel_nm1, d, grid):
    """One CH step.  vel_* = (u, v, w) coarse.  Returns dict(phi, psi, G, gb, gt)."""
    h, dim, r, ry = grid.h, grid.dim, grid.r, grid.ry
    eta = d.eta
    phis = 2.0 * phi_n - phi_nm1
    phih = 2.0 * phi_n - 0.5 * phi_nm1
    us = [2.0 * a - b for a, b in zip(vel_n, vel_nm1)]
    uf, vf, wf = op.prolong_velocity(us[0], us[1], us[2], r, ry, dim)
    if getattr(d, "advection", "central") == "weno5z":  # the paper's scheme (Section 3.2.1)
        A = weno.advection(phis, uf, vf, wf, h, dim)
    else:
        A = advection(phis, uf, vf, wf, h, dim)
    hh = f_bulk(phis, eta) - d.S / eta ** 2 * phis
    if d.dw > 0:  # Eq. NS34 with D_w > 0: a Robin condition coupling the two solves
        Eb, Et = wall_explicit(phis, phih, d, grid)
        Q = (phih / d.dt - A) / d.Ml + op.lap_neumann(hh, h, dim)
        psi, phi = spectral.solve_ch_robin(Q, Eb, Et, d.c, d.alpha, d.kappa, h)
        gb = Eb - d.kappa * (1.5 * phi[0] - 0.5 * phi[1])
        gt = Et - d.kappa * (1.5 * phi[-1] - 0.5 * phi[-2])
        B = wall_term(phis.shape, gb, gt, h)
        R1 = Q - d.c * B
    else:
        gb, gt = wall_flux(phis, d)
        B = wall_term(phis.shape, gb, gt, h)
        R1 = (phih / d.dt - A) / d.Ml + op.lap_neumann(hh, h, dim) - d.c * B
        psi = spectral.solve(R1, d.c, h, "neumann")
        phi = spectral.solve(psi - B, -d.alpha, h, "neumann")
    G = d.lam * (-(op.lap_neumann(phi, h, dim) + B) + f_bulk(phi, eta))
    return dict(phi=phi, psi=psi, G=G, gb=gb, gt=gt, A=A, R1=R1, phis=phis, phih=phih)


def ch_step_two_ghost(phi_n, phi_nm1, vel_n, vel_nm1, d, grid, ghb, ght):
    """The same step written with both wall ghosts of Eq. NS33 explicit.

    ghb/ght are arbitrary discrete wall gradients n.grad(f(phi*) - S/eta^2 phi*)
    used both inside Q (Eq. NS28) and in the Psi wall flux (Eq. NS33).  The
    solution does not depend on them (the resolved ambiguity)."""
    h, dim, r, ry = grid.h, grid.dim, grid.r, grid.ry
    eta = d.eta
    phis = 2.0 * phi_n - phi_nm1
    phih = 2.0 * phi_n - 0.5 * phi_nm1
    us = [2.0 * a - b for a, b in zip(vel_n, vel_nm1)]
    uf, vf, wf = op.prolong_velocity(us[0], us[1], us[2], r, ry, dim)
    if getattr(d, "advection", "central") == "weno5z":  # the paper's scheme (Section 3.2.1)
        A = weno.advection(phis, uf, vf, wf, h, dim)
    else:
        A = advection(phis, uf, vf, wf, h, dim)
    hh = f_bulk(phis, eta) - d.S / eta ** 2 * phis
    gb, gt = wall_flux(phis, d)
    Bh = wall_term(phis.shape, ghb, ght, h)
    Q = (phih / d.dt - A) / d.Ml + op.lap_neumann(hh, h, dim) + Bh
    # Psi ghost: n.grad Psi = g_h + c g (Eq. NS33); lap Psi = L_N Psi + B(g_h + c g)
    Bpsi = wall_term(phis.shape, ghb + d.c * gb, ght + d.c * gt, h)
    psi = spectral.solve(Q - Bpsi, d.c, h, "neumann")
    B = wall_term(phis.shape, gb, gt, h)
    phi = spectral.solve(psi - B, -d.alpha, h, "neumann")
    return phi
