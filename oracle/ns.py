"""Navier-Stokes step on the coarse MAC mesh (oracle; test infrastructure only).

Section 3.2.2, Eqs. NS35-NS39 (Dong's constant-coefficient splitting, BDF2):

 step 1 (Eq. NS36, with the -u_hat/dt of Eq. NS35 restored on the right side):
   nu_m lap(u~) - (gamma0/dt) u~ = -u_hat/dt + div(u* u*) + (1/rho) J . grad(u*)
        + (1/rho0) grad p^n + (1/rho - 1/rho0) grad p* + nu_m lap(u*)
        - (1/rho) div(tau*) - (1/rho) div(mu (grad u* + grad u*^T))
        - (1/rho) G grad(phi) - g
 step 2 (Eq. NS37, coefficient read as gamma0 rho0/dt so that Eq. NS38 gives
   div u^{n+1} = 0):  lap p' = (gamma0 rho0/dt) div(u~),  dp'/dn = 0, zero mode 0
 step 3 (Eqs. NS38, NS39): u = u~ - dt/(gamma0 rho0) grad p',  p = p^n + p'

rho, mu at the faces/centres/edges come from the restricted phi^{n+1} through
Eq. dual3; G at centres (for J = -(rho1 - rho2)/2 M grad G, Eq. NS10) and at
faces (surface force G grad phi) from the restricted chemical potential.

Readings: J . grad u is taken at u* (a constant-coefficient solve cannot hold it
implicit); J's tangential components at a face are 4-point MAC averages; the
surface force at an x-face is G_face (phi_c[i] - phi_c[i-1])/dx; tangential
no-slip through the ghost u_g = 2 u_w - u_0; the polymer stress gets mirror
ghosts at the walls (homogeneous Neumann, text after Eq. NS46); the external
force enters as a body acceleration g.
"""
import numpy as np

from . import operators as op
from . import spectral
from .operators import xp, xm, yp, ym


def zpad_dir(a, wb, wt):
    """Cell-centred tangential velocity with no-slip ghosts 2 u_w - u."""
    return np.concatenate([2.0 * wb - a[:1], a, 2.0 * wt - a[-1:]], axis=0)


def _edge_xz(t):
    """Centre field -> x-z edges (x = i dx, z = k dx), k = 0..nz, mirror ghosts."""
    g = op.zpad_mirror(t)
    a = g[:-1] + g[1:]
    return 0.25 * (a + xm(a))


def _edge_yz(t):
    g = op.zpad_mirror(t)
    a = g[:-1] + g[1:]
    return 0.25 * (a + ym(a))


def _edge_xy(t):
    a = t + ym(t)
    return 0.25 * (a + xm(a))


def momentum_rhs(vel_n, vel_nm1, p_n, p_nm1, tau_s, rphi, rG, d, grid):
    """Right-hand sides of Eq. NS36 (u, v, w); w is returned on all nz+1 faces."""
    D = grid.dx
    dim = grid.dim
    dt = d.dt
    u_n, v_n, w_n = vel_n
    u_o, v_o, w_o = vel_nm1
    us, vs, ws = 2 * u_n - u_o, 2 * v_n - v_o, 2 * w_n - w_o
    uh, vh, wh = 2 * u_n - 0.5 * u_o, 2 * v_n - 0.5 * v_o, 2 * w_n - 0.5 * w_o
    ps = 2 * p_n - p_nm1
    nz = us.shape[0]
    rho0 = d.rho0
    cj = -0.5 * (d.rho1 - d.rho2) * d.mob
    phic, Gc = rphi["c"], rG["c"]
    mu_c = d.mu(phic)
    mu_exz = d.mu(rphi["exz"])
    usz = zpad_dir(us, d.uw_bot, d.uw_top)
    zero = np.zeros_like(us)
    vsz = zpad_dir(vs, zero[:1], zero[:1])

    # J at its natural faces (Eq. NS10 with the chemical potential G)
    Jx = cj * (Gc - xm(Gc)) / D
    Jz = np.zeros_like(ws)
    Jz[1:-1] = cj * (Gc[1:] - Gc[:-1]) / D
    Jy = cj * (Gc - ym(Gc)) / D if dim == 3 else None

    # shared edge products and stresses
    Exz = 0.5 * (usz[:-1] + usz[1:]) * 0.5 * (xm(ws) + ws)          # u w at x-z edges
    Sxz = mu_exz * ((usz[1:] - usz[:-1]) / D + (ws - xm(ws)) / D)    # mu(du/dz + dw/dx)
    if tau_s is not None:
        Txz = _edge_xz(tau_s["xz"])
    if dim == 3:
        mu_exy = d.mu(rphi["exy"])
        mu_eyz = d.mu(rphi["eyz"])
        Exy = 0.5 * (ym(us) + us) * 0.5 * (xm(vs) + vs)               # u v at x-y edges
        Eyz = 0.5 * (vsz[:-1] + vsz[1:]) * 0.5 * (ym(ws) + ws)        # v w at y-z edges
        Sxy = mu_exy * ((us - ym(us)) / D + (vs - xm(vs)) / D)
        Syz = mu_eyz * ((vsz[1:] - vsz[:-1]) / D + (ws - ym(ws)) / D)
        if tau_s is not None:
            Txy = _edge_xy(tau_s["xy"])
            Tyz = _edge_yz(tau_s["yz"])

    # ---------------- x momentum at u-faces ----------------
    rho_u = d.rho(rphi["fx"])
    Cxx = (0.5 * (us + xp(us))) ** 2
    adv = (Cxx - xm(Cxx)) / D + (Exz[1:] - Exz[:-1]) / D
    Jzu = 0.25 * (Jz[:-1] + Jz[1:] + xm(Jz[:-1]) + xm(Jz[1:]))
    jg = Jx * (xp(us) - xm(us)) / (2 * D) + Jzu * (usz[2:] - usz[:-2]) / (2 * D)
    lap = op.lap_periodic(us, D, dim) + (usz[2:] - 2 * us + usz[:-2]) / D ** 2
    Sxx = 2 * mu_c * (xp(us) - us) / D
    visc = (Sxx - xm(Sxx)) / D + (Sxz[1:] - Sxz[:-1]) / D
    divt = zero.copy()
    if tau_s is not None:
        divt = (tau_s["xx"] - xm(tau_s["xx"])) / D + (Txz[1:] - Txz[:-1]) / D
    if dim == 3:
        adv = adv + (yp(Exy) - Exy) / D
        Jyu = 0.25 * (Jy + yp(Jy) + xm(Jy) + xm(yp(Jy)))
        jg = jg + Jyu * (yp(us) - ym(us)) / (2 * D)
        visc = visc + (yp(Sxy) - Sxy) / D
        if tau_s is not None:
            divt = divt + (yp(Txy) - Txy) / D
    st = rG["fx"] * (phic - xm(phic)) / D
    gp = (p_n - xm(p_n)) / D / rho0 + (1 / rho_u - 1 / rho0) * (ps - xm(ps)) / D
    Ru = (-uh / dt + adv + jg / rho_u + gp + d.nu_m * lap - divt / rho_u - visc / rho_u
          - st / rho_u - d.g[0])

    # ---------------- z momentum at interior w-faces ----------------
    Rw = np.zeros_like(ws)
    rho_w = d.rho(rphi["fz"])[1:-1]
    Czz = (0.5 * (ws[:-1] + ws[1:])) ** 2
    adv = (xp(Exz) - Exz)[1:-1] / D + (Czz[1:] - Czz[:-1]) / D
    Jxw = 0.25 * (Jx[:-1] + xp(Jx[:-1]) + Jx[1:] + xp(Jx[1:]))
    wi = ws[1:-1]
    jg = Jxw * (xp(wi) - xm(wi)) / (2 * D) + Jz[1:-1] * (ws[2:] - ws[:-2]) / (2 * D)
    lap = op.lap_periodic(wi, D, dim) + (ws[2:] - 2 * wi + ws[:-2]) / D ** 2
    Szz = 2 * mu_c * (ws[1:] - ws[:-1]) / D
    visc = (xp(Sxz) - Sxz)[1:-1] / D + (Szz[1:] - Szz[:-1]) / D
    divt = np.zeros_like(wi)
    if tau_s is not None:
        divt = (xp(Txz) - Txz)[1:-1] / D + (tau_s["zz"][1:] - tau_s["zz"][:-1]) / D
    if dim == 3:
        adv = adv + (yp(Eyz) - Eyz)[1:-1] / D
        Jyw = 0.25 * (Jy[:-1] + yp(Jy[:-1]) + Jy[1:] + yp(Jy[1:]))
        jg = jg + Jyw * (yp(wi) - ym(wi)) / (2 * D)
        visc = visc + (yp(Syz) - Syz)[1:-1] / D
        if tau_s is not None:
            divt = divt + (yp(Tyz) - Tyz)[1:-1] / D
    st = rG["fz"][1:-1] * (phic[1:] - phic[:-1]) / D
    gp = ((p_n[1:] - p_n[:-1]) / D / rho0
          + (1 / rho_w - 1 / rho0) * (ps[1:] - ps[:-1]) / D)
    Rw[1:-1] = (-wh[1:-1] / dt + adv + jg / rho_w + gp + d.nu_m * lap - divt / rho_w
                - visc / rho_w - st / rho_w - d.g[2])

    # ---------------- y momentum at v-faces (3D) ----------------
    Rv = np.zeros_like(vs)
    if dim == 3:
        rho_v = d.rho(rphi["fy"])
        Cyy = (0.5 * (vs + yp(vs))) ** 2
        adv = (Cyy - ym(Cyy)) / D + (xp(Exy) - Exy) / D + (Eyz[1:] - Eyz[:-1]) / D
        Jxv = 0.25 * (ym(Jx) + xp(ym(Jx)) + Jx + xp(Jx))
        Jzv = 0.25 * (Jz[:-1] + Jz[1:] + ym(Jz[:-1]) + ym(Jz[1:]))
        jg = (Jxv * (xp(vs) - xm(vs)) / (2 * D) + Jy * (yp(vs) - ym(vs)) / (2 * D)
              + Jzv * (vsz[2:] - vsz[:-2]) / (2 * D))
        lap = op.lap_periodic(vs, D, dim) + (vsz[2:] - 2 * vs + vsz[:-2]) / D ** 2
        Syy = 2 * mu_c * (yp(vs) - vs) / D
        visc = (Syy - ym(Syy)) / D + (xp(Sxy) - Sxy) / D + (Syz[1:] - Syz[:-1]) / D
        divt = zero.copy()
        if tau_s is not None:
            divt = ((tau_s["yy"] - ym(tau_s["yy"])) / D + (xp(Txy) - Txy) / D
                    + (Tyz[1:] - Tyz[:-1]) / D)
        st = rG["fy"] * (phic - ym(phic)) / D
        gp = (p_n - ym(p_n)) / D / rho0 + (1 / rho_v - 1 / rho0) * (ps - ym(ps)) / D
        Rv = (-vh / dt + adv + jg / rho_v + gp + d.nu_m * lap - divt / rho_v
              - visc / rho_v - st / rho_v - d.g[1])
    return Ru, Rv, Rw


def ns_step(vel_n, vel_nm1, p_n, p_nm1, tau_s, rphi, rG, d, grid):
    """Steps 1-3.  tau_s: extrapolated weighted polymer stress dict or None."""
    D = grid.dx
    dim = grid.dim
    nz = vel_n[0].shape[0]
    Ru, Rv, Rw = momentum_rhs(vel_n, vel_nm1, p_n, p_nm1, tau_s, rphi, rG, d, grid)
    k = d.gamma0 / (d.dt * d.nu_m)
    # tangential components: Dirichlet ghost 2 u_w - u moves 2 u_w/D^2 to the right side
    bu = np.zeros_like(Ru)
    bu[0] += 2 * d.uw_bot / D ** 2
    bu[-1] += 2 * d.uw_top / D ** 2
    ut = spectral.solve(Ru / d.nu_m - bu, k, D, "dirichlet")
    vt = spectral.solve(Rv / d.nu_m, k, D, "dirichlet") if dim == 3 else np.zeros_like(ut)
    wt = np.zeros_like(Rw)
    wt[1:-1] = spectral.solve(Rw[1:-1] / d.nu_m, k, D, "faces", nz_cells=nz)
    div = op.div_faces(ut, vt, wt, D, dim)
    pp = spectral.solve(d.gamma0 * d.rho0 / d.dt * div, 0.0, D, "neumann")
    cf = d.dt / (d.gamma0 * d.rho0)
    u = ut - cf * (pp - xm(pp)) / D
    v = vt - cf * (pp - ym(pp)) / D if dim == 3 else np.zeros_like(ut)
    w = wt.copy()
    w[1:-1] = wt[1:-1] - cf * (pp[1:] - pp[:-1]) / D
    p = p_n + pp
    return dict(u=u, v=v, w=w, p=p, pp=pp, ut=ut, vt=vt, wt=wt)
