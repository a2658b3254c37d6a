"""Differentiable FP64 restatement of the oracle's coupled 2D step (test
infrastructure only).

The same dual-resolution step as oracle.step.State.step -- the Cahn-Hilliard
update (Section 3.2.1, Eqs. NS25-NS34, literal form with the NS33/NS34 ghosts),
the restriction (Eqs. dual2, dual3), the Navier-Stokes projection (Section
3.2.2, Eqs. NS35-NS39 with the readings of oracle.ns) and the log-conformation
polymer update (Section 3.2.3, Eqs. NS40-NS46, relaxing sign) -- written with
plain PyTorch CPU ops in float64, so that torch.autograd yields the exact
discrete adjoint of N coupled steps: gradients of the wetted length or the
z-centroid with respect to phi0, the bottom contact angle, the mobility M and
the Weissenberg number (lambda_H).  Every constant-coefficient solve is a dense
solve of the assembled operator (the pressure Poisson operator through its
pseudo-inverse, which is the oracle's zero-mode convention), so it is meant for
tiny two-dimensional grids.  The polymer's eigen-decomposition is
torch.linalg.eigh, whose derivative needs distinct eigenvalues: start from a
log-conformation with distinct eigenvalues.  S takes the smallest value allowed
by Eq. NS30 and moves with M; nu_m and rho0 take their defaults.
"""
import math

import numpy as np
import torch

from .ch_torch import _lap_matrix

F64 = torch.float64


def _xp(a):
    return torch.roll(a, -1, dims=-1)


def _xm(a):
    return torch.roll(a, 1, dims=-1)


def _coarse_matrix(nz, nx, D, kind):
    """Dense (periodic x) Laplacian on coarse unknowns [k, i]:
    'dirichlet' cell centres with odd ghosts at the walls, 'faces' interior
    z-faces with zero walls, 'neumann' cell centres with mirror ghosts."""
    rows = nz - 1 if kind == "faces" else nz
    n = rows * nx
    A = np.zeros((n, n))
    idx = lambda k, i: k * nx + i
    for k in range(rows):
        for i in range(nx):
            r = idx(k, i)
            A[r, idx(k, (i + 1) % nx)] += 1
            A[r, idx(k, (i - 1) % nx)] += 1
            A[r, r] -= 2
            for dk in (-1, 1):
                kk = k + dk
                if 0 <= kk < rows:
                    A[r, idx(kk, i)] += 1
                    A[r, r] -= 1
                elif kind == "dirichlet":
                    A[r, r] -= 2  # ghost -u_0: (-u_0) - u_0
                elif kind == "faces":
                    A[r, r] -= 1  # zero wall face
                # neumann: mirror ghost, no contribution
    return A / D ** 2


class CoupledTorch2D:
    def __init__(self, grid, prm):
        if grid.dim != 2:
            raise ValueError("two-dimensional grids only")
        self.g = grid
        self.p = dict(prm)
        p = self.p
        self.r = grid.r
        nzf, _, nxf = grid.fine_shape
        nz, _, nx = grid.coarse_shape
        self.fshape = (nzf, 1, nxf)
        self.cshape = (nz, 1, nx)
        self.h, self.D = grid.h, grid.dx
        self.Lf = _lap_matrix(nzf, 1, nxf, self.h)
        self.If = torch.eye(nzf * nxf, dtype=F64)
        D = self.D
        self.rho1, self.rho2 = p["rho1"], p["rho2"]
        self.rho0 = min(self.rho1, self.rho2)
        self.visco = p.get("wi", 0.0) > 0.0 and p.get("beta", 1.0) < 1.0
        beta = p.get("beta", 1.0) if self.visco else 1.0
        self.mu_s1, self.mu_p1, self.mu_s2 = beta * p["mu1"], (1.0 - beta) * p["mu1"], p["mu2"]
        self.nu_m = p.get("nu_m", 0.0) or 0.5 * max(self.mu_s1, self.mu_s2) / self.rho0
        self.gamma0 = 1.5
        self.dt = p["dt"]
        k = self.gamma0 / (self.dt * self.nu_m)
        self.Hu = torch.tensor(_coarse_matrix(nz, nx, D, "dirichlet") - k * np.eye(nz * nx))
        self.Hw = torch.tensor(_coarse_matrix(nz, nx, D, "faces") - k * np.eye((nz - 1) * nx))
        # pseudo-inverse of the singular Neumann operator (null space: the constant
        # vector 1): L+ = (L + 1 1^T/n)^{-1} - 1 1^T/n, exactly
        Ln = _coarse_matrix(nz, nx, D, "neumann")
        E = np.full(Ln.shape, 1.0 / Ln.shape[0])
        self.Pinv = torch.tensor(np.linalg.inv(Ln + E) - E)
        self.lam = 3.0 * p["sigma"] * p["eta"] / (2.0 * math.sqrt(2.0))

    # ---------------- transfers (Eqs. dual1, dual2) ----------------
    def prolong(self, u, w):
        if self.r == 1:
            return u, w
        uf = torch.stack([u, 0.5 * (u + _xp(u))], dim=-1).reshape(u.shape[:-1] + (-1,))
        uf = torch.repeat_interleave(uf, 2, dim=0)
        wx = torch.repeat_interleave(w, 2, dim=-1)
        mid = 0.5 * (wx[:-1] + wx[1:])
        wf = torch.stack([wx[:-1], mid], dim=1).reshape((-1,) + wx.shape[1:])
        wf = torch.cat([wf, wx[-1:]], dim=0)
        return uf, wf

    def restrict(self, a):
        r = self.r
        nzf, ny, nxf = a.shape
        if r == 1:
            pad = torch.cat([a[:1], a, a[-1:]], 0)
            fz = 0.5 * (pad[:-1] + pad[1:])
            return {"c": a, "fx": 0.5 * (_xm(a) + a), "fz": fz,
                    "exz": 0.5 * (fz + _xm(fz))}
        c = a.reshape(nzf // 2, 2, ny, nxf // 2, 2).mean(dim=(1, 4))
        px = (0.5 * (_xm(a) + a))[..., 0::2]                      # pairs straddling x-faces
        fx = px.reshape(nzf // 2, 2, ny, -1).mean(dim=1)
        g = torch.cat([a[:1], a, a[-1:]], 0)
        pz = 0.5 * (g[0::2] + g[1::2])                            # pairs straddling z-faces k = 0..nz
        fz = pz.reshape(pz.shape[0], ny, nxf // 2, 2).mean(dim=-1)
        exz = (0.5 * (_xm(pz) + pz))[..., 0::2]
        return {"c": c, "fx": fx, "fz": fz, "exz": exz}

    # ---------------- Cahn-Hilliard (Eqs. NS25-NS34) ----------------
    def ch(self, pn, po, us, ws, theta_bot, mob):
        """mob: the mobility, or copies (M_a, M_b, M_s) of it entering the time
        term 1/(M lambda dt), the advection term 1/(M lambda) and S."""
        p, h = self.p, self.h
        eta, dt, g0 = p["eta"], self.dt, self.gamma0
        lam = self.lam
        Ma, Mb, Ms = mob if isinstance(mob, tuple) else (mob,) * 3
        S = eta ** 2 * torch.sqrt(4.0 * g0 / (Ms * lam * dt))   # Eq. NS30, equality
        alpha = -S / (2.0 * eta ** 2)
        c = alpha + S / eta ** 2
        phs = 2 * pn - po
        phh = 2 * pn - 0.5 * po
        uf, wf = self.prolong(us, ws)
        Fx = uf * 0.5 * (_xm(phs) + phs)
        A = (_xp(Fx) - Fx) / h
        inner = wf[1:-1] * 0.5 * (phs[:-1] + phs[1:])
        z = torch.zeros((1,) + phs.shape[1:], dtype=F64)
        Fz = torch.cat([z, inner, z], 0)
        A = A + (Fz[1:] - Fz[:-1]) / h
        hh = phs * (phs * phs - 1) / eta ** 2 - S / eta ** 2 * phs
        s2 = math.sqrt(2.0)
        cb = torch.cos(theta_bot * math.pi / 180.0)
        ct = math.cos(math.radians(p["theta_top_deg"]))
        wb = 1.5 * phs[0] - 0.5 * phs[1]
        wt = 1.5 * phs[-1] - 0.5 * phs[-2]
        gb = cb * (1 - wb * wb) / (s2 * eta)
        gt = ct * (1 - wt * wt) / (s2 * eta)
        zero = torch.zeros_like(phs[1:-1])
        B = torch.cat([(gb / h)[None], zero, (gt / h)[None]], 0)
        lap = lambda a: (self.Lf @ a.reshape(-1)).reshape(self.fshape)
        R1 = phh / (dt * Ma * lam) - A / (Mb * lam) + lap(hh) - c * B
        psi = torch.linalg.solve(self.Lf - c * self.If, R1.reshape(-1)).reshape(self.fshape)
        phi = torch.linalg.solve(self.Lf + alpha * self.If, (psi - B).reshape(-1)).reshape(self.fshape)
        G = lam * (-(lap(phi) + B) + phi * (phi * phi - 1) / eta ** 2)
        return phi, G

    # ---------------- Navier-Stokes (Eqs. NS35-NS39) ----------------
    def mu(self, ph):
        return 0.5 * (1 + ph) * self.mu_s1 + 0.5 * (1 - ph) * self.mu_s2

    def rho(self, ph):
        return 0.5 * (1 + ph) * self.rho1 + 0.5 * (1 - ph) * self.rho2

    def ns(self, un, uo, wn, wo, pn, po, tau_s, rphi, rG, mob, record=None):
        p, D, dt = self.p, self.D, self.dt
        uw_b, uw_t = p.get("uw_bot", 0.0), p.get("uw_top", 0.0)
        us, ws = 2 * un - uo, 2 * wn - wo
        uh, wh = 2 * un - 0.5 * uo, 2 * wn - 0.5 * wo
        ps = 2 * pn - po
        rho0 = self.rho0
        cj = -0.5 * (self.rho1 - self.rho2) * mob
        phic, Gc = rphi["c"], rG["c"]
        mu_c = self.mu(phic)
        mu_exz = self.mu(rphi["exz"])
        usz = torch.cat([2 * uw_b - us[:1], us, 2 * uw_t - us[-1:]], 0)
        Jx = cj * (Gc - _xm(Gc)) / D
        zrow = torch.zeros_like(Gc[:1])
        Jz = torch.cat([zrow, cj * (Gc[1:] - Gc[:-1]) / D, zrow], 0)
        Exz = 0.5 * (usz[:-1] + usz[1:]) * 0.5 * (_xm(ws) + ws)
        Sxz = mu_exz * ((usz[1:] - usz[:-1]) / D + (ws - _xm(ws)) / D)
        Txz = None
        if tau_s is not None:
            g = torch.cat([tau_s["xz"][:1], tau_s["xz"], tau_s["xz"][-1:]], 0)
            a = g[:-1] + g[1:]
            Txz = 0.25 * (a + _xm(a))
        # x momentum at u-faces
        rho_u = self.rho(rphi["fx"])
        Cxx = (0.5 * (us + _xp(us))) ** 2
        adv = (Cxx - _xm(Cxx)) / D + (Exz[1:] - Exz[:-1]) / D
        Jzu = 0.25 * (Jz[:-1] + Jz[1:] + _xm(Jz[:-1]) + _xm(Jz[1:]))
        jg = Jx * (_xp(us) - _xm(us)) / (2 * D) + Jzu * (usz[2:] - usz[:-2]) / (2 * D)
        lap = (_xp(us) - 2 * us + _xm(us)) / D ** 2 + (usz[2:] - 2 * us + usz[:-2]) / D ** 2
        Sxx = 2 * mu_c * (_xp(us) - us) / D
        visc = (Sxx - _xm(Sxx)) / D + (Sxz[1:] - Sxz[:-1]) / D
        divt = torch.zeros_like(us)
        if tau_s is not None:
            divt = (tau_s["xx"] - _xm(tau_s["xx"])) / D + (Txz[1:] - Txz[:-1]) / D
        st = rG["fx"] * (phic - _xm(phic)) / D
        gp = (pn - _xm(pn)) / D / rho0 + (1 / rho_u - 1 / rho0) * (ps - _xm(ps)) / D
        Ru = (-uh / dt + adv + jg / rho_u + gp + self.nu_m * lap - divt / rho_u - visc / rho_u
              - st / rho_u - p.get("gx", 0.0))
        # z momentum at interior w-faces
        rho_w = self.rho(rphi["fz"])[1:-1]
        Czz = (0.5 * (ws[:-1] + ws[1:])) ** 2
        adv = (_xp(Exz) - Exz)[1:-1] / D + (Czz[1:] - Czz[:-1]) / D
        Jxw = 0.25 * (Jx[:-1] + _xp(Jx[:-1]) + Jx[1:] + _xp(Jx[1:]))
        wi = ws[1:-1]
        jg = Jxw * (_xp(wi) - _xm(wi)) / (2 * D) + Jz[1:-1] * (ws[2:] - ws[:-2]) / (2 * D)
        lap = (_xp(wi) - 2 * wi + _xm(wi)) / D ** 2 + (ws[2:] - 2 * wi + ws[:-2]) / D ** 2
        Szz = 2 * mu_c * (ws[1:] - ws[:-1]) / D
        visc = (_xp(Sxz) - Sxz)[1:-1] / D + (Szz[1:] - Szz[:-1]) / D
        divt = torch.zeros_like(wi)
        if tau_s is not None:
            divt = (_xp(Txz) - Txz)[1:-1] / D + (tau_s["zz"][1:] - tau_s["zz"][:-1]) / D
        st = rG["fz"][1:-1] * (phic[1:] - phic[:-1]) / D
        gp = (pn[1:] - pn[:-1]) / D / rho0 + (1 / rho_w - 1 / rho0) * (ps[1:] - ps[:-1]) / D
        Rw = (-wh[1:-1] / dt + adv + jg / rho_w + gp + self.nu_m * lap - divt / rho_w
              - visc / rho_w - st / rho_w - p.get("gz", 0.0))
        # step 1: Helmholtz solves; step 2: Poisson; step 3: correction
        nz, _, nx = self.cshape
        bu = torch.zeros_like(Ru)
        bu[0] = bu[0] + 2 * uw_b / D ** 2
        bu[-1] = bu[-1] + 2 * uw_t / D ** 2
        ut = torch.linalg.solve(self.Hu, (Ru / self.nu_m - bu).reshape(-1)).reshape(self.cshape)
        wti = torch.linalg.solve(self.Hw, (Rw / self.nu_m).reshape(-1)).reshape((nz - 1, 1, nx))
        wt = torch.cat([torch.zeros_like(wti[:1]), wti, torch.zeros_like(wti[:1])], 0)
        div = (_xp(ut) - ut) / D + (wt[1:] - wt[:-1]) / D
        pp = (self.Pinv @ (self.gamma0 * rho0 / dt * div).reshape(-1)).reshape(self.cshape)
        cf = dt / (self.gamma0 * rho0)
        if record is not None:
            record.update(Ru=Ru, Rw=Rw, ut=ut, wt=wt, pp=pp)
        u = ut - cf * (pp - _xm(pp)) / D
        w = torch.cat([torch.zeros_like(wti[:1]), wti - cf * (pp[1:] - pp[:-1]) / D,
                       torch.zeros_like(wti[:1])], 0)
        return u, w, pn + pp

    # ---------------- polymer (Eqs. NS40-NS46) ----------------
    def _grad_u(self, u, w):
        D = self.D
        p = self.p
        uc = 0.5 * (u + _xp(u))
        wc = 0.5 * (w[:-1] + w[1:])
        ucz = torch.cat([2 * p.get("uw_bot", 0.0) - uc[:1], uc, 2 * p.get("uw_top", 0.0) - uc[-1:]], 0)
        dudx = (_xp(u) - u) / D
        dwdz = (w[1:] - w[:-1]) / D
        dudz = (ucz[2:] - ucz[:-2]) / (2 * D)
        dwdx = (_xp(wc) - _xm(wc)) / (2 * D)
        return torch.stack([torch.stack([dudx, dudz], -1), torch.stack([dwdx, dwdz], -1)], -2)

    def _adv(self, T, u, w):
        D = self.D
        ex = (Ellipsis, None, None)
        Fx = u[ex] * 0.5 * (torch.roll(T, 1, dims=2) + T)
        A = (torch.roll(Fx, -1, dims=2) - Fx) / D
        inner = w[1:-1][ex] * 0.5 * (T[:-1] + T[1:])
        z = torch.zeros_like(T[:1])
        Fz = torch.cat([z, inner, z], 0)
        return A + (Fz[1:] - Fz[:-1]) / D

    def _rh(self, T, L, adv, lam_h):
        th, R = torch.linalg.eigh(T)
        lam = torch.exp(th)
        RT = R.transpose(-1, -2)
        Mt = RT @ L @ R
        la, lb = lam[..., 0], lam[..., 1]
        om = (lb * Mt[..., 0, 1] + la * Mt[..., 1, 0]) / (lb - la)
        z = torch.zeros_like(om)
        Om = torch.stack([torch.stack([z, om], -1), torch.stack([-om, z], -1)], -2)
        Bt = torch.stack([torch.stack([Mt[..., 0, 0], z], -1), torch.stack([z, Mt[..., 1, 1]], -1)], -2)
        Omega = R @ Om @ RT
        Bm = R @ Bt @ RT
        relax = R @ (torch.exp(-th)[..., :, None] * RT) - torch.eye(2, dtype=F64)
        return -adv + (Omega @ T - T @ Omega) + 2.0 * Bm + relax / lam_h

    def polymer(self, T, u, w, phic, lam_h):
        dt = self.dt
        L = self._grad_u(u, w)
        T1 = T + dt * self._rh(T, L, self._adv(T, u, w), lam_h)
        T2 = 0.5 * T + 0.5 * (T1 + dt * self._rh(T1, L, self._adv(T1, u, w), lam_h))
        th, R = torch.linalg.eigh(T2)
        c = R @ (torch.exp(th)[..., :, None] * R.transpose(-1, -2))
        taup = self.mu_p1 / lam_h * (c - torch.eye(2, dtype=F64))
        tau = 0.5 * (1.0 + phic)[..., None, None] * taup
        return T2, tau

    # ---------------- one coupled step (oracle.step.State.step) ----------------
    def step(self, s, theta_bot, mob, lam_h):
        """mob: the mobility, or four copies of it (CH time term, CH advection, S,
        the flux J of the momentum equation)."""
        mch, mj = (mob[:3], mob[3]) if isinstance(mob, tuple) else (mob, mob)
        phi, G = self.ch(s["phi"], s["phi_old"], 2 * s["u"] - s["u_old"], 2 * s["w"] - s["w_old"], theta_bot, mch)
        rphi, rG = self.restrict(phi), self.restrict(G)
        tau_s = None
        if self.visco:
            t = 2 * s["tau"] - s["tau_old"]
            tau_s = {"xx": t[..., 0, 0], "xz": t[..., 0, 1], "zz": t[..., 1, 1]}
        u, w, p = self.ns(s["u"], s["u_old"], s["w"], s["w_old"], s["p"], s["p_old"], tau_s, rphi, rG, mj)
        n = dict(phi=phi, phi_old=s["phi"], u=u, u_old=s["u"], w=w, w_old=s["w"], p=p, p_old=s["p"],
                 theta=s["theta"], tau=s["tau"], tau_old=s["tau_old"])
        if self.visco:
            th, tau = self.polymer(s["theta"], u, w, rphi["c"], lam_h)
            n.update(theta=th, tau=tau, tau_old=s["tau"])
        return n


def objective(phi, grid, which):
    h = grid.h
    if which == "wetted":
        wb = 1.5 * phi[0] - 0.5 * phi[1]
        return torch.sum(0.5 * (1 + wb)) * h ** (grid.dim - 1)
    nz = phi.shape[0]
    z = (torch.arange(nz, dtype=F64) + 0.5) * h
    wgt = 0.5 * (1 + phi)
    return torch.sum(wgt * z[:, None, None]) / torch.sum(wgt)


def run(grid, prm, phi0, steps, which, vel0=None, theta0=None, split_mobility=False):
    """J after `steps` coupled steps from phi^{-1} = phi^0 (u^{-1} = u^0, ...),
    and the leaf tensors (phi0, theta_bot, M, lambda_H) whose .grad are dJ/d*.
    With split_mobility, M is four leaves (see CoupledTorch2D.step): dJ/dM is
    the sum of their gradients, and their sizes show its cancellation."""
    m = CoupledTorch2D(grid, prm)
    nz, _, nx = grid.coarse_shape
    ph0 = torch.tensor(phi0, dtype=F64, requires_grad=True)
    th = torch.tensor(float(prm["theta_bot_deg"]), dtype=F64, requires_grad=True)
    if split_mobility:
        mob = tuple(torch.tensor(float(prm["mobility"]), dtype=F64, requires_grad=True) for _ in range(4))
    else:
        mob = torch.tensor(float(prm["mobility"]), dtype=F64, requires_grad=True)
    lh = torch.tensor(float(prm.get("wi", 0.0)) or 1.0, dtype=F64, requires_grad=True)
    if vel0 is None:
        u0, w0 = np.zeros((nz, 1, nx)), np.zeros((nz + 1, 1, nx))
    else:
        u0, w0 = vel0[0], vel0[2]
    u0 = torch.tensor(u0, dtype=F64)
    w0 = torch.tensor(w0, dtype=F64)
    T0 = torch.zeros((nz, 1, nx, 2, 2), dtype=F64) if theta0 is None else torch.tensor(theta0, dtype=F64)
    z = torch.zeros((nz, 1, nx), dtype=F64)
    tau0 = torch.zeros((nz, 1, nx, 2, 2), dtype=F64)
    s = dict(phi=ph0, phi_old=ph0, u=u0, u_old=u0, w=w0, w_old=w0, p=z, p_old=z, theta=T0, tau=tau0,
             tau_old=tau0)
    for _ in range(steps):
        s = m.step(s, th, mob, lh)
    J = objective(s["phi"], grid, which)
    return J, dict(phi0=ph0, theta=th, mobility=mob, wi=lh), s
