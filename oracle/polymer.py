"""Log-conformation Giesekus / Oldroyd-B update on coarse centres (oracle; test infrastructure only).

Section 2.2 (Eqs. NS17-NS24) and Section 3.2.3 (Eqs. NS40-NS46):
  tau_p = (mu_p/lambda_H)(c - I)                                         NS17
  c = R Lambda R^T, Theta = log c = R log(Lambda) R^T                      NS19, NS20
  M~ = R^T (grad u)^T R, omega_ab = (l_b m_ab + l_a m_ba)/(l_b - l_a),
  Omega = R [omega] R^T (antisymmetric), B = R diag(m_aa) R^T              NS23, NS24
  dTheta/dt = RH = -div(u Theta) + (Omega Theta - Theta Omega) + 2 B
                   - (1/lambda_H) e^{-Theta} [I + alpha (e^Theta - I)] (e^Theta - I)
  (Eqs. NS22, NS41, Giesekus mobility alpha; alpha = 0 is Oldroyd-B, whose
  relaxation is (1/lambda_H)(e^{-Theta} - I)).  The three factors are functions
  of Theta, so the term is diagonal in its eigenbasis:
  (1/lambda_H) [(e^{-theta} - 1) - alpha (e^{theta} - 1)(1 - e^{-theta})].
  RK2-TVD: Theta1 = Theta^n + dt RH(Theta^n; R^n, Lambda^n)                NS42
           diagonalise Theta1                                             NS43
           Theta^{n+1} = Theta^n/2 + (Theta1 + dt RH(Theta1; R1, Lambda1))/2 NS44
           diagonalise, tau_p^{n+1} = (mu_p/lambda_H)(R Lambda R^T - I)   NS45, NS46
  tau = (1 + phi)/2 tau_p  (approach 2, Eq. NS12: the droplet phi = +1 is viscoelastic);
  approach 1 (Eq. NS11): mu_p, lambda_H and alpha are linear in phi at each
  centre (the restricted phi^{n+1}) in both stages, and tau = tau_p.

Readings: the printed sign of the relaxation term in Eqs. NS18/NS22/NS41 is
reversed (as printed it would grow, not relax); the oracle relaxes.  For
(near-)equal eigenvalues, |l_a - l_b| <= 1e-10 max(1, |l_a|), omega_ab = 0 and
B takes the symmetric off-diagonal (m_ab + m_ba)/2 in the R basis (the limit of
the commutator term; with tau_p = 0 this is Omega = 0, B = sym(grad u^T), as the
paper states).  The convective term is the central conservative flux with zero
flux through the walls (w = 0 there).  The velocity gradient at the centre uses
face differences along the face normal and, across, central differences of the
centre-averaged velocity (no-slip ghosts 2 u_w - u at the walls).  With the
paper's WENO5-Z option (advection "weno5z") the convective term takes the
WENO5-Z face values of oracle.weno per component instead of the central flux.
(grad u)^T has entries L[a, b] = d u_a / d x_b.
"""
import numpy as np

from . import operators as op
from .operators import xp, xm, yp, ym
from .ns import zpad_dir

DEG_TOL = 1e-10


def velocity_gradient(u, v, w, d, grid):
    """L[..., a, b] = du_a/dx_b at coarse centres; axes (x, z) in 2D, (x, y, z) in 3D."""
    D = grid.dx
    uc = 0.5 * (u + xp(u))
    wc = 0.5 * (w[:-1] + w[1:])
    ucz = zpad_dir(uc, d.uw_bot, d.uw_top)
    dudx = (xp(u) - u) / D
    dwdz = (w[1:] - w[:-1]) / D
    dudz = (ucz[2:] - ucz[:-2]) / (2 * D)
    dwdx = (xp(wc) - xm(wc)) / (2 * D)
    if grid.dim == 2:
        L = np.stack([np.stack([dudx, dudz], -1), np.stack([dwdx, dwdz], -1)], -2)
        return L
    vc = 0.5 * (v + yp(v))
    vcz = zpad_dir(vc, np.zeros_like(vc[:1]), np.zeros_like(vc[:1]))
    dudy = (yp(uc) - ym(uc)) / (2 * D)
    dvdx = (xp(vc) - xm(vc)) / (2 * D)
    dvdy = (yp(v) - v) / D
    dvdz = (vcz[2:] - vcz[:-2]) / (2 * D)
    dwdy = (yp(wc) - ym(wc)) / (2 * D)
    L = np.stack([np.stack([dudx, dudy, dudz], -1),
                  np.stack([dvdx, dvdy, dvdz], -1),
                  np.stack([dwdx, dwdy, dwdz], -1)], -2)
    return L


def advection_weno(T, u, v, w, grid):
    """div(u Theta) per component with the WENO5-Z face values of oracle.weno
    (the paper's scheme for the convective term, before Eq. NS40): u, v, w are
    the coarse face velocities (left x face and y face of each cell, z faces
    with both walls), the same arrays the central flux takes."""
    from . import weno
    out = np.empty_like(T)
    n = T.shape[-1]
    for a in range(n):
        for b in range(a, n):
            out[..., a, b] = weno.advection(T[..., a, b], u, v if grid.dim == 3 else None, w, grid.dx, grid.dim)
            out[..., b, a] = out[..., a, b]
    return out


def advection(T, u, v, w, grid, scheme="central"):
    """div(u Theta) per component; T has shape (nz, ny, nx, n, n)."""
    if scheme == "weno5z":
        return advection_weno(T, u, v, w, grid)
    D = grid.dx
    ex = (Ellipsis, None, None)
    Fx = u[ex] * 0.5 * (np.roll(T, 1, axis=2) + T)
    A = (np.roll(Fx, -1, axis=2) - Fx) / D
    if grid.dim == 3:
        Fy = v[ex] * 0.5 * (np.roll(T, 1, axis=1) + T)
        A = A + (np.roll(Fy, -1, axis=1) - Fy) / D
    nz = T.shape[0]
    Fz = np.zeros((nz + 1,) + T.shape[1:])
    Fz[1:-1] = w[1:-1][ex] * 0.5 * (T[:-1] + T[1:])
    return A + (Fz[1:] - Fz[:-1]) / D


def decompose(T):
    th, R = np.linalg.eigh(T)
    return th, R


def rh(T, L, adv, lam_h, alpha_g=0.0):
    """Right-hand side RH of Eq. NS41 with the diagonalisation of T (Eq. NS23-NS24)."""
    n = T.shape[-1]
    th, R = decompose(T)
    lam = np.exp(th)
    Mt = np.einsum("...ba,...bc,...cd->...ad", R, L, R)  # R^T L R
    Om = np.zeros_like(Mt)
    Bt = np.zeros_like(Mt)
    for a in range(n):
        Bt[..., a, a] = Mt[..., a, a]
    for a in range(n):
        for b in range(a + 1, n):
            la, lb = lam[..., a], lam[..., b]
            dl = lb - la
            deg = np.abs(dl) <= DEG_TOL * np.maximum(1.0, np.abs(la))
            om = np.where(deg, 0.0, (lb * Mt[..., a, b] + la * Mt[..., b, a]) / np.where(deg, 1.0, dl))
            Om[..., a, b] = om
            Om[..., b, a] = -om
            sym = np.where(deg, 0.5 * (Mt[..., a, b] + Mt[..., b, a]), 0.0)
            Bt[..., a, b] = sym
            Bt[..., b, a] = sym
    RT = np.swapaxes(R, -1, -2)
    Omega = R @ Om @ RT
    B = R @ Bt @ RT
    I = np.eye(n)
    lam_h = np.asarray(lam_h, dtype=np.float64)[..., None, None]
    if np.ndim(alpha_g) == 0 and alpha_g == 0.0:
        relax = R @ (np.exp(-th)[..., :, None] * RT) - I
    else:
        ag = np.asarray(alpha_g, dtype=np.float64)[..., None]
        em, ep = np.exp(-th), np.exp(th)
        relax = R @ (((em - 1.0) - ag * (ep - 1.0) * (1.0 - em))[..., :, None] * RT)
    return -adv + (Omega @ T - T @ Omega) + 2.0 * B + relax / lam_h


def polymer_step(T, u, v, w, phic, d, grid):
    """RK2-TVD of Eqs. NS42-NS46.  Returns (Theta^{n+1}, weighted tau tensor)."""
    L = velocity_gradient(u, v, w, d, grid)
    dt = d.dt
    mu_p, lam_h, ag = d.polymer_props(phic)
    sch = getattr(d, "advection", "central")
    T1 = T + dt * rh(T, L, advection(T, u, v, w, grid, sch), lam_h, ag)
    T2 = 0.5 * T + 0.5 * (T1 + dt * rh(T1, L, advection(T1, u, v, w, grid, sch), lam_h, ag))
    th, R = decompose(T2)
    n = T.shape[-1]
    c = R @ (np.exp(th)[..., :, None] * np.swapaxes(R, -1, -2))
    taup = np.asarray(mu_p / lam_h)[..., None, None] * (c - np.eye(n))
    if d.approach1:
        return T2, taup
    tau = 0.5 * (1.0 + phic)[..., None, None] * taup
    return T2, tau


def tau_components(tau, dim):
    """Tensor (..., n, n) -> dict of named components (zeros where absent in 2D)."""
    if tau is None:
        return None
    if dim == 2:
        z = np.zeros_like(tau[..., 0, 0])
        return dict(xx=tau[..., 0, 0], xz=tau[..., 0, 1], zz=tau[..., 1, 1], yy=z, xy=z, yz=z)
    return dict(xx=tau[..., 0, 0], yy=tau[..., 1, 1], zz=tau[..., 2, 2],
                xy=tau[..., 0, 1], xz=tau[..., 0, 2], yz=tau[..., 1, 2])
