"""Pins of the oracle's Navier-Stokes coupling terms (Section 3.2.2, Eqs. NS2,
NS5-NS10, NS12, NS35-NS36; Section 4.4, Eq. NS48; the observables).

Each pin is fixed by something other than the oracle's own formulas:
  * the momentum right side of Eq. NS36 (with the -u_hat/dt of Eq. NS35) on
    smooth manufactured fields converges at second order to the continuous
    expression, written here from Eqs. NS2 and NS8-NS10 and differentiated
    symbolically: advection, J . grad u, both pressure terms, nu_m lap u*,
    div tau, div(mu (grad u + grad u^T)) with variable mu, G grad phi, the body
    force -- a dropped term, a wrong sign or a transposed index leaves an O(1)
    error that does not converge;
  * a static droplet carries the Laplace pressure jump sigma/R (2D) or
    2 sigma/R (3D) (G grad phi with its sign and factor);
  * a two-layer Couette flow with mu1 != mu2 reaches the steady state of an
    independent 1D balance of edge fluxes (the variable viscosity at edges);
  * a body-force-driven Oldroyd-B channel reaches Poiseuille flow with the
    total viscosity mu_s + mu_p in the droplet phase, and the solvent viscosity
    alone in the other phase (div tau and the (1 + phi)/2 weighting of NS12);
  * a 3D sessile droplet relaxes to the spherical cap of its volume at the
    contact angle;
  * a flat equilibrium interface carries a free energy of sigma per unit
    length (Eqs. NS5-NS7);
  * translating phi translates its centroid.
Each pin is also run once with a mistake planted in the oracle (a sign flip,
a swapped phase, a wrong weight) and must then fail.
"""
import math

import numpy as np
import pytest
import sympy as sp

from paper_2111_04577_gb300 import workloads as wl
from oracle import ns, observables as ob, polymer, step
from oracle.params import Derived
from mutate import mutated


# ---------------------------------------------------------------------------
# manufactured momentum right side
# ---------------------------------------------------------------------------
X, Y, Z = sp.symbols("x y z")
PI = sp.pi


def _fields(dim):
    """Smooth periodic-in-x,y test fields on Lx = Ly = 2, Lz = 1."""
    yy = (lambda e: e) if dim == 3 else (lambda e: 0)
    f = dict(
        U1=0.3 * sp.sin(PI * X + 0.4) * sp.cos(PI * Z / 2 + 0.3) + yy(0.2 * sp.cos(PI * Y)),
        U0=0.2 * sp.cos(PI * X) * sp.sin(PI * Z + 0.5),
        V1=yy(0.2 * sp.cos(PI * Y + 0.1) * sp.sin(PI * Z + 0.2) + 0.1 * sp.sin(PI * X)),
        V0=yy(0.1 * sp.sin(PI * Y) * sp.cos(PI * X)),
        W1=0.25 * sp.cos(PI * X + 0.2) * sp.sin(PI * Z) + yy(0.1 * sp.sin(PI * Y)),
        W0=0.15 * sp.sin(PI * X) * sp.cos(PI * Z / 2),
        P1=0.7 * sp.cos(PI * X) * sp.cos(PI * Z) + yy(0.2 * sp.sin(PI * Y)),
        P0=0.5 * sp.sin(PI * X + 0.3) * sp.cos(PI * Z),
        PHI=0.8 * sp.sin(PI * X + 0.3) * sp.cos(PI * Z / 2 + 0.2) * (sp.cos(PI * Y - 0.2) if dim == 3 else 1),
        G=2.0 * sp.cos(PI * X - 0.5) * sp.sin(PI * Z + 0.1) + yy(0.5 * sp.cos(PI * Y)),
        Txx=0.3 * sp.cos(PI * X) * sp.sin(PI * Z),
        Txz=0.2 * sp.sin(PI * X + 0.1) * sp.cos(PI * Z),
        Tzz=0.1 * sp.cos(PI * X + 0.4) * sp.cos(PI * Z / 2),
        Tyy=yy(0.2 * sp.sin(PI * Y + 0.3) * sp.cos(PI * Z)),
        Txy=yy(0.15 * sp.cos(PI * X + PI * Y)),
        Tyz=yy(0.1 * sp.sin(PI * Y) * sp.sin(PI * Z + 0.2)),
    )
    return {k: sp.sympify(v) for k, v in f.items()}


PRM = dict(rho1=1.0, rho2=0.25, mu1=0.08, mu2=0.03, sigma=1.0, eta=0.05, mobility=0.2,
           theta_bot_deg=90.0, theta_top_deg=90.0, dt=0.01, nu_m=0.3, gx=0.1, gy=0.05, gz=-0.2)


def continuous_rhs(dim, prm=PRM):
    """The right side of Eq. NS36 (u~ on the left), from Eqs. NS2, NS8-NS10 and
    NS35: R = -u_hat/dt + div(u* u*) + (1/rho) J . grad u* + (1/rho0) grad p^n
    + (1/rho - 1/rho0) grad p* + nu_m lap u* - (1/rho) div tau*
    - (1/rho) div(mu (grad u* + grad u*^T)) - (1/rho) G grad phi - g."""
    f = _fields(dim)
    axes = (X, Y, Z) if dim == 3 else (X, Z)
    comp = ("x", "y", "z") if dim == 3 else ("x", "z")
    us = {"x": 2 * f["U1"] - f["U0"], "y": 2 * f["V1"] - f["V0"], "z": 2 * f["W1"] - f["W0"]}
    uh = {"x": 2 * f["U1"] - f["U0"] / 2, "y": 2 * f["V1"] - f["V0"] / 2, "z": 2 * f["W1"] - f["W0"] / 2}
    ps = 2 * f["P1"] - f["P0"]
    phi = f["PHI"]
    rho1, rho2 = prm["rho1"], prm["rho2"]
    rho = (1 + phi) / 2 * rho1 + (1 - phi) / 2 * rho2                 # NS8
    mu = (1 + phi) / 2 * prm["mu1"] + (1 - phi) / 2 * prm["mu2"]      # NS9
    rho0 = min(rho1, rho2)
    J = {c: -(rho1 - rho2) / 2 * prm["mobility"] * sp.diff(f["G"], a) for c, a in zip(comp, axes)}  # NS10
    tau = {("x", "x"): f["Txx"], ("x", "z"): f["Txz"], ("z", "z"): f["Tzz"],
           ("y", "y"): f["Tyy"], ("x", "y"): f["Txy"], ("y", "z"): f["Tyz"]}
    T = lambda a, b: tau.get((a, b), tau.get((b, a)))
    grav = {"x": prm["gx"], "y": prm["gy"], "z": prm["gz"]}
    out = {}
    for c, a in zip(comp, axes):
        adv = sum(sp.diff(us[c] * us[e], b) for e, b in zip(comp, axes))
        jg = sum(J[e] * sp.diff(us[c], b) for e, b in zip(comp, axes))
        lap = sum(sp.diff(us[c], b, 2) for b in axes)
        divt = sum(sp.diff(T(c, e), b) for e, b in zip(comp, axes))
        visc = sum(sp.diff(mu * (sp.diff(us[c], b) + sp.diff(us[e], a)), b) for e, b in zip(comp, axes))
        r = (-uh[c] / prm["dt"] + adv + jg / rho + sp.diff(f["P1"], a) / rho0
             + (1 / rho - 1 / rho0) * sp.diff(ps, a) + prm["nu_m"] * lap - divt / rho
             - visc / rho - f["G"] * sp.diff(phi, a) / rho - grav[c])
        out[c] = sp.lambdify((X, Y, Z), r, "numpy")
    return out


def _sample(expr, x, y, z):
    fn = sp.lambdify((X, Y, Z), expr, "numpy")
    return np.broadcast_to(np.asarray(fn(x, y, z), dtype=float), np.broadcast(x, y, z).shape).copy()


def discrete_rhs(dim, n, rhs=None):
    """The oracle's momentum_rhs on the manufactured fields sampled where the
    MAC mesh stores them (coarse nx = n, nz = n/2, dx = 2/n)."""
    rhs = rhs or ns.momentum_rhs
    f = _fields(dim)
    nx, nz = n, n // 2
    ny = n if dim == 3 else 1
    D = 2.0 / n
    g = wl.Grid(nx, ny, nz, 2.0, 2.0 if dim == 3 else D, 1.0, 1)
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    kf = np.arange(nz + 1)[:, None, None]
    xc, xf = (i + 0.5) * D, i * D
    yc, yf = ((j + 0.5) * D, j * D) if dim == 3 else (0 * j, 0 * j)
    zc, zf = (k + 0.5) * D, kf * D
    S = _sample
    vel1 = (S(f["U1"], xf, yc, zc), S(f["V1"], xc, yf, zc), S(f["W1"], xc, yc, zf))
    vel0 = (S(f["U0"], xf, yc, zc), S(f["V0"], xc, yf, zc), S(f["W0"], xc, yc, zf))
    rphi = {"c": S(f["PHI"], xc, yc, zc), "fx": S(f["PHI"], xf, yc, zc), "fz": S(f["PHI"], xc, yc, zf),
            "exz": S(f["PHI"], xf, yc, zf)}
    rG = {"c": S(f["G"], xc, yc, zc), "fx": S(f["G"], xf, yc, zc), "fz": S(f["G"], xc, yc, zf)}
    if dim == 3:
        rphi.update(fy=S(f["PHI"], xc, yf, zc), exy=S(f["PHI"], xf, yf, zc), eyz=S(f["PHI"], xc, yf, zf))
        rG["fy"] = S(f["G"], xc, yf, zc)
    tau = {c: S(f["T" + c], xc, yc, zc) for c in ("xx", "xz", "zz", "yy", "xy", "yz")}
    prm = dict(wl.Params().as_dict(), **PRM)
    d = Derived(prm)
    Ru, Rv, Rw = rhs(vel1, vel0, S(f["P1"], xc, yc, zc), S(f["P0"], xc, yc, zc), tau, rphi, rG, d, g)
    return dict(Ru=Ru, Rv=Rv, Rw=Rw, at=dict(u=(xf, yc, zc), v=(xc, yf, zc), w=(xc, yc, zf)), nz=nz)


def manufactured_errors(dim, sizes, rhs=None):
    """Max interior error of each momentum component at each size (rows that
    touch a wall ghost are left out: the wall closures are pinned elsewhere)."""
    exact = continuous_rhs(dim)
    errs = []
    for n in sizes:
        o = discrete_rhs(dim, n, rhs)
        nz = o["nz"]
        e = []
        eu = exact["x"](*o["at"]["u"])
        e.append(np.max(np.abs(o["Ru"] - eu)[2:nz - 2]))
        ew = exact["z"](*o["at"]["w"])
        e.append(np.max(np.abs(o["Rw"] - ew)[2:nz - 1]))
        if dim == 3:
            ev = exact["y"](*o["at"]["v"])
            e.append(np.max(np.abs(o["Rv"] - ev)[2:nz - 2]))
        errs.append(e)
    return np.array(errs)


def second_order(errs):
    slopes = np.log2(errs[:-1] / errs[1:])
    return bool(np.all(slopes > 1.7) and np.all(slopes < 2.4)), slopes


SIZES = {2: (16, 32, 64), 3: (12, 24, 48)}


@pytest.mark.parametrize("dim", [2, 3])
def test_momentum_rhs_converges_to_the_continuous_equation(dim):
    errs = manufactured_errors(dim, SIZES[dim])
    ok, slopes = second_order(errs)
    assert ok, (errs, slopes)


MOMENTUM_MUTATIONS = [
    # J . grad u with the wrong sign
    ("Ru = (-uh / dt + adv + jg / rho_u", "Ru = (-uh / dt + adv - jg / rho_u"),
    # the transposed gradient of the x-z shear stress with the wrong sign
    ("Sxz = mu_exz * ((usz[1:] - usz[:-1]) / D + (ws - xm(ws)) / D)",
     "Sxz = mu_exz * ((usz[1:] - usz[:-1]) / D - (ws - xm(ws)) / D)"),
    # the polymer stress pushing the wrong way
    ("+ d.nu_m * lap - divt / rho_u", "+ d.nu_m * lap + divt / rho_u"),
    # the surface force with the wrong sign
    ("- st / rho_u - d.g[0])", "+ st / rho_u - d.g[0])"),
    # the explicit pressure with rho0 in place of rho
    ("gp = (p_n - xm(p_n)) / D / rho0 + (1 / rho_u - 1 / rho0)", "gp = (p_n - xm(p_n)) / D / rho0 + (1 / rho0 - 1 / rho0)"),
    # mu(grad u) without the factor 2 of the normal stress
    ("Sxx = 2 * mu_c * (xp(us) - us) / D", "Sxx = mu_c * (xp(us) - us) / D"),
]


@pytest.mark.parametrize("old,new", MOMENTUM_MUTATIONS)
def test_planted_momentum_mistakes_fail_the_manufactured_pin(old, new):
    bad = mutated(ns, "momentum_rhs", old, new)
    ok, _ = second_order(manufactured_errors(2, SIZES[2], bad))
    assert not ok


# ---------------------------------------------------------------------------
# static droplet: Laplace pressure jump (G grad phi, Eqs. NS2, NS5, NS7)
# ---------------------------------------------------------------------------
def laplace_jump(dim):
    """p(centre) - p(far field) of a resting droplet of radius R = 1 after a few
    steps; sigma = 1.  Returns (measured, sharp-interface value (dim - 1) sigma/R)."""
    n, L = (64, 4.0) if dim == 2 else (32, 4.0)
    eta = 0.05 if dim == 2 else 0.1
    dx = L / n
    g = wl.Grid(n, n if dim == 3 else 1, n, L, L if dim == 3 else dx, L, 1)
    prm = wl.Params(rho1=1.0, rho2=1.0, mu1=0.1, mu2=0.1, sigma=1.0, eta=eta, mobility=1e-3, dt=1e-3)
    w = wl.Workload("laplace", g, prm, 1, R0=1.0, amp=0.0)
    st = step.State(g, prm.as_dict(), wl.initial_phi(w, centre=(L / 2, L / 2, L / 2)))
    for _ in range(20):
        st.step()
    p = st.p
    nz, ny, nx = p.shape
    jy = slice(ny // 2 - 1, ny // 2 + 1) if dim == 3 else slice(0, 1)
    pin = p[nz // 2 - 1:nz // 2 + 1, jy, nx // 2 - 1:nx // 2 + 1].mean()
    pout = p[0:2, 0:2 if dim == 3 else 1, 0:2].mean()
    return pin - pout, (dim - 1) * 1.0 / 1.0


LAPLACE_TOL = {2: 0.06, 3: 0.08}   # diffuse-interface corrections O(eta/R): eta/R = 0.05, 0.1


@pytest.mark.parametrize("dim", [2, 3])
def test_static_droplet_laplace_jump(dim):
    dp, ref = laplace_jump(dim)
    assert abs(dp / ref - 1) < LAPLACE_TOL[dim], (dp, ref)


def test_planted_surface_force_sign_fails_the_laplace_pin(monkeypatch):
    bad = mutated(ns, "momentum_rhs", [("- st / rho_u - d.g[0])", "+ st / rho_u - d.g[0])"),
                                       ("- st / rho_w - d.g[2])", "+ st / rho_w - d.g[2])")])
    monkeypatch.setattr(ns, "momentum_rhs", bad)
    dp, ref = laplace_jump(2)
    assert not abs(dp / ref - 1) < LAPLACE_TOL[2]


# ---------------------------------------------------------------------------
# two-layer Couette flow: variable viscosity at the x-z edges
# ---------------------------------------------------------------------------
def two_layer_couette():
    """Droplet phase (mu1 = 1) below z = 1/2, ambient (mu2 = 1/4) above, top wall
    at U = 1.  Returns (oracle's steady u(z), independent steady u(z)).

    The independent state solves the 1D balance of the discrete shear flux:
    mu_e(k) (u_k - u_{k-1})/dx = F for every edge k = 0..nz, with the no-slip
    ghosts u_{-1} = -u_0 and u_nz = 2U - u_{nz-1}; mu_e(k) is Eq. NS9 of phi at
    the edge, phi there being the mean of the fine cells that meet at the edge
    (Eq. dual2), computed here from the oracle's final phi."""
    nz, nx, Lz, U = 16, 4, 1.0, 1.0
    dx = Lz / nz
    g = wl.Grid(nx, 1, nz, nx * dx, dx, Lz, 1)
    m1, m2, eta = 1.0, 0.25, 0.04
    prm = wl.Params(rho1=1.0, rho2=1.0, mu1=m1, mu2=m2, sigma=1.0, eta=eta, mobility=1e-4, dt=5e-3,
                    nu_m=1.0, uw_top=U)
    zf = (np.arange(2 * nz) + 0.5) * dx / 2
    phi0 = np.broadcast_to(np.tanh((0.5 - zf) / (math.sqrt(2) * eta))[:, None, None], g.fine_shape).copy()
    st = step.State(g, prm.as_dict(), phi0)
    for _ in range(1200):
        st.step()
    pf = st.phi[:, 0, 0]
    pad = np.concatenate([pf[:1], pf, pf[-1:]])             # mirror rows beyond the walls
    phie = 0.5 * (pad[0:2 * nz + 1:2] + pad[1:2 * nz + 2:2])  # edge k: fine rows 2k-1 and 2k
    mue = 0.5 * (1 + phie) * m1 + 0.5 * (1 - phie) * m2
    A = np.zeros((nz + 1, nz + 1))
    b = np.zeros(nz + 1)
    for k in range(nz + 1):
        c = mue[k] / dx
        if k == 0:
            A[k, 0] = 2 * c
        elif k == nz:
            A[k, nz - 1] = -2 * c
            b[k] = -2 * c * U
        else:
            A[k, k], A[k, k - 1] = c, -c
        A[k, nz] = -1.0
    sol = np.linalg.solve(A, b)
    return st.vel[0][:, 0, 0], sol[:nz]


def test_two_layer_couette_reaches_the_edge_flux_balance():
    u, ref = two_layer_couette()
    assert np.max(np.abs(u - ref)) < 1e-5 * np.max(np.abs(ref)), np.max(np.abs(u - ref))


def test_planted_phase_swap_fails_the_couette_pin(monkeypatch):
    bad = mutated(ns, "momentum_rhs", 'mu_exz = d.mu(rphi["exz"])', 'mu_exz = d.mu(-rphi["exz"])')
    monkeypatch.setattr(ns, "momentum_rhs", bad)
    u, ref = two_layer_couette()
    assert not np.max(np.abs(u - ref)) < 1e-5 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------
# Oldroyd-B channel: div tau and the (1 + phi)/2 weighting of Eq. NS12
# ---------------------------------------------------------------------------
def oldroyd_channel(sign):
    """Body force g = 1 between resting walls, phi = sign everywhere; the droplet
    phase (phi = +1) is Oldroyd-B with mu_s = mu_p = 1/2, lambda_H = 0.2; the
    other phase is Newtonian with mu2 = 1/4.  At steady state the polymer shear
    stress is mu_p du/dz, so the profile is Poiseuille's with the phase's total
    viscosity, u = g z (Lz - z)/(2 mu_t).  Returns max relative deviation."""
    nz, nx, Lz = 16, 4, 1.0
    dx = Lz / nz
    g = wl.Grid(nx, 1, nz, nx * dx, dx, Lz, 1)
    prm = wl.Params(rho1=1.0, rho2=1.0, mu1=1.0, mu2=0.25, sigma=1.0, eta=0.04, mobility=1e-4, dt=2e-3,
                    nu_m=1.0, wi=0.2, beta=0.5, gx=1.0)
    st = step.State(g, prm.as_dict(), np.full(g.fine_shape, float(sign)))
    with np.errstate(all="ignore"):
        for _ in range(2000):
            st.step()
    u = st.vel[0][:, 0, 0]
    z = (np.arange(nz) + 0.5) * dx
    ref = z * (Lz - z) / (2 * (1.0 if sign > 0 else 0.25))
    return float(np.max(np.abs(u - ref)) / np.max(ref))


CHANNEL_TOL = 0.02   # O(dx^2) of the cell-centred profile at nz = 16 (measured 0.95 % and 0.39 %)


@pytest.mark.parametrize("sign", [1, -1])
def test_oldroyd_b_channel_reaches_poiseuille_with_the_phase_viscosity(sign):
    assert oldroyd_channel(sign) < CHANNEL_TOL


def test_planted_polymer_mistakes_fail_the_channel_pin(monkeypatch):
    wrong_weight = mutated(polymer, "polymer_step", "tau = 0.5 * (1.0 + phic)", "tau = 0.5 * (1.0 - phic)")
    monkeypatch.setattr(polymer, "polymer_step", wrong_weight)
    assert not oldroyd_channel(1) < CHANNEL_TOL
    monkeypatch.undo()
    wrong_sign = mutated(ns, "momentum_rhs", "+ d.nu_m * lap - divt / rho_u", "+ d.nu_m * lap + divt / rho_u")
    monkeypatch.setattr(ns, "momentum_rhs", wrong_sign)
    assert not oldroyd_channel(1) < CHANNEL_TOL


# ---------------------------------------------------------------------------
# 3D sessile droplet: spherical cap at the contact angle
# ---------------------------------------------------------------------------
def cap3d(theta):
    """A hemisphere of radius 1 on the bottom wall relaxes without flow (CH only,
    large mobility) on a 64 x 64 x 24 fine mesh.  Returns the cap height and
    base radius over those of the spherical cap of the same volume at theta:
    R (1 - cos theta) and R sin theta with V = pi/3 R^3 (2 - 3 cos + cos^3)."""
    n, nz, L, eta = 32, 12, 4.0, 0.1
    dx = L / n
    g = wl.Grid(n, n, nz, L, L, nz * dx, 1)
    lam = 3 * eta / (2 * math.sqrt(2))
    prm = wl.Params(eta=eta, sigma=1.0, mobility=1e-2 / lam, theta_bot_deg=theta, dt=1e-2, S=4.0)
    w = wl.Workload("cap3d", g, prm, 1, amp=0.0)
    st = step.State(g, prm.as_dict(), wl.initial_phi(w, centre=(L / 2, L / 2, 0.0)))
    for _ in range(1500):
        st.step(with_ns=False)
    h = g.h
    t = math.radians(theta)
    vol = np.count_nonzero(st.phi > 0) * h ** 3
    R = (3 * vol / (math.pi * (2 - 3 * math.cos(t) + math.cos(t) ** 3))) ** (1 / 3)
    nzf, nyf, nxf = st.phi.shape
    c = st.phi[:, nyf // 2 - 1:nyf // 2 + 1, nxf // 2 - 1:nxf // 2 + 1].mean(axis=(1, 2))  # axis of the cap
    k = np.where(c > 0)[0].max()
    H = (k + 0.5 + c[k] / (c[k] - c[k + 1])) * h
    wall = 1.5 * st.phi[0] - 0.5 * st.phi[1]
    rb = math.sqrt(np.count_nonzero(wall > 0) * h * h / math.pi)
    return H / (R * (1 - math.cos(t))), rb / (R * math.sin(t))


@pytest.mark.slow
@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_3d_equilibrium_is_the_spherical_cap(theta):
    hr, br = cap3d(theta)
    assert abs(hr - 1) < 0.03 and abs(br - 1) < 0.03, (hr, br)


@pytest.mark.slow
def test_planted_wall_flux_sign_fails_the_cap_pin(monkeypatch):
    from oracle import ch
    bad = mutated(ch, "wall_flux", "gb = d.cos_bot * (1.0 - wb * wb)", "gb = -d.cos_bot * (1.0 - wb * wb)")
    monkeypatch.setattr(ch, "wall_flux", bad)
    hr, br = cap3d(60.0)
    assert not (abs(hr - 1) < 0.03 and abs(br - 1) < 0.03)


# ---------------------------------------------------------------------------
# free energy of a flat interface; centroid
# ---------------------------------------------------------------------------
def flat_interface_energy(ratio, energy=None):
    """Two flat interfaces x = 1 and x = 3 (tanh profile, Eq. NS5 in 1D) in a
    4 x 1 box with 90 deg walls, eta/h = ratio.  The free energy of Eqs. NS5-NS7
    is sigma per unit length of interface: E -> 2 sigma Lz.  Returns E/(2 sigma Lz)."""
    energy = energy or ob.energy
    eta, L, Lz, sigma = 0.1, 4.0, 1.0, 1.7
    h = eta / ratio
    nx, nz = int(round(L / h)), int(round(Lz / h))
    g = wl.Grid(nx // 2, 1, nz // 2, L, 2 * h, Lz, 1)
    x = (np.arange(nx) + 0.5) * h
    s = math.sqrt(2) * eta
    phi = np.tanh((x - 1.0) / s) - np.tanh((x - 3.0) / s) - 1.0
    phi = np.broadcast_to(phi[None, None, :], g.fine_shape).copy()
    d = Derived(dict(wl.Params(sigma=sigma, eta=eta, mobility=1e-3).as_dict()))
    return energy(phi, d, g) / (2 * sigma * Lz)


def test_flat_interface_energy_is_sigma_per_length():
    e = np.array([flat_interface_energy(r) for r in (2, 4, 8)])
    err = np.abs(e - 1)
    assert err[-1] < 2e-3, e
    assert np.all(np.log2(err[:-1] / err[1:]) > 1.8), e


def test_planted_energy_factor_fails_the_energy_pin():
    bad = mutated(ob, "energy", "e += np.sum((phi * phi - 1.0) ** 2) / (4.0 * d.eta ** 2)",
                  "e += np.sum((phi * phi - 1.0) ** 2) / (2.0 * d.eta ** 2)")
    assert not abs(flat_interface_energy(8, bad) - 1) < 2e-3


def test_centroid_follows_translations():
    """A droplet moved by whole fine cells moves its centroid by as much; a
    droplet symmetric about its centre has its centroid there."""
    g = wl.Grid(32, 32, 16, 4.0, 4.0, 2.0, 1)
    w = wl.Workload("c", g, wl.params_from_groups(), 1, R0=0.5, amp=0.0)
    h = g.h
    base = wl.initial_phi(w, centre=(1.5, 2.0, 1.0))
    c0 = ob.centroid(base, g)
    assert np.allclose(c0, (1.5, 2.0, 1.0), atol=1e-10)
    moved = np.roll(np.roll(base, 5, axis=2), -3, axis=1)
    up = np.concatenate([np.full((2,) + base.shape[1:], base[0, 0, 0]), moved[:-2]], axis=0)
    c1 = ob.centroid(up, g)
    assert np.allclose(c1, (c0[0] + 5 * h, c0[1] - 3 * h, c0[2] + 2 * h), atol=1e-10)
    bad = mutated(ob, "centroid", "wgt = 0.5 * (1.0 + phi)", "wgt = 0.5 * (1.0 - phi)")
    assert not np.allclose(bad(base, g), (1.5, 2.0, 1.0), atol=1e-3)
