"""Pins of the oracle's Cahn-Hilliard step (Section 3.2.1, Eqs. NS25-NS34, NS48).

What fixes each part, independently of the oracle's own formulas:
  * the un-split Eq. NS25 with the discrete no-flux condition Eq. NS14 must hold
    for the result of the two split solves (pins alpha, c, Q, B(g), the solves);
  * the choice of the wall gradient of f(phi*) - S/eta^2 phi* in Eq. NS33 cancels;
  * sum(phi) is conserved to round-off (Eq. NS1 with NS14 and no penetration);
  * theta = 90 deg walls equal a mirror (homogeneous Neumann) boundary;
  * a planar interface relaxes to tanh(s/(sqrt(2) eta)) (Eqs. NS5-NS6) at O(h^2);
  * the equilibrium 2D cap obeys Eq. NS48 (Section 4.4);
  * the stabilised scheme decreases the free energy without flow;
  * BDF2 (Eq. NS31) is second order in time.
"""
import math

import numpy as np
import pytest

from paper_2111_04577_gb300 import workloads as wl
from oracle import ch, step, observables as ob
from oracle.params import Derived


# --- independent helpers written for the tests (periodic x/y, walls in z) ----
def lapN(a, h):
    out = np.zeros_like(a)
    out += (np.roll(a, -1, 2) - 2 * a + np.roll(a, 1, 2)) / h ** 2
    if a.shape[1] > 1:
        out += (np.roll(a, -1, 1) - 2 * a + np.roll(a, 1, 1)) / h ** 2
    up = np.concatenate([a[1:], a[-1:]], 0)
    dn = np.concatenate([a[:1], a[:-1]], 0)
    return out + (up - 2 * a + dn) / h ** 2


def small(dim=2, dual=1, theta=60.0, n=16, **kw):
    if dim == 2:
        g = wl.Grid(n, 1, n // 2, 4.0, 4.0 / n, 2.0, dual)
    else:
        g = wl.Grid(n, n, n // 2, 4.0, 4.0, 2.0, dual)
    prm = wl.params_from_groups(theta_deg=theta, **kw)
    prm.theta_top_deg = 75.0
    w = wl.Workload("t", g, prm, 1)
    return w


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("dual", [1, 0])
def test_unsplit_ns25_residual(dim, dual):
    w = small(dim, dual)
    g = w.grid
    d = Derived(w.params.as_dict())
    phi0 = wl.initial_phi(w)
    rng = np.random.default_rng(3)
    phim = phi0 + 0.01 * rng.uniform(-1, 1, phi0.shape)
    vel = wl.random_velocity(g, 5)
    velm = wl.random_velocity(g, 6)
    o = ch.ch_step(phi0, phim, vel, velm, d, g)
    phi, h = o["phi"], g.h
    phis, phih = 2 * phi0 - phim, 2 * phi0 - 0.5 * phim
    # wetting ghost of Eq. NS34: n.grad(phi) = g on both walls
    s2 = math.sqrt(2)
    wb, wt = 1.5 * phis[0] - 0.5 * phis[1], 1.5 * phis[-1] - 0.5 * phis[-2]
    gb = math.cos(math.radians(60.0)) * (1 - wb ** 2) / (s2 * d.eta)
    gt = math.cos(math.radians(75.0)) * (1 - wt ** 2) / (s2 * d.eta)
    lap_g = lapN(phi, h)
    lap_g[0] += gb / h
    lap_g[-1] += gt / h
    fstar = phis * (phis ** 2 - 1) / d.eta ** 2
    q = lap_g - d.S / d.eta ** 2 * (phi - phis) - fstar       # bracket of Eq. NS25
    lhs = (1.5 * phi - phih) / d.dt + o["A"]
    rhs = -d.Ml * lapN(q, h)                                  # n.grad q = 0  (Eq. NS14)
    scale = np.max(np.abs(phih / d.dt))
    assert np.max(np.abs(lhs - rhs)) < 1e-11 * scale
    # split constants: NS26 x NS27 reproduce NS25's operator
    assert abs(d.alpha ** 2 + d.S / d.eta ** 2 * d.alpha + 1.5 / (d.Ml * d.dt)) < 1e-9 * d.alpha ** 2


def test_two_ghost_form_is_independent_of_the_wall_gradient():
    w = small(2)
    g = w.grid
    d = Derived(w.params.as_dict())
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 1)
    ref = ch.ch_step(phi0, phi0, vel, vel, d, g)["phi"]
    rng = np.random.default_rng(0)
    nx = g.fine_shape[2]
    for _ in range(3):
        ghb = rng.standard_normal((1, nx)) * 1e3
        ght = rng.standard_normal((1, nx)) * 1e3
        got = ch.ch_step_two_ghost(phi0, phi0, vel, vel, d, g, ghb, ght)
        assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_conserved_coupled(dim):
    w = small(dim, 1, ratio_rho=10.0, ratio_mu=5.0)
    g = w.grid
    st = step.State(g, w.params.as_dict(), wl.initial_phi(w), vel0=wl.random_velocity(g, 2, 0.3))
    m0 = np.sum(st.phi)
    for _ in range(15):
        st.step()
    scale = np.sum(np.abs(st.phi))
    assert abs(np.sum(st.phi) - m0) < 1e-13 * scale


def test_theta90_equals_mirror():
    """A theta = 90 deg wall is a mirror: the solution on [0, Lz] equals the lower
    half of the mirror-symmetric solution on [0, 2 Lz]."""
    n = 16
    g1 = wl.Grid(n, 1, n // 2, 4.0, 4.0 / n, 2.0, 1)
    g2 = wl.Grid(n, 1, n, 4.0, 4.0 / n, 4.0, 1)
    prm = wl.params_from_groups(theta_deg=90.0)
    d = Derived(prm.as_dict())
    w1 = wl.Workload("a", g1, prm, 1)
    phi0 = wl.initial_phi(w1, centre=(2.0, 0, 0.7))
    phim = phi0 + 1e-3 * np.sin(np.arange(phi0.size).reshape(phi0.shape))
    big0 = np.concatenate([phi0, phi0[::-1]], 0)
    bigm = np.concatenate([phim, phim[::-1]], 0)
    z1 = wl.zero_state(g1)
    z2 = wl.zero_state(g2)
    v1 = (z1["u"], z1["v"], z1["w"])
    v2 = (z2["u"], z2["v"], z2["w"])
    a = ch.ch_step(phi0, phim, v1, v1, d, g1)["phi"]
    b = ch.ch_step(big0, bigm, v2, v2, d, g2)["phi"]
    assert np.max(np.abs(b[: a.shape[0]] - a)) < 1e-12
    assert np.max(np.abs(b[::-1][: a.shape[0]] - a)) < 1e-12


def test_tanh_profile_second_order():
    """Planar interfaces at rest: the discrete equilibrium approaches
    tanh(s/(sqrt(2) eta)) (Eqs. NS5-NS6, G = 0 in 1D) with error O((h/eta)^2)."""
    errs = []
    eta, lx = 0.1, 4.0
    for ratio in (2, 4, 8):
        h = eta / ratio
        nx = int(round(lx / h))
        g = wl.Grid(nx // 2, 1, 2, lx, lx / (nx // 2), 4 * h, 1)
        prm = wl.Params(eta=eta, sigma=1.0, mobility=1.0, dt=2e-3, S=4.0).as_dict()
        x = (np.arange(nx) + 0.5) * h
        ex = np.tanh((1.0 - np.abs(x - 2.0)) / (math.sqrt(2) * eta))
        # a zero-mean perturbation, symmetric about the droplet centre
        pert = 0.05 * np.cos(2 * np.pi * 3 * (x - 2.0) / lx)
        phi0 = np.broadcast_to(ex + pert, g.fine_shape).copy()
        st = step.State(g, prm, phi0)
        for _ in range(3000):
            st.step(with_ns=False)
        errs.append(np.max(np.abs(st.phi[0, 0] - ex)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - 2.0) < 0.15), (errs, slopes)


def _cap_measure(phi, h):
    nz, ny, nx = phi.shape
    col = phi[:, 0, nx // 2]
    k = np.where(col > 0)[0].max()
    H = (k + 0.5 + col[k] / (col[k] - col[k + 1])) * h
    wb = 1.5 * phi[0, 0] - 0.5 * phi[1, 0]
    idx = np.where(wb > 0)[0]
    i0, i1 = idx.min(), idx.max()
    xl = (i0 - 0.5 + (0 - wb[i0 - 1]) / (wb[i0] - wb[i0 - 1])) * h
    xr = (i1 + 0.5 + wb[i1] / (wb[i1] - wb[i1 + 1])) * h
    return H, xr - xl


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_equilibrium_cap_ns48(theta):
    """Section 4.4: at equilibrium H = R(1 - cos t) sqrt(pi/(2(t - sin t cos t))),
    L = 2 R sin t sqrt(...), with R the radius of the initial half-disc of equal
    area; R is measured on the phi = 0 contour so that the diffuse-interface
    shrinkage (Section 1) does not enter the comparison."""
    eta, n = 0.05, 240
    g = wl.Grid(n, 1, n // 3, 6.0, 6.0 / n, 2.0, 1)
    lam = 3 * eta / (2 * math.sqrt(2))
    prm = wl.Params(eta=eta, sigma=1.0, mobility=1e-2 / lam, theta_bot_deg=theta, dt=1e-2, S=4.0)
    w = wl.Workload("cap", g, prm, 1, amp=0.0)
    st = step.State(g, prm.as_dict(), wl.initial_phi(w, centre=(3.0, 0, 0.0)))
    energies = []
    for s in range(1500):
        st.step(with_ns=False)
        if s % 100 == 0:
            energies.append(ob.energy(st.phi, st.d, g))
    assert np.all(np.diff(energies) <= 1e-12 * abs(energies[0]))
    # radius of the half-disc with the area enclosed by the phi = 0 contour
    area = np.count_nonzero(st.phi > 0) * g.h ** 2
    R = math.sqrt(2 * area / math.pi)
    t = math.radians(theta)
    fac = math.sqrt(math.pi / (2 * (t - math.sin(t) * math.cos(t))))
    H, L = _cap_measure(st.phi, g.h)
    assert abs(H / (R * (1 - math.cos(t)) * fac) - 1) < 0.03
    assert abs(L / (2 * R * math.sin(t) * fac) - 1) < 0.03


def test_bdf2_second_order_in_time():
    """Self-convergence under dt halving (Eq. NS31): successive differences of the
    solution at a fixed time fall with a least-squares slope of 2 +- 0.2."""
    n = 16
    g = wl.Grid(n, 1, n // 2, 4.0, 4.0 / n, 2.0, 1)
    prm = wl.params_from_groups(theta_deg=60.0).as_dict()
    prm.update(eta=0.3, mobility=2e-2, theta_top_deg=75.0)
    lam = 3 * 0.3 / (2 * math.sqrt(2))
    T = 0.02
    # one S for all dt, admissible (Eq. NS30) at the smallest step
    prm["S"] = 1.01 * 0.09 * math.sqrt(6 / (prm["mobility"] * lam * T / 160))
    x, y, z = wl.fine_centres(g)
    phi0 = np.broadcast_to(0.6 * np.cos(2 * np.pi * x / 4.0) * np.cos(np.pi * z / 2.0) + 0.1,
                           g.fine_shape).copy()
    vel = wl.random_velocity(g, 4, 0.2)
    sols = []
    for m in (10, 20, 40, 80, 160):
        prm["dt"] = T / m
        st = step.State(g, prm, phi0, vel0=vel)
        for _ in range(m):
            st.step(with_ns=False)
        sols.append(st.phi)
    diffs = np.array([np.max(np.abs(sols[i] - sols[i + 1])) for i in range(4)])
    slope = np.polyfit(np.log2([1, 0.5, 0.25, 0.125]), np.log2(diffs), 1)[0]
    assert abs(slope - 2.0) < 0.2, (diffs, slope)


def test_contact_angle_sign():
    """theta < 90 deg spreads (wetted length grows), theta > 90 deg recoils."""
    res = {}
    for th in (45.0, 135.0):
        w = small(2, 1, theta=th, n=32)
        prm = w.params.as_dict()
        prm.update(eta=0.08, mobility=1e-1, dt=1e-3, S=0.0)
        g = w.grid
        st = step.State(g, prm, wl.initial_phi(wl.Workload("t", g, wl.Params(**prm), 1, amp=0)))
        l0 = ob.wetted(st.phi, g)
        for _ in range(100):
            st.step(with_ns=False)
        res[th] = ob.wetted(st.phi, g) - l0
    assert res[45.0] > 0 > res[135.0]
