"""Pins of the oracle's Navier-Stokes step (Section 3.2.2, Eqs. NS35-NS39)."""
import math

import numpy as np
import pytest

from paper_2111_04577_gb300 import workloads as wl
from oracle import step, operators as op
from oracle.params import Derived


def grid(dim, n=16):
    if dim == 2:
        return wl.Grid(n, 1, n // 2, 2.0, 2.0 / n, 1.0, 1)
    return wl.Grid(n, n // 2, n // 2, 2.0, 1.0, 1.0, 1)


@pytest.mark.parametrize("dim", [2, 3])
def test_projection_gives_zero_divergence(dim):
    g = grid(dim)
    prm = wl.params_from_groups(ratio_rho=20.0, ratio_mu=10.0, theta_deg=70.0)
    w = wl.Workload("t", g, prm, 1)
    st = step.State(g, prm.as_dict(), wl.initial_phi(w), vel0=wl.random_velocity(g, 7, 0.3))
    for _ in range(3):
        st.step()
        u, v, ww = st.vel
        div = op.div_faces(u, v, ww, g.dx, dim)
        assert np.max(np.abs(div)) < 1e-11 * np.max(np.abs(u)) / g.dx
        assert np.all(ww[0] == 0) and np.all(ww[-1] == 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_couette_is_an_exact_steady_state(dim):
    """One phase (phi = +1), walls moving at -U and +U: the linear profile is a
    discrete steady solution of Eqs. NS35-NS39 and phi stays 1."""
    g = grid(dim)
    U = 0.7
    prm = wl.params_from_groups(ratio_rho=1000.0, ratio_mu=30.0)
    prm.uw_bot, prm.uw_top = -U, U
    nz, ny, nx = g.coarse_shape
    z = (np.arange(nz) + 0.5) * g.dx
    u = np.broadcast_to((U * (2 * z / g.lz - 1))[:, None, None], (nz, ny, nx)).copy()
    vel0 = (u, np.zeros_like(u), np.zeros((nz + 1, ny, nx)))
    st = step.State(g, prm.as_dict(), np.ones(g.fine_shape), vel0=vel0)
    for _ in range(5):
        st.step()
    assert np.max(np.abs(st.vel[0] - u)) < 1e-12
    assert np.max(np.abs(st.vel[2])) < 1e-12
    assert np.max(np.abs(st.phi - 1)) < 1e-13
    assert np.max(np.abs(st.p - st.p.mean())) < 1e-10


def test_shear_wave_decay_matches_the_bdf2_recurrence():
    """u = A sin(pi z/Lz) in one phase is a discrete Dirichlet eigenmode (eigenvalue
    lz1); Eq. NS35's split (implicit nu_m, explicit nu) gives the amplitude
    recurrence (g0 a' - a_hat)/dt = nu_m lz1 a' - nu_m lz1 a* + nu lz1 a*,
    which pins the restored -u_hat/dt and both viscous terms."""
    g = grid(2)
    prm = wl.params_from_groups(Re=2.0, ratio_rho=5.0, ratio_mu=3.0)
    d = Derived(prm.as_dict())
    nz, ny, nx = g.coarse_shape
    D = g.dx
    z = (np.arange(nz) + 0.5) / nz
    mode = np.sin(np.pi * z)[:, None, None] * np.ones((nz, ny, nx))
    A0 = 0.3
    st = step.State(g, prm.as_dict(), np.ones(g.fine_shape),
                    vel0=(A0 * mode, np.zeros_like(mode), np.zeros((nz + 1, ny, nx))))
    lz1 = -4 / D ** 2 * math.sin(math.pi / (2 * nz)) ** 2
    nu = d.mu_s1 / d.rho1
    a, ao = A0, A0
    for _ in range(20):
        st.step()
        ah, ast = 2 * a - 0.5 * ao, 2 * a - ao
        an = (ah / d.dt + (nu - d.nu_m) * lz1 * ast) / (1.5 / d.dt - d.nu_m * lz1)
        ao, a = a, an
        assert np.max(np.abs(st.vel[0] - a * mode)) < 1e-12 * A0
    # and the continuous decay exp(-nu pi^2 t / Lz^2) to within O(dt^2 + dx^2)
    t = 20 * d.dt
    assert abs(a / A0 - math.exp(-nu * math.pi ** 2 * t / g.lz ** 2)) < 5e-4


def test_hydrostatic_rest_stays_at_rest():
    """One heavy phase under gravity: every explicit term is a pure z-gradient, the
    projection removes it, and the fluid stays at rest while p tends to
    hydrostatic."""
    g = grid(2)
    prm = wl.params_from_groups(ratio_rho=2.0, ratio_mu=10.0)
    prm.gz = -9.81
    st = step.State(g, prm.as_dict(), np.ones(g.fine_shape))
    for _ in range(150):
        st.step()
        assert np.max(np.abs(st.vel[0])) < 1e-11
        assert np.max(np.abs(st.vel[2])) < 1e-11
    dpdz = (st.p[1:] - st.p[:-1]) / g.dx
    assert np.max(np.abs(dpdz / (st.d.rho1 * -9.81) - 1)) < 1e-3


def test_advection_conserves_momentum():
    """The conservative central fluxes telescope: with periodic x, y and walls at
    rest, the advective part of each momentum right side sums to zero."""
    from oracle import ns
    g = grid(3)
    u, v, w = wl.random_velocity(g, 9)
    rphi = op.restrict(np.ones(g.fine_shape), 2, 2, 3)
    rG = op.restrict(np.zeros(g.fine_shape), 2, 2, 3)
    z = np.zeros_like(u)
    lin = wl.params_from_groups()
    lin.mu1 = lin.mu2 = 0.0          # no viscous terms, nu_m = 0
    d0 = Derived(lin.as_dict())
    assert d0.nu_m == 0.0
    Ru, Rv, Rw = ns.momentum_rhs((u, v, w), (u, v, w), z, z, None, rphi, rG, d0, g)
    # u^{n-1} = u^n: u_hat = 1.5 u, so R + 1.5 u/dt is the advection alone.
    # (Wall-normal momentum is not conserved: the walls take its flux.)
    for R, a in ((Ru, u), (Rv, v)):
        adv = R + 1.5 * a / d0.dt
        assert abs(adv.sum()) < 1e-11 * np.abs(adv).sum()
