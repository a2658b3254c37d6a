"""Pins of the oracle's log-conformation update (Eqs. NS17-NS24, NS40-NS46)."""
import math

import numpy as np
import pytest

from paper_2111_04577_gb300 import workloads as wl
from oracle import polymer
from oracle.params import Derived


def rand_spd_log(rng, shape, n, scale=0.5):
    A = rng.standard_normal(shape + (n, n)) * scale
    return 0.5 * (A + np.swapaxes(A, -1, -2))


@pytest.mark.parametrize("n", [2, 3])
def test_rigid_rotation_is_frame_indifferent(n):
    """For an antisymmetric grad u^T = W the decomposition of Eq. NS21 gives
    B = 0 and Omega = W (omega_ab = m_ab), so RH = W Theta - Theta W + relaxation."""
    rng = np.random.default_rng(0)
    T = rand_spd_log(rng, (5,), n)
    Wm = rng.standard_normal((5, n, n))
    Wm = Wm - np.swapaxes(Wm, -1, -2)
    lam_h = 0.7
    got = polymer.rh(T, Wm, np.zeros_like(T), lam_h)
    th, R = np.linalg.eigh(T)
    einv = R @ (np.exp(-th)[..., :, None] * np.swapaxes(R, -1, -2))
    want = Wm @ T - T @ Wm + (einv - np.eye(n)) / lam_h
    assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("n", [2, 3])
def test_coaxial_extension(n):
    """Theta and a symmetric grad u^T sharing eigenvectors: Omega = 0, B = L."""
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    th = rng.standard_normal(n)
    T = (Q * th) @ Q.T
    L = (Q * rng.standard_normal(n)) @ Q.T
    got = polymer.rh(T[None], L[None], np.zeros((1, n, n)), 2.0)[0]
    want = 2 * L + ((Q * np.exp(-th)) @ Q.T - np.eye(n)) / 2.0
    assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("n", [2, 3])
def test_zero_stress_rule_and_degenerate_limit(n):
    """Theta = 0 (tau_p = 0): Omega = 0, B = sym(grad u^T) (text after Eq. NS24);
    nearly equal eigenvalues approach the same limit continuously."""
    rng = np.random.default_rng(2)
    L = rng.standard_normal((1, n, n))
    got = polymer.rh(np.zeros((1, n, n)), L, np.zeros((1, n, n)), 1.0)
    assert np.max(np.abs(got - (L + np.swapaxes(L, -1, -2)))) < 1e-14
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    for eps in (1e-4, 1e-6):
        T = (Q * (0.3 + eps * np.arange(n))) @ Q.T
        T0 = (Q * np.full(n, 0.3)) @ Q.T
        a = polymer.rh(T[None], L, np.zeros((1, n, n)), 1.0)
        b = polymer.rh(T0[None], L, np.zeros((1, n, n)), 1.0)
        assert np.max(np.abs(a - b)) < 20 * eps


def _startup(dim, dt, t_end, gam=1.3, lam_h=0.8, alpha_g=0.0):
    n = 8
    g = wl.Grid(4, 1 if dim == 2 else 4, n, 0.5, 0.125 if dim == 2 else 0.5, 1.0, 1)
    prm = wl.params_from_groups(Wi=lam_h, beta=0.4, dt=dt)
    prm.alpha_giesekus = alpha_g
    prm.uw_bot, prm.uw_top = -gam * 0.5, gam * 0.5
    d = Derived(prm.as_dict())
    nz, ny, nx = g.coarse_shape
    z = (np.arange(nz) + 0.5) * g.dx
    u = np.broadcast_to((gam * (z - 0.5))[:, None, None], (nz, ny, nx)).copy()
    v = np.zeros_like(u)
    w = np.zeros((nz + 1, ny, nx))
    m = 2 if dim == 2 else 3
    T = np.zeros((nz, ny, nx, m, m))
    phic = np.ones((nz, ny, nx))
    steps = int(round(t_end / dt))
    for _ in range(steps):
        T, tau = polymer.polymer_step(T, u, v, w, phic, d, g)
    return tau, d


@pytest.mark.parametrize("dim", [2, 3])
def test_oldroyd_b_startup_shear(dim):
    """Uniform shear from rest: tau_xz = mu_p g (1 - e^{-t/l}),
    tau_xx = 2 mu_p l g^2 (1 - (1 + t/l) e^{-t/l}), tau_zz = 0 (Eqs. NS17-NS18
    with the relaxation sign that makes c relax to I).  RK2-TVD error O(dt^2)."""
    gam, lam_h, t = 1.3, 0.8, 1.6
    errs = []
    for dt in (0.04, 0.02, 0.01):
        tau, d = _startup(dim, dt, t, gam, lam_h)
        mp = d.mu_p1
        e = math.exp(-t / lam_h)
        xz = mp * gam * (1 - e)
        xx = 2 * mp * lam_h * gam ** 2 * (1 - (1 + t / lam_h) * e)
        iz = 1 if dim == 2 else 2
        err = max(np.max(np.abs(tau[..., 0, iz] - xz)) / xz,
                  np.max(np.abs(tau[..., 0, 0] - xx)) / xx,
                  np.max(np.abs(tau[..., iz, iz])) / xx)
        errs.append(err)
    assert errs[-1] < 2e-4
    r = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(r - 2) < 0.2), (errs, r)


def _giesekus_steady_shear(gam, lam_h, alpha_g):
    """Steady conformation of homogeneous shear u = gam z, solved as an
    algebraic system independent of the log-conformation scheme: with
    L = grad u^T = [[0, gam], [0, 0]] (x, z), the steady Eq. NS18 (relaxing
    sign) reads L c + c L^T = (1/lambda_H)[(c - I) + alpha (c - I)^2]."""
    from scipy.optimize import fsolve

    def F(x):
        cxx, cxz, czz = x
        c = np.array([[cxx, cxz], [cxz, czz]])
        L = np.array([[0.0, gam], [0.0, 0.0]])
        e = c - np.eye(2)
        r = L @ c + c @ L.T - (e + alpha_g * e @ e) / lam_h
        return [r[0, 0], r[0, 1], r[1, 1]]

    wi = gam * lam_h
    x0 = [1.0 + 2.0 * wi * wi, wi, 1.0]  # the Oldroyd-B solution
    x = fsolve(F, x0, xtol=1e-13)
    assert max(abs(r) for r in F(x)) < 1e-12  # converged to round-off
    return x


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("alpha_g", [0.2, 0.5])
def test_giesekus_shear_reaches_the_algebraic_steady_state(dim, alpha_g):
    """Giesekus mobility (Eqs. NS18, NS22): uniform shear from rest, run to
    steady state by the RK2-TVD log-conformation scheme, gives the stress of the
    steady algebraic solution; the shear-thinning (tau_xz below mu_p gam) and
    tau_zz != 0 separate it from Oldroyd-B.  A fixed point of the RK2 map is a
    zero of RH, so only the decaying transient remains."""
    gam, lam_h = 1.3, 0.8
    tau, d = _startup(dim, 0.02, 24.0, gam, lam_h, alpha_g)
    cxx, cxz, czz = _giesekus_steady_shear(gam, lam_h, alpha_g)
    mp = d.mu_p1
    iz = 1 if dim == 2 else 2
    want = {"xx": mp / lam_h * (cxx - 1), "xz": mp / lam_h * cxz, "zz": mp / lam_h * (czz - 1)}
    got = {"xx": tau[..., 0, 0], "xz": tau[..., 0, iz], "zz": tau[..., iz, iz]}
    scale = abs(want["xx"])
    for k in want:
        assert np.max(np.abs(got[k] - want[k])) < 1e-8 * scale, (k, got[k].ravel()[:2], want[k])
    assert want["xz"] < mp * gam * (1 - 1e-3)   # shear thinning
    assert abs(want["zz"]) > 1e-3 * scale       # second normal stress difference
