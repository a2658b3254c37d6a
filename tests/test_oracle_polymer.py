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


def _startup(dim, dt, t_end, gam=1.3, lam_h=0.8, alpha_g=0.0, phi=1.0, **extra):
    n = 8
    g = wl.Grid(4, 1 if dim == 2 else 4, n, 0.5, 0.125 if dim == 2 else 0.5, 1.0, 1)
    prm = wl.params_from_groups(Wi=lam_h, beta=0.4, dt=dt)
    prm.alpha_giesekus = alpha_g
    for k, val in extra.items():
        setattr(prm, k, val)
    prm.uw_bot, prm.uw_top = -gam * 0.5, gam * 0.5
    d = Derived(prm.as_dict())
    nz, ny, nx = g.coarse_shape
    z = (np.arange(nz) + 0.5) * g.dx
    u = np.broadcast_to((gam * (z - 0.5))[:, None, None], (nz, ny, nx)).copy()
    v = np.zeros_like(u)
    w = np.zeros((nz + 1, ny, nx))
    m = 2 if dim == 2 else 3
    T = np.zeros((nz, ny, nx, m, m))
    phic = np.full((nz, ny, nx), float(phi))
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


# Approach 1 of Section 2.1 (Eq. NS11): mu_p, lambda_H and alpha linear in phi,
# tau = tau_p unweighted.  Phase 2 gets its own polymer: mu_p2, wi2, alpha2.
AP1 = dict(polymer_approach=1, mu_p2=0.05, wi2=0.3)


@pytest.mark.parametrize("dim", [2, 3])
def test_approach1_startup_shear_uses_the_phase_averaged_parameters(dim):
    """Uniform shear from rest at a constant phi = 0.4: the closed-form
    Oldroyd-B start-up with lambda_H = 0.7 lambda_1 + 0.3 lambda_2 and
    mu_p = 0.7 mu_p1 + 0.3 mu_p2 (Eq. NS11), and no (1 + phi)/2 weight.
    Swapped phases (lambda_H 0.45, mu_p 0.3/0.7 mix) or the weight of Eq. NS12
    (0.7) miss it by tens of per cent."""
    gam, lam1, t, phi = 1.3, 0.8, 1.6, 0.4
    a, b = 0.5 * (1 + phi), 0.5 * (1 - phi)
    tau, d = _startup(dim, 0.005, t, gam, lam1, phi=phi, **AP1)
    lam = a * lam1 + b * AP1["wi2"]
    mp = a * d.mu_p1 + b * AP1["mu_p2"]
    e = math.exp(-t / lam)
    xz = mp * gam * (1 - e)
    xx = 2 * mp * lam * gam ** 2 * (1 - (1 + t / lam) * e)
    iz = 1 if dim == 2 else 2
    assert np.max(np.abs(tau[..., 0, iz] - xz)) < 1e-4 * xz
    assert np.max(np.abs(tau[..., 0, 0] - xx)) < 1e-4 * xx
    assert np.max(np.abs(tau[..., iz, iz])) < 1e-4 * xx


@pytest.mark.parametrize("dim", [2, 3])
def test_approach1_giesekus_steady_shear_at_intermediate_phi(dim):
    """The algebraic Giesekus steady state (independent fsolve) with the
    interpolated alpha = 0.4 alpha_1 + 0.6 alpha_2 and lambda_H at phi = -0.2."""
    gam, lam1, phi = 1.3, 0.8, -0.2
    a, b = 0.5 * (1 + phi), 0.5 * (1 - phi)
    extra = dict(AP1, alpha_giesekus2=0.1)
    tau, d = _startup(dim, 0.02, 24.0, gam, lam1, 0.5, phi=phi, **extra)
    lam = a * lam1 + b * extra["wi2"]
    ag = a * 0.5 + b * 0.1
    mp = a * d.mu_p1 + b * extra["mu_p2"]
    cxx, cxz, czz = _giesekus_steady_shear(gam, lam, ag)
    iz = 1 if dim == 2 else 2
    want = {"xx": mp / lam * (cxx - 1), "xz": mp / lam * cxz, "zz": mp / lam * (czz - 1)}
    got = {"xx": tau[..., 0, 0], "xz": tau[..., 0, iz], "zz": tau[..., iz, iz]}
    for k in want:
        assert np.max(np.abs(got[k] - want[k])) < 1e-8 * abs(want["xx"]), k


@pytest.mark.parametrize("dim", [2, 3])
def test_approach1_reduces_to_approach2_in_the_droplet_and_vanishes_in_a_newtonian_ambient(dim):
    """phi = +1: both approaches give tau_p of the droplet's constants; phi = -1
    with mu_p2 = 0: no stress at all, whatever the ambient's relaxation time."""
    t1, _ = _startup(dim, 0.02, 0.4, phi=1.0, **AP1)
    t2, _ = _startup(dim, 0.02, 0.4, phi=1.0)
    assert np.allclose(t1, t2, rtol=0, atol=1e-14 * np.max(np.abs(t2)))
    t3, _ = _startup(dim, 0.02, 0.4, phi=-1.0, **dict(AP1, mu_p2=0.0))
    assert np.max(np.abs(t3)) == 0.0


@pytest.mark.parametrize("plant", ["swap_phases", "weight"])
def test_approach1_pin_catches_planted_mistakes(monkeypatch, plant):
    """The start-up pin fails with the phases swapped in Eq. NS11, and with the
    (1 + phi)/2 weight of Eq. NS12 applied in approach 1."""
    from mutate import mutated
    from oracle.params import Derived as D
    if plant == "swap_phases":
        bad = mutated(D, "polymer_props", "a, b = 0.5 * (1.0 + phic), 0.5 * (1.0 - phic)",
                      "b, a = 0.5 * (1.0 + phic), 0.5 * (1.0 - phic)")
        monkeypatch.setattr(D, "polymer_props", bad)
    else:
        bad = mutated(polymer, "polymer_step", "if d.approach1:", "if False:")
        monkeypatch.setattr(polymer, "polymer_step", bad)
    with pytest.raises(AssertionError):
        test_approach1_startup_shear_uses_the_phase_averaged_parameters(2)
