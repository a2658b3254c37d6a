"""Pins of the differentiable CH restatement (the FP64 CPU adjoint reference).

Its forward must equal the oracle's CH step, and its autograd gradients must
equal central finite differences of the oracle itself, for the wetted length
and the z-centroid, with respect to the bottom contact angle, the mobility and
phi0 (a seeded direction)."""
import numpy as np
import pytest
import torch

from paper_2111_04577_gb300 import workloads as wl
from oracle import ch_torch, step as ostep, observables as ob


def tiny():
    g = wl.Grid(8, 1, 4, 4.0, 0.5, 2.0, 1)
    prm = wl.params_from_groups(theta_deg=60.0, Pe=50.0, Cn=0.2)
    prm.theta_top_deg = 80.0
    w = wl.Workload("tiny", g, prm, 1)
    return w


def oracle_J(w, vel, phi0, steps, which, theta=None, mob=None):
    prm = w.params.as_dict()
    if theta is not None:
        prm["theta_bot_deg"] = theta
    if mob is not None:
        prm["mobility"] = mob
    st = ostep.State(w.grid, prm, phi0, vel0=vel)
    for _ in range(steps):
        st.step(with_ns=False)
    if which == "wetted":
        return ob.wetted(st.phi, w.grid)
    return ob.centroid(st.phi, w.grid)[2]


def test_forward_equals_oracle():
    w = tiny()
    vel = wl.random_velocity(w.grid, 3, 0.3)
    phi0 = wl.initial_phi(w)
    J, *_rest, pn = ch_torch.run(w.grid, w.params.as_dict(), vel, phi0, 4, "wetted")
    st = ostep.State(w.grid, w.params.as_dict(), phi0, vel0=vel)
    for _ in range(4):
        st.step(with_ns=False)
    assert np.max(np.abs(pn.detach().numpy() - st.phi)) < 1e-12
    assert abs(J.item() - ob.wetted(st.phi, w.grid)) < 1e-12


@pytest.mark.parametrize("which", ["wetted", "centroid"])
def test_gradients_equal_finite_differences(which):
    w = tiny()
    vel = wl.random_velocity(w.grid, 3, 0.3)
    phi0 = wl.initial_phi(w)
    steps = 4
    J, ph0, th, mob, _ = ch_torch.run(w.grid, w.params.as_dict(), vel, phi0, steps, which)
    J.backward()
    t0, m0 = w.params.theta_bot_deg, w.params.mobility
    dt_ = 1e-3
    fd_t = (oracle_J(w, vel, phi0, steps, which, theta=t0 + dt_) - oracle_J(w, vel, phi0, steps, which, theta=t0 - dt_)) / (2 * dt_)
    dm = 1e-2 * m0  # the FD rounding error dominates below ~1e-3
    fd_m = (oracle_J(w, vel, phi0, steps, which, mob=m0 + dm) - oracle_J(w, vel, phi0, steps, which, mob=m0 - dm)) / (2 * dm)
    rng = np.random.default_rng(5)
    dirn = rng.standard_normal(phi0.shape)
    eps = 1e-5
    fd_p = (oracle_J(w, vel, phi0 + eps * dirn, steps, which) - oracle_J(w, vel, phi0 - eps * dirn, steps, which)) / (2 * eps)
    ad_p = float(np.sum(ph0.grad.numpy() * dirn))
    assert abs(th.grad.item() - fd_t) <= 1e-6 * max(1e-8, abs(fd_t)) + 1e-10
    assert abs(mob.grad.item() - fd_m) <= 1e-5 * max(1e-8, abs(fd_m)) + 1e-10
    assert abs(ad_p - fd_p) <= 1e-6 * max(1e-8, abs(fd_p)) + 1e-10


def test_split_mobility_parts_add_up():
    """The three copies of M in the split form carry gradients that add up to dJ/dM."""
    w = tiny()
    vel = wl.random_velocity(w.grid, 3, 0.3)
    phi0 = wl.initial_phi(w)
    prm = w.params.as_dict()
    J, _, _, mob, _ = ch_torch.run(w.grid, prm, vel, phi0, 4, "centroid")
    J.backward()
    J2, _, _, parts, _ = ch_torch.run(w.grid, prm, vel, phi0, 4, "centroid", split_mobility=True)
    J2.backward()
    assert abs(J2.item() - J.item()) < 1e-15
    total = sum(p.grad.item() for p in parts)
    assert abs(total - mob.grad.item()) < 1e-12 * sum(abs(p.grad.item()) for p in parts)


# ---------------------------------------------------------------------------
# the coupled 2D step (CH, restriction, NS, polymer) in torch: oracle.step_torch
# ---------------------------------------------------------------------------
def _coupled_case():
    from paper_2111_04577_gb300 import workloads as wl
    w = wl.scaled(wl.config("c2"), 8, 4)
    w.params.dt = 1e-3
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 3, 0.2)
    nz, ny, nx = g.coarse_shape
    rng = np.random.default_rng(5)
    a = 0.3 * rng.standard_normal((nz, ny, nx, 2, 2))
    th0 = a + np.swapaxes(a, -1, -2)  # distinct eigenvalues (torch.linalg.eigh's derivative)
    return g, w.params.as_dict(), phi0, vel, th0


def test_coupled_torch_forward_equals_oracle():
    from oracle import step as ostep, step_torch as stt
    g, prm, phi0, vel, th0 = _coupled_case()
    _, _, s = stt.run(g, prm, phi0, 5, "wetted", vel0=vel, theta0=th0)
    ref = ostep.State(g, prm, phi0, vel0=vel, theta0=th0)
    for _ in range(5):
        ref.step()
    rel = lambda a, b: np.max(np.abs(a.detach().numpy() - b)) / np.max(np.abs(b))
    assert rel(s["phi"], ref.phi) < 1e-12
    assert rel(s["u"], ref.vel[0]) < 1e-11 and rel(s["w"], ref.vel[2]) < 1e-11
    assert rel(s["p"], ref.p) < 1e-11
    assert rel(s["theta"], ref.theta) < 1e-12 and rel(s["tau"], ref.tau) < 1e-12


@pytest.mark.parametrize("which", ["wetted", "centroid"])
def test_coupled_torch_gradients_equal_oracle_central_differences(which):
    """dJ/dtheta_s, dJ/dM, dJ/dWi and <dJ/dphi0, v> of the coupled step's
    autograd adjoint against central differences of the FP64 oracle."""
    from oracle import step as ostep, step_torch as stt
    g, prm, phi0, vel, th0 = _coupled_case()
    J, leaves, _ = stt.run(g, prm, phi0, 5, which, vel0=vel, theta0=th0)
    J.backward()

    def Jor(p0=phi0, **kw):
        p2 = dict(prm)
        p2.update(kw)
        r = ostep.State(g, p2, p0, vel0=vel, theta0=th0)
        for _ in range(5):
            r.step()
        return ob.wetted(r.phi, g) if which == "wetted" else ob.centroid(r.phi, g)[2]

    assert abs(J.item() - Jor()) < 1e-12 * abs(J.item())
    # dJ/dM is a small difference of large parts (the 1/(M lambda dt) term against
    # S(M)): its differences take a wider step (truncation O(h^2)) and 1e-3
    for key, h, ad, tol in (("theta_bot_deg", 0.1, leaves["theta"].grad.item(), 1e-4),
                            ("wi", 1e-4, leaves["wi"].grad.item(), 1e-4),
                            ("mobility", prm["mobility"] * 1e-2, leaves["mobility"].grad.item(), 1e-3)):
        fd = (Jor(**{key: prm[key] + h}) - Jor(**{key: prm[key] - h})) / (2 * h)
        assert abs(fd - ad) <= tol * abs(fd), (key, fd, ad)
    v = np.random.default_rng(8).uniform(-1, 1, phi0.shape)
    eps = 1e-6
    fd = (Jor(phi0 + eps * v) - Jor(phi0 - eps * v)) / (2 * eps)
    ad = float(np.sum(leaves["phi0"].grad.numpy() * v))
    assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)
