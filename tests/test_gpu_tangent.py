"""Forward-mode sensitivities through the whole coupled step (pf_tangent)
against central finite differences of the FP64 oracle (tolerance
1e-3 for finite differences) and of the GPU's own FP64 path; the objective's
value against the oracle at the FP64 parity tolerance."""
import numpy as np
import pytest

from paper_2111_04577_gb300 import binding, build, workloads as wl
from oracle import step as ostep, observables as ob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def case(dim):
    """Small viscoelastic droplets with a seeded rough velocity: 20 steps of
    dt = 1e-3 keep the oracle's finite differences converged to about 1e-4."""
    if dim == 2:
        w = wl.scaled(wl.config("c2"), 16, 8)
    else:
        w = wl.scaled(wl.config("c4"), 8, 4)
    w.params.dt = 1e-3
    vel = wl.random_velocity(w.grid, 3, 0.3)
    return w, vel, 20


def oracle_J(w, vel, n, **over):
    prm = w.params.as_dict()
    prm.update(over)
    st = ostep.State(w.grid, prm, wl.initial_phi(w), vel0=vel)
    for _ in range(n):
        st.step()
    return np.array([ob.wetted(st.phi, w.grid), ob.centroid(st.phi, w.grid)[2]])


def gpu_J(w, vel, n, prec=binding.PF_FP64, **over):
    prm = wl.Params(**{**w.params.as_dict(), **over})
    s = binding.Solver(w.grid, prm, prec)
    s.load_state(wl.initial_phi(w), vel)
    s.step(n)
    d = s.diagnostics()
    return np.array([d["wetted"], d["centroid"][2]])


def tangents(w, vel, n, param, prec=binding.PF_FP64):
    s = binding.Solver(w.grid, w.params, prec)
    s.load_state(wl.initial_phi(w), vel)
    out = [s.tangent(n, param, obj) for obj in (binding.PF_OBJ_WETTED, binding.PF_OBJ_CENTROID_Z)]
    return np.array([o[0] for o in out]), np.array([o[1] for o in out])


def close(a, b, tol):
    return np.all(np.abs(a - b) <= tol * np.maximum(np.abs(b), 1e-300))


@pytest.mark.parametrize("dim", [2, 3])
def test_wi_sensitivity_equals_oracle_central_difference(dim):
    w, vel, n = case(dim)
    J, dJ = tangents(w, vel, n, binding.PF_PARAM_WI)
    wi = w.params.wi
    h = 1e-3 * wi
    fd = (oracle_J(w, vel, n, wi=wi + h) - oracle_J(w, vel, n, wi=wi - h)) / (2 * h)
    assert close(J, oracle_J(w, vel, n), 1e-10), (J, oracle_J(w, vel, n))
    assert np.all(np.abs(dJ) > 0)
    assert close(dJ, fd, 1e-3), (dJ, fd)


@pytest.mark.parametrize("dim", [2, 3])
def test_theta_sensitivity_equals_oracle_central_difference(dim):
    w, vel, n = case(dim)
    J, dJ = tangents(w, vel, n, binding.PF_PARAM_THETA_BOT)
    th = w.params.theta_bot_deg
    hd = 1e-2  # degrees
    fd = (oracle_J(w, vel, n, theta_bot_deg=th + hd) - oracle_J(w, vel, n, theta_bot_deg=th - hd)) / (2 * hd)
    assert close(dJ, fd, 1e-3), (dJ, fd)


def test_wi_sensitivity_equals_gpu_fp64_central_difference():
    """The same derivative by differencing the GPU's own FP64 step (its
    kernels, not the derivative-carrying ones)."""
    w, vel, n = case(3)
    _, dJ = tangents(w, vel, n, binding.PF_PARAM_WI)
    wi = w.params.wi
    h = 1e-3 * wi
    fd = (gpu_J(w, vel, n, wi=wi + h) - gpu_J(w, vel, n, wi=wi - h)) / (2 * h)
    assert close(dJ, fd, 1e-3), (dJ, fd)


def test_tangent_from_a_mixed_context_and_context_untouched():
    """A PF_MIXED context gives its (rounded) state to the FP64 copy; the
    context itself is not advanced."""
    w, vel, n = case(2)
    s = binding.Solver(w.grid, w.params, binding.PF_MIXED)
    s.load_state(wl.initial_phi(w), vel)
    phi_before = s.fine("phi").copy()
    J, dJ = s.tangent(n, binding.PF_PARAM_WI, binding.PF_OBJ_WETTED)
    assert np.array_equal(s.fine("phi"), phi_before)
    J64, dJ64 = tangents(w, vel, n, binding.PF_PARAM_WI)
    assert abs(J - J64[0]) < 1e-5 * abs(J64[0])
    assert abs(dJ - dJ64[0]) < 1e-2 * abs(dJ64[0])


def test_tangent_errors():
    w, vel, n = case(2)
    s = binding.Solver(w.grid, w.params, binding.PF_FP64)
    s.load_state(wl.initial_phi(w), vel)
    for bad in [(0, binding.PF_PARAM_WI, binding.PF_OBJ_WETTED), (n, 7, binding.PF_OBJ_WETTED),
                (n, binding.PF_PARAM_WI, 5)]:
        with pytest.raises(binding.PFError) as e:
            s.tangent(*bad)
        assert e.value.code == -1
    newt = wl.scaled(wl.config("c1"), 16, 8)
    s2 = binding.Solver(newt.grid, newt.params, binding.PF_FP64)
    s2.load_state(wl.initial_phi(newt))
    with pytest.raises(binding.PFError):
        s2.tangent(2, binding.PF_PARAM_WI, binding.PF_OBJ_WETTED)


def test_coupled_objective_autograd():
    """torch.autograd through the coupled step: the gradients pf_tangent gives."""
    import torch
    from paper_2111_04577_gb300 import adjoint as padj
    w, vel, n = case(2)
    s = binding.Solver(w.grid, w.params, binding.PF_FP64)
    s.load_state(wl.initial_phi(w), vel)
    wi = torch.tensor(w.params.wi, dtype=torch.float64, requires_grad=True)
    th = torch.tensor(w.params.theta_bot_deg, dtype=torch.float64, requires_grad=True)
    J = padj.CoupledObjective.apply(wi, th, s, w.params, n, binding.PF_OBJ_WETTED)
    (2.0 * J).backward()
    Jt, dwi = s.tangent(n, binding.PF_PARAM_WI, binding.PF_OBJ_WETTED)
    _, dth = s.tangent(n, binding.PF_PARAM_THETA_BOT, binding.PF_OBJ_WETTED)
    assert float(J.detach()) == Jt
    assert float(wi.grad) == 2.0 * dwi and float(th.grad) == 2.0 * dth


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_dot_product_with_tangent(dim):
    """The classical adjoint check, between two independent codes: the
    hand-written reverse sweep of the CH step (velocity fixed) and forward-mode
    derivatives of the forward kernels.  <dJ/dphi^0, v> and dJ/dtheta agree to
    FP64 rounding (tolerance 1e-10 for adjoint against adjoint)."""
    w, vel, _ = case(dim)
    n = 8
    rng = np.random.default_rng(5)
    for obj in (binding.PF_OBJ_WETTED, binding.PF_OBJ_CENTROID_Z):
        s = binding.Solver(w.grid, w.params, binding.PF_FP64)
        s.load_state(wl.initial_phi(w), vel)
        v = rng.standard_normal(w.grid.fine_shape)
        J_t, dv = s.tangent(n, binding.PF_PARAM_PHI0, obj, binding.PF_STEP_CH_ONLY, v)
        _, dth_t = s.tangent(n, binding.PF_PARAM_THETA_BOT, obj, binding.PF_STEP_CH_ONLY)
        J_a, dth_a, _, dphi = s.adjoint(n, 3, obj)
        assert abs(J_t - J_a) <= 1e-12 * abs(J_a)
        dot = float(np.sum(dphi.astype(np.float64) * v))
        assert abs(dv - dot) <= 1e-10 * max(abs(dot), 1e-300), (dv, dot)
        assert abs(dth_t - dth_a) <= 1e-10 * abs(dth_a), (dth_t, dth_a)


@pytest.mark.parametrize("dim", [2, 3])
def test_mobility_sensitivity_equals_oracle_central_difference(dim):
    """dJ/dM through the whole coupled step: M enters the CH right side, both
    shifts of the paired solve (through S, which follows M at the Eq. NS30
    bound) and the flux J of the momentum equation."""
    w, vel, n = case(dim)
    J, dJ = tangents(w, vel, n, binding.PF_PARAM_MOBILITY)
    M = w.params.mobility
    h = 1e-3 * M
    fd = (oracle_J(w, vel, n, mobility=M + h) - oracle_J(w, vel, n, mobility=M - h)) / (2 * h)
    assert close(dJ, fd, 1e-3), (dJ, fd)


def test_mobility_tangent_equals_adjoint_velocity_fixed():
    """With the velocity fixed, dJ/dM by forward mode equals the reverse
    sweep's.  dJ/dM is a difference of parts ~1e7 times larger than itself
    (the 1/(M lambda dt) term against the S(M) term), so FP64 rounding of
    either code leaves ~1e-9 relative: the bound is 1e-6."""
    w, vel, _ = case(3)
    n = 6
    for obj in (binding.PF_OBJ_WETTED, binding.PF_OBJ_CENTROID_Z):
        s = binding.Solver(w.grid, w.params, binding.PF_FP64)
        s.load_state(wl.initial_phi(w), vel)
        _, dm_t = s.tangent(n, binding.PF_PARAM_MOBILITY, obj, binding.PF_STEP_CH_ONLY)
        _, _, dm_a, _ = s.adjoint(n, 2, obj, want_phi=False)
        assert abs(dm_t - dm_a) <= 1e-6 * abs(dm_a), (dm_t, dm_a)


def test_wi_sensitivity_in_polymer_approach1():
    """Eq. NS11 (approach 1): d/dWi moves the droplet's relaxation time, which
    the polymer update mixes with phase 2's at every centre; against central
    differences of the oracle."""
    w, vel, n = case(2)
    w.params.polymer_approach = 1
    w.params.mu_p2 = 0.02
    w.params.wi2 = 0.4
    J, dJ = tangents(w, vel, n, binding.PF_PARAM_WI)
    wi = w.params.wi
    h = 1e-3 * wi
    fd = (oracle_J(w, vel, n, wi=wi + h) - oracle_J(w, vel, n, wi=wi - h)) / (2 * h)
    assert close(J, oracle_J(w, vel, n), 1e-10)
    assert close(dJ, fd, 1e-3), (dJ, fd)


def test_theta_sensitivity_with_weno5z_advection():
    """Forward mode through the WENO5-Z fluxes (phi and Theta): dJ/dtheta_s
    against central differences of the oracle with the same scheme."""
    w, vel, n = case(2)
    w.params.advection = 1
    J, dJ = tangents(w, vel, n, binding.PF_PARAM_THETA_BOT)
    th = w.params.theta_bot_deg
    hd = 1e-2
    fd = (oracle_J(w, vel, n, theta_bot_deg=th + hd) - oracle_J(w, vel, n, theta_bot_deg=th - hd)) / (2 * hd)
    assert close(J, oracle_J(w, vel, n), 1e-10)
    assert close(dJ, fd, 1e-3), (dJ, fd)
