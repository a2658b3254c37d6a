"""The hand-written GPU adjoint of the CH step (velocity fixed) against the FP64
CPU adjoint (autograd of the oracle restatement) and central finite
differences of the GPU forward (tolerance 1e-3 for finite differences)."""
import numpy as np
import pytest
import torch

from paper_2111_04577_gb300 import adjoint as padj, binding, build, workloads as wl
from oracle import ch_torch

pytestmark = pytest.mark.gpu

OBJ = {"wetted": binding.PF_OBJ_WETTED, "centroid": binding.PF_OBJ_CENTROID_Z}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def tiny():
    g = wl.Grid(8, 1, 4, 4.0, 0.5, 2.0, 1)
    prm = wl.params_from_groups(theta_deg=60.0, Pe=50.0, Cn=0.2)
    prm.theta_top_deg = 80.0
    return wl.Workload("tiny", g, prm, 1)


def solver_for(w, vel, prec=binding.PF_FP64):
    s = binding.Solver(w.grid, w.params, prec)
    s.load_state(wl.initial_phi(w), vel)
    return s


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("which", ["wetted", "centroid"])
def test_gpu_adjoint_equals_cpu_adjoint(which):
    w = tiny()
    vel = wl.random_velocity(w.grid, 3, 0.3)
    phi0 = wl.initial_phi(w)
    steps = 5
    J, ph0, th, mob, _ = ch_torch.run(w.grid, w.params.as_dict(), vel, phi0, steps, which, split_mobility=True)
    J.backward()
    s = solver_for(w, vel)
    Jg, dth, dm, dphi = s.adjoint(steps, 2, OBJ[which])
    assert rel(Jg, J.item()) < 1e-12
    # per-degree contact-angle derivative; autograd differentiated w.r.t. degrees too
    assert rel(dth, th.grad.item()) < 1e-9
    # dJ/dM is a difference of the 1/(M lambda dt) part and the S part of Eq. NS30,
    # each up to ~3e7 times larger than their sum: the tolerance scales with the parts
    parts = [m.grad.item() for m in mob]
    assert abs(dm - sum(parts)) < 1e-12 * sum(abs(v) for v in parts)
    ref = ph0.grad.numpy()
    assert np.max(np.abs(dphi - ref)) < 1e-9 * np.max(np.abs(ref))


def _J(w, vel, phi0, steps, which, theta=None, mob=None, prec=binding.PF_FP64):
    prm = wl.Params(**w.params.as_dict())
    if theta is not None:
        prm.theta_bot_deg = theta
    if mob is not None:
        prm.mobility = mob
    s = binding.Solver(w.grid, prm, prec)
    s.load_state(phi0, vel)
    s.step(steps, binding.PF_STEP_CH_ONLY)
    dg = s.diagnostics()
    s.close()
    return dg["wetted"] if which == "wetted" else dg["centroid"][2]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("which", ["wetted", "centroid"])
def test_gpu_adjoint_equals_finite_differences(dim, which):
    if dim == 2:
        g = wl.Grid(32, 1, 16, 4.0, 4.0 / 32, 2.0, 1)
    else:
        g = wl.Grid(12, 12, 6, 4.0, 4.0, 2.0, 1)
    prm = wl.params_from_groups(theta_deg=50.0, Pe=100.0, Cn=0.1)
    w = wl.Workload("fd", g, prm, 1)
    vel = wl.random_velocity(g, 7, 0.2)
    phi0 = wl.initial_phi(w)
    steps = 6
    s = solver_for(w, vel)
    _, dth, dm, dphi = s.adjoint(steps, 4, OBJ[which])
    t0, m0 = prm.theta_bot_deg, prm.mobility
    fd_t = (_J(w, vel, phi0, steps, which, theta=t0 + 1e-2) - _J(w, vel, phi0, steps, which, theta=t0 - 1e-2)) / 2e-2
    dmm = 1e-2 * m0
    fd_m = (_J(w, vel, phi0, steps, which, mob=m0 + dmm) - _J(w, vel, phi0, steps, which, mob=m0 - dmm)) / (2 * dmm)
    rng = np.random.default_rng(2)
    dirn = rng.standard_normal(phi0.shape)
    eps = 1e-5
    fd_p = (_J(w, vel, phi0 + eps * dirn, steps, which) - _J(w, vel, phi0 - eps * dirn, steps, which)) / (2 * eps)
    assert rel(dth, fd_t) < 1e-3, (dth, fd_t)
    assert rel(dm, fd_m) < 1e-3, (dm, fd_m)
    assert rel(float(np.sum(dphi * dirn)), fd_p) < 1e-3


def test_checkpoint_interval_does_not_change_gradients():
    w = tiny()
    vel = wl.random_velocity(w.grid, 3, 0.3)
    res = []
    for K in (1, 3, 10):
        s = solver_for(w, vel)
        res.append(s.adjoint(7, K, binding.PF_OBJ_WETTED))
    for r in res[1:]:
        assert abs(r[1] - res[0][1]) <= 1e-12 * abs(res[0][1])
        assert abs(r[2] - res[0][2]) <= 1e-12 * abs(res[0][2])
        assert np.max(np.abs(r[3] - res[0][3])) <= 1e-12 * np.max(np.abs(res[0][3]))


def test_mixed_adjoint_close_to_fp64():
    g = wl.Grid(32, 1, 16, 4.0, 4.0 / 32, 2.0, 1)
    prm = wl.params_from_groups(theta_deg=50.0, Pe=100.0, Cn=0.1)
    w = wl.Workload("mx", g, prm, 1)
    vel = wl.random_velocity(g, 7, 0.2)
    a = solver_for(w, vel, binding.PF_FP64).adjoint(10, 5, binding.PF_OBJ_WETTED)
    b = solver_for(w, vel, binding.PF_MIXED).adjoint(10, 5, binding.PF_OBJ_WETTED)
    assert rel(b[1], a[1]) < 1e-3 and rel(b[2], a[2]) < 1e-3


def test_autograd_function_matches_direct_adjoint():
    w = tiny()
    vel = wl.random_velocity(w.grid, 3, 0.3)
    s = solver_for(w, vel)
    phi0 = torch.tensor(wl.initial_phi(w), dtype=torch.float64, requires_grad=True)
    th = torch.tensor(w.params.theta_bot_deg, dtype=torch.float64, requires_grad=True)
    mob = torch.tensor(w.params.mobility, dtype=torch.float64, requires_grad=True)
    J = padj.CHObjective.apply(phi0, th, mob, s, w.params, 5, 2, binding.PF_OBJ_CENTROID_Z)
    gphi, gth, gm = torch.autograd.grad(J, (phi0, th, mob))
    s2 = solver_for(w, vel)
    _, dth, dm, dphi = s2.adjoint(5, 2, binding.PF_OBJ_CENTROID_Z)
    assert rel(gth.item(), dth) < 1e-12 and rel(gm.item(), dm) < 1e-12
    assert np.max(np.abs(gphi.numpy() - dphi)) <= 1e-12 * np.max(np.abs(dphi))
