"""The batched persistent sweep against the single-problem GPU path and the oracle.

Uneven 2D problems (radix-2, 3, 5 and 7 sizes, different contact angles and
Weissenberg numbers, Newtonian, Oldroyd-B and one problem in polymer
approach 1 with a Giesekus ambient) advanced together by one
persistent launch per step must reproduce, problem by problem, the fields of
the single-problem path (same device code: agreement to round-off) and the
FP64 oracle (1e-10 relative).
"""
import numpy as np
import pytest

from paper_2111_04577_gb300 import binding, build, workloads as wl
from oracle import step as ostep

pytestmark = pytest.mark.gpu


def problems():
    sizes = [(32, 16), (48, 24), (40, 20), (56, 28), (64, 32)]
    thetas = [45.0, 120.0, 60.0, 150.0, 90.0]
    wis = [0.0, 1.0, 0.5, 2.0, 0.3]
    out = []
    for b, ((nx, nz), th, wi) in enumerate(zip(sizes, thetas, wis)):
        g = wl.Grid(nx, 1, nz, 4.0, 4.0 / nx, 2.0, 1)
        prm = wl.params_from_groups(theta_deg=th, Wi=wi, beta=0.5 if wi > 0 else 1.0, ratio_rho=10.0, ratio_mu=5.0)
        if b == 3:  # polymer approach 1 (Eq. NS11): both phases viscoelastic, parameters linear in phi
            prm.polymer_approach, prm.mu_p2, prm.wi2, prm.alpha_giesekus2 = 1, 0.01, 0.7, 0.2
        out.append(wl.Workload(f"b{b}", g, prm, 3, seed=b))
    return out


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


@pytest.mark.parametrize("prec", [binding.PF_FP64, binding.PF_MIXED])
def test_batch_matches_single_problem_path(prec):
    ws = problems()
    bt = binding.Batch([w.grid for w in ws], [w.params for w in ws], prec)
    singles = []
    for b, w in enumerate(ws):
        phi0 = wl.initial_phi(w)
        vel = wl.random_velocity(w.grid, 10 + b, 0.05)
        bt.set(b, "phi", phi0)
        bt.set(b, "u", vel[0])
        bt.set(b, "w", vel[2])
        s = binding.Solver(w.grid, w.params, prec)
        s.load_state(phi0, vel)
        singles.append(s)
    nsteps = 4
    bt.step(nsteps)
    for s in singles:
        s.step(nsteps)
    tol = 1e-12 if prec == binding.PF_FP64 else 1e-5
    for b, (w, s) in enumerate(zip(ws, singles)):
        for name in ("phi", "u", "w", "p"):
            a = bt.get(b, name).astype(np.float64)
            ref = s.get(name).astype(np.float64)
            assert rel(a, ref) < tol, (b, name, rel(a, ref))
        if w.params.wi > 0:
            assert rel(bt.get(b, "theta").astype(np.float64), s.get("theta").astype(np.float64)) < tol * 10
    bt.close()


def test_batch_fp64_matches_oracle():
    ws = problems()
    bt = binding.Batch([w.grid for w in ws], [w.params for w in ws], binding.PF_FP64)
    refs = []
    for b, w in enumerate(ws):
        phi0 = wl.initial_phi(w)
        bt.set(b, "phi", phi0)
        refs.append(ostep.State(w.grid, w.params.as_dict(), phi0))
    for _ in range(3):
        bt.step(1)
        for r in refs:
            r.step()
    for b, (w, r) in enumerate(zip(ws, refs)):
        g = w.grid
        nz, ny, nx = g.coarse_shape
        assert rel(bt.get(b, "phi").reshape(g.fine_shape), r.phi) < 1e-10, b
        assert rel(bt.get(b, "u").reshape(nz, ny, nx), r.vel[0]) < 1e-10, b
        assert rel(bt.get(b, "w").reshape(nz + 1, ny, nx), r.vel[2]) < 1e-10, b
    bt.close()


def test_batch_adjoint_matches_single_problem_adjoint():
    """pf_batch_adjoint on each problem equals pf_adjoint on a standalone
    context holding the same state (the same kernels: bitwise in FP64)."""
    ws = problems()[:3]
    bt = binding.Batch([w.grid for w in ws], [w.params for w in ws], binding.PF_FP64)
    for b, w in enumerate(ws):
        vel = wl.random_velocity(w.grid, 20 + b, 0.2)
        phi0 = wl.initial_phi(w)
        bt.set(b, "phi", phi0)
        bt.set(b, "phi_old", phi0)
        for name, a in zip(("u", "w"), (vel[0], vel[2])):
            bt.set(b, name, a)
            bt.set(b, name + "_old", a)
        s = binding.Solver(w.grid, w.params, binding.PF_FP64)
        s.load_state(phi0, vel)
        ref = s.adjoint(6, 2, binding.PF_OBJ_WETTED)
        got = bt.adjoint(b, 6, 2, binding.PF_OBJ_WETTED)
        assert got[0] == ref[0] and got[1] == ref[1] and got[2] == ref[2]
        assert np.array_equal(got[3], ref[3])
        s.close()
    bt.close()


def test_batch_tangent_matches_single_problem_tangent():
    """pf_batch_tangent on a problem of the batch equals pf_tangent_ex on a
    standalone context holding the same state, for each parameter: the
    derivative-carrying copy is built from the same fields and parameters."""
    ws = problems()[:2]
    bt = binding.Batch([w.grid for w in ws], [w.params for w in ws], binding.PF_FP64)
    for b, w in enumerate(ws):
        vel = wl.random_velocity(w.grid, 30 + b, 0.2)
        phi0 = wl.initial_phi(w)
        bt.set(b, "phi", phi0)
        bt.set(b, "phi_old", phi0)
        for name, a in zip(("u", "w"), (vel[0], vel[2])):
            bt.set(b, name, a)
            bt.set(b, name + "_old", a)
        s = binding.Solver(w.grid, w.params, binding.PF_FP64)
        s.load_state(phi0, vel)
        params = [binding.PF_PARAM_THETA_BOT, binding.PF_PARAM_MOBILITY]
        if w.params.wi > 0 and w.params.beta < 1:
            params.append(binding.PF_PARAM_WI)
        for prm in params:
            assert bt.tangent(b, 4, prm) == s.tangent(4, prm), prm
        s.close()
    bt.close()
