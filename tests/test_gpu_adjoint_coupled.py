"""The reverse sweep through the whole coupled 2D step (pf_adjoint_ex with
PF_ADJ_COUPLED: CH, restriction, NS projection, log-conformation update).

Checked against:
 - the FP64 CPU adjoint of the same discrete step (oracle.step_torch: torch
   autograd through a restatement of the oracle, itself pinned to the oracle's
   forward and to its central differences) on a tiny grid: J, dJ/dtheta_s,
   dJ/dM, dJ/dWi and dJ/dphi0;
 - forward-mode derivatives of the GPU step (pf_tangent_ex, dual numbers
   through the forward kernels), an independent code: the dot-product test
   <dJ/dphi0, v> and each parameter's derivative, at 1e-10;
 - itself across checkpoint intervals, and the mixed-precision sweep against
   the FP64 one.
"""
import numpy as np
import pytest

from paper_2111_04577_gb300 import adjoint as padj, binding, build, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def case(nx=8, nz=4, dt=1e-3, seed=5):
    w = wl.scaled(wl.config("c2"), nx, nz)
    w.params.dt = dt
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 3, 0.2)
    nzc, ny, nxc = g.coarse_shape
    rng = np.random.default_rng(seed)
    a = 0.3 * rng.standard_normal((nzc, ny, nxc, 2, 2))
    th0 = a + np.swapaxes(a, -1, -2)  # distinct eigenvalues
    return w, g, phi0, vel, th0


def solver(w, g, phi0, vel, th0, prec=binding.PF_FP64):
    s = binding.Solver(g, w.params, prec)
    s.load_state(phi0, vel)
    s.set("theta", np.stack([th0[..., 0, 0], th0[..., 0, 1], th0[..., 1, 1]]))
    return s


def relerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(np.asarray(b))), 1e-300))


@pytest.mark.parametrize("which", [binding.PF_OBJ_WETTED, binding.PF_OBJ_CENTROID_Z])
def test_coupled_adjoint_equals_the_cpu_adjoint(which):
    from oracle import step_torch as stt
    w, g, phi0, vel, th0 = case()
    n = 5
    J_t, leaves, _ = stt.run(g, w.params.as_dict(), phi0, n, "wetted" if which == 0 else "centroid", vel0=vel,
                             theta0=th0, split_mobility=True)
    J_t.backward()
    parts = [m.grad.item() for m in leaves["mobility"]]
    dm_ref, dm_scale = sum(parts), sum(abs(x) for x in parts)
    s = solver(w, g, phi0, vel, th0)
    J, dth, dm, dwi, dphi = s.adjoint_coupled(n, 2, which)
    s.close()
    assert abs(J - J_t.item()) <= 1e-12 * abs(J_t.item())
    assert abs(dth - leaves["theta"].grad.item()) <= 1e-9 * abs(leaves["theta"].grad.item()), (dth,)
    assert abs(dwi - leaves["wi"].grad.item()) <= 1e-9 * abs(leaves["wi"].grad.item()), (dwi,)
    # dJ/dM is a difference of parts up to ~1e7 times larger than itself (the
    # 1/(M lambda dt) term against S(M)): bounded against the size of the parts
    assert abs(dm - dm_ref) <= 1e-12 * dm_scale, (dm, dm_ref, dm_scale)
    assert relerr(dphi, leaves["phi0"].grad.numpy()) < 1e-9


def test_coupled_adjoint_dot_product_with_forward_mode():
    """<dJ/dphi0, v> and dJ/dtheta, dJ/dWi, dJ/dM of one reverse sweep against
    forward-mode derivatives through the coupled GPU step (one run each)."""
    w, g, phi0, vel, th0 = case(16, 8)
    n = 8
    s = solver(w, g, phi0, vel, th0)
    J, dth, dm, dwi, dphi = s.adjoint_coupled(n, 3, binding.PF_OBJ_WETTED)
    v = np.random.default_rng(2).uniform(-1, 1, phi0.shape)
    res = {}
    for name, param, direction in (("phi0", binding.PF_PARAM_PHI0, v), ("theta", binding.PF_PARAM_THETA_BOT, None),
                                   ("wi", binding.PF_PARAM_WI, None), ("mob", binding.PF_PARAM_MOBILITY, None)):
        t = solver(w, g, phi0, vel, th0)
        Jt, dJ = t.tangent(n, param, binding.PF_OBJ_WETTED, 0, direction)
        t.close()
        res[name] = (Jt, dJ)
    s.close()
    assert abs(res["theta"][0] - J) <= 1e-12 * abs(J)
    dot = float(np.sum(dphi * v))
    assert abs(dot - res["phi0"][1]) <= 1e-10 * abs(res["phi0"][1]), (dot, res["phi0"][1])
    assert abs(dth - res["theta"][1]) <= 1e-10 * abs(res["theta"][1]), (dth, res["theta"][1])
    assert abs(dwi - res["wi"][1]) <= 1e-10 * abs(res["wi"][1]), (dwi, res["wi"][1])
    assert abs(dm - res["mob"][1]) <= 1e-7 * abs(res["mob"][1]), (dm, res["mob"][1])


def test_coupled_adjoint_does_not_depend_on_the_checkpoint_interval():
    w, g, phi0, vel, th0 = case(16, 8)
    out = []
    for K in (1, 4, 10):
        s = solver(w, g, phi0, vel, th0)
        out.append(s.adjoint_coupled(10, K, binding.PF_OBJ_CENTROID_Z))
        s.close()
    for o in out[1:]:
        for a, b in zip(o[:4], out[0][:4]):
            assert abs(a - b) <= 1e-12 * abs(b) + 1e-300
        assert relerr(o[4], out[0][4]) < 1e-12


def test_coupled_adjoint_leaves_the_context_at_step_n():
    w, g, phi0, vel, th0 = case(16, 8)
    a = solver(w, g, phi0, vel, th0)
    b = solver(w, g, phi0, vel, th0)
    a.adjoint_coupled(6, 4, binding.PF_OBJ_WETTED, want_phi=False)
    b.step(6)
    for name in ("phi", "u", "w", "p", "theta", "tau"):
        assert np.array_equal(a.get(name), b.get(name)), name
    a.close()
    b.close()


def test_mixed_coupled_adjoint_against_fp64():
    """The same sweep in PF_MIXED (FP32 fields, dual-number Jacobians in FP64,
    FP64 reductions) against PF_FP64 on the 64 x 32 2D droplet."""
    w, g, phi0, vel, th0 = case(64, 32, dt=1e-4)
    res = {}
    for prec in (binding.PF_FP64, binding.PF_MIXED):
        s = solver(w, g, phi0, vel, th0, prec)
        res[prec] = s.adjoint_coupled(20, 5, binding.PF_OBJ_WETTED)
        s.close()
    d, m = res[binding.PF_FP64], res[binding.PF_MIXED]
    assert abs(m[0] - d[0]) <= 1e-6 * abs(d[0])
    for q in (1, 3):
        assert abs(m[q] - d[q]) <= 1e-3 * abs(d[q]), (q, m[q], d[q])
    assert relerr(m[4], d[4]) < 1e-3


def test_coupled_autograd_function():
    import torch
    w, g, phi0, vel, th0 = case(16, 8)
    s = solver(w, g, phi0, vel, th0)
    ph = torch.tensor(phi0, requires_grad=True)
    th = torch.tensor(w.params.theta_bot_deg, dtype=torch.float64, requires_grad=True)
    mob = torch.tensor(w.params.mobility, dtype=torch.float64, requires_grad=True)
    wi = torch.tensor(w.params.wi, dtype=torch.float64, requires_grad=True)
    J = padj.CoupledAdjointObjective.apply(ph, th, mob, wi, s, w.params, 6, 3, binding.PF_OBJ_WETTED)
    J.backward()
    s.close()
    r = solver(w, g, phi0, vel, th0)
    J2, dth, dm, dwi, dphi = r.adjoint_coupled(6, 3, binding.PF_OBJ_WETTED)
    r.close()
    assert abs(J.item() - J2) <= 1e-13 * abs(J2)
    assert abs(th.grad.item() - dth) <= 1e-13 * abs(dth)
    assert abs(wi.grad.item() - dwi) <= 1e-13 * abs(dwi)
    assert np.allclose(ph.grad.numpy(), dphi, rtol=0, atol=1e-13 * np.max(np.abs(dphi)))


def test_coupled_adjoint_equals_oracle_central_differences():
    """dJ/dtheta_s, dJ/dWi and <dJ/dphi0, v> of the GPU sweep against central
    differences of the FP64 oracle (1e-3, the gradients' stated tolerance)."""
    from oracle import step as ostep, observables as ob
    w, g, phi0, vel, th0 = case(16, 8)
    n = 6
    prm = w.params.as_dict()
    s = solver(w, g, phi0, vel, th0)
    J, dth, dm, dwi, dphi = s.adjoint_coupled(n, 3, binding.PF_OBJ_CENTROID_Z)
    s.close()

    def Jor(p0=phi0, **kw):
        p2 = dict(prm)
        p2.update(kw)
        r = ostep.State(g, p2, p0, vel0=vel, theta0=th0)
        for _ in range(n):
            r.step()
        return ob.centroid(r.phi, g)[2]

    assert abs(J - Jor()) <= 1e-10 * abs(J)
    for key, h, ad in (("theta_bot_deg", 0.1, dth), ("wi", 1e-4, dwi)):
        fd = (Jor(**{key: prm[key] + h}) - Jor(**{key: prm[key] - h})) / (2 * h)
        assert abs(fd - ad) <= 1e-3 * abs(fd), (key, fd, ad)
    v = np.random.default_rng(4).uniform(-1, 1, phi0.shape)
    eps = 1e-6
    fd = (Jor(phi0 + eps * v) - Jor(phi0 - eps * v)) / (2 * eps)
    assert abs(fd - float(np.sum(dphi * v))) <= 1e-3 * abs(fd)


def test_batch_coupled_adjoint_equals_a_standalone_context():
    ws = []
    for b, (nx, th) in enumerate(((16, 60.0), (24, 120.0))):
        w = wl.scaled(wl.config("c2"), nx, nx // 2)
        w.params.dt = 1e-3
        w.params.theta_bot_deg = th
        ws.append(w)
    bt = binding.Batch([w.grid for w in ws], [w.params for w in ws], binding.PF_FP64)
    for b, w in enumerate(ws):
        bt.set(b, "phi", wl.initial_phi(w))
    got = bt.adjoint_coupled(1, 5, 2, binding.PF_OBJ_WETTED)
    bt.close()
    s = binding.Solver(ws[1].grid, ws[1].params, binding.PF_FP64)
    s.load_state(wl.initial_phi(ws[1]))
    ref = s.adjoint_coupled(5, 2, binding.PF_OBJ_WETTED)
    s.close()
    for a, b in zip(got[:4], ref[:4]):
        assert a == b
    assert np.array_equal(got[4], ref[4])
