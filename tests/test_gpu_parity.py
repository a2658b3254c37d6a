"""GPU path vs the CPU oracle, element by element, through the C ABI.

Tolerances (stated for the FP64 GPU path): 1e-10 relative per field (max
|gpu - oracle| / max |oracle|).  Mixed path: 2e-4 max-abs on phi and 1e-3
relative on velocity and stress after the stated number of steps.
Sizes span several FFT/solve tiles, odd radices (3, 5, 7) and ragged tails.
"""
import numpy as np
import pytest

from paper_2111_04577_gb300 import binding, build, workloads as wl
from oracle import step as ostep, observables as ob

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def grid(dim, nx, nz, dual=1, lx=4.0):
    dx = lx / nx
    if dim == 2:
        return wl.Grid(nx, 1, nz, lx, dx, nz * dx, dual)
    return wl.Grid(nx, nx, nz, lx, lx, nz * dx, dual)


def workload(g, **kw):
    prm = wl.params_from_groups(**kw)
    prm.theta_top_deg = 75.0
    return wl.Workload("t", g, prm, 1)


CH_CASES = [
    (2, 16, 8, 1), (2, 24, 12, 1), (2, 20, 10, 0), (2, 28, 6, 1),
    (3, 16, 8, 1), (3, 12, 6, 1), (3, 10, 4, 0),
    # deep z: several 32-row solve segments with a ragged last one
    (2, 12, 40, 1), (2, 16, 48, 0), (3, 8, 20, 1),
    # power-of-two lines >= 64: the register-resident transforms
    (3, 32, 8, 1), (2, 64, 8, 1),
]


@pytest.mark.parametrize("dim,nx,nz,dual", CH_CASES)
def test_ch_step_fp64(dim, nx, nz, dual):
    g = grid(dim, nx, nz, dual)
    w = workload(g, theta_deg=60.0)
    phi0 = wl.initial_phi(w)
    rng = np.random.default_rng(7)
    phim = phi0 + 1e-2 * rng.uniform(-1, 1, phi0.shape)
    vel = wl.random_velocity(g, 3, 0.2)
    s = binding.Solver(g, w.params, binding.PF_FP64)
    s.load_state(phi0, vel, phi_old=phim)
    ref = ostep.State(g, w.params.as_dict(), phi0, vel0=vel)
    ref.phi_old = phim.copy()
    for n in range(4):
        s.step(1, binding.PF_STEP_CH_ONLY)
        ref.step(with_ns=False)
        assert rel(s.fine("phi"), ref.phi) < FP64_TOL, n
    assert rel(s.fine("G"), ref.G) < FP64_TOL


@pytest.mark.parametrize("dim,nx,nz,dual", [(2, 16, 8, 1), (3, 12, 6, 1)])
def test_ch_step_without_graph_matches_graph(dim, nx, nz, dual):
    g = grid(dim, nx, nz, dual)
    w = workload(g, theta_deg=45.0)
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 3, 0.2)
    a = binding.Solver(g, w.params, binding.PF_FP64)
    b = binding.Solver(g, w.params, binding.PF_FP64)
    for s in (a, b):
        s.load_state(phi0, vel)
    a.step(3, binding.PF_STEP_CH_ONLY)
    b.step(3, binding.PF_STEP_CH_ONLY | binding.PF_STEP_NO_GRAPH)
    assert np.array_equal(a.fine("phi"), b.fine("phi"))


FULL_CASES = [
    # dim, nx, nz, dual, groups
    (2, 32, 16, 1, dict(ratio_rho=1000.0, ratio_mu=100.0, theta_deg=120.0, Wi=1.0, beta=0.5)),
    (2, 24, 12, 0, dict(ratio_rho=10.0, ratio_mu=5.0, theta_deg=60.0)),
    (3, 16, 8, 1, dict(ratio_rho=1000.0, ratio_mu=20.0, theta_deg=90.0, Wi=2.0, beta=0.3)),
    (3, 12, 6, 1, dict(ratio_rho=1000.0, ratio_mu=50.0, theta_deg=45.0)),
    # deep z: coarse u/p 40 rows, w 39 faces, fine 80 rows
    (2, 16, 40, 1, dict(ratio_rho=100.0, ratio_mu=10.0, theta_deg=70.0, Wi=0.5, beta=0.5)),
    # coarse and fine lines of 64 and 128 points (register-resident transforms)
    (3, 64, 4, 1, dict(ratio_rho=1000.0, ratio_mu=20.0, theta_deg=80.0, Wi=1.0, beta=0.3)),
]


@pytest.mark.parametrize("dim,nx,nz,dual,groups", FULL_CASES)
def test_full_step_fp64(dim, nx, nz, dual, groups):
    g = grid(dim, nx, nz, dual, lx=4.0 if dim == 2 else 5.0)
    w = workload(g, **groups)
    w.params.uw_top = 0.3
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 5, 0.1)
    s = binding.Solver(g, w.params, binding.PF_FP64)
    s.load_state(phi0, vel)
    ref = ostep.State(g, w.params.as_dict(), phi0, vel0=vel)
    for n in range(4):
        s.step(1)
        ref.step()
    assert rel(s.fine("phi"), ref.phi) < FP64_TOL
    assert rel(s.coarse("u"), ref.vel[0]) < FP64_TOL
    assert rel(s.coarse("w"), ref.vel[2]) < FP64_TOL
    if dim == 3:
        assert rel(s.coarse("v"), ref.vel[1]) < FP64_TOL
    assert rel(s.coarse("p"), ref.p) < FP64_TOL
    if ref.d.visco:
        th = s.coarse("theta")
        idx = [(0, 0), (0, 1), (1, 1)] if dim == 2 else [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
        for q, (a, b) in enumerate(idx):
            assert rel(th[q], ref.theta[..., a, b]) < FP64_TOL, q


def test_config1_fp64_full_run():
    """2D sessile droplet, coarse 64x32 / fine 128x64, 200 steps, FP64."""
    w = wl.config("c1")
    g = w.grid
    phi0 = wl.initial_phi(w)
    s = binding.Solver(g, w.params, binding.PF_FP64)
    s.load_state(phi0)
    s.step(w.steps)
    ref = ostep.run(g, w.params.as_dict(), phi0, w.steps)
    assert rel(s.fine("phi"), ref.phi) < FP64_TOL
    assert rel(s.coarse("u"), ref.vel[0]) < FP64_TOL
    assert rel(s.coarse("w"), ref.vel[2]) < FP64_TOL
    assert rel(s.coarse("p"), ref.p) < FP64_TOL
    dg = s.diagnostics()
    assert abs(dg["mass"] - ob.mass(ref.phi, g)) < 1e-12 * np.sum(np.abs(ref.phi)) * g.h ** 2
    assert abs(dg["energy"] / ob.energy(ref.phi, ref.d, g) - 1) < 1e-10
    assert abs(dg["wetted"] / ob.wetted(ref.phi, g) - 1) < 1e-10
    assert np.allclose(dg["centroid"], ob.centroid(ref.phi, g), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("prec", [binding.PF_MIXED, binding.PF_MIXED_Z64, binding.PF_MIXED_Z2F])
def test_config1_mixed_full_run(prec):
    """Mixed paths on config 1: 2e-4 max-abs on phi, 1e-3 relative on u, w."""
    w = wl.config("c1")
    g = w.grid
    phi0 = wl.initial_phi(w)
    s = binding.Solver(g, w.params, prec)
    s.load_state(phi0)
    s.step(w.steps)
    ref = ostep.run(g, w.params.as_dict(), phi0, w.steps)
    assert np.max(np.abs(s.fine("phi") - ref.phi)) < 2e-4
    assert rel(s.coarse("u"), ref.vel[0]) < 1e-3
    assert rel(s.coarse("w"), ref.vel[2]) < 1e-3


@pytest.mark.parametrize("cfg,nx,nz,steps", [("c2", 32, 16, 40), ("c4", 16, 8, 20)])
def test_viscoelastic_mixed_vs_oracle(cfg, nx, nz, steps):
    """Mixed path with the Oldroyd-B polymer: 2e-4 max-abs on phi, 1e-3 relative
    on velocity and on every Theta component."""
    w = wl.scaled(wl.config(cfg), nx, nz)
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 11, 0.2)
    s = binding.Solver(g, w.params, binding.PF_MIXED)
    s.load_state(phi0, vel)
    s.step(steps)
    ref = ostep.State(g, w.params.as_dict(), phi0, vel0=vel)
    for _ in range(steps):
        ref.step()
    assert np.max(np.abs(s.fine("phi") - ref.phi)) < 2e-4
    assert rel(s.coarse("u"), ref.vel[0]) < 1e-3
    assert rel(s.coarse("w"), ref.vel[2]) < 1e-3
    th = s.coarse("theta")
    idx = [(0, 0), (0, 1), (1, 1)] if g.dim == 2 else [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    scale = max(np.max(np.abs(ref.theta)), 1e-300)
    for q, (a, b) in enumerate(idx):
        assert np.max(np.abs(th[q] - ref.theta[..., a, b])) < 1e-3 * scale, q


def test_mass_conservation_gpu_fp64_and_mixed():
    w = wl.scaled(wl.config("c2"), 32, 16)
    g = w.grid
    phi0 = wl.initial_phi(w)
    for prec, tol in ((binding.PF_FP64, 1e-13), (binding.PF_MIXED, 1e-9), (binding.PF_MIXED_Z64, 1e-9),
                      (binding.PF_MIXED_Z2F, 1e-9)):
        s = binding.Solver(g, w.params, prec)
        s.load_state(phi0)
        m0 = s.diagnostics()["mass"]
        s.step(20)
        m1 = s.diagnostics()["mass"]
        assert abs(m1 - m0) < tol * np.sum(np.abs(phi0)) * g.h ** 2, prec


@pytest.mark.parametrize("prec", [binding.PF_MIXED, binding.PF_MIXED_Z64, binding.PF_MIXED_Z2F, binding.PF_FP64])
def test_mixed_mass_is_the_stored_fields_own_sum(prec):
    """The FP64 mass reduction of every path is the exact sum of the stored
    field: the compensated FP32 phi's values plus remainders (PF_PHI_REM),
    summed on the host in FP64, to 1e-13 relative.  So the mass drift is the
    field's own; over 200 steps of the 2D droplet it stays below 1e-9 of
    sum |phi| (an FP32 summation alone would err by about 1e-7 of it)."""
    w = wl.scaled(wl.config("c2"), 32, 16)
    g = w.grid
    s = binding.Solver(g, w.params, prec)
    s.load_state(wl.initial_phi(w))
    h2 = g.h ** 2
    masses = []
    for n in (0, 100, 100):
        if n:
            s.step(n)
        m = s.diagnostics()["mass"]
        ph = s.get("phi").astype(np.float64) + s.get("phi_rem").astype(np.float64)
        ref = np.sum(ph) * h2
        scale = np.sum(np.abs(ph)) * h2
        assert abs(m - ref) <= 1e-13 * scale, (prec, m, ref)
        masses.append(m)
    if prec == binding.PF_FP64:
        assert not np.any(s.get("phi_rem"))
    assert max(abs(x - masses[0]) for x in masses) < 1e-9 * scale, masses
    with pytest.raises(binding.PFError):
        s.set("phi_rem", np.zeros(g.fine_cells(), dtype=s.dtype))
    s.close()


@pytest.mark.parametrize("prec", [binding.PF_FP64, binding.PF_MIXED])
def test_overlapped_polymer_update_matches_sequential_order(prec):
    """Within one pf_step call the LCR update of a step runs beside the next
    step's CH transforms; calling pf_step one step at a time keeps the strict
    order.  Both must give the same bits."""
    w = wl.scaled(wl.config("c4"), 16, 8)
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 4, 0.2)
    a = binding.Solver(g, w.params, prec)
    b = binding.Solver(g, w.params, prec)
    for s in (a, b):
        s.load_state(phi0, vel)
    a.step(6)
    for _ in range(6):
        b.step(1)
    for name in ("phi", "u", "v", "w", "p", "theta", "tau"):
        assert np.array_equal(a.get(name), b.get(name)), name


@pytest.mark.parametrize("dim,nx,nz,theta", [(2, 16, 8, 0.0), (2, 16, 8, 180.0), (3, 12, 6, 0.0), (2, 20, 2, 30.0)])
def test_degenerate_cases_fp64(dim, nx, nz, theta):
    """Contact angles at the ends of the range (cos = +-1, full wetting and
    non-wetting), and the thinnest wall-to-wall mesh (two coarse rows, four
    fine ones, so every fine row touches a wall or its neighbour)."""
    g = grid(dim, nx, nz, 1)
    w = workload(g, theta_deg=theta, ratio_rho=10.0, ratio_mu=5.0, Wi=0.5, beta=0.5)
    w.params.theta_top_deg = 180.0 - theta
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 8, 0.1)
    s = binding.Solver(g, w.params, binding.PF_FP64)
    s.load_state(phi0, vel)
    ref = ostep.State(g, w.params.as_dict(), phi0, vel0=vel)
    for _ in range(3):
        s.step(1)
        ref.step()
    assert rel(s.fine("phi"), ref.phi) < FP64_TOL
    assert rel(s.coarse("u"), ref.vel[0]) < FP64_TOL
    assert rel(s.coarse("w"), ref.vel[2]) < FP64_TOL


@pytest.mark.parametrize("cfg,nx,nz", [("c2", 16, 8), ("c4", 12, 6)])
@pytest.mark.parametrize("alpha_g", [0.3])
def test_giesekus_fp64_and_mixed_vs_oracle(cfg, nx, nz, alpha_g):
    """Giesekus mobility (Eqs. NS18, NS22) in the polymer update: FP64 GPU path
    against the oracle at 1e-10, mixed at the viscoelastic
    tolerances, after steps from a seeded velocity and a seeded Theta of order
    one (so that the alpha term, quadratic in e^Theta - I, is not small)."""
    w = wl.scaled(wl.config(cfg), nx, nz)
    w.params.alpha_giesekus = alpha_g
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 13, 0.2)
    nz_, ny_, nx_ = g.coarse_shape
    m = 2 if g.dim == 2 else 3
    rng = np.random.default_rng(21)
    a = 0.25 * rng.standard_normal((nz_, ny_, nx_, m, m))
    theta0 = a + np.swapaxes(a, -1, -2)
    idx = [(0, 0), (0, 1), (1, 1)] if g.dim == 2 else [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    theta_comp = np.stack([theta0[..., i, j] for i, j in idx])
    n = 6

    def oracle(params):
        ref = ostep.State(g, params.as_dict(), phi0, vel0=vel, theta0=theta0)
        for _ in range(n):
            ref.step()
        return ref

    ref = oracle(w.params)
    for prec in (binding.PF_FP64, binding.PF_MIXED):
        s = binding.Solver(g, w.params, prec)
        s.load_state(phi0, vel)
        s.set("theta", theta_comp)
        s.step(n)
        th = s.coarse("theta")
        if prec == binding.PF_FP64:
            assert rel(s.fine("phi"), ref.phi) < FP64_TOL
            assert rel(s.coarse("u"), ref.vel[0]) < FP64_TOL
            assert rel(s.coarse("w"), ref.vel[2]) < FP64_TOL
            for q, (i, j) in enumerate(idx):
                assert rel(th[q], ref.theta[..., i, j]) < FP64_TOL, q
        else:
            assert np.max(np.abs(s.fine("phi") - ref.phi)) < 2e-4
            assert rel(s.coarse("u"), ref.vel[0]) < 1e-3
            scale = max(np.max(np.abs(ref.theta)), 1e-300)
            for q, (i, j) in enumerate(idx):
                assert np.max(np.abs(th[q] - ref.theta[..., i, j])) < 1e-3 * scale, q
        s.close()
    # the mobility changes the answer: Oldroyd-B (alpha = 0) gives another Theta
    ref0 = oracle(wl.scaled(wl.config(cfg), nx, nz).params)
    assert rel(ref0.theta, ref.theta) > 1e-4


@pytest.mark.parametrize("visco", [True, False])
def test_coalescing_drops_case_fp64(visco):
    """The performance case of Section 4.5 (two tangent drops on a 180 deg wall,
    Oh = 0.118, Cn = 0.015, density ratio 1/0.00119, Wi = 10, beta = 0.1) at
    coarse 16^3 / fine 32^3 on its 6 x 6 x 6 box, FP64 against the oracle."""
    w = wl.scaled(wl.config("e9", visco=visco), 16, 16)
    g = w.grid
    phi0 = wl.drops_phi(w)
    vel = wl.random_velocity(g, 12, 0.05)
    s = binding.Solver(g, w.params, binding.PF_FP64)
    s.load_state(phi0, vel)
    ref = ostep.State(g, w.params.as_dict(), phi0, vel0=vel)
    for _ in range(3):
        s.step(1)
        ref.step()
    assert rel(s.fine("phi"), ref.phi) < FP64_TOL
    for name, a in (("u", ref.vel[0]), ("v", ref.vel[1]), ("w", ref.vel[2]), ("p", ref.p)):
        assert rel(s.coarse(name), a) < FP64_TOL, name
    if visco:
        th = s.coarse("theta")
        for q, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
            assert rel(th[q], ref.theta[..., a, b]) < FP64_TOL, q


@pytest.mark.parametrize("dim,nx,nz", [(2, 8, 400), (3, 4, 384)])
def test_long_z_lines_vs_oracle(dim, nx, nz):
    """z lines of 800 and 768 fine rows (400 and 384 coarse): more 16-row
    segments than a 16-column CTA holds, so the solves run with the columns per
    CTA halved (8 and 4).  FP64 at 1e-10, both mixed paths at the mixed
    tolerances, against the oracle after 3 steps from a seeded velocity."""
    g = grid(dim, nx, nz, 1, lx=2.0)
    w = workload(g, ratio_rho=1000.0, ratio_mu=20.0, theta_deg=120.0, Wi=1.0, beta=0.3)
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 9, 0.1)
    ref = ostep.State(g, w.params.as_dict(), phi0, vel0=vel)
    for _ in range(3):
        ref.step()
    names = ["u", "w", "p"] + (["v"] if dim == 3 else [])
    refs = {"u": ref.vel[0], "v": ref.vel[1] if dim == 3 else None, "w": ref.vel[2], "p": ref.p}
    for prec in (binding.PF_FP64, binding.PF_MIXED, binding.PF_MIXED_Z64, binding.PF_MIXED_Z2F):
        s = binding.Solver(g, w.params, prec)
        s.load_state(phi0, vel)
        s.step(3)
        phi = s.fine("phi").astype(np.float64)
        out = {n: s.coarse(n).astype(np.float64) for n in names}
        s.close()
        if prec == binding.PF_FP64:
            assert rel(phi, ref.phi) < FP64_TOL
            for n in names:
                assert rel(out[n], refs[n]) < FP64_TOL, n
        else:
            assert np.max(np.abs(phi - ref.phi)) < 2e-4, prec
            for n in ("u", "w"):
                assert rel(out[n], refs[n]) < 1e-3, (prec, n)


AP1 = dict(polymer_approach=1, mu_p2=0.02, wi2=0.4, alpha_giesekus2=0.1)


@pytest.mark.parametrize("cfg,nx,nz", [("c2", 16, 8), ("c4", 12, 6)])
def test_polymer_approach1_fp64_and_mixed_vs_oracle(cfg, nx, nz):
    """Approach 1 of Section 2.1 (Eq. NS11): mu_p, lambda_H and alpha linear in
    the restricted phi at every centre, both phases viscoelastic, tau = tau_p.
    FP64 against the oracle at 1e-10, mixed at the viscoelastic tolerances,
    after 6 steps from a seeded velocity and Theta; the answer differs from
    approach 2 (Eq. NS12) on the same inputs."""
    w = wl.scaled(wl.config(cfg), nx, nz)
    w.params.alpha_giesekus = 0.2
    for k, v in AP1.items():
        setattr(w.params, k, v)
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 14, 0.2)
    nz_, ny_, nx_ = g.coarse_shape
    m = 2 if g.dim == 2 else 3
    a = 0.25 * np.random.default_rng(22).standard_normal((nz_, ny_, nx_, m, m))
    theta0 = a + np.swapaxes(a, -1, -2)
    idx = [(0, 0), (0, 1), (1, 1)] if g.dim == 2 else [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    theta_comp = np.stack([theta0[..., i, j] for i, j in idx])
    n = 6

    def oracle(params):
        ref = ostep.State(g, params.as_dict(), phi0, vel0=vel, theta0=theta0)
        for _ in range(n):
            ref.step()
        return ref

    ref = oracle(w.params)
    for prec in (binding.PF_FP64, binding.PF_MIXED):
        s = binding.Solver(g, w.params, prec)
        s.load_state(phi0, vel)
        s.set("theta", theta_comp)
        s.step(n)
        th = s.coarse("theta")
        if prec == binding.PF_FP64:
            assert rel(s.fine("phi"), ref.phi) < FP64_TOL
            for name, r in (("u", ref.vel[0]), ("w", ref.vel[2]), ("p", ref.p)):
                assert rel(s.coarse(name), r) < FP64_TOL, name
            for q, (i, j) in enumerate(idx):
                assert rel(th[q], ref.theta[..., i, j]) < FP64_TOL, q
        else:
            assert np.max(np.abs(s.fine("phi") - ref.phi)) < 2e-4
            assert rel(s.coarse("u"), ref.vel[0]) < 1e-3
            scale = max(np.max(np.abs(ref.theta)), 1e-300)
            for q, (i, j) in enumerate(idx):
                assert np.max(np.abs(th[q] - ref.theta[..., i, j])) < 1e-3 * scale, q
        s.close()
    p2 = wl.Params(**{**w.params.as_dict(), "polymer_approach": 0})
    assert rel(oracle(p2).vel[0], ref.vel[0]) > 1e-6


def test_polymer_approach1_argument_errors():
    w = wl.scaled(wl.config("c2"), 16, 8)
    for over in (dict(polymer_approach=2), dict(polymer_approach=1, wi2=0.0, mu_p2=0.1),
                 dict(polymer_approach=1, wi2=0.5, alpha_giesekus2=1.0)):
        prm = wl.Params(**{**w.params.as_dict(), **over})
        with pytest.raises(binding.PFError) as e:
            binding.Solver(w.grid, prm, binding.PF_FP64)
        assert e.value.code == -1, over


@pytest.mark.parametrize("cfg,nx,nz", [("c2", 16, 8), ("c4", 12, 6), ("c4", 16, 4)])
def test_weno5z_advection_fp64_and_mixed_vs_oracle(cfg, nx, nz):
    """The paper's WENO5-Z convective fluxes (advection = 1) for phi in the CH
    step (2D tiled, 3D scalar march in FP64, 3D float4 march in FP32) and for
    Theta in the polymer update: FP64 against the oracle at 1e-10, mixed at
    the mixed tolerances, after 4 steps from a seeded velocity and Theta; the
    fluxes change the answer against the central scheme."""
    w = wl.scaled(wl.config(cfg), nx, nz)
    w.params.advection = 1
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 15, 0.3)
    nz_, ny_, nx_ = g.coarse_shape
    m = 2 if g.dim == 2 else 3
    a = 0.25 * np.random.default_rng(23).standard_normal((nz_, ny_, nx_, m, m))
    theta0 = a + np.swapaxes(a, -1, -2)
    idx = [(0, 0), (0, 1), (1, 1)] if g.dim == 2 else [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    theta_comp = np.stack([theta0[..., i, j] for i, j in idx])
    n = 4

    def oracle(params):
        ref = ostep.State(g, params.as_dict(), phi0, vel0=vel, theta0=theta0)
        for _ in range(n):
            ref.step()
        return ref

    ref = oracle(w.params)
    for prec in (binding.PF_FP64, binding.PF_MIXED):
        s = binding.Solver(g, w.params, prec)
        s.load_state(phi0, vel)
        s.set("theta", theta_comp)
        s.step(n)
        th = s.coarse("theta")
        if prec == binding.PF_FP64:
            assert rel(s.fine("phi"), ref.phi) < FP64_TOL
            for name, r in (("u", ref.vel[0]), ("w", ref.vel[2]), ("p", ref.p)):
                assert rel(s.coarse(name), r) < FP64_TOL, name
            for q, (i, j) in enumerate(idx):
                assert rel(th[q], ref.theta[..., i, j]) < FP64_TOL, q
        else:
            assert np.max(np.abs(s.fine("phi") - ref.phi)) < 2e-4
            assert rel(s.coarse("u"), ref.vel[0]) < 1e-3
            scale = max(np.max(np.abs(ref.theta)), 1e-300)
            for q, (i, j) in enumerate(idx):
                assert np.max(np.abs(th[q] - ref.theta[..., i, j])) < 1e-3 * scale, q
        s.close()
    central = oracle(wl.Params(**{**w.params.as_dict(), "advection": 0}))
    assert rel(central.phi, ref.phi) > 1e-9
    assert rel(central.theta, ref.theta) > 1e-6


def test_weno5z_argument_errors():
    w = wl.scaled(wl.config("c2"), 16, 8)
    bad = wl.Params(**{**w.params.as_dict(), "advection": 2})
    with pytest.raises(binding.PFError) as e:
        binding.Solver(w.grid, bad, binding.PF_FP64)
    assert e.value.code == -1
    thin = wl.scaled(wl.config("c2"), 16, 2)
    with pytest.raises(binding.PFError) as e:
        binding.Solver(thin.grid, wl.Params(**{**thin.params.as_dict(), "advection": 1}), binding.PF_FP64)
    assert e.value.code == -1
    we = wl.Params(**{**w.params.as_dict(), "advection": 1})
    s = binding.Solver(w.grid, we, binding.PF_FP64)
    s.load_state(wl.initial_phi(w))
    with pytest.raises(binding.PFError) as e:
        s.adjoint(2, 1, binding.PF_OBJ_WETTED)
    assert e.value.code == -3
    s.close()
    with pytest.raises(binding.PFError) as e:
        binding.Batch([w.grid], [we], binding.PF_FP64)
    assert e.value.code == -3


@pytest.mark.parametrize("cfg,nx,nz", [("c1", 32, 16), ("c3", 12, 6), ("c2", 16, 8)])
def test_dynamic_contact_angle_fp64_and_mixed_vs_oracle(cfg, nx, nz):
    """Eq. NS15 / NS34 with D_w = 10 (the Robin walls that couple the two CH
    solves: the BDF2 time derivative of the wall value, implicit) and a
    moving top wall (the wall advection term), faster CH dynamics (100x
    mobility): 4 full steps, FP64 against the oracle at 1e-10 (phi, G and the
    flow), mixed at the mixed tolerances; 2D tiled, 3D scalar march (FP64)
    and float4 march (FP32) right sides.  D_w changes the answer."""
    w = wl.scaled(wl.config(cfg), nx, nz)
    w.params.mobility *= 100
    w.params.uw_top = 0.4
    w.params.dw = 10.0
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 5, 0.1)
    n = 4
    ref = ostep.State(g, w.params.as_dict(), phi0, vel0=vel)
    for _ in range(n):
        ref.step()
    for prec in (binding.PF_FP64, binding.PF_MIXED, binding.PF_MIXED_Z64, binding.PF_MIXED_Z2F):
        s = binding.Solver(g, w.params, prec)
        s.load_state(phi0, vel)
        s.step(n)
        phi = s.fine("phi").astype(np.float64)
        if prec == binding.PF_FP64:
            assert rel(phi, ref.phi) < FP64_TOL
            assert rel(s.fine("G"), ref.G) < FP64_TOL
            for name, r in (("u", ref.vel[0]), ("w", ref.vel[2]), ("p", ref.p)):
                assert rel(s.coarse(name), r) < FP64_TOL, name
        else:
            assert np.max(np.abs(phi - ref.phi)) < 2e-4, prec
            assert rel(s.coarse("u").astype(np.float64), ref.vel[0]) < 1e-3, prec
        s.close()
    st = ostep.State(g, {**w.params.as_dict(), "dw": 0.0}, phi0, vel0=vel)
    for _ in range(n):
        st.step()
    assert rel(st.G, ref.G) > 1e-2


def test_dynamic_contact_angle_ch_only_and_errors():
    """CH-only steps with D_w > 0 keep G (with the flux of phi^{n+1}) equal to
    the oracle's; D_w < 0 is an argument error; the batch, forward mode and
    the reverse sweep reject D_w > 0."""
    w = wl.scaled(wl.config("c1"), 32, 16)
    w.params.mobility *= 100
    w.params.dw = 3.0
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 6, 0.2)
    s = binding.Solver(g, w.params, binding.PF_FP64)
    s.load_state(phi0, vel)
    ref = ostep.State(g, w.params.as_dict(), phi0, vel0=vel)
    for k in range(3):
        s.step(1, binding.PF_STEP_CH_ONLY)
        ref.step(with_ns=False)
        assert rel(s.fine("phi"), ref.phi) < FP64_TOL, k
        assert rel(s.fine("G"), ref.G) < FP64_TOL, k
    for call in (lambda: s.adjoint(2, 1, binding.PF_OBJ_WETTED), lambda: s.tangent(2, binding.PF_PARAM_THETA_BOT, 0)):
        with pytest.raises(binding.PFError) as e:
            call()
        assert e.value.code == -3
    s.close()
    with pytest.raises(binding.PFError) as e:
        binding.Batch([g], [w.params], binding.PF_FP64)
    assert e.value.code == -3
    with pytest.raises(binding.PFError) as e:
        binding.Solver(g, wl.Params(**{**w.params.as_dict(), "dw": -1.0}), binding.PF_FP64)
    assert e.value.code == -1



def test_double_float_eliminations_track_the_fp64_ones():
    """PF_MIXED_Z2F runs the wall-normal eliminations in double-float (two FP32
    words, 48-bit significand).  After one full step from a seeded state, the
    only arithmetic that differs between PF_MIXED, PF_MIXED_Z64 and
    PF_MIXED_Z2F is those eliminations, whose results are stored in FP32: the
    double-float results round to the same FP32 values as the FP64 ones except
    at ties, while FP32 eliminations lose digits in the ill-conditioned low
    modes of the pressure solve.  So the Z2F fields sit at least ten times
    closer to the Z64 ones than the PF_MIXED fields do."""
    w = wl.scaled(wl.config("c2"), 64, 64)
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 17, 0.2)
    out = {}
    for prec in (binding.PF_MIXED_Z64, binding.PF_MIXED_Z2F, binding.PF_MIXED):
        s = binding.Solver(g, w.params, prec)
        s.load_state(phi0, vel)
        s.step(1)
        out[prec] = {n: s.coarse(n) for n in ("u", "w", "p")}
        out[prec]["phi"] = s.fine("phi") + s.fine("phi_rem")
        s.close()
    z64 = out[binding.PF_MIXED_Z64]
    dist = {prec: max(np.max(np.abs(out[prec][n] - z64[n])) / max(np.max(np.abs(z64[n])), 1e-300)
                      for n in ("u", "w", "p"))
            for prec in (binding.PF_MIXED_Z2F, binding.PF_MIXED)}
    print("distance to the FP64-elimination fields:", dist)
    assert dist[binding.PF_MIXED] > 0
    assert dist[binding.PF_MIXED_Z2F] <= 0.1 * dist[binding.PF_MIXED], dist
