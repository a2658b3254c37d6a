"""Pins of the WENO5-Z fluxes (oracle/weno.py): fifth-order accuracy on
smooth data, exact conservation, near-boundedness at a step, and the mirror
symmetry between the two upwind directions."""
import numpy as np
import pytest

from oracle import weno


def test_fifth_order_on_smooth_periodic_data():
    """Cell averages of sin in, face values out: the face-value error of the
    WENO-Z reconstruction is O(h^5) for smooth data (the ideal-weight limit)."""
    errs = []
    for n in (16, 32, 64, 128):
        h = 1.0 / n
        xl = np.arange(n) * h
        avg = (np.cos(2 * np.pi * xl) - np.cos(2 * np.pi * (xl + h))) / (2 * np.pi * h)  # exact cell averages
        left, right = weno.face_values(avg[None, None, :], axis=2, periodic=True)
        xf = (np.arange(n) + 1) * h
        exact = np.sin(2 * np.pi * xf)
        errs.append(max(np.max(np.abs(left[0, 0] - exact)), np.max(np.abs(right[0, 0] - exact))))
    r = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(r[1:] > 4.6), (errs, r)


def test_conservation_periodic_and_walls():
    rng = np.random.default_rng(3)
    nz, ny, nx = 8, 6, 10
    h = 0.1
    q = rng.standard_normal((nz, ny, nx))
    uf = rng.standard_normal((nz, ny, nx))
    vf = rng.standard_normal((nz, ny, nx))
    wf = rng.standard_normal((nz + 1, ny, nx))
    wf[0] = wf[-1] = 0.0
    for dim in (2, 3):
        div = weno.advection(q, uf, vf if dim == 3 else None, wf, h, dim)
        assert abs(np.sum(div)) < 1e-12 * np.sum(np.abs(div))


def test_bounded_at_a_step():
    """Essentially non-oscillatory: at a unit step the face values leave
    [0, 1] by at most 1e-3 (the linear fifth-order scheme overshoots by ~10 %)."""
    n = 64
    v = (np.arange(n) >= n // 2).astype(float)
    left, right = weno.face_values(v[None, None, :], axis=2, periodic=True)
    for f in (left, right):
        assert f.min() > -1e-3 and f.max() < 1 + 1e-3
    # the ideal-weight (linear) combination does overshoot: the weights matter
    g = lambda o: np.roll(v, -o)
    lin = (0.1 * (2 * g(-2) - 7 * g(-1) + 11 * g(0)) + 0.6 * (-g(-1) + 5 * g(0) + 2 * g(1))
           + 0.3 * (2 * g(0) + 5 * g(1) - g(2))) / 6
    assert lin.max() > 1.05 or lin.min() < -0.05


def test_upwind_direction_mirror_symmetry():
    """Reversing the velocity and mirroring the data mirrors the fluxes."""
    rng = np.random.default_rng(4)
    n = 20
    v = rng.standard_normal(n)
    u = np.abs(rng.standard_normal(n))
    f = weno.upwind_flux(v[None, None, :], u[None, None, :], axis=2, periodic=True)[0, 0]
    # mirrored problem: cell j -> n-1-j, face i+1/2 -> face (n-2-i)+1/2, velocity -> -velocity
    vm = v[::-1]
    um = -np.roll(u[::-1], -1)
    fm = weno.upwind_flux(vm[None, None, :], um[None, None, :], axis=2, periodic=True)[0, 0]
    assert np.allclose(np.roll(fm[::-1], -1), -f, rtol=1e-13, atol=1e-14)


def test_ch_step_with_weno_conserves_mass_and_stays_close_to_central():
    """The oracle's CH step with the paper's WENO5-Z advection: the phi integral
    is conserved to round-off (a conservative flux with zero wall flux), and on
    a resolved smooth state it differs from the central-flux step by the
    truncation of the advection only."""
    from paper_2111_04577_gb300 import workloads as wl
    from oracle import step as ostep

    w = wl.scaled(wl.config("c1"), 32, 16)
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 7, 0.3)
    out = {}
    for adv in ("central", "weno5z"):
        prm = w.params.as_dict()
        prm["advection"] = adv
        st = ostep.State(g, prm, phi0, vel0=vel)
        m0 = np.sum(st.phi)
        for _ in range(5):
            st.step(with_ns=False)
        assert abs(np.sum(st.phi) - m0) < 1e-11 * np.sum(np.abs(phi0))
        out[adv] = st.phi
    d = np.max(np.abs(out["weno5z"] - out["central"]))
    assert 0 < d < 1e-2


def _theta_case(n, axis):
    """One Theta component varying along x (periodic) or z (walls), with a
    non-uniform face velocity along that axis; the exact d(u Theta)/dx_axis at
    the centres.  3D coarse grid n cells along the axis, 4 across."""
    from paper_2111_04577_gb300 import workloads as wl
    L = 1.0
    h = L / n
    if axis == "x":
        g = wl.Grid(n, 4, 4, L, 4 * h, 4 * h, 1)
        xc = (np.arange(n) + 0.5) * h
        xf = np.arange(n) * h  # left faces
        th = np.sin(2 * np.pi * xc)
        T = np.zeros((4, 4, n, 3, 3))
        T[..., 0, 1] = T[..., 1, 0] = th[None, None, :]
        u = np.broadcast_to(1.0 + 0.5 * np.cos(2 * np.pi * xf), (4, 4, n)).copy()
        v = np.zeros((4, 4, n))
        w = np.zeros((5, 4, n))
        exact = (-np.pi * np.sin(2 * np.pi * xc) * np.sin(2 * np.pi * xc)
                 + 2 * np.pi * np.cos(2 * np.pi * xc) * (1.0 + 0.5 * np.cos(2 * np.pi * xc)))
        return g, T, u, v, w, exact[None, None, :], (0, 1)
    g = wl.Grid(4, 4, n, 4 * h, 4 * h, L, 1)
    zc = (np.arange(n) + 0.5) * h
    zf = np.arange(n + 1) * h
    s = 0.08
    th = np.exp(-((zc - 0.5) / s) ** 2)
    T = np.zeros((n, 4, 4, 3, 3))
    T[..., 2, 2] = th[:, None, None]
    u = np.zeros((n, 4, 4))
    v = np.zeros((n, 4, 4))
    w = np.broadcast_to(np.sin(np.pi * zf)[:, None, None], (n + 1, 4, 4)).copy()
    wc, dwc = np.sin(np.pi * zc), np.pi * np.cos(np.pi * zc)
    dth = -2 * (zc - 0.5) / s ** 2 * th
    exact = dwc * th + wc * dth
    return g, T, u, v, w, exact[:, None, None], (2, 2)


@pytest.mark.parametrize("axis", ["x", "z"])
def test_theta_weno_advection_converges_to_the_divergence(axis):
    """The polymer's WENO5-Z convective term, per component with the coarse
    face velocities: with a non-uniform face velocity it converges to the
    exact d(u Theta)/dx at (at least) second order along x (periodic) and z
    (walls, mirror ghosts); a face velocity taken one face off converges at
    first order only (see the planted-mistake test)."""
    from oracle import polymer
    errs = []
    for n in (32, 64, 128):
        g, T, u, v, w, exact, (a, b) = _theta_case(n, axis)
        A = polymer.advection(T, u, v, w, g, "weno5z")
        errs.append(np.max(np.abs(A[..., a, b] - exact)))
    r = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(r > 1.8), (errs, r)


def test_theta_weno_advection_of_a_uniform_state_is_zero():
    """A uniform Theta under a discretely divergence-free velocity (uniform
    along x, zero w) is not advected: every face value is the constant."""
    from oracle import polymer
    from paper_2111_04577_gb300 import workloads as wl
    g = wl.Grid(8, 8, 8, 1.0, 1.0, 1.0, 1)
    T = np.broadcast_to(np.array([[0.3, 0.1, -0.2], [0.1, 0.5, 0.05], [-0.2, 0.05, -0.4]]), (8, 8, 8, 3, 3)).copy()
    u = np.full((8, 8, 8), 0.7)
    v = np.full((8, 8, 8), -0.3)
    w = np.zeros((9, 8, 8))
    assert np.max(np.abs(polymer.advection(T, u, v, w, g, "weno5z"))) < 1e-13


def test_theta_weno_pin_catches_a_shifted_face_velocity(monkeypatch):
    from mutate import mutated
    from oracle import polymer
    bad = mutated(polymer, "advection_weno", "weno.advection(T[..., a, b], u,",
                  "weno.advection(T[..., a, b], np.roll(u, 1, axis=2),")
    monkeypatch.setattr(polymer, "advection_weno", bad)
    with pytest.raises(AssertionError):
        test_theta_weno_advection_converges_to_the_divergence("x")
