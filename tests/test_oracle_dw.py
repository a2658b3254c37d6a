"""Pins of the dynamic contact-angle condition (Eq. NS15, discrete Eq. NS34
with D_w > 0) in the oracle's CH step.

With D_w > 0 the wall flux of phi^{n+1} depends on phi^{n+1} itself (the BDF2
time derivative at the wall), so the two Helmholtz solves become one linear
system per Fourier mode (oracle.spectral.solve_ch_robin).  Checked against:
 - the D_w = 0 path (DCT along z), in the limit D_w -> 0;
 - the D_w = 0 path given the step's own final wall flux: it must reproduce
   phi^{n+1} (the dense per-mode system and the DCT diagonalisation share no
   arithmetic);
 - conservation of the phi integral (Eq. NS33 keeps the chemical-potential
   flux through the walls zero for any wall flux of phi);
 - the decrease of the free energy, and the retardation of the contact line
   that Section 2.1 states: the larger D_w, the less the wetted length moves
   in the same time;
 - planted mistakes (the relaxation's sign, the c of the Psi wall flux).
"""
import numpy as np
import pytest

from paper_2111_04577_gb300 import workloads as wl
from oracle import ch, observables as ob, operators as op, spectral, step as ostep
from oracle.params import Derived


def case(dim=2, mob_factor=100.0):
    """The 2D sessile droplet (60 deg), faster CH dynamics so that the contact
    line moves within a few steps."""
    if dim == 2:
        w = wl.scaled(wl.config("c1"), 32, 16)
    else:
        w = wl.scaled(wl.config("c3"), 12, 6)
    w.params.mobility *= mob_factor
    return w


def run(w, dw, steps, uw_top=0.0):
    prm = w.params.as_dict()
    prm["dw"] = dw
    prm["uw_top"] = uw_top
    st = ostep.State(w.grid, prm, wl.initial_phi(w))
    W, E, M = [ob.wetted(st.phi, w.grid)], [ob.energy(st.phi, st.d, w.grid)], [np.sum(st.phi)]
    for _ in range(steps):
        st.step(with_ns=False)
        W.append(ob.wetted(st.phi, w.grid))
        E.append(ob.energy(st.phi, st.d, w.grid))
        M.append(np.sum(st.phi))
    return st, np.array(W), np.array(E), np.array(M)


@pytest.mark.parametrize("dim", [2, 3])
def test_dw_to_zero_equals_the_static_condition(dim):
    w = case(dim)
    a, *_ = run(w, 0.0, 3)
    b, *_ = run(w, 1e-300, 3)
    assert np.max(np.abs(a.phi - b.phi)) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_dw_step_equals_the_static_solves_given_its_own_wall_flux(dim):
    """One step with D_w = 10 and a moving top wall; then the D_w = 0 solves
    (DCT along z) with the step's final wall flux g = n.grad(phi^{n+1}) as an
    explicit flux give the same Psi and phi^{n+1}."""
    w = case(dim)
    prm = w.params.as_dict()
    prm.update(dw=10.0, uw_top=0.4)
    d = Derived(prm)
    g = w.grid
    rng = np.random.default_rng(3)
    phi_n = wl.initial_phi(w)
    phi_o = phi_n + 1e-2 * rng.uniform(-1, 1, phi_n.shape)
    vel = wl.random_velocity(g, 4, 0.2)
    out = ch.ch_step(phi_n, phi_o, vel, vel, d, g)
    B = ch.wall_term(phi_n.shape, out["gb"], out["gt"], g.h)
    psi = spectral.solve(out["R1"], d.c, g.h, "neumann")
    phi = spectral.solve(psi - B, -d.alpha, g.h, "neumann")
    scale = np.max(np.abs(out["phi"]))
    assert np.max(np.abs(psi - out["psi"])) < 1e-10 * np.max(np.abs(psi))
    assert np.max(np.abs(phi - out["phi"])) < 1e-10 * scale
    # and the flux differs from the static one by the implicit relaxation term
    gs, _ = ch.wall_flux(out["phis"], d)
    assert np.max(np.abs(out["gb"] - gs)) > 1e-3 * np.max(np.abs(gs))


@pytest.mark.parametrize("dim", [2, 3])
def test_dw_conserves_mass_and_dissipates_energy(dim):
    w = case(dim)
    _, _, E, M = run(w, 10.0, 40 if dim == 2 else 10)
    assert np.max(np.abs(M - M[0])) < 1e-11 * np.sum(np.abs(wl.initial_phi(w)))
    assert np.all(np.diff(E) < 0)


def test_dw_retards_the_contact_line():
    """Section 2.1: relaxation at the wall retards the contact line.  Over the
    same 100 steps the wetted length moves less, the larger D_w."""
    w = case(2)
    moves = []
    for dw in (0.0, 1.0, 10.0):
        _, W, _, _ = run(w, dw, 100)
        moves.append(W[-1] - W[0])
    moves = np.array(moves)
    assert np.all(np.sign(moves) == np.sign(moves[0])) and abs(moves[0]) > 1e-4
    assert abs(moves[0]) > abs(moves[1]) > abs(moves[2])
    assert abs(moves[2]) < 0.3 * abs(moves[0])


def test_dw_pins_catch_planted_mistakes(monkeypatch):
    """The relaxation with the wrong sign (anti-dissipative) fails the
    retardation pin; the Psi wall flux without its factor c fails mass
    conservation."""
    from mutate import mutated
    bad = mutated(ch, "wall_explicit", "+ d.dw / d.dt * wh", "- d.dw / d.dt * wh")
    monkeypatch.setattr(ch, "wall_explicit", bad)
    orig = Derived.__init__

    def flipped(self, prm):
        orig(self, prm)
        self.kappa = -self.kappa

    monkeypatch.setattr(Derived, "__init__", flipped)
    with pytest.raises((AssertionError, FloatingPointError, np.linalg.LinAlgError)):
        test_dw_retards_the_contact_line()
    monkeypatch.undo()
    bad = mutated(spectral, "solve_ch_robin", "for o, coef in ((0, c), (nz, 1.0)):",
                  "for o, coef in ((0, 0.0), (nz, 1.0)):")
    monkeypatch.setattr(spectral, "solve_ch_robin", bad)
    with pytest.raises(AssertionError):
        test_dw_conserves_mass_and_dissipates_energy(2)
