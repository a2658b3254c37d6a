"""The 3D viscoelastic droplet at its full size (coarse 256x256x128 / fine
512x512x256), in the launch configuration the bench times (autotuned shapes).

The oracle cannot step 67 M fine cells in a test, so the full-size checks use
what holds at any size and a reference that is itself pinned to the oracle:
 - the mixed path against the FP64 GPU path (parity-tested against the oracle
   at smaller sizes) after a few steps: 2e-4 max-abs on phi, 1e-3 relative on
   velocity and on every Theta component;
 - the phi integral conserved to round-off by the FP64 path.
"""
import numpy as np
import pytest

from paper_2111_04577_gb300 import autotune, binding, build, workloads as wl

pytestmark = pytest.mark.gpu

STEPS = 4


@pytest.fixture(scope="module")
def runs():
    build.build()
    w = wl.config("c4")
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 9, 0.1)
    out = {}
    for prec in (binding.PF_FP64, binding.PF_MIXED):
        s = binding.Solver(g, w.params, prec)
        if prec == binding.PF_MIXED:
            autotune.apply(s, autotune.tuned(g, w.params, prec, phi0=phi0.astype(np.float32)))
        s.load_state(phi0, vel)
        m0 = s.diagnostics()["mass"]
        s.step(STEPS)
        out[prec] = {name: s.get(name).astype(np.float64) for name in ("phi", "u", "v", "w", "theta")}
        out[prec]["mass"] = (m0, s.diagnostics()["mass"])
        s.close()
        del s
    return w, out


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_fullsize_mixed_matches_fp64(runs):
    w, out = runs
    m, d = out[binding.PF_MIXED], out[binding.PF_FP64]
    assert np.max(np.abs(m["phi"] - d["phi"])) < 2e-4
    for name in ("u", "v", "w"):
        assert rel(m[name], d[name]) < 1e-3, name
    assert rel(m["theta"], d["theta"]) < 1e-3


def test_fullsize_fp64_conserves_mass(runs):
    w, out = runs
    m0, m1 = out[binding.PF_FP64]["mass"]
    g = w.grid
    scale = g.fine_cells() * g.h ** 3  # sum |phi| h^3 <= this
    assert abs(m1 - m0) < 1e-12 * scale


def test_tangent_at_full_size():
    """pf_tangent on the full 512x512x256 workload (the derivative-carrying
    copy: 16 bytes a value; tiles clamped to the shared-memory limit): J equals
    the FP64 path's, and dJ/dtheta equals central differences of the FP64 GPU
    path; dJ/dWi is finite (after 3 steps from rest it is tiny)."""
    w = wl.config("c4")
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = wl.random_velocity(g, 9, 0.1)
    n = 3

    def fp64_J(theta):
        prm = wl.Params(**{**w.params.as_dict(), "theta_bot_deg": theta})
        s = binding.Solver(g, prm, binding.PF_FP64)
        s.load_state(phi0, vel)
        s.step(n)
        J = s.diagnostics()["wetted"]
        s.close()
        return J

    s = binding.Solver(g, w.params, binding.PF_FP64)
    s.load_state(phi0, vel)
    J, dth = s.tangent(n, binding.PF_PARAM_THETA_BOT, binding.PF_OBJ_WETTED)
    _, dwi = s.tangent(n, binding.PF_PARAM_WI, binding.PF_OBJ_WETTED)
    s.close()
    th = w.params.theta_bot_deg
    assert abs(J - fp64_J(th)) <= 1e-12 * abs(J)
    hd = 0.05
    fd = (fp64_J(th + hd) - fp64_J(th - hd)) / (2 * hd)
    assert abs(dth - fd) <= 1e-3 * abs(fd), (dth, fd)
    assert np.isfinite(dwi)
