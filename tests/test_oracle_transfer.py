"""Pins of the oracle's inter-grid transfers (Section 3.1, Eqs. dual1-dual3)."""
import numpy as np
import pytest

from paper_2111_04577_gb300 import workloads as wl
from oracle import operators as op
from oracle.params import Derived


def grid(dim, dual, n=8):
    if dim == 2:
        return wl.Grid(n, 1, n // 2, 2.0, 2.0 / n, 1.0, dual)
    return wl.Grid(n, n // 2, n // 2, 2.0, 1.0, 1.0, dual)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("dual", [1, 0])
def test_prolongation_divergence_equals_parent(dim, dual):
    """Eq. dual1 is exactly divergence-free: every fine cell inherits the coarse
    divergence of its parent (Rudman 1998, Section 3.1)."""
    g = grid(dim, dual)
    u, v, w = wl.random_velocity(g, 11)
    uf, vf, wf = op.prolong_velocity(u, v, w, g.r, g.ry, dim)
    dc = op.div_faces(u, v, w, g.dx, dim)
    df = op.div_faces(uf, vf, wf, g.h, dim)
    parent = np.repeat(np.repeat(np.repeat(dc, g.r, 0), g.ry, 1), g.r, 2)
    assert np.max(np.abs(df - parent)) < 1e-12 * np.max(np.abs(dc))


def test_prolongation_values_dual1():
    """The coincident fine face copies the coarse face; the mid-cell face averages."""
    g = grid(2, 1)
    u, v, w = wl.random_velocity(g, 3)
    uf, vf, wf = op.prolong_velocity(u, v, w, 2, 1, 2)
    i, k = 3, 1
    assert uf[2 * k, 0, 2 * i] == u[k, 0, i] and uf[2 * k + 1, 0, 2 * i] == u[k, 0, i]
    assert np.isclose(uf[2 * k + 1, 0, 2 * i + 1], 0.5 * (u[k, 0, i] + u[k, 0, i + 1]))
    assert np.isclose(wf[2 * k + 1, 0, 2 * i], 0.5 * (w[k, 0, i] + w[k + 1, 0, i]))
    assert wf[0].max() == 0 and wf[-1].max() == 0


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("dual", [1, 0])
def test_restriction_exact_for_linear_fields(dim, dual):
    """Each average of Eq. dual2 is centred on its coarse location, so it returns a
    linear field's value there (away from the periodic seam and the walls)."""
    g = grid(dim, dual)
    x, y, z = wl.fine_centres(g)
    a, b, c, e = 0.3, 1.7, -0.9, 2.3
    f = a + b * x + c * y + e * z + 0 * (x + y + z)
    f = np.broadcast_to(f, g.fine_shape).copy()
    if dim == 2:
        c = 0.0
        f = a + b * x + e * z + 0 * y
        f = np.broadcast_to(f, g.fine_shape).copy()
    R = op.restrict(f, g.r, g.ry, dim)
    D = g.dx
    dy = g.ly / g.ny
    nz, ny, nx = g.coarse_shape
    K, J, I = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx), indexing="ij")
    lin = lambda X, Y, Z: a + b * X + c * Y + e * Z
    loc = {
        "c": (I + 0.5, J + 0.5, K + 0.5), "fx": (I, J + 0.5, K + 0.5),
        "fz": (I + 0.5, J + 0.5, K), "exz": (I, J + 0.5, K),
        "fy": (I + 0.5, J, K + 0.5), "exy": (I, J, K + 0.5), "eyz": (I + 0.5, J, K),
    }
    for key, arr in R.items():
        X, Y, Z = loc[key]
        want = lin(X * D, Y * dy, Z * D)[: arr.shape[0]]
        sel = np.ones(arr.shape, bool)
        sel[..., 0] = False                      # periodic seam in x
        if dim == 3:
            sel[:, 0, :] = False                 # periodic seam in y
        if key in ("fz", "exz", "eyz"):
            sel[0] = False
            sel[-1] = False                      # mirror ghosts at the walls
        assert np.max(np.abs(arr[sel] - want[sel])) < 1e-12, key


def test_restriction_conserves_the_mean():
    g = grid(3, 1)
    rng = np.random.default_rng(0)
    f = rng.standard_normal(g.fine_shape)
    R = op.restrict(f, 2, 2, 3)
    assert abs(R["c"].mean() - f.mean()) < 1e-14
    assert abs(R["fx"].mean() - f.mean()) < 1e-14


def test_properties_dual3():
    d = Derived(wl.Params(rho1=3.0, rho2=0.5, mu1=2.0, mu2=0.1, eta=0.05, mobility=1e-3).as_dict())
    assert d.rho(1.0) == 3.0 and d.rho(-1.0) == 0.5 and d.rho(0.0) == 1.75
    assert d.mu(1.0) == 2.0 and d.mu(-1.0) == 0.1
