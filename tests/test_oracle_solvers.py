"""Pins of the oracle's constant-coefficient solves (Eqs. NS26, NS27, NS36, NS37).

Each solve is checked against (1) a dense solve of the operator assembled cell by
cell from its second-order stencil and wall ghost, (2) discrete eigenfunctions,
for which the answer is known in closed form, and (3) second-order convergence
to a continuous manufactured solution.
"""
import numpy as np
import pytest

from oracle import spectral


def assemble(nz, ny, nx, h, shift, zbc):
    """Dense matrix of (L - shift) with L the 5/7-point Laplacian; x, y periodic."""
    nzu = nz - 1 if zbc == "faces" else nz
    n = nzu * ny * nx
    A = np.zeros((n, n))
    idx = lambda k, j, i: (k * ny + j) * nx + i
    for k in range(nzu):
        for j in range(ny):
            for i in range(nx):
                r = idx(k, j, i)
                A[r, r] -= shift
                for di in (-1, 1):
                    A[r, idx(k, j, (i + di) % nx)] += 1 / h ** 2
                    A[r, r] -= 1 / h ** 2
                if ny > 1:
                    for dj in (-1, 1):
                        A[r, idx(k, (j + dj) % ny, i)] += 1 / h ** 2
                        A[r, r] -= 1 / h ** 2
                for dk in (-1, 1):
                    kk = k + dk
                    A[r, r] -= 1 / h ** 2
                    if 0 <= kk < nzu:
                        A[r, idx(kk, j, i)] += 1 / h ** 2
                    elif zbc == "neumann":
                        A[r, r] += 1 / h ** 2      # ghost = self
                    elif zbc == "dirichlet":
                        A[r, r] -= 1 / h ** 2      # ghost = -self
                    # faces: neighbour is a wall face with value 0
    return A


CASES = [(4, 1, 6), (4, 3, 4), (5, 4, 2), (6, 1, 8)]


@pytest.mark.parametrize("shape", CASES)
@pytest.mark.parametrize("zbc", ["neumann", "dirichlet", "faces"])
@pytest.mark.parametrize("shift", [0.0, 3.7, 250.0])
def test_dense_operator(shape, zbc, shift):
    nz, ny, nx = shape
    h = 0.37
    rng = np.random.default_rng(1)
    nzu = nz - 1 if zbc == "faces" else nz
    b = rng.standard_normal((nzu, ny, nx))
    A = assemble(nz, ny, nx, h, shift, zbc)
    if zbc == "neumann" and shift == 0.0:
        b -= b.mean()
        ref = np.linalg.lstsq(A, b.ravel(), rcond=None)[0]
    else:
        ref = np.linalg.solve(A, b.ravel())
    got = spectral.solve(b, shift, h, zbc, nz_cells=nz)
    assert np.max(np.abs(got.ravel() - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_discrete_eigenfunctions_exact():
    """cos(pi m (k+1/2)/N) e^{2 pi i (kx x)} are eigenvectors of the Neumann operator."""
    nz, ny, nx, h = 16, 8, 32, 0.1
    k = np.arange(nz)[:, None, None]
    j = np.arange(ny)[None, :, None]
    i = np.arange(nx)[None, None, :]
    for (m, ky, kx) in [(0, 0, 1), (3, 2, 5), (15, 7, 16), (1, 0, 0)]:
        f = np.cos(np.pi * m * (k + 0.5) / nz) * np.cos(2 * np.pi * (kx * i / nx + ky * j / ny))
        lam = -4 / h ** 2 * (np.sin(np.pi * m / (2 * nz)) ** 2 + np.sin(np.pi * kx / nx) ** 2
                             + np.sin(np.pi * ky / ny) ** 2)
        for shift in (5.0, 1234.5):
            got = spectral.solve(f, shift, h, "neumann")
            assert np.max(np.abs(got - f / (lam - shift))) < 1e-13 * np.max(np.abs(f / (lam - shift)))
    # Dirichlet (odd ghost): sin(pi (m+1) (k+1/2)/N)
    for m in (0, 4, nz - 1):
        f = np.sin(np.pi * (m + 1) * (k + 0.5) / nz) * np.cos(2 * np.pi * 3 * i / nx) + 0 * j
        lam = -4 / h ** 2 * (np.sin(np.pi * (m + 1) / (2 * nz)) ** 2 + np.sin(np.pi * 3 / nx) ** 2)
        got = spectral.solve(f, 7.0, h, "dirichlet")
        assert np.max(np.abs(got - f / (lam - 7.0))) < 1e-13 * np.max(np.abs(f / (lam - 7.0)))
    # faces (zero walls): sin(pi m k/N), k = 1..N-1
    kf = np.arange(1, nz)[:, None, None]
    for m in (1, 5, nz - 1):
        f = np.sin(np.pi * m * kf / nz) * np.cos(2 * np.pi * 2 * i / nx) + 0 * j
        lam = -4 / h ** 2 * (np.sin(np.pi * m / (2 * nz)) ** 2 + np.sin(np.pi * 2 / nx) ** 2)
        got = spectral.solve(f, 7.0, h, "faces", nz_cells=nz)
        assert np.max(np.abs(got - f / (lam - 7.0))) < 1e-13 * np.max(np.abs(f / (lam - 7.0)))


@pytest.mark.parametrize("zbc", ["neumann", "dirichlet", "faces"])
def test_second_order_convergence(zbc):
    """Manufactured continuous solution on [0,1]x[0,1]x[0,1]: slope 2 +- 0.1."""
    errs = []
    shift = 3.0
    for n in (16, 32, 64, 128):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        y = x
        if zbc == "faces":
            z = np.arange(1, n) * h
        else:
            z = (np.arange(n) + 0.5) * h
        X, Y, Z = x[None, None, :], y[None, :, None], z[:, None, None]
        if zbc == "neumann":
            zf, lz = np.cos(np.pi * Z) + 0.3 * np.cos(2 * np.pi * Z), None
            ex = np.cos(2 * np.pi * X) * np.sin(2 * np.pi * Y) * zf
            lap = np.cos(2 * np.pi * X) * np.sin(2 * np.pi * Y) * (
                -8 * np.pi ** 2 * zf - np.pi ** 2 * np.cos(np.pi * Z) - 1.2 * np.pi ** 2 * np.cos(2 * np.pi * Z))
        else:
            zf = np.sin(np.pi * Z) + 0.3 * np.sin(3 * np.pi * Z)
            ex = np.cos(2 * np.pi * X) * np.sin(2 * np.pi * Y) * zf
            lap = np.cos(2 * np.pi * X) * np.sin(2 * np.pi * Y) * (
                -8 * np.pi ** 2 * zf - np.pi ** 2 * np.sin(np.pi * Z) - 2.7 * np.pi ** 2 * np.sin(3 * np.pi * Z))
        got = spectral.solve(lap - shift * ex, shift, h, zbc, nz_cells=n)
        errs.append(np.max(np.abs(got - ex)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - 2.0) < 0.1), (errs, slopes)
