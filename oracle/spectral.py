"""Constant-coefficient Helmholtz / Poisson solves (oracle; test infrastructure only).

The paper solves Eqs. NS26, NS27, NS36 and NS37 with an FFT-based direct solver
(Section 3.2.1, end; Section 3.2.2, end).  This oracle diagonalises the discrete
second-order central Laplacian exactly: a DFT along the periodic x (and y) axes
and, along the wall-normal z axis, the real trigonometric transform whose basis
satisfies the wall condition:

  zbc="neumann"   cell-centred unknowns, mirror ghost  -> DCT-II,  eig m = 0..N-1
  zbc="dirichlet" cell-centred unknowns, odd ghost      -> DST-II,  eig m = 1..N
  zbc="faces"     face unknowns k = 1..N-1, zero walls   -> DST-I,   eig m = 1..N-1

with the one-dimensional eigenvalues -(4/h^2) sin^2(pi m/(2N)) along z and
-(4/h^2) sin^2(pi k/N) along a periodic axis of N cells.

solve(rhs, shift, ...) returns x with (L - shift) x = rhs.  For shift = 0 with
Neumann walls the zero mode is singular and set to zero (pressure, Eq. NS37).
"""
import os

import numpy as np
import scipy.fft as sf

_W = os.cpu_count() or 1


def eig_periodic(n, h):
    k = np.arange(n)
    return -4.0 / h ** 2 * np.sin(np.pi * k / n) ** 2


def eig_z(nz, h, zbc):
    if zbc == "neumann":
        m = np.arange(nz)
    elif zbc == "dirichlet":
        m = np.arange(1, nz + 1)
    elif zbc == "faces":
        m = np.arange(1, nz)
    else:
        raise ValueError(zbc)
    return -4.0 / h ** 2 * np.sin(np.pi * m / (2.0 * nz)) ** 2


def _zfwd(a, zbc):
    if zbc == "neumann":
        return sf.dct(a, type=2, axis=0, norm="ortho", workers=_W)
    if zbc == "dirichlet":
        return sf.dst(a, type=2, axis=0, norm="ortho", workers=_W)
    return sf.dst(a, type=1, axis=0, norm="ortho", workers=_W)


def _zinv(a, zbc):
    if zbc == "neumann":
        return sf.idct(a, type=2, axis=0, norm="ortho", workers=_W)
    if zbc == "dirichlet":
        return sf.idst(a, type=2, axis=0, norm="ortho", workers=_W)
    return sf.idst(a, type=1, axis=0, norm="ortho", workers=_W)


def solve(rhs, shift, h, zbc="neumann", nz_cells=None):
    """(Lx + Ly + Lz - shift) x = rhs on a uniform grid of spacing h.

    rhs has shape (Nz', Ny, Nx); Nz' = Nz for cell unknowns, Nz - 1 for "faces"
    (then nz_cells = Nz must be given).
    """
    rhs = np.asarray(rhs, dtype=np.float64)
    nzp, ny, nx = rhs.shape
    nz = nz_cells if zbc == "faces" else nzp
    t = _zfwd(rhs, zbc)
    t = sf.rfft(t, axis=2, workers=_W)
    if ny > 1:
        t = sf.fft(t, axis=1, workers=_W)
    lx = eig_periodic(nx, h)[: nx // 2 + 1]
    ly = eig_periodic(ny, h) if ny > 1 else np.zeros(1)
    lz = eig_z(nz, h, zbc)
    den = lz[:, None, None] + ly[None, :, None] + lx[None, None, :] - shift
    zero = den == 0.0
    den = np.where(zero, 1.0, den)
    t = np.where(zero, 0.0, t / den)
    if ny > 1:
        t = sf.ifft(t, axis=1, workers=_W)
    t = sf.irfft(t, n=nx, axis=2, workers=_W)
    return _zinv(t, zbc)


def solve_ch_robin(Q, Eb, Et, c, alpha, kappa, h):
    """The CH pair of Eqs. NS26-NS27 with the dynamic contact-angle walls of
    Eqs. NS33-NS34 (D_w > 0), solved as one linear system per Fourier mode.

    Unknowns Psi and phi = phi^{n+1} (cell-centred, shape (nz, ny, nx)); with
    the wall flux g = n.grad(phi^{n+1}) at each wall column,
        (L_N - c) Psi + c B(g) = Q            (Eq. NS26 with Eq. NS33's ghost)
        (L_N + alpha) phi + B(g) = Psi        (Eq. NS27 with Eq. NS34's ghost)
        g = E - kappa (1.5 phi_0 - 0.5 phi_1)  per wall (Eq. NS34),
    B(g) = g/h on the wall layer, L_N the homogeneous-Neumann Laplacian; E
    (Eb, Et: shape (ny, nx)) holds the explicit part of Eq. NS34 and kappa =
    D_w gamma0/dt its implicit coefficient.  The x (and y) DFT diagonalises the
    periodic directions; along z each mode is a dense 2 nz x 2 nz solve.
    Returns (Psi, phi)."""
    Q = np.asarray(Q, dtype=np.float64)
    nz, ny, nx = Q.shape
    nxr = nx // 2 + 1

    def fwd(a):
        t = sf.rfft(a, axis=-1, workers=_W)
        return sf.fft(t, axis=-2, workers=_W) if ny > 1 else t

    def inv(a):
        t = sf.ifft(a, axis=-2, workers=_W) if ny > 1 else a
        return sf.irfft(t, n=nx, axis=-1, workers=_W)

    Qh, Ebh, Eth = fwd(Q), fwd(np.asarray(Eb, dtype=np.float64)), fwd(np.asarray(Et, dtype=np.float64))
    lam = eig_periodic(nx, h)[:nxr][None, :] + (eig_periodic(ny, h) if ny > 1 else np.zeros(1))[:, None]
    n2 = 2 * nz
    M = np.zeros((ny, nxr, n2, n2))
    k = np.arange(nz)
    for blk, diag in ((0, -c), (1, alpha)):
        o = blk * nz
        M[..., o + k, o + k] = (-2.0 / h ** 2) + lam[..., None] + diag
        M[..., o + k[:-1], o + k[:-1] + 1] = 1.0 / h ** 2
        M[..., o + k[1:], o + k[1:] - 1] = 1.0 / h ** 2
        M[..., o, o] += 1.0 / h ** 2            # mirror ghost of L_N at both walls
        M[..., o + nz - 1, o + nz - 1] += 1.0 / h ** 2
    M[..., nz + k, k] = -1.0                     # - Psi in the phi rows
    rhs = np.zeros((ny, nxr, n2), dtype=complex)
    rhs[..., :nz] = np.moveaxis(Qh, 0, -1)
    # B(g) with g = E - kappa w(phi): enters the Psi rows times c, the phi rows once
    for row, wall, E in ((0, (0, 1), Ebh), (nz - 1, (nz - 1, nz - 2), Eth)):
        for o, coef in ((0, c), (nz, 1.0)):
            M[..., o + row, nz + wall[0]] += -coef * kappa * 1.5 / h
            M[..., o + row, nz + wall[1]] += coef * kappa * 0.5 / h
            rhs[..., o + row] -= coef * E / h
    sol = np.linalg.solve(M, rhs[..., None])[..., 0]
    psi = inv(np.moveaxis(sol[..., :nz], -1, 0))
    phi = inv(np.moveaxis(sol[..., nz:], -1, 0))
    return psi, phi
