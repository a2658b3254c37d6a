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
