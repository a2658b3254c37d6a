"""FP64 CPU oracle of the dual-resolution phase-field step (arXiv 2111.04577).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library: its own
index conventions, NumPy stencils written from the paper's equations, and
spectral solves built on scipy.fft (FFT along the periodic axes, DCT/DST along
the wall-normal axis) instead of the library's batched FFT + Thomas kernels.

Array convention: every field is a NumPy array indexed [k, j, i] = (z, y, x), x
fastest.  A two-dimensional problem has ny = 1 and no y terms.  Coarse MAC
layout (0-based): p, Theta at cell centres; u[k, j, i] on the x-face at
x = i*dx; v on the y-face y = j*dx; w[k, j, i] on the z-face z = k*dx for
k = 0..nz (w = 0 on both walls).  Fine cells: coarse cell i holds fine cells
r*i .. r*i + r - 1 (r = 2 dual resolution, r = 1 single resolution).

Modules:
  params     derived constants (Eqs. NS7, NS29-NS31, text after NS39)
  spectral   constant-coefficient Helmholtz/Poisson solves (Eqs. NS26, NS27, NS36, NS37)
  operators  stencils, prolongation (Eq. dual1), restriction (Eq. dual2), properties (dual3)
  ch         Cahn-Hilliard step (Eqs. NS25-NS34)
  ns         Navier-Stokes step (Eqs. NS35-NS39)
  polymer    log-conformation RK2-TVD (Eqs. NS17-NS24, NS40-NS46)
  step       the coupled time step in the paper's order
  observables mass, free energy, wetted length, centroid
"""
