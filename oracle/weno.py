"""WENO5-Z convective fluxes (oracle; test infrastructure only).

The paper advects phi (CH) and Theta (LCR) with the fifth-order WENO-Z
scheme of Borges et al. (2008) (Section 3.2.1 and the text before Eq. NS40);
the GPU path uses second-order central fluxes.  This is the oracle form of
the WENO-Z alternative; the oracle's CH step takes it when the parameter
"advection" is "weno5z" (default "central", as the GPU path).

Face value at i+1/2 from the upwind side (velocity > 0: cells i-2..i+2):
  candidates  q0 = ( 2 v[i-2] - 7 v[i-1] + 11 v[i]) / 6
              q1 = (  -v[i-1] + 5 v[i]   +  2 v[i+1]) / 6
              q2 = ( 2 v[i]   + 5 v[i+1] -    v[i+2]) / 6
  smoothness  b0 = 13/12 (v[i-2] - 2 v[i-1] + v[i])^2   + 1/4 (v[i-2] - 4 v[i-1] + 3 v[i])^2
              b1 = 13/12 (v[i-1] - 2 v[i]   + v[i+1])^2 + 1/4 (v[i-1] - v[i+1])^2
              b2 = 13/12 (v[i]   - 2 v[i+1] + v[i+2])^2 + 1/4 (3 v[i] - 4 v[i+1] + v[i+2])^2
  WENO-Z      tau5 = |b0 - b2|,  a_k = d_k (1 + tau5 / (b_k + eps)),
              (d0, d1, d2) = (1/10, 6/10, 3/10),  w_k = a_k / sum a
  value       sum w_k q_k
and the mirror image of the stencil for velocity < 0.  The flux through the
face is u_face times that value.

Boundaries (readings; the paper does not state them): periodic directions
wrap; at the walls (z) the face flux is zero (w = 0 there) and the stencil
reads mirror ghosts v[-1-m] = v[m], v[n+m] = v[n-1-m] (homogeneous Neumann).
"""
import numpy as np

EPS = 1e-40
D = (0.1, 0.6, 0.3)


def _face_from_left(vm2, vm1, v0, vp1, vp2):
    q0 = (2 * vm2 - 7 * vm1 + 11 * v0) / 6
    q1 = (-vm1 + 5 * v0 + 2 * vp1) / 6
    q2 = (2 * v0 + 5 * vp1 - vp2) / 6
    b0 = 13 / 12 * (vm2 - 2 * vm1 + v0) ** 2 + 0.25 * (vm2 - 4 * vm1 + 3 * v0) ** 2
    b1 = 13 / 12 * (vm1 - 2 * v0 + vp1) ** 2 + 0.25 * (vm1 - vp1) ** 2
    b2 = 13 / 12 * (v0 - 2 * vp1 + vp2) ** 2 + 0.25 * (3 * v0 - 4 * vp1 + vp2) ** 2
    tau5 = np.abs(b0 - b2)
    a0 = D[0] * (1 + tau5 / (b0 + EPS))
    a1 = D[1] * (1 + tau5 / (b1 + EPS))
    a2 = D[2] * (1 + tau5 / (b2 + EPS))
    s = a0 + a1 + a2
    return (a0 * q0 + a1 * q1 + a2 * q2) / s


def face_values(v, axis, periodic):
    """Left- and right-biased WENO5-Z values at the faces i+1/2 between cells i
    and i+1 along `axis`.  Periodic: n faces (the last one wraps).  Walls: the
    n-1 interior faces, with mirror ghosts."""
    v = np.moveaxis(np.asarray(v, dtype=np.float64), axis, 0)
    n = v.shape[0]
    if periodic:
        ext = np.concatenate([v[-3:], v, v[:3]], axis=0)
        idx = np.arange(n) + 3  # cell i of face i+1/2
    else:
        ext = np.concatenate([v[2::-1], v, v[:-4:-1]], axis=0)
        idx = np.arange(n - 1) + 3
    g = lambda o: ext[idx + o]
    left = _face_from_left(g(-2), g(-1), g(0), g(1), g(2))
    right = _face_from_left(g(3), g(2), g(1), g(0), g(-1))  # mirror stencil around the face
    return np.moveaxis(left, 0, axis), np.moveaxis(right, 0, axis)


def upwind_flux(v, u_face, axis, periodic):
    """u_face * (WENO5-Z upwind value) at the faces of face_values."""
    left, right = face_values(v, axis, periodic)
    return np.where(u_face >= 0, u_face * left, u_face * right)


def advection(q, uf, vf, wf, h, dim):
    """div(u q) at cell centres, conservative, with WENO5-Z face values.
    q: (nz, ny, nx); uf: x faces (left face of each cell, periodic, (nz, ny, nx));
    vf: y faces (3D, (nz, ny, nx)); wf: z faces (nz+1, ny, nx), zero at the walls."""
    fx = upwind_flux(q, np.roll(uf, -1, axis=2), axis=2, periodic=True)  # face i+1/2 carries u at i+1
    div = (fx - np.roll(fx, 1, axis=2)) / h
    if dim == 3:
        fy = upwind_flux(q, np.roll(vf, -1, axis=1), axis=1, periodic=True)
        div += (fy - np.roll(fy, 1, axis=1)) / h
    fz = upwind_flux(q, wf[1:-1], axis=0, periodic=False)  # interior faces 1..nz-1
    zero = np.zeros_like(q[:1])
    fz = np.concatenate([zero, fz, zero], axis=0)
    div += (fz[1:] - fz[:-1]) / h
    return div
