"""Stencils and inter-grid transfers (oracle; test infrastructure only).

Second-order central differences (Section 3.2.1: "second-order central
difference to approximate spatial derivatives").  x and y are periodic; z is
bounded by walls.  Arrays are [k, j, i]; a 2D array has a y extent of 1 and its
y differences vanish identically.
"""
import numpy as np


def xp(a):
    """a[..., i+1] (periodic)."""
    return np.roll(a, -1, axis=-1)


def xm(a):
    return np.roll(a, 1, axis=-1)


def yp(a):
    return np.roll(a, -1, axis=-2)


def ym(a):
    return np.roll(a, 1, axis=-2)


def zpad_mirror(a):
    """Append mirror ghosts a[-1] := a[0], a[N] := a[N-1] along z (axis 0)."""
    return np.concatenate([a[:1], a, a[-1:]], axis=0)


def lap_periodic(a, h, dim):
    out = (xp(a) - 2.0 * a + xm(a)) / h ** 2
    if dim == 3:
        out = out + (yp(a) - 2.0 * a + ym(a)) / h ** 2
    return out


def lap_neumann(a, h, dim):
    """L_N: periodic x,y; homogeneous Neumann (mirror ghost) on both z walls."""
    g = zpad_mirror(a)
    return lap_periodic(a, h, dim) + (g[2:] - 2.0 * a + g[:-2]) / h ** 2


# ----------------------------------------------------------------------------
# Eq. dual1: divergence-free first-order prolongation of the MAC velocity
# ----------------------------------------------------------------------------
def prolong_velocity(u, v, w, r, ry, dim):
    """Coarse face velocities -> fine face velocities (Eq. dual1, after Rudman 1998).

    0-based: the fine face r*i coincides with coarse face i and copies it; the
    fine face r*i + 1 (r = 2) sits mid-cell and takes the mean of coarse faces i
    and i+1.  Tangentially every fine row of coarse row k copies it.
    Returns (uf, vf, wf) with shapes (r nz, ry ny, r nx), same, (r nz + 1, ...).
    """
    nz, ny, nx = u.shape

    def along_x(a):  # a at x-faces -> fine x-faces, then tangential copies
        out = np.empty(a.shape[:-1] + (r * nx,))
        out[..., 0::r] = a
        if r == 2:
            out[..., 1::2] = 0.5 * (a + xp(a))
        return out

    def along_y(a):
        out = np.empty(a.shape[:-2] + (ry * ny, a.shape[-1]))
        out[..., 0::ry, :] = a
        if ry == 2:
            out[..., 1::2, :] = 0.5 * (a + yp(a))
        return out

    def rep_x(a):
        return np.repeat(a, r, axis=-1)

    def rep_y(a):
        return np.repeat(a, ry, axis=-2)

    def rep_z(a):
        return np.repeat(a, r, axis=0)

    uf = rep_z(rep_y(along_x(u)))
    if dim == 3:
        vf = rep_z(along_y(rep_x(v)))
    else:
        vf = np.zeros_like(uf)
    # w: nz+1 coarse faces -> r nz + 1 fine faces
    wx = rep_y(rep_x(w))
    wf = np.empty((r * nz + 1,) + wx.shape[1:])
    wf[0::r] = wx
    if r == 2:
        wf[1::2] = 0.5 * (wx[:-1] + wx[1:])
    return uf, vf, wf


def div_faces(u, v, w, h, dim):
    """Cell divergence of a face field (u, v at x/y faces, w with both wall faces)."""
    d = (xp(u) - u) / h + (w[1:] - w[:-1]) / h
    if dim == 3:
        d = d + (yp(v) - v) / h
    return d


# ----------------------------------------------------------------------------
# Eq. dual2: restriction by averaging over fine cell centres
# ----------------------------------------------------------------------------
def _block_mean_z(a, r):
    nzf = a.shape[0]
    return a.reshape(nzf // r, r, *a.shape[1:]).mean(axis=1)


def _block_mean_y(a, ry):
    s = a.shape
    return a.reshape(s[0], s[1] // ry, ry, s[2]).mean(axis=2)


def _block_mean_x(a, r):
    s = a.shape
    return a.reshape(s[0], s[1], s[2] // r, r).mean(axis=3)


def _pair_x(a, r):
    """Mean of fine cells r*i - 1 and r*i (the pair straddling coarse x-face i)."""
    return 0.5 * (xm(a) + a)[..., 0::r]


def _pair_y(a, ry):
    return 0.5 * (ym(a) + a)[..., 0::ry, :]


def _pair_z(a, r):
    """Mean of fine cells r*k - 1 and r*k for k = 0..nz (mirror ghosts at walls)."""
    g = zpad_mirror(a)  # g[K+1] = a[K]
    nzf = a.shape[0]
    ks = np.arange(0, nzf + 1, r)
    return 0.5 * (g[ks] + g[ks + 1])


def restrict(g, r, ry, dim):
    """All coarse samples of a fine cell-centred field g (Eq. dual2).

    Returns a dict:
      c   : coarse centres, mean of the r^d fine cells inside            (nz, ny, nx)
      fx  : x-faces, the r^(d-1) x 2 fine cells straddling the face     (nz, ny, nx)
      fy  : y-faces (3D)                                                 (nz, ny, nx)
      fz  : z-faces k = 0..nz (mirror ghost at the walls)                (nz+1, ny, nx)
      exz : x-z edges (x = i dx, z = k dx), 2 x 2 (x ry) cells           (nz+1, ny, nx)
      exy : x-y edges (3D)                                               (nz, ny, nx)
      eyz : y-z edges (3D)                                               (nz+1, ny, nx)
    The v-face row of Eq. dual2 is read as the mirror image of the u-face row
    (the printed row mixes index pairs; see the readings of the paper).
    """
    out = {}
    bx = _block_mean_x
    by = _block_mean_y
    bz = _block_mean_z
    out["c"] = bz(by(bx(g, r), ry), r)
    out["fx"] = bz(by(_pair_x(g, r), ry), r)
    out["fz"] = by(bx(_pair_z(g, r), r), ry)
    out["exz"] = by(_pair_z(_pair_x(g, r), r), ry)
    if dim == 3:
        out["fy"] = bz(_pair_y(bx(g, r), ry), r)
        out["exy"] = bz(_pair_y(_pair_x(g, r), ry), r)
        out["eyz"] = _pair_z(_pair_y(bx(g, r), ry), r)
    return out
