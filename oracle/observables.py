"""Global diagnostics in FP64 (oracle; test infrastructure only).

mass        sum(phi) h^d (conserved by Eqs. NS1 + NS14, Section 3.2.1)
energy      lambda sum(|grad phi|^2/2 + (phi^2-1)^2/(4 eta^2)) h^d
            + sum over wall faces f_w(phi_w) h^(d-1)  (Eqs. NS5-NS7, NS16; the
            constant (sigma_1w + sigma_2w)/2 of NS16 is dropped)
wetted      sum over bottom-wall faces (1 + phi_w)/2 h^(d-1): the wetted length
            (2D) or area (3D) of the droplet phase
centroid    sum(x (1 + phi)/2) / sum((1 + phi)/2), per axis (Section 4.3)
phi_w is the wall value 1.5 phi_0 - 0.5 phi_1 used by the contact-angle law.
Gradient terms use face differences; wall faces contribute no |grad phi|^2.
"""
import numpy as np


def mass(phi, grid):
    return float(np.sum(phi) * grid.h ** grid.dim)


def wall_values(phi):
    return 1.5 * phi[0] - 0.5 * phi[1], 1.5 * phi[-1] - 0.5 * phi[-2]


def energy(phi, d, grid):
    h = grid.h
    gx = (phi - np.roll(phi, 1, axis=2)) / h
    e = 0.5 * np.sum(gx * gx)
    if grid.dim == 3:
        gy = (phi - np.roll(phi, 1, axis=1)) / h
        e += 0.5 * np.sum(gy * gy)
    gz = (phi[1:] - phi[:-1]) / h
    e += 0.5 * np.sum(gz * gz)
    e += np.sum((phi * phi - 1.0) ** 2) / (4.0 * d.eta ** 2)
    e *= d.lam * h ** grid.dim
    wb, wt = wall_values(phi)
    sig = d.p["sigma"]
    fw = lambda c, p: sig * c * p * (p * p - 3.0) / 4.0
    e += (np.sum(fw(d.cos_bot, wb)) + np.sum(fw(d.cos_top, wt))) * h ** (grid.dim - 1)
    return float(e)


def wetted(phi, grid):
    wb, _ = wall_values(phi)
    return float(np.sum(0.5 * (1.0 + wb)) * grid.h ** (grid.dim - 1))


def centroid(phi, grid):
    nz, ny, nx = phi.shape
    h = grid.h
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * (grid.ly / ny)
    z = (np.arange(nz) + 0.5) * h
    wgt = 0.5 * (1.0 + phi)
    s = np.sum(wgt)
    return (float(np.sum(wgt * x[None, None, :]) / s),
            float(np.sum(wgt * y[None, :, None]) / s),
            float(np.sum(wgt * z[:, None, None]) / s))
