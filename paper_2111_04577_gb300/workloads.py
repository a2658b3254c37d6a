"""Seeded synthetic workloads: grids, physical parameters and initial fields.

This module only *describes* inputs.  It holds none of the method's arithmetic
(no transfer, stencil, solve or derived constant of the scheme); it is the one
module that both the CUDA path and the CPU oracle are fed from, so that both
sides see byte-identical inputs.

Parameter mapping from dimensionless groups (R0 = 1, U = 1, rho1 = 1, fluid 1 is
the droplet, phi = +1):

* mu1 = 1/Re, sigma = 1/We, eta = Cn * R0, lambda_H = Wi;
* mobility M from the Peclet number of the Couette case (Section 4.1):
  Pe = 2 sqrt(2) U R0 eta / (3 M sigma)  =>  M = 2 sqrt(2) eta / (3 sigma Pe);
* density and viscosity ratios are read droplet/ambient (droplet heavier and more
  viscous, as in the coalescence case of Section 4.5): rho2 = rho1/ratio_rho,
  mu2 = mu1/ratio_mu;
* viscoelastic droplet: beta = mu_s1/(mu_s1 + mu_p1) (Section 4.1); beta = 1 and
  wi = 0 mean Newtonian.

Initial state (Section 4.4, initial contact angle 90 deg): a droplet of radius R0
centred on the bottom wall, phi0 = tanh((R0 - r)/(sqrt(2) eta)) at fine cell
centres plus an i.i.d. U(-1, 1) perturbation of amplitude 1e-3 drawn from
numpy.random.default_rng(seed); velocities, pressure and log-conformation zero.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

# field identifiers shared by the C-ABI, the binding and the tests
PHI, PHI_OLD, U, U_OLD, V, V_OLD, W, W_OLD, P, P_OLD, THETA, TAU, TAU_OLD, G_FINE, PHI_REM = range(15)


@dataclass
class Grid:
    """Coarse (flow) mesh; the phase-field mesh is 2x finer per direction when dual."""
    nx: int
    ny: int          # 1 => two-dimensional (x-z plane)
    nz: int
    lx: float
    ly: float
    lz: float
    dual: int = 1    # 1: phi on the 2x finer mesh; 0: phi on the coarse mesh

    def __post_init__(self):
        dx = self.lx / self.nx
        if abs(self.lz / self.nz - dx) > 1e-12 * dx or (
                self.ny > 1 and abs(self.ly / self.ny - dx) > 1e-12 * dx):
            raise ValueError("cells must be square/cubic: lx/nx = ly/ny = lz/nz")

    @property
    def dim(self) -> int:
        return 2 if self.ny == 1 else 3

    @property
    def r(self) -> int:
        return 2 if self.dual else 1

    @property
    def ry(self) -> int:
        return self.r if self.dim == 3 else 1

    @property
    def fine_shape(self):
        """(Nz, Ny, Nx) of the phase-field mesh, x fastest."""
        return (self.r * self.nz, self.ry * self.ny, self.r * self.nx)

    @property
    def coarse_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def dx(self) -> float:
        return self.lx / self.nx

    @property
    def h(self) -> float:
        return self.dx / self.r

    def fine_cells(self) -> int:
        a, b, c = self.fine_shape
        return a * b * c


@dataclass
class Params:
    """Physical parameters, field-for-field the `pf_params` struct of the C-ABI."""
    rho1: float = 1.0
    rho2: float = 1.0
    mu1: float = 0.1
    mu2: float = 0.1
    sigma: float = 1.0
    eta: float = 0.02
    mobility: float = 0.0
    theta_bot_deg: float = 90.0
    theta_top_deg: float = 90.0
    dw: float = 0.0
    wi: float = 0.0
    beta: float = 1.0
    alpha_giesekus: float = 0.0
    dt: float = 1e-4
    S: float = 0.0           # 0 => the smallest S allowed by Eq. (NS30)
    nu_m: float = 0.0        # 0 => 1/2 max(mu)/min(rho)
    uw_bot: float = 0.0
    uw_top: float = 0.0
    gx: float = 0.0
    gy: float = 0.0
    gz: float = 0.0
    mu_p2: float = 0.0            # approach 1: polymer viscosity of phase 2
    wi2: float = 0.0              # approach 1: relaxation time of phase 2
    alpha_giesekus2: float = 0.0  # approach 1: Giesekus mobility of phase 2
    polymer_approach: int = 0     # 0: Eq. NS12 (droplet only), 1: Eq. NS11 (linear in phi)
    advection: int = 0            # 0: central second order, 1: WENO5-Z (phi and Theta)

    def as_dict(self):
        return asdict(self)


def params_from_groups(Re=10.0, We=1.0, Pe=1e3, Cn=0.02, ratio_rho=1.0, ratio_mu=1.0,
                       theta_deg=90.0, theta_top_deg=90.0, Wi=0.0, beta=1.0, dt=1e-4,
                       R0=1.0) -> Params:
    rho1 = 1.0
    mu1 = 1.0 / Re
    sigma = 1.0 / We
    eta = Cn * R0
    mob = 2.0 * math.sqrt(2.0) * eta / (3.0 * sigma * Pe)
    return Params(rho1=rho1, rho2=rho1 / ratio_rho, mu1=mu1, mu2=mu1 / ratio_mu,
                  sigma=sigma, eta=eta, mobility=mob, theta_bot_deg=theta_deg,
                  theta_top_deg=theta_top_deg, wi=Wi, beta=beta, dt=dt)


@dataclass
class Workload:
    name: str
    grid: Grid
    params: Params
    steps: int
    R0: float = 1.0
    seed: int = 0
    amp: float = 1e-3
    extra: dict = field(default_factory=dict)


def _c1(dual=1):
    return Workload("2d-sessile-newtonian-64x32", Grid(64, 1, 32, 4.0, 4.0 / 64, 2.0, dual),
                    params_from_groups(theta_deg=60.0), steps=200)


def _c2(dual=1):
    # The configuration states no time step.  With the 1e-4 of the Newtonian 2D
    # droplet this density-ratio-1000 case is unstable in the scheme (the
    # velocity doubles about every 100 steps from step 300 on and overflows near
    # step 825, in the FP64 oracle as in every GPU path); 5e-5 stays bounded over
    # 4000 steps, so the 2000 stated steps run at 5e-5.
    return Workload("2d-viscoelastic-oldroydb-256x128",
                    Grid(256, 1, 128, 4.0, 4.0 / 256, 2.0, dual),
                    params_from_groups(ratio_rho=1000.0, ratio_mu=100.0, theta_deg=120.0,
                                       Wi=1.0, beta=0.5, dt=5e-5), steps=2000)


def _c3(dual=1):
    return Workload("3d-newtonian-128x128x64", Grid(128, 128, 64, 5.0, 5.0, 2.5, dual),
                    params_from_groups(ratio_rho=1000.0, ratio_mu=50.0, theta_deg=45.0),
                    steps=1000)


def _c4(dual=1, wi=2.0):
    return Workload(f"3d-viscoelastic-oldroydb-256x256x128-wi{wi:g}",
                    Grid(256, 256, 128, 5.0, 5.0, 2.5, dual),
                    params_from_groups(ratio_rho=1000.0, ratio_mu=20.0, theta_deg=90.0,
                                       Wi=wi, beta=0.3), steps=500)


def e9_params(visco=True) -> Params:
    """The coalescing-drops case of Section 4.5 in the units r0 = rho_d = sigma = 1
    (velocity scale u_ci = sqrt(sigma/(rho_d r0)) = 1): Oh = mu_d = 0.118 (droplet
    solvent + polymer viscosity), Wi = lambda_H = 10, beta = 0.1, Cn = eta = 0.015,
    Pe = 2 sqrt(2) eta/(3 M) = 6/Cn, air/drop ratios 0.017 (viscosity) and
    0.00119 (density); bottom wall 180 deg, top 90 deg.  The section states no
    time step: 5e-5 (below the capillary bound sqrt(rho h^3/(2 pi sigma)) of the
    fine mesh, 1.9e-4)."""
    eta = 0.015
    pe = 6.0 / eta
    mob = 2.0 * math.sqrt(2.0) * eta / (3.0 * 1.0 * pe)
    mu_d = 0.118
    return Params(rho1=1.0, rho2=0.00119, mu1=mu_d, mu2=0.017 * mu_d, sigma=1.0, eta=eta, mobility=mob,
                  theta_bot_deg=180.0, theta_top_deg=90.0, wi=10.0 if visco else 0.0,
                  beta=0.1 if visco else 1.0, dt=5e-5)


def _e9(dual=1, visco=True, n=384):
    """Section 4.5: two tangent drops of radius r0 = 1 on a superhydrophobic
    wall in a 6 x 6 x 6 box; dual resolution 384^3 (phase field 768^3) against
    single resolution 768^3; 100 steps."""
    return Workload(f"e9-coalescing-drops-{'viscoelastic' if visco else 'newtonian'}-{n}^3",
                    Grid(n, n, n, 6.0, 6.0, 6.0, dual), e9_params(visco), steps=100,
                    extra={"drops": ((2.0, 3.0, 1.0), (4.0, 3.0, 1.0))})


CONFIGS = {"c1": _c1, "c2": _c2, "c3": _c3, "c4": _c4, "e9": _e9}


def config(name: str, **kw) -> Workload:
    return CONFIGS[name](**kw)


def scaled(w: Workload, nx: int, nz: int, ny: int | None = None) -> Workload:
    """Same physics and x/y domain, another coarse resolution (tests use small
    copies); lz follows nz so that cells stay cubic."""
    g = w.grid
    ny = (1 if g.dim == 2 else nx) if ny is None else ny
    ly = g.ly if g.dim == 3 else g.lx / nx
    lz = nz * g.lx / nx
    return Workload(w.name + f"@{nx}x{ny}x{nz}", Grid(nx, ny, nz, g.lx, ly, lz, g.dual),
                    Params(**w.params.as_dict()), w.steps, w.R0, w.seed, w.amp, dict(w.extra))


def fine_centres(grid: Grid):
    """Coordinates of the phase-field cell centres, each broadcastable to fine_shape."""
    nz, ny, nx = grid.fine_shape
    h = grid.h
    x = (np.arange(nx) + 0.5) * h
    z = (np.arange(nz) + 0.5) * h
    y = (np.arange(ny) + 0.5) * (grid.ly / ny)
    return x[None, None, :], y[None, :, None], z[:, None, None]


def initial_phi(w: Workload, centre=None) -> np.ndarray:
    """Droplet of radius R0 sitting on the bottom wall (90 deg initial angle)."""
    g = w.grid
    x, y, z = fine_centres(g)
    if centre is None:
        centre = (g.lx / 2, g.ly / 2, 0.0)
    r2 = (x - centre[0]) ** 2 + (z - centre[2]) ** 2
    if g.dim == 3:
        r2 = r2 + (y - centre[1]) ** 2
    r = np.sqrt(r2)
    phi = np.tanh((w.R0 - r) / (math.sqrt(2.0) * w.params.eta))
    rng = np.random.default_rng(w.seed)
    phi = phi + w.amp * rng.uniform(-1.0, 1.0, size=g.fine_shape)
    return np.ascontiguousarray(phi, dtype=np.float64)


def drops_phi(w: Workload, dtype=np.float64) -> np.ndarray:
    """Several drops of radius R0 (centres w.extra['drops'], box coordinates):
    phi0 = tanh((R0 - d)/(sqrt(2) eta)) with d the distance to the nearest
    centre (a reading: Section 4.5 places two tangent spheres on the wall; their
    centres sit one radius above it), plus the seeded perturbation.  Built one
    z-layer at a time, so meshes of several hundred million cells stay within a
    few host-memory copies of the field."""
    g = w.grid
    x, y, z = fine_centres(g)
    nz, ny, nx = g.fine_shape
    rng = np.random.default_rng(w.seed)
    out = np.empty(g.fine_shape, dtype=dtype)
    s = math.sqrt(2.0) * w.params.eta
    for k in range(nz):
        d = None
        for (cx, cy, cz) in w.extra["drops"]:
            r = np.sqrt((x[0, 0] - cx) ** 2 + (y[0, :, 0][:, None] - cy) ** 2 + (z[k, 0, 0] - cz) ** 2)
            d = r if d is None else np.minimum(d, r)
        layer = np.tanh((w.R0 - d) / s)
        if w.amp:
            layer = layer + w.amp * rng.uniform(-1.0, 1.0, size=(ny, nx))
        out[k] = layer
    return out


def zero_state(grid: Grid):
    """Coarse fields at rest: u, v at x/y faces, w at z faces incl. both walls."""
    nz, ny, nx = grid.coarse_shape
    st = {
        "u": np.zeros((nz, ny, nx)),
        "v": np.zeros((nz, ny, nx)),
        "w": np.zeros((nz + 1, ny, nx)),
        "p": np.zeros((nz, ny, nx)),
    }
    return st


def random_velocity(grid: Grid, seed: int, amp: float = 0.1):
    """A seeded, smooth-ish, wall-compatible coarse velocity (for unit-level parity)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = grid.coarse_shape
    u = amp * rng.uniform(-1, 1, (nz, ny, nx))
    v = amp * rng.uniform(-1, 1, (nz, ny, nx)) if grid.dim == 3 else np.zeros((nz, ny, nx))
    w = amp * rng.uniform(-1, 1, (nz + 1, ny, nx))
    w[0] = 0.0
    w[-1] = 0.0
    return u, v, w


def batch_problems(n=64, seed=0):
    """Uneven 2D droplets for the batched sweep: coarse nx in {64..256}, nz = nx/2,
    contact angle ~ U(30, 150) deg, Wi ~ U(0, 2), beta = 0.5, Lx = 4, Lz = 2."""
    rng = np.random.default_rng(seed)
    sizes = [64, 96, 128, 160, 192, 224, 256]
    out = []
    for b in range(n):
        nx = int(sizes[rng.integers(0, len(sizes))])
        th = float(rng.uniform(30.0, 150.0))
        wi = float(rng.uniform(0.0, 2.0))
        w = Workload(f"batch{b}-{nx}", Grid(nx, 1, nx // 2, 4.0, 4.0 / nx, 2.0, 1),
                     params_from_groups(theta_deg=th, Wi=wi, beta=0.5), steps=500, seed=b)
        out.append(w)
    return out
