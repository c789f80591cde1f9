"""Seeded synthetic inputs: meshes, initial fields and parameter sets.

This module builds the *inputs* of a two-phase DUGKS run (Zhang, Yang & Guo,
"A discrete unified gas-kinetic scheme for immiscible two-phase flows"): cell
widths of tensor-product meshes, initial order-parameter fields and raw
parameter sets for the paper's test problems (Sec. 3).  It holds none of the
scheme's arithmetic; both the CPU oracle and the CUDA library consume what it
returns, so it must import neither.

Conventions
-----------
* Fluid A is marked by ``phiA`` (default 1), fluid B by ``phiB`` (default 0).
* Arrays of cell fields are row-major ``[ny, nx]`` (x fastest), float64.
* ``Params`` carries the raw model parameters; ``beta`` and ``kappa`` are the
  free-energy coefficients, ``mobility`` is lambda, ``tau_g`` the relaxation
  time of the order-parameter equation, ``(gx, gy)`` the body-force
  acceleration and ``rho_ref`` the reference density of the body force
  ``F_b = (rho - rho_ref) * g``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PERIODIC = 0
WALL = 1


@dataclasses.dataclass
class Params:
    phiA: float = 1.0
    phiB: float = 0.0
    rhoA: float = 1.0
    rhoB: float = 1.0
    nuA: float = 0.1
    nuB: float = 0.1
    mobility: float = 0.1
    tau_g: float = 0.5
    beta: float = 0.0
    kappa: float = 0.0
    gx: float = 0.0
    gy: float = 0.0
    rho_ref: float = 0.0
    cfl: float = 0.5

    def as_list(self):
        return [self.phiA, self.phiB, self.rhoA, self.rhoB, self.nuA, self.nuB,
                self.mobility, self.tau_g, self.beta, self.kappa, self.gx,
                self.gy, self.rho_ref, self.cfl]


@dataclasses.dataclass
class Mesh:
    dx: np.ndarray          # [nx] cell widths
    dy: np.ndarray          # [ny] cell heights
    bc_x: int = PERIODIC
    bc_y: int = PERIODIC

    @property
    def nx(self):
        return int(self.dx.shape[0])

    @property
    def ny(self):
        return int(self.dy.shape[0])

    @property
    def ncells(self):
        return self.nx * self.ny

    def centres(self):
        """Cell-centre coordinates (xc[nx], yc[ny]); the low faces sit at 0."""
        xc = np.cumsum(self.dx) - 0.5 * self.dx
        yc = np.cumsum(self.dy) - 0.5 * self.dy
        return xc, yc


@dataclasses.dataclass
class Case:
    """One run: mesh, parameters and initial fields (u = p = 0 unless given)."""
    name: str
    mesh: Mesh
    params: Params
    phi0: np.ndarray
    ux0: np.ndarray | None = None
    uy0: np.ndarray | None = None
    p0: np.ndarray | None = None
    steps: int = 0


def params_from_sigma_width(sigma, width, phiA=1.0, phiB=0.0):
    """(beta, kappa) giving surface tension ``sigma`` and interface width
    ``width``: the inverse of Eqs. (thickness) and (sigma) of Sec. 2.1,
    beta = 12 sigma / (W (phiA-phiB)^4), kappa = 3 sigma W / (2 (phiA-phiB)^2)."""
    d = abs(phiA - phiB)
    beta = 12.0 * sigma / (width * d ** 4)
    kappa = 1.5 * sigma * width / d ** 2
    return beta, kappa


def uniform_mesh(nx, ny, bc_x=PERIODIC, bc_y=PERIODIC, dx=1.0, dy=1.0):
    return Mesh(np.full(nx, float(dx)), np.full(ny, float(dy)), bc_x, bc_y)


def tanh_nodes(n_half, eps=2.5):
    """Nodes xi_k, k = -n_half..n_half, of the locally refined channel mesh of
    Sec. 3.2 (refined toward the walls at -1, +1 and the interface at 0)."""
    k = np.arange(-n_half, n_half + 1, dtype=np.float64)
    t = 2.0 * math.tanh(eps / 2.0)
    xi = np.where(k >= 0,
                  0.5 + np.tanh(eps * (k / n_half - 0.5)) / t,
                  -0.5 + np.tanh(eps * (k / n_half + 0.5)) / t)
    xi[n_half] = 0.0
    return xi


def tanh_channel_heights(ny, height, eps=2.5):
    """Cell heights of a channel of total height ``height`` with ``ny`` (even)
    cells, built from ``tanh_nodes`` on each half channel."""
    if ny % 2:
        raise ValueError("ny must be even for the two-sided tanh mesh")
    xi = tanh_nodes(ny // 2, eps)
    nodes = 0.5 * height * (xi + 1.0)
    return np.diff(nodes)


def drop_field(mesh, radius, centre, width, phiA=1.0, phiB=0.0):
    """Circular drop of fluid A (Eq. droplet, Sec. 3.1)."""
    xc, yc = mesh.centres()
    X, Y = np.meshgrid(xc, yc)
    r = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2)
    return 0.5 * (phiA + phiB) + 0.5 * (phiA - phiB) * np.tanh(2.0 * (radius - r) / width)


def layered_field(mesh, y_interface, width, phiA=1.0, phiB=0.0):
    """Fluid A below ``y_interface``, fluid B above (flat tanh interface)."""
    xc, yc = mesh.centres()
    Y = np.broadcast_to(yc[:, None], (mesh.ny, mesh.nx))
    return 0.5 * (phiA + phiB) + 0.5 * (phiA - phiB) * np.tanh(2.0 * (y_interface - Y) / width)


def rt_field(mesh, wavelength, y0, amplitudes, width, phiA=1.0, phiB=0.0):
    """Heavy fluid A above the perturbed interface
    y = y0 + sum_k a_k cos(2 pi k x / L)."""
    xc, yc = mesh.centres()
    eta = np.full_like(xc, float(y0))
    for k, a in enumerate(amplitudes, start=1):
        eta = eta + a * np.cos(2.0 * math.pi * k * xc / wavelength)
    X, Y = np.meshgrid(xc, yc)
    H = np.broadcast_to(eta[None, :], X.shape)
    return 0.5 * (phiA + phiB) + 0.5 * (phiA - phiB) * np.tanh(2.0 * (Y - H) / width)


# ----------------------------------------------------------------------------
# Workloads shaped like the paper's tests (Sec. 3) at the sizes this library is
# benchmarked and checked on.
# ----------------------------------------------------------------------------

def stationary_drop(n=64, radius=16.0, sigma=1e-3, width=4.0, density_ratio=10.0,
                    nu=0.1, mobility=0.1, cfl=0.5, steps=2000):
    """64x64 periodic stationary drop, rhoA/rhoB = 10, plain FP64 workload."""
    beta, kappa = params_from_sigma_width(sigma, width)
    mesh = uniform_mesh(n, n)
    prm = Params(rhoA=1.0, rhoB=1.0 / density_ratio, nuA=nu, nuB=nu, mobility=mobility,
                 beta=beta, kappa=kappa, cfl=cfl)
    phi0 = drop_field(mesh, radius, (0.5 * n, 0.5 * n), width)
    return Case("stationary_drop_%dx%d" % (n, n), mesh, prm, phi0, steps=steps)


def droplet_sec31(radius=25.0, n=100, mobility=0.1, cfl=0.4, sigma=1e-3, width=4.0):
    """The stationary droplet of Sec. 3.1: rhoA = 1, rhoB = 0.2, tau_f = tau_g
    = 0.5 (nu = c_s^2 tau_f = 1/6 in both fluids), W = 4, sigma = 1e-3,
    CFL = 0.4, an n x n periodic mesh, centred on a cell centre."""
    beta, kappa = params_from_sigma_width(sigma, width)
    mesh = uniform_mesh(n, n)
    prm = Params(rhoA=1.0, rhoB=0.2, nuA=1.0 / 6.0, nuB=1.0 / 6.0, mobility=mobility, tau_g=0.5,
                 beta=beta, kappa=kappa, cfl=cfl)
    c = 0.5 * n + 0.5
    phi0 = drop_field(mesh, radius, (c, c), width)
    return Case("droplet_R%g_lam%g_cfl%g" % (radius, mobility, cfl), mesh, prm, phi0)


def mobility_sweep(mobilities=(0.01, 0.1, 1.0), **kw):
    """Sec. 3.1, the density profile against the mobility (one batch)."""
    return [droplet_sec31(mobility=m, **kw) for m in mobilities]


def cfl_sweep(cfls=(0.1, 0.2, 0.4, 0.8), mobility=0.1, **kw):
    """Sec. 3.1, the density profile against the CFL number at lambda = 0.1
    (one batch; each CFL has its own time step)."""
    return [droplet_sec31(mobility=mobility, cfl=c, **kw) for c in cfls]


def viscosity_ratio_sweep(ratios=(3.0, 10.0, 100.0, 1000.0), **kw):
    """Sec. 3.2, the layered Poiseuille flow over viscosity ratios (one batch)."""
    return [layered_poiseuille(nu_ratio=r, **kw) for r in ratios]


def layered_poiseuille(nx=4, ny=256, height=256.0, nu_ratio=1.0, nuB=0.05, force=1e-6,
                       sigma=1e-3, width=4.0, mobility=0.1, cfl=0.5, eps=2.5, steps=50000):
    """Two-layer channel: walls at y=0 and y=height, fluid A below y=height/2,
    tanh-refined in y, body force ``force`` along x, equal densities."""
    beta, kappa = params_from_sigma_width(sigma, width)
    mesh = Mesh(np.ones(nx), tanh_channel_heights(ny, height, eps), PERIODIC, WALL)
    prm = Params(rhoA=1.0, rhoB=1.0, nuA=nuB * nu_ratio, nuB=nuB, mobility=mobility,
                 beta=beta, kappa=kappa, gx=force, gy=0.0, rho_ref=0.0, cfl=cfl)
    phi0 = layered_field(mesh, 0.5 * height, width)
    return Case("layered_poiseuille_%dx%d_nu%g" % (nx, ny, nu_ratio), mesh, prm, phi0, steps=steps)


def rayleigh_taylor(nx=256, ny=1024, atwood=0.5, reynolds=3000.0, sqrt_gl=0.04,
                    peclet=1000.0, sigma=5e-5, width=4.0, cfl=0.5, amplitudes=None, steps=20000):
    """Rayleigh-Taylor: L = nx, domain L x 4L style (ny rows), heavy A on top,
    periodic in x, walls in y, interface y = ny/2 + 0.1 L cos(2 pi x / L)."""
    L = float(nx)
    g = sqrt_gl ** 2 / L
    rhoB = 1.0
    rhoA = rhoB * (1.0 + atwood) / (1.0 - atwood)
    nu = sqrt_gl * L / reynolds
    lam = sqrt_gl * L / peclet
    beta, kappa = params_from_sigma_width(sigma, width)
    mesh = uniform_mesh(nx, ny, PERIODIC, WALL)
    prm = Params(rhoA=rhoA, rhoB=rhoB, nuA=nu, nuB=nu, mobility=lam, beta=beta, kappa=kappa,
                 gx=0.0, gy=-g, rho_ref=0.5 * (rhoA + rhoB), cfl=cfl)
    if amplitudes is None:
        amplitudes = [0.1 * L]
    phi0 = rt_field(mesh, L, 0.5 * ny, amplitudes, width)
    return Case("rayleigh_taylor_%dx%d" % (nx, ny), mesh, prm, phi0, steps=steps)


def roofline_drop(n=4096, steps=200):
    """Large periodic drop whose state is far larger than L2 (FP32 ~1.2 GB)."""
    c = stationary_drop(n=n, radius=n / 4.0, steps=steps)
    c.name = "roofline_drop_%dx%d" % (n, n)
    return c


BATCH_SIDES = (64, 96, 128, 192, 256, 384, 512)


def batched_ensemble(n_instances=512, seed=1802, sides=BATCH_SIDES, sigma=1e-3, width=4.0,
                     eotvos=10.0, nuB=0.1, mobility=0.1, cfl=0.5, max_density_ratio=20.0):
    """Ensemble of rising-bubble and stationary-drop instances on square periodic
    meshes of uneven size (side drawn from ``sides``), seeded.  The density
    ratio is log-uniform in [2, max_density_ratio]: the scheme as printed is
    stable to about 20 here and diverges from about 50 on (the paper shows
    bubbles up to a ratio of 5)."""
    rng = np.random.default_rng(seed)
    beta, kappa = params_from_sigma_width(sigma, width)
    cases = []
    for k in range(n_instances):
        side = int(rng.choice(np.asarray(sides)))
        radius = float(rng.uniform(0.1, 0.25)) * side
        ratio = float(np.exp(rng.uniform(math.log(2.0), math.log(max_density_ratio))))
        nu_ratio = float(rng.uniform(1.0, 100.0))
        bubble = bool(rng.integers(0, 2))
        rhoB = 1.0
        rhoA = rhoB / ratio               # fluid A is the light bubble / drop
        mesh = uniform_mesh(side, side)
        if bubble:
            G = eotvos * sigma / ((rhoB - rhoA) * (2.0 * radius) ** 2)
            centre = (0.5 * side, side / 3.0)
            gy, rho_ref = -G, rhoB
        else:
            centre = (0.5 * side, 0.5 * side)
            gy, rho_ref = 0.0, 0.0
        prm = Params(rhoA=rhoA, rhoB=rhoB, nuA=nuB * nu_ratio, nuB=nuB, mobility=mobility,
                     beta=beta, kappa=kappa, gx=0.0, gy=gy, rho_ref=rho_ref, cfl=cfl)
        phi0 = drop_field(mesh, radius, centre, width)
        cases.append(Case("%s_%d_s%d" % ("bubble" if bubble else "drop", k, side), mesh, prm, phi0))
    return cases


def rising_bubble_numbers(G, sigma, D, rhoA, rhoB, muB):
    """Eotvos, Morton and Reynolds numbers of the rising bubble (Sec. 3.3)."""
    drho = rhoB - rhoA
    Eo = G * drho * D ** 2 / sigma
    Mo = G * drho * muB ** 4 / (rhoB ** 2 * sigma ** 3)
    Re = math.sqrt(G * rhoB * drho * D ** 3) / muB
    return Eo, Mo, Re


def random_state(rng, shape, scale=1.0):
    """Seeded smooth-ish random perturbation field (for parity tests)."""
    return scale * rng.standard_normal(shape)
