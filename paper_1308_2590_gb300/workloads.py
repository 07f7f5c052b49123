"""Seeded synthetic workloads for the implicit 2D3V PIC particle loop.

This module only describes runs and draws their initial particles: grid and
time step, species, plasma slab, Maxwellian momenta, laser parameters.  It holds
none of the method's arithmetic (no gather, push, deposit or field solve), so
both the CUDA path and the CPU oracle can be fed from it.

Units are normalised: c = eps0 = mu0 = 1, charge in e, mass in m_e, time in
1/omega_r, length in c/omega_r, density in n_r with omega_r^2 = n_r e^2/(eps0 m_e).
The uniform-plasma workloads take omega_r = omega_pe (n_e = 1); the laser-foil
workloads take omega_r = omega_0 of the laser, so that n_r is the critical
density n_c and the laser wavelength is 2*pi.

The paper's own runs (Section 4) use a 1200x1200 grid of 25 nm cells, a 1 um
laser with dt = 0.01 lambda/c and carbon foils; the laser-foil workloads here
keep its resolution ratios (40 cells per wavelength, dt = 0.01 lambda/c) on the
grid sizes stated per workload, with protons in place of carbon and no
ionisation.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

BC_PERIODIC = 0
BC_ABSORBING = 1
FIELD_LITERAL = 0
FIELD_CN = 1
PREC_FP64 = 0
PREC_FP32 = 1
DEPOSIT_ATOMIC = 0
DEPOSIT_DETERMINISTIC = 1
CN_PRECOND_AUTO, CN_PRECOND_JACOBI, CN_PRECOND_FFT = 0, 1, 2

ME_C2_KEV = 510.99895  # electron rest energy, keV
M_PROTON = 1836.15267343  # proton mass in m_e
M_PROTON_ROUND = 1836.0  # the uniform-plasma workloads state m_i/m_e = 1836


@dataclasses.dataclass
class Species:
    q: float
    m: float
    ppc: int               # macro-particles per cell (inside the slab)
    density: float         # in n_r
    temperature_kev: float


@dataclasses.dataclass
class Laser:
    a0: float = 0.0        # peak normalised vector potential (E in m_e c omega_0/e)
    omega: float = 1.0     # laser angular frequency in omega_r units
    tau: float = 0.0       # FWHM of intensity, in 1/omega_r
    t0: float = 0.0        # time of the envelope peak at x = 0
    pol: int = 0           # 0: E along y (in-plane), 1: E along z


@dataclasses.dataclass
class RunConfig:
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    steps: int
    bc_x: int = BC_PERIODIC
    field_mode: int = FIELD_LITERAL
    precision: int = PREC_FP64
    deposit: int = DEPOSIT_ATOMIC
    species: List[Species] = dataclasses.field(default_factory=list)
    slab: Optional[Tuple[int, int]] = None   # [first, last) cell columns in x holding plasma; None = all
    laser: Laser = dataclasses.field(default_factory=Laser)
    tile_nx: int = 16
    tile_ny: int = 16
    cn_tol: float = 1e-12
    cn_max_iter: int = 400
    seed: int = 1234
    shape: int = 1   # particle shape order: 1 area weighting (the paper's), 2-4 B-splines of that degree
    cn_precond: int = 0   # CN preconditioner: 0 automatic, 1 block-Jacobi, 2 spectral / line

    @property
    def n_particles(self) -> int:
        x0, x1 = self.slab if self.slab is not None else (0, self.nx)
        return sum(s.ppc for s in self.species) * (x1 - x0) * self.ny

    def scaled(self, **kw) -> "RunConfig":
        return dataclasses.replace(self, **kw)


def u_thermal(temperature_kev: float, m: float) -> float:
    """Non-relativistic thermal spread of u = p/(m c): sqrt(T / (m c^2))."""
    return math.sqrt(temperature_kev / (ME_C2_KEV * m))


def laser_units_au(wavelength_um: float):
    """The laser-foil runs' field unit m_e c omega_0 / e and time unit 1/omega_0 in atomic units
    (5.14220674763e11 V/m and 2.4188843265857e-17 s), for the field-ionisation pass."""
    omega0 = 2.0 * math.pi * 299792458.0 / (wavelength_um * 1e-6)
    e_unit = 9.1093837015e-31 * 299792458.0 * omega0 / 1.602176634e-19
    return e_unit / 5.14220674763e11, (1.0 / omega0) / 2.4188843265857e-17


M_CARBON = 12.0 * M_PROTON_ROUND   # carbon ions in m_e (nucleon mass taken as the proton's)
CARBON_IP_EV = (11.2603, 24.3833, 47.8878, 64.4939, 392.087, 489.993)   # C0 -> C1+ ... C5+ -> C6+


def carbon_foil(name: str, nx: int, ny: int, foil_x0: int, foil_cells: int, density_nc: float, ppc: int,
                steps: int, a0: float, seed: int, charge_states: int = 2, precision: int = PREC_FP64,
                tile: int = 8) -> RunConfig:
    """A laser foil of neutral carbon that ionises (species 0: electrons, 1: C0, 2..: C1+ ...), as the
    paper's targets do; the ion density is density_nc / 6 (fully ionised it gives density_nc electrons)."""
    cfg = laser_foil(name, nx, ny, foil_x0, foil_cells, density_nc, ppc, steps, a0, seed, precision, tile)
    n_ion = density_nc / 6.0
    cfg.species = ([Species(-1.0, 1.0, ppc, n_ion, 1.0)] +
                   [Species(float(z), M_CARBON, ppc, n_ion, 1.0) for z in range(charge_states + 1)])
    return cfg


def carbon_chains(charge_states: int = 2):
    """Ionisation chains of carbon_foil: (ion species, target species, electron species, potential in eV)."""
    return [(1 + z, 2 + z, 0, CARBON_IP_EV[z]) for z in range(charge_states)]


def laser_tau_fs_to_norm(tau_fs: float, wavelength_um: float) -> float:
    omega0 = 2.0 * math.pi * 299792458.0 / (wavelength_um * 1e-6)
    return tau_fs * 1e-15 * omega0


def uniform_plasma(name: str, n: int, ppc: int, steps: int, seed: int,
                   precision: int = PREC_FP64, tile: int = 16) -> RunConfig:
    """Periodic uniform e- + p plasma, n_e = 1, dx = dy = 0.02, dt = 0.5 (omega_pe units), 1 keV."""
    return RunConfig(
        name=name, nx=n, ny=n, dx=0.02, dy=0.02, dt=0.5, steps=steps,
        bc_x=BC_PERIODIC, field_mode=FIELD_CN, precision=precision,
        species=[Species(-1.0, 1.0, ppc, 1.0, 1.0), Species(1.0, M_PROTON_ROUND, ppc, 1.0, 1.0)],
        slab=None, tile_nx=tile, tile_ny=tile, seed=seed)


def laser_foil(name: str, nx: int, ny: int, foil_x0: int, foil_cells: int, density_nc: float,
               ppc: int, steps: int, a0: float, seed: int, precision: int = PREC_FP64,
               tile: int = 8) -> RunConfig:
    """Absorbing-x / periodic-y box, 0.8 um plane wave from x = 0, proton-electron foil.

    lambda/40 cells and dt = 0.01 lambda/c as in the paper's runs (Section 4);
    lengths in c/omega_0, so lambda = 2 pi.
    """
    lam = 2.0 * math.pi
    tau = laser_tau_fs_to_norm(30.0, 0.8)
    return RunConfig(
        name=name, nx=nx, ny=ny, dx=lam / 40.0, dy=lam / 40.0, dt=0.01 * lam, steps=steps,
        bc_x=BC_ABSORBING, field_mode=FIELD_LITERAL, precision=precision,
        species=[Species(-1.0, 1.0, ppc, density_nc, 1.0), Species(1.0, M_PROTON_ROUND, ppc, density_nc, 1.0)],
        slab=(foil_x0, foil_x0 + foil_cells),
        laser=Laser(a0=a0, omega=1.0, tau=tau, t0=tau, pol=0),
        tile_nx=tile, tile_ny=tile, seed=seed)


def config(idx: int) -> RunConfig:
    """The five workloads, by index 1..5 (5 returns one representative serving run)."""
    if idx == 1:
        return uniform_plasma("uniform-64x64-16ppc-cn", 64, 16, 50, seed=1234 + 1)
    if idx == 2:
        return laser_foil("laser-foil-1024x512-64ppc", 1024, 512, 150, 100, 100.0, 64, 1000, 5.0, seed=1234 + 2)
    if idx == 3:
        return laser_foil("laser-foil-4096x2048-4ppc", 4096, 2048, 150, 20, 50.0, 4, 500, 5.0, seed=1234 + 3)
    if idx == 4:
        return uniform_plasma("uniform-2048x2048-32ppc-cn", 2048, 32, 200, seed=1234 + 4,
                              precision=PREC_FP32, tile=16)
    if idx == 5:
        return serving_stream(1)[0][1]
    raise ValueError(idx)


def serving_stream(n_runs: int = 256, rate_per_s: float = 20.0, seed: int = 1234 + 5,
                   steps: int = 200) -> List[Tuple[float, RunConfig]]:
    """Poisson stream of independent laser-foil runs: (arrival time in s, config).

    Grids uniform in {64..512}^2 in steps of 64, 4-64 particles/cell/species,
    foil density 10-200 n_c, a0 1-20, foil round(nx/10) cells starting at
    x = 3 um (150 cells) or, in small boxes, centred.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n_runs):
        t += float(rng.exponential(1.0 / rate_per_s))
        nx = int(rng.integers(1, 9)) * 64
        ny = int(rng.integers(1, 9)) * 64
        ppc = int(rng.integers(4, 65))
        dens = float(rng.uniform(10.0, 200.0))
        a0 = float(rng.uniform(1.0, 20.0))
        thick = max(1, int(round(nx / 10)))
        x0 = min(150, (nx - thick) // 2)
        cfg = laser_foil(f"serve-{k}-{nx}x{ny}-{ppc}ppc", nx, ny, x0, thick, dens, ppc, steps, a0,
                         seed=seed * 1000 + k, precision=PREC_FP32, tile=8)
        out.append((t, cfg))
    return out


def generate_particles(cfg: RunConfig, seed: Optional[int] = None):
    """Initial macro-particles of every species, in cell-major order.

    Returns a list (one entry per species) of dicts with float64 arrays
    x, y, ux, uy, uz, w.  Cells are visited row by row (y outer, x inner),
    ppc particles each; positions are uniform in the cell, momenta Maxwellian
    (u_i = sqrt(T/(m c^2)) N(0,1)), and every species uses the same positions
    so that the initial charge density is zero where the species' charges
    cancel.  w = n dx dy / ppc (particles per unit length in z).
    """
    rng = np.random.default_rng(cfg.seed if seed is None else seed)
    x0, x1 = cfg.slab if cfg.slab is not None else (0, cfg.nx)
    ncx = x1 - x0
    ppc = cfg.species[0].ppc
    assert all(s.ppc == ppc for s in cfg.species), "species share positions, so ppc must agree"
    jj, ii = np.meshgrid(np.arange(cfg.ny, dtype=np.float64), np.arange(x0, x1, dtype=np.float64), indexing="ij")
    ci = np.repeat(ii.ravel(), ppc)
    cj = np.repeat(jj.ravel(), ppc)
    n = ci.size
    fx = rng.random(n)
    fy = rng.random(n)
    x = (ci + fx) * cfg.dx
    y = (cj + fy) * cfg.dy
    # keep every position strictly inside its drawn cell despite rounding
    Lx = cfg.nx * cfg.dx
    Ly = cfg.ny * cfg.dy
    x = np.minimum(x, np.nextafter(Lx, 0.0))
    y = np.minimum(y, np.nextafter(Ly, 0.0))
    out = []
    for s in cfg.species:
        uth = u_thermal(s.temperature_kev, s.m)
        u = rng.standard_normal((3, n)) * uth
        w = np.full(n, s.density * cfg.dx * cfg.dy / s.ppc)
        out.append(dict(x=x.copy(), y=y.copy(), ux=u[0].copy(), uy=u[1].copy(), uz=u[2].copy(), w=w))
    return out


def lattice_particles(cfg: RunConfig, species_idx: int, offsets=((0.25, 0.25),), drift=(0.0, 0.0, 0.0),
                      density: float = 1.0):
    """Cold lattice load: the same in-cell offsets in every cell, uniform drift."""
    pts = []
    for (ox, oy) in offsets:
        jj, ii = np.meshgrid(np.arange(cfg.ny), np.arange(cfg.nx), indexing="ij")
        pts.append(((ii.ravel() + ox) * cfg.dx, (jj.ravel() + oy) * cfg.dy))
    x = np.concatenate([p[0] for p in pts])
    y = np.concatenate([p[1] for p in pts])
    n = x.size
    w = np.full(n, density * cfg.dx * cfg.dy / len(offsets))
    return dict(x=x, y=y, ux=np.full(n, drift[0]), uy=np.full(n, drift[1]), uz=np.full(n, drift[2]), w=w)
