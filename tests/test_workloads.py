"""The seeded synthetic inputs match their stated recipes (CPU only).

Every workload is synthetic: the paper's runs (Section 4) are not a public
dataset.  These tests pin the generator to the recipe each workload states:
grid, step, boundaries, species, particle counts, thermal spreads, the foil's
place and the laser's timing (40 cells per wavelength and dt = 0.01 lambda/c as
in Section 4), the serving stream's distributions, and the properties both
sides rely on (zero initial charge density, weights, reproducibility).
"""
import math

import numpy as np
import pytest

from paper_1308_2590_gb300 import workloads as W


def test_uniform_plasma_64x64():
    c = W.config(1)
    assert (c.nx, c.ny, c.dx, c.dy, c.dt, c.steps) == (64, 64, 0.02, 0.02, 0.5, 50)
    assert c.bc_x == W.BC_PERIODIC and c.field_mode == W.FIELD_CN and c.slab is None
    e, p = c.species
    assert (e.q, e.m, p.q, p.m) == (-1.0, 1.0, 1.0, 1836.0)
    assert e.ppc == p.ppc == 16 and e.density == p.density == 1.0
    assert c.n_particles == 131072
    # 1 keV: u_th = sqrt(T / (m c^2)) with m_e c^2 = 511.0 keV
    assert W.u_thermal(e.temperature_kev, e.m) == pytest.approx(0.04424, rel=1e-3)
    assert W.u_thermal(p.temperature_kev, p.m) == pytest.approx(0.001032, rel=1e-3)


def test_laser_foil_1024x512():
    c = W.config(2)
    lam = 2.0 * math.pi                       # lengths in c / omega_0
    assert (c.nx, c.ny, c.steps) == (1024, 512, 1000)
    assert c.dx == pytest.approx(lam / 40) and c.dy == pytest.approx(lam / 40)
    assert c.dt == pytest.approx(0.01 * lam)
    assert c.bc_x == W.BC_ABSORBING and c.field_mode == W.FIELD_LITERAL
    assert c.slab == (150, 250)               # 3 um from x = 0 at 0.8 um / 40 per cell, 100 cells thick
    assert all(s.density == 100.0 and s.ppc == 64 for s in c.species)
    assert c.n_particles == 6553600
    # 30 fs intensity FWHM of a 0.8 um wave, in 1/omega_0; the envelope peaks one tau in
    omega0 = 2.0 * math.pi * 299792458.0 / 0.8e-6
    assert c.laser.tau == pytest.approx(30e-15 * omega0) and c.laser.t0 == c.laser.tau
    assert c.laser.a0 == 5.0 and c.laser.omega == 1.0


def test_laser_foil_4096x2048_and_uniform_2048():
    c3 = W.config(3)
    assert (c3.nx, c3.ny, c3.steps, c3.slab) == (4096, 2048, 500, (150, 170))
    assert all(s.density == 50.0 and s.ppc == 4 for s in c3.species)
    assert c3.n_particles == 327680
    c4 = W.config(4)
    assert (c4.nx, c4.ny, c4.steps, c4.field_mode, c4.precision) == (2048, 2048, 200, W.FIELD_CN, W.PREC_FP32)
    assert c4.n_particles == 268435456


def test_serving_stream_distributions():
    runs = W.serving_stream()
    assert len(runs) == 256
    t = np.array([a for a, _ in runs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    # exponential inter-arrivals at 20/s: mean 0.05 s (256 draws: standard error 0.05/16)
    assert abs(gaps.mean() - 0.05) < 4 * 0.05 / 16
    sizes = set()
    for _, c in runs:
        assert c.nx in range(64, 513, 64) and c.ny in range(64, 513, 64)
        sizes.add((c.nx, c.ny))
        s = c.species[0]
        assert 4 <= s.ppc <= 64 and 10.0 <= s.density <= 200.0 and 1.0 <= c.laser.a0 <= 20.0
        thick = max(1, round(c.nx / 10))
        x0 = min(150, (c.nx - thick) // 2)
        assert c.slab == (x0, x0 + thick) and c.slab[1] <= c.nx
        assert c.steps == 200 and c.precision == W.PREC_FP32
        assert c.n_particles <= 3_400_000
    assert len(sizes) > 30                      # the 64 grid shapes are well spread
    assert W.serving_stream() == runs          # seeded


def test_generated_particles_follow_the_recipe():
    c = W.config(2).scaled(ny=16)              # the foil of the 1024x512 workload, 16 rows
    parts = W.generate_particles(c)
    e, p = parts
    n = c.n_particles // 2
    for P in parts:
        assert all(P[k].shape == (n,) and P[k].dtype == np.float64 for k in ("x", "y", "ux", "uy", "uz", "w"))
    # electrons and ions share positions: zero charge density at t = 0
    assert np.array_equal(e["x"], p["x"]) and np.array_equal(e["y"], p["y"])
    cx = np.floor(e["x"] / c.dx).astype(int)
    cy = np.floor(e["y"] / c.dy).astype(int)
    assert cx.min() == 150 and cx.max() == 249 and cy.min() == 0 and cy.max() == 15
    counts = np.bincount((cy * c.nx + cx), minlength=c.nx * c.ny).reshape(c.ny, c.nx)
    assert np.all(counts[:, 150:250] == 64) and counts.sum() == n
    # weight: density x cell area / particles per cell
    assert np.all(e["w"] == 100.0 * c.dx * c.dy / 64)
    # Maxwellian momenta with the species' thermal spread (n = 102,400 draws per component)
    for P, s in zip(parts, c.species):
        uth = W.u_thermal(s.temperature_kev, s.m)
        u = np.stack([P["ux"], P["uy"], P["uz"]])
        assert np.all(np.abs(u.mean(axis=1)) < 5 * uth / math.sqrt(n))
        assert np.all(np.abs(u.std(axis=1) / uth - 1.0) < 0.02)
    # seeded: the same seed gives the same particles, another seed others
    again = W.generate_particles(c)
    assert all(np.array_equal(a[k], b[k]) for a, b in zip(parts, again) for k in a)
    other = W.generate_particles(c, seed=c.seed + 1)
    assert not np.array_equal(other[0]["x"], e["x"])
