"""GPU (through the C ABI) versus the FP64 CPU oracle on the same seeded inputs.

FP64 form: particle state within 1e-10 relative, moments and fields within
1e-9 relative (normwise, see tests/parity.py), cells and particle order exact.
Cases span several tiles with ragged tails, empty and single-particle inputs,
particles leaving through walls, multi-cell moves and both field modes.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1308_2590_gb300 import pic, workloads as W
from tests.parity import (compare_grid, compare_particles, density_scale, normwise, run_pair, stream)

pytestmark = pytest.mark.gpu


def small_foil(nx=70, ny=37, ppc=6, tile=8, steps=12, a0=3.0, precision=W.PREC_FP64):
    cfg = W.laser_foil("foil-small", nx, ny, 3, 17, 40.0, ppc, steps, a0, seed=77, precision=precision, tile=tile)
    # a short pulse so that it reaches the foil within the test
    cfg.laser.tau = 6.0
    cfg.laser.t0 = 6.0
    return cfg


def small_uniform(n=24, ppc=5, tile=8, field_mode=W.FIELD_CN, dt=0.5, precision=W.PREC_FP64):
    cfg = W.uniform_plasma("uniform-small", n, ppc, 10, seed=99, precision=precision, tile=tile)
    cfg.ny = n - 5      # ragged: not a multiple of the tile
    cfg.field_mode = field_mode
    cfg.dt = dt
    cfg.cn_tol = 1e-14
    cfg.cn_max_iter = 2000
    return cfg


def hot(cfg, kev):
    cfg.species = [W.Species(s.q, s.m, s.ppc, s.density, kev) for s in cfg.species]
    return cfg


def test_load_order_and_initial_moments_match():
    cfg = hot(small_uniform(), 50.0)
    rng = np.random.default_rng(5)
    ny, nx = cfg.ny, cfg.nx
    H = rng.standard_normal((3, ny, nx)) * 0.3
    E = rng.standard_normal((3, ny, nx)) * 0.1
    g, o = run_pair(cfg, 0, fields=(E, H))
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    d = g.pic_diagnostics()
    assert abs(d["charge_grid"] - o.diagnostics()["charge_grid"]) < 1e-12 * density_scale(cfg) * nx * ny * cfg.dx * cfg.dy
    g.close()


def test_literal_laser_foil_steps_match():
    cfg = small_foil()
    g, o = run_pair(cfg, cfg.steps)
    compare_particles(g, o, cfg)
    errs = compare_grid(g, o, rho_scale=density_scale(cfg))
    dg, do = g.pic_diagnostics(), o.diagnostics()
    assert dg["count"] == do["count"] and dg["removed"] == do["removed"]
    for k in ("kinetic", "field"):
        assert abs(dg[k] - do[k]) <= 1e-9 * abs(do[k]) + 1e-15, (k, dg[k], do[k])
    g.close()


def test_literal_walls_remove_fast_particles():
    """Hot electrons next to both walls: removals counted identically, survivors match."""
    cfg = small_foil(nx=40, ny=16, ppc=4, steps=8, a0=0.0)
    cfg.slab = (0, 40)
    cfg.species = [W.Species(-1.0, 1.0, 4, 5.0, 200.0), W.Species(1.0, 1836.0, 4, 5.0, 1.0)]
    g, o = run_pair(cfg, cfg.steps)
    dg, do = g.pic_diagnostics(), o.diagnostics()
    assert do["removed"] > 0
    assert dg["removed"] == do["removed"] and dg["count"] == do["count"]
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    g.close()


@pytest.mark.parametrize("tile", [4, 8])
def test_cn_uniform_plasma_steps_match(tile):
    """Time-centred field mode at c dt / dx = 25 (the uniform-plasma workloads), multi-cell moves."""
    cfg = hot(small_uniform(tile=tile), 30.0)
    g, o = run_pair(cfg, 6)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    d = g.pic_diagnostics()
    assert d["cn_residual"] < 1e-12, d
    g.close()


def test_uniform_plasma_workload_full_size_matches():
    """The 64x64, 16 particles/cell/species uniform workload, 10 of its 50 steps."""
    cfg = W.config(1).scaled(cn_tol=1e-14, cn_max_iter=2000)
    g, o = run_pair(cfg, 10)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    dg, do = g.pic_diagnostics(), o.diagnostics()
    assert abs(dg["total"] - do["total"]) <= 1e-9 * abs(do["total"])
    g.close()


def wall_edge_particles(cfg, moving=False):
    """Particles at x = nextafter(Lx, 0) (x/dx rounds to nx), one at x = 0 and one inside, in a walled
    box.  At rest (with no laser every field stays exactly zero, so nobody moves), or, with moving set,
    the two at the far wall drifting inward fast enough to leave the wall cell in one step (a particle
    left at the wall edge with a tiny outward push is removed or kept by rounding alone)."""
    Lx = cfg.nx * cfg.dx
    top = np.nextafter(Lx, 0.0)
    ux = np.array([-0.3, -0.2, 0.0, 0.1]) if moving else np.zeros(4)
    P = dict(x=np.array([top, top, 0.0, 0.5 * Lx]), y=np.array([0.3, 2.1, 1.0, 4.0]) * cfg.dy,
             ux=ux, uy=np.zeros(4), uz=np.zeros(4), w=np.full(4, 0.5))
    return [P, {k: v[:0] for k, v in P.items()}]


@pytest.mark.parametrize("moving", [False, True])
@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32])
def test_particle_just_inside_the_far_wall(precision, moving):
    """Reading 18 at a wall: x < Lx whose x/dx rounds to nx lies in the last cell at the largest offset
    below 1 of the form's precision.  Such a particle is kept (by the oracle and by both forms, which
    the checks build also accepts: tests/checks_run.py), deposits on the wall node, and moves off it."""
    cfg = small_foil(nx=20, ny=8, ppc=1, steps=3, a0=0.0, precision=precision)
    g, o = run_pair(cfg, 3, parts=wall_edge_particles(cfg, moving))
    dg, do = g.pic_diagnostics(), o.diagnostics()
    assert dg["count"] == do["count"] == 4 and dg["removed"] == do["removed"] == 0
    assert not (dg["flags"] & 32)
    rs = 0.5 / (cfg.dx * cfg.dy)
    if precision == W.PREC_FP64:
        compare_particles(g, o, cfg)
        compare_grid(g, o, rho_scale=rs)
    else:
        compare_particles(g, o, cfg, rtol=1e-5)
        compare_grid(g, o, rtol=1e-5, rho_scale=rs)
    g.close()


@pytest.mark.slow
def test_field_dominated_workload_full_size_matches():
    """The field-dominated laser foil at full size (4096x2048 cells, 20-cell foil at 50 n_c,
    4 particles/cell/species: 327,680 particles; walls, laser, literal solve), 4 steps: every
    particle, node and cell against the oracle.  Almost every tile is vacuum, so this covers the
    field solve's vacuum path and the clear of only the tiles the deposit touched."""
    cfg = W.config(3)
    g, o = run_pair(cfg, 4)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    dg, do = g.pic_diagnostics(), o.diagnostics()
    assert dg["count"] == do["count"] and dg["removed"] == do["removed"]
    for k in ("kinetic", "field"):
        assert abs(dg[k] - do[k]) <= 1e-9 * abs(do[k]) + 1e-15, (k, dg[k], do[k])
    g.close()


def test_particles_entering_vacuum_tiles_match():
    """A hot thin foil in a wide walled box: particles leave the occupied tiles each step, so the
    tiles whose moments are cleared and solved in full change every step (tile 4, 16 steps)."""
    cfg = small_foil(nx=96, ny=24, ppc=4, tile=4, steps=16, a0=2.0)
    cfg.slab = (44, 48)
    cfg.species = [W.Species(-1.0, 1.0, 4, 20.0, 300.0), W.Species(1.0, 1836.0, 4, 20.0, 5.0)]
    g, o = run_pair(cfg, cfg.steps)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    g.close()


def test_empty_and_single_particle():
    cfg = small_foil(nx=20, ny=8, ppc=1, steps=3, a0=1.0)
    empty = [dict(x=np.zeros(0), y=np.zeros(0), ux=np.zeros(0), uy=np.zeros(0), uz=np.zeros(0), w=np.zeros(0))] * 2
    g, o = run_pair(cfg, 3, parts=empty)
    compare_grid(g, o, rho_scale=1.0)
    assert g.pic_diagnostics()["count"] == 0
    g.close()
    one = [dict(x=np.array([1.0 * cfg.dx * 7.3]), y=np.array([cfg.dy * 3.9]), ux=np.array([0.5]),
                uy=np.array([-0.2]), uz=np.array([0.1]), w=np.array([0.7])),
           dict(x=np.zeros(0), y=np.zeros(0), ux=np.zeros(0), uy=np.zeros(0), uz=np.zeros(0), w=np.zeros(0))]
    g, o = run_pair(cfg, 3, parts=one)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=1.0)
    g.close()


def test_particles_on_cell_and_tile_edges():
    """Particles placed exactly on node lines, tile borders and the periodic seam."""
    cfg = small_uniform(n=16, ppc=1, tile=4, field_mode=W.FIELD_LITERAL, dt=0.01)
    xs = np.array([0.0, 4 * cfg.dx, 8 * cfg.dx, 15.5 * cfg.dx, 3.999999 * cfg.dx])
    ys = np.array([0.0, 4 * cfg.dy, 10.25 * cfg.dy, 0.5 * cfg.dy, 7.0 * cfg.dy])
    P = dict(x=xs, y=ys, ux=np.array([0.3, -0.3, 0.0, 0.9, 0.01]), uy=np.array([0.0, 0.2, -0.6, 0.0, 0.0]),
             uz=np.zeros(5), w=np.array([1.0, 1.5, 2.0, 0.5, 0.25]))
    g, o = run_pair(cfg, 5, parts=[P, dict((k, v[:0]) for k, v in P.items())])
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=1.0 / (cfg.dx * cfg.dy))
    g.close()


@pytest.mark.parametrize("field_mode,dt,ny", [(W.FIELD_LITERAL, 0.5, 12), (W.FIELD_CN, 3.0, 12), (W.FIELD_CN, 3.0, 16)])
def test_vacuum_dispersion_on_gpu(field_mode, dt, ny):
    """Pin P5 through the GPU path: one eigenmode, exact discrete phase per step
    (CN on 16x16 runs the spectral preconditioner, on 16x12 block-Jacobi)."""
    nx, dx, dy = 16, 1.0, 0.8
    cfg = W.RunConfig(name="vac", nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, steps=20, field_mode=field_mode,
                      species=[W.Species(-1.0, 1.0, 1, 1.0, 0.0)], tile_nx=4, tile_ny=4, cn_tol=1e-14,
                      cn_max_iter=500)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    E0 = np.zeros((3, ny, nx))
    E0[2] = np.cos(2 * np.pi * (2 * ii / nx + 3 * jj / ny))
    with pic.Pic(cfg, stream=stream()) as g:
        g.pic_set_fields(E0, np.zeros((3, ny, nx)))
        a, b = math.pi * 2 / nx, math.pi * 3 / ny
        keff = math.sqrt(4 * (math.sin(a) ** 2 * math.cos(b) ** 2 / dx ** 2 + math.cos(a) ** 2 * math.sin(b) ** 2 / dy ** 2))
        th = dt * keff / 2
        cos_wdt = 1 - 2 * th * th if field_mode == W.FIELD_LITERAL else (1 - th * th) / (1 + th * th)
        amps = [1.0]
        for _ in range(20):
            g.pic_step(1)
            E, _ = g.pic_fields()
            amp = np.sum(E[2] * E0[2]) / np.sum(E0[2] ** 2)
            assert np.max(np.abs(E[2] - amp * E0[2])) < 1e-11
            amps.append(amp)
        a_ = np.array(amps)
        n = np.arange(1, len(a_) - 1)
        big = np.abs(a_[n]) > 0.2
        c = (a_[n + 1] + a_[n - 1])[big] / a_[n][big]
        assert np.max(np.abs(c - 2 * cos_wdt)) < 1e-10
        if field_mode == W.FIELD_CN and ny == 16:
            # in vacuum the spectral preconditioner is the exact inverse
            assert g.pic_diagnostics()["cn_iterations"] <= 6


def test_bad_inputs_are_rejected():
    cfg = small_foil(nx=20, ny=8, ppc=1, steps=1)
    with pic.Pic(cfg, stream=stream()) as g:
        with pytest.raises(pic.PicError):
            g.pic_load_particles(0, [cfg.nx * cfg.dx + 1.0], [0.1], [0], [0], [0], [1.0])
        with pytest.raises(pic.PicError):
            g.pic_load_particles(5, [0.1], [0.1], [0], [0], [0], [1.0])
        assert g.pic_particle_count(0) == 0
    bad = small_foil(nx=20, ny=8, ppc=1, steps=1)
    bad.tile_nx = 200             # tiles of at most 128 cells a side
    with pytest.raises(pic.PicError):
        pic.Pic(bad, stream=stream())


@pytest.mark.parametrize("cdt", [0.4, 2.0])
def test_cn_laser_foil_with_walls_matches(cdt):
    """The implicit-curl field solve in a box with walls (Mur condition in the wall nodes' y and z rows,
    the laser injected through the x = 0 wall): laser foil at the paper's c dt/dx = 0.4 and at 2 (where
    the leapfrog curls of Eqs. 4-5 are unstable), 12 steps, every particle, node and cell against the
    oracle; the solver reaches the FP64 tolerance in a few block-Jacobi iterations per step."""
    cfg = small_foil(a0=4.0)
    cfg.field_mode = W.FIELD_CN
    cfg.dt = cdt * cfg.dx
    cfg.cn_tol = 1e-13
    cfg.cn_max_iter = 2000
    g, o = run_pair(cfg, cfg.steps)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    dg, do = g.pic_diagnostics(), o.diagnostics()
    assert dg["count"] == do["count"] and dg["removed"] == do["removed"]
    for k in ("kinetic", "field"):
        assert abs(dg[k] - do[k]) <= 1e-9 * abs(do[k]) + 1e-15, (k, dg[k], do[k])
    assert dg["cn_residual"] < 1e-12, dg
    assert 0 < dg["cn_iterations"] <= 60, dg
    g.close()


@pytest.mark.slow
def test_laser_foil_workload_full_size_matches():
    """The 1024x512, 6.55M-particle laser-foil workload: 3 full steps, every particle and node compared."""
    cfg = W.config(2)
    g, o = run_pair(cfg, 3)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    g.close()


def test_regroup_overflow_and_far_moves_fall_back_to_full_sort():
    """A dense beam leaves its tile for an empty neighbour (bin overflow) and a few fast
    particles cross more than one tile: the order and state must still match the oracle."""
    cfg = small_uniform(n=32, ppc=1, tile=4, field_mode=W.FIELD_LITERAL, dt=0.01)
    cfg.ny = 32
    cfg.dx = cfg.dy = 0.02
    n = 400
    rng = np.random.default_rng(3)
    x = (1.0 + 2.0 * rng.random(n)) * cfg.dx          # all in cells 1..2 of tile (0, 0)
    y = (0.5 + 3.0 * rng.random(n)) * cfg.dy
    ux = np.full(n, 3.0)                               # ~2.8 cells per step: into tile (1, 0)
    ux[:5] = 40.0                                      # ~5 cells per step: two tiles away
    P = dict(x=x, y=y, ux=ux, uy=0.01 * rng.standard_normal(n), uz=np.zeros(n), w=np.full(n, 0.01))
    empty = dict((k, v[:0]) for k, v in P.items())
    g, o = run_pair(cfg, 4, parts=[P, empty])
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=1.0)
    # the full regroup (decided on the device) ran in the steps whose tile regroup could not place everyone
    assert g.pic_diagnostics()["full_regroups"] >= 1
    g.close()


@pytest.mark.parametrize("maker,tile", [("foil", 8), ("uniform", 4), ("uniform", 16)])
def test_per_step_cell_order_matches_oracle(maker, tile):
    """Every step sorts each tile's particles by cell, stayers before arrivals
    inside a cell; a hot plasma makes many particles change cell and tile."""
    if maker == "foil":
        cfg = small_foil(steps=8, tile=tile)
    else:
        cfg = hot(small_uniform(tile=tile), 30.0)
    g, o = run_pair(cfg, 7)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    for s in range(len(cfg.species)):
        P = g.pic_get_particles(s)
        cx = P["cell"] % cfg.nx
        cy = P["cell"] // cfg.nx
        t = (cy // cfg.tile_ny) * (-(-cfg.nx // cfg.tile_nx)) + cx // cfg.tile_nx
        key = t * (cfg.tile_nx * cfg.tile_ny) + (cy % cfg.tile_ny) * cfg.tile_nx + cx % cfg.tile_nx
        assert np.all(np.diff(key) >= 0)
    g.close()


@pytest.mark.parametrize("nx,ny", [(32, 16), (64, 32)])
def test_cn_spectral_preconditioner_matches_oracle(nx, ny):
    """Power-of-two periodic grids: the CN solve runs BiCGSTAB with the FFT
    preconditioner; the result matches the oracle's sparse LU solve, in far
    fewer inner iterations than the block-Jacobi form needs."""
    cfg = hot(small_uniform(tile=8), 20.0)
    cfg.nx, cfg.ny = nx, ny
    g, o = run_pair(cfg, 6)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    d = g.pic_diagnostics()
    assert d["cn_residual"] < 1e-12   # the target 1e-14 sits at the FP64 rounding floor of the residual
    assert d["cn_iterations"] <= 40, d
    g.close()
