"""Spline shapes of degree 2, 3, 4 (the centred B-spline over the nearest (n + 1) x (n + 1) nodes,
PIC_SHAPE_QUADRATIC .. PIC_SHAPE_QUARTIC; the higher-order weightings up to fourth order of Section
3.3's last paragraph) on the GPU against the FP64 oracle with the same shape.

FP64 form: particle state within 1e-10, moments and fields within 1e-9 (normwise), cells and order
exact -- the laser foil with walls and the source, hot particles at both walls, a hot periodic
plasma in CN mode with tiles of 2 cells (the touched-tile map reaches two or more tiles).
FP32 form: the workload tolerances (1e-5).  Deterministic deposit: bitwise reproducible, and a run
resumed from a checkpoint continues bitwise in both forms (the deposit at rest and the push add the
same per-lane products).  Ionisation and batched steps refuse the shape."""
import numpy as np
import pytest

from paper_1308_2590_gb300 import pic, workloads as W
from tests.parity import compare_grid, compare_particles, density_scale, normwise, run_pair, stream
from tests.test_gpu_parity import hot, small_foil, small_uniform

pytestmark = pytest.mark.gpu


def _s2(cfg, order=2):
    cfg.shape = order
    return cfg


ORDERS = [2, 3, 4]


@pytest.mark.parametrize("order", ORDERS)
def test_spline_shape_literal_laser_foil_matches(order):
    cfg = _s2(small_foil(), order)
    g, o = run_pair(cfg, cfg.steps)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    # the shape matters: the linear-shape oracle's moments are far from these
    import oracle
    o1 = oracle.OracleSim.from_config(cfg.scaled(shape=1))
    for s, P in enumerate(W.generate_particles(cfg)):
        o1.load_particles(s, **P)
    o1.step(cfg.steps)
    assert normwise(g.pic_moments()[0], o1.M[0], density_scale(cfg)) > 1e-3
    dg, do = g.pic_diagnostics(), o.diagnostics()
    assert dg["count"] == do["count"] and dg["removed"] == do["removed"]
    for k in ("kinetic", "field"):
        assert abs(dg[k] - do[k]) <= 1e-9 * abs(do[k]) + 1e-15, (k, dg[k], do[k])
    g.close()


@pytest.mark.parametrize("order", ORDERS)
def test_spline_shape_hot_particles_at_both_walls(order):
    cfg = _s2(small_foil(nx=40, ny=16, ppc=4, steps=8, a0=0.0), order)
    cfg.slab = (0, 40)
    cfg.species = [W.Species(-1.0, 1.0, 4, 5.0, 200.0), W.Species(1.0, 1836.0, 4, 5.0, 1.0)]
    g, o = run_pair(cfg, cfg.steps)
    dg, do = g.pic_diagnostics(), o.diagnostics()
    assert do["removed"] > 0
    assert dg["removed"] == do["removed"] and dg["count"] == do["count"]
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    g.close()


@pytest.mark.parametrize("order,tile", [(2, 2), (2, 8), (3, 2), (4, 2), (4, 8)])
def test_spline_shape_cn_periodic_plasma_matches(order, tile):
    cfg = _s2(hot(small_uniform(tile=tile), 20.0), order)
    g, o = run_pair(cfg, 6)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    g.close()


@pytest.mark.parametrize("order", ORDERS)
def test_spline_shape_fp32_form_within_targets(order):
    cfg = _s2(small_foil(precision=W.PREC_FP32), order)
    g, o = run_pair(cfg, cfg.steps)
    Mg, Mo = g.pic_moments(), o.M
    assert normwise(Mg[0], Mo[0], density_scale(cfg)) < 1e-5
    assert normwise(Mg[1:10], Mo[1:10]) < 1e-5 and normwise(Mg[10:13], Mo[10:13]) < 1e-5
    Lx = cfg.nx * cfg.dx
    for s in range(len(cfg.species)):
        a, b = g.pic_get_particles(s), o.particles(s)
        assert a["x"].size == b["x"].size
        assert np.max(np.abs(a["x"] - b["x"])) / Lx < 1e-5
        us = max(np.max(np.abs(b[k])) for k in ("ux", "uy", "uz"))
        assert max(normwise(a[k], b[k], us) for k in ("ux", "uy", "uz")) < 1e-5
    dg, do = g.pic_diagnostics(), o.diagnostics()
    assert dg["count"] == do["count"] and abs(dg["total"] - do["total"]) <= 1e-3 * abs(do["total"])
    g.close()


def _state(g, nsp):
    out = [g.pic_moments(), *g.pic_fields()]
    for s in range(nsp):
        P = g.pic_save_particles(s)
        out += [P[k] for k in ("cell", "ox", "oy", "ux", "uy", "uz", "w")]
    return out


def _equal(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x.shape == y.shape and np.array_equal(x.view(np.uint8), y.view(np.uint8))


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32])
def test_spline_shape_deterministic_reproducible_and_resumes_bitwise(precision, order):
    cfg = _s2(small_foil(precision=precision), order)
    cfg.laser.t0 = 2.0
    cfg.deposit = W.DEPOSIT_DETERMINISTIC
    parts = W.generate_particles(cfg)
    nsp = len(parts)
    k, total = 5, 10
    runs = []
    for _ in range(2):
        whole = pic.Pic(cfg, stream=stream())
        whole.pic_load_species(parts)
        whole.pic_step(total)
        runs.append(_state(whole, nsp))
        whole.close()
    _equal(runs[0], runs[1])
    first = pic.Pic(cfg, stream=stream())
    first.pic_load_species(parts)
    first.pic_step(k)
    E, H = first.pic_fields()
    saved = [first.pic_save_particles(s) for s in range(nsp)]
    first.close()
    resumed = pic.Pic(cfg, stream=stream())
    for s, P in enumerate(saved):
        resumed.pic_restore_particles(s, P)
    resumed.pic_set_fields(E, H)
    resumed.pic_set_step(k)
    resumed.pic_step(total - k)
    _equal(runs[0], _state(resumed, nsp))
    resumed.close()


@pytest.mark.parametrize("order", ORDERS)
def test_spline_shape_deterministic_matches_oracle(order):
    cfg = _s2(small_foil(), order)
    cfg.deposit = W.DEPOSIT_DETERMINISTIC
    g, o = run_pair(cfg, cfg.steps)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    g.close()


def test_spline_shape_refused_by_ionisation_and_batched_steps():
    cfg = _s2(small_foil(steps=1))
    g = pic.Pic(cfg, stream=stream())
    g.pic_load_species(W.generate_particles(cfg))
    with pytest.raises(pic.PicError, match="shape"):
        g.pic_ionize([(1, 0, 0, 11.26)], 1, 1.0, 1.0)
    b = pic.Batch(4, stream=stream())
    with pytest.raises(pic.PicError, match="shape"):
        b.step([g], 1)
    b.close()
    g.close()
