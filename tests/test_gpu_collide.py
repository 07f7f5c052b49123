"""Binary-collision pass on the GPU (pic_collide) against the oracle's (oracle/collide.py): the same
pairs in the same order with the same Philox draws, so in the FP64 form every particle's u after a
pass matches the oracle's to rounding (1e-12 relative to the largest |u|) and the redeposited
moments to 1e-9; the FP32 form within its 1e-5; the pass conserves momentum and the kinetic energy
sum m |u|^2 / 2 (equal weights); steps after a pass still match the oracle.  Cases: like-particle
collisions with odd and even cell counts, electron-ion pairs with either species driving, a hot
laser foil (several species and collision entries at once), empty species."""
import numpy as np
import pytest

import oracle
from oracle import collide as ocol
from paper_1308_2590_gb300 import pic, workloads as W
from tests.parity import compare_grid, compare_particles, density_scale, normwise, run_pair, stream
from tests.test_gpu_parity import hot, small_foil, small_uniform

pytestmark = pytest.mark.gpu

KAPPA = 2.2e-5     # a large collision strength, so that a pass moves particles visibly
LNL = 10.0


def _u(P):
    return np.stack([P["ux"], P["uy"], P["uz"]])


def _compare_u(g, o, nsp, rtol):
    for s in range(nsp):
        a, b = g.pic_get_particles(s), o.particles(s)
        assert a["x"].size == b["x"].size
        # the order: weights equal (FP64) or equal to FP32 rounding (the FP32 form stores w in FP32)
        assert np.array_equal(a["w"], b["w"]) if rtol < 1e-9 else np.allclose(a["w"], b["w"], rtol=1e-7, atol=0)
        if a["x"].size:
            assert normwise(_u(a), _u(b)) < rtol, (s, normwise(_u(a), _u(b)))


@pytest.mark.parametrize("pairs", [[(0, 0)], [(0, 1)], [(1, 0)], [(0, 0), (1, 1), (0, 1)]])
def test_collision_pass_matches_oracle_fp64(pairs):
    cfg = hot(small_uniform(ppc=7, tile=8), 5.0)     # 7 per cell: odd counts and the triple rule
    cfg.species[1] = W.Species(1.0, 4.0, 7, cfg.species[1].density, 5.0)   # light ions
    parts = W.generate_particles(cfg)
    keep = np.random.default_rng(8).random(parts[0]["x"].size) < 0.7    # fewer electrons: ions drive somewhere
    parts[0] = {k: np.ascontiguousarray(v[keep]) for k, v in parts[0].items()}
    g, o = run_pair(cfg, 2, parts=parts)
    n_g = g.pic_collide(pairs, 11, LNL, KAPPA)
    n_o = ocol.collide(o, pairs, 11, LNL, KAPPA)
    assert n_g == n_o > 0
    _compare_u(g, o, len(cfg.species), 1e-12)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    # and the run goes on equal
    g.pic_step(2)
    o.step(2)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    g.close()


def test_collision_pass_conserves_momentum_and_energy():
    cfg = hot(small_uniform(ppc=9, tile=8), 20.0)
    parts = W.generate_particles(cfg)
    for P in parts:
        P["w"] = np.full(P["w"].size, P["w"][0])      # equal weights: every pair conserves exactly
    g = pic.Pic(cfg, stream=stream())
    g.pic_load_species(parts)
    masses = [s.m for s in cfg.species]

    def totals():
        p = np.zeros(3)
        e = 0.0
        for s, m in enumerate(masses):
            P = g.pic_get_particles(s)
            u = _u(P)
            p += m * P["w"][0] * u.sum(axis=1)
            e += 0.5 * m * P["w"][0] * np.sum(u * u)
        return p, e

    p0, e0 = totals()
    g.pic_collide([(0, 0), (1, 1), (0, 1)], 3, LNL, 100 * KAPPA)
    p1, e1 = totals()
    assert np.max(np.abs(p1 - p0)) < 1e-12 * e0 ** 0.5 * 10 and abs(e1 - e0) < 1e-12 * e0
    g.close()


def test_collision_pass_on_the_laser_foil_matches_and_fp32_within_targets():
    cfg = small_foil(steps=3)
    g, o = run_pair(cfg, 3)
    pairs = [(0, 0), (0, 1), (1, 1)]
    assert g.pic_collide(pairs, 5, LNL, KAPPA) == ocol.collide(o, pairs, 5, LNL, KAPPA)
    _compare_u(g, o, 2, 1e-12)
    g.close()
    cfg32 = small_foil(steps=3, precision=W.PREC_FP32)
    g, o = run_pair(cfg32, 3)
    g.pic_collide(pairs, 5, LNL, KAPPA)
    ocol.collide(o, pairs, 5, LNL, KAPPA)
    _compare_u(g, o, 2, 1e-5)
    Mg, Mo = g.pic_moments(), o.M
    assert normwise(Mg[0], Mo[0], density_scale(cfg32)) < 1e-5 and normwise(Mg[10:13], Mo[10:13]) < 1e-5
    g.close()


def test_collision_pass_with_an_empty_species_and_bad_arguments():
    cfg = small_uniform(tile=8)
    parts = W.generate_particles(cfg)
    parts[1] = {k: v[:0] for k, v in parts[1].items()}
    g = pic.Pic(cfg, stream=stream())
    g.pic_load_species(parts)
    assert g.pic_collide([(0, 1), (1, 1)], 1, LNL, KAPPA) == 0
    with pytest.raises(pic.PicError):
        g.pic_collide([(0, 5)], 1, LNL, KAPPA)
    with pytest.raises(pic.PicError):
        g.pic_collide([(0, 0)], 1, -1.0, KAPPA)
    g.close()
