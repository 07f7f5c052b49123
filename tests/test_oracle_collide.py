"""Pins of the oracle's binary-collision pass (oracle/collide.py; Takizuka and Abe's model, the reading
for the collisions the paper names beside ionisation, Sections 4-5).

Pinned against what mechanics and the kinetic theory of a Lorentz gas fix: every pair conserves
momentum and kinetic energy m |u|^2 / 2 exactly and keeps |g|; the angle between g and g' is the
2 atan|delta| of the pair's draws (taken here from numpy's Philox, an independent generator); a cold
electron beam crossing cold heavy ions slows at the textbook momentum-transfer rate
nu = n Z^2 e^4 lnL / (4 pi eps0^2 m^2 v^3) (converted here to the code's units); like-particle
collisions isotropise an anisotropic plasma with its momentum and energy unchanged.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import collide as col
from paper_1308_2590_gb300 import workloads as W


def _philox_uniforms(index, spec, step, seed):
    # numpy's Philox(counter=c) produces its first block from c + 1 (a 256-bit increment: at index 0 the
    # carry reaches the second word)
    c0 = (index - 1) % 2 ** 64
    c1 = 16 + spec - (1 if index == 0 else 0)
    bg = np.random.Philox(key=np.array([seed, 0], dtype=np.uint64),
                          counter=np.array([c0, c1, step, 1], dtype=np.uint64))
    return [float(int(v) >> 11) * 2.0 ** -53 for v in bg.random_raw(4)]


def test_draws_match_numpys_philox():
    for idx, spec, step, seed in [(0, 0, 0, 1), (12345, 2, 17, 99), (2 ** 40 + 3, 5, 1000, 2 ** 61)]:
        assert col.draws(idx, spec, step, seed) == _philox_uniforms(idx, spec, step, seed)


def test_pair_conserves_momentum_energy_and_relative_speed():
    rng = np.random.default_rng(21)
    for _ in range(200):
        m1, m2 = rng.choice([1.0, 1836.0, 7.3]), rng.choice([1.0, 12.0 * 1836])
        q1, q2 = rng.choice([-1.0, 1.0, 3.0]), rng.choice([-1.0, 2.0])
        u1, u2 = rng.standard_normal(3) * 0.05, rng.standard_normal(3) * 0.01
        v = list(rng.random(4))
        n1, n2 = col.scatter(u1, u2, m1, m2, q1, q2, 1.0, 1.0, 50.0, 0.5, 10.0, 1e-4, v)
        p0 = m1 * u1 + m2 * u2
        assert np.max(np.abs(m1 * n1 + m2 * n2 - p0)) < 1e-14 * (np.max(np.abs(m1 * u1)) + np.max(np.abs(m2 * u2)))
        e0 = 0.5 * m1 * u1 @ u1 + 0.5 * m2 * u2 @ u2
        e1 = 0.5 * m1 * n1 @ n1 + 0.5 * m2 * n2 @ n2
        assert abs(e1 - e0) < 1e-13 * e0
        assert abs(np.linalg.norm(n1 - n2) - np.linalg.norm(u1 - u2)) < 1e-13 * np.linalg.norm(u1 - u2)


def test_scattering_angle_is_that_of_the_draws():
    """cos(g, g') = (1 - delta^2) / (1 + delta^2) with delta from the Box-Muller of the pair's draws."""
    rng = np.random.default_rng(22)
    for k in range(100):
        u1, u2 = rng.standard_normal(3) * 0.03, rng.standard_normal(3) * 0.03
        v = _philox_uniforms(k, 0, 5, 77)
        nL, dt, lnL, kap = 30.0, 0.2, 8.0, 3e-4
        n1, n2 = col.scatter(u1, u2, 1.0, 1.0, -1.0, -1.0, 1.0, 1.0, nL, dt, lnL, kap, v)
        g, gn = u1 - u2, n1 - n2
        gm = np.linalg.norm(g)
        s2 = nL * lnL * kap * dt / (2 * 0.25 * gm ** 3)
        delta = math.sqrt(s2) * math.sqrt(-2 * math.log(1 - v[0])) * math.cos(2 * math.pi * v[1])
        cosT = (g @ gn) / (gm * np.linalg.norm(gn))
        assert abs(cosT - (1 - delta ** 2) / (1 + delta ** 2)) < 1e-12


def test_unequal_weights_update_the_lighter_partner_always():
    """Nanbu-Yonemura: with w1 = 2 w2 particle 2 always moves, particle 1 only when v3 < 1/2."""
    u1, u2 = np.array([0.02, 0.0, 0.0]), np.array([0.0, 0.01, 0.0])
    for v3, moved1 in [(0.3, True), (0.7, False)]:
        n1, n2 = col.scatter(u1, u2, 1.0, 1.0, -1.0, -1.0, 2.0, 1.0, 10.0, 1.0, 10.0, 1e-3, [0.4, 0.1, 0.2, v3])
        assert (not np.array_equal(n1, u1)) == moved1
        assert not np.array_equal(n2, u2)


def _beam_on_heavy_ions(g0, n_hat, ppc, lnL, kappa, dt):
    cfg = W.RunConfig(name="beam", nx=8, ny=8, dx=1.0, dy=1.0, dt=dt, steps=1, bc_x=W.BC_PERIODIC,
                      species=[W.Species(-1.0, 1.0, 1, 1.0, 0.0), W.Species(1.0, 1e8, 1, 1.0, 0.0)],
                      tile_nx=8, tile_ny=8)
    sim = oracle.OracleSim.from_config(cfg)
    rng = np.random.default_rng(23)
    n = ppc * cfg.nx * cfg.ny
    w = n_hat * cfg.dx * cfg.dy / ppc
    for s, u in ((0, g0), (1, 0.0)):
        sim.load_particles(s, x=rng.random(n) * cfg.nx, y=rng.random(n) * cfg.ny, ux=np.full(n, u),
                           uy=np.zeros(n), uz=np.zeros(n), w=np.full(n, w))
    return sim


def test_electron_beam_slows_at_the_lorentz_gas_rate():
    """Cold electrons (speed v) through cold ions of huge mass: <du_x>/v = -nu dt, with the textbook
    momentum-transfer rate nu = n e^4 lnL / (4 pi eps0^2 m_e^2 v^3), which in units c = omega = n_c = 1
    reads n lnL (r_e omega / c) / v^3."""
    v0, n_hat, lnL, kappa, dt = 0.05, 1.0, 10.0, 2.2e-8, 1.0
    sim = _beam_on_heavy_ions(v0, n_hat, 400, lnL, kappa, dt)
    col.collide(sim, [(0, 1)], seed=5, lnL=lnL, kappa=kappa)
    du = sim.parts[0]["ux"] - v0
    nu_dt = n_hat * lnL * kappa / v0 ** 3 * dt
    assert nu_dt < 0.01      # small-angle regime
    assert abs(np.mean(du) / v0 / (-nu_dt) - 1.0) < 0.03
    # the ions took the electrons' momentum
    p = 1.0 * np.sum(sim.parts[0]["ux"]) + 1e8 * np.sum(sim.parts[1]["ux"])
    assert abs(p - v0 * sim.parts[0]["ux"].size) < 1e-9 * v0 * sim.parts[0]["ux"].size


def test_like_collisions_isotropise_and_conserve():
    cfg = W.RunConfig(name="aniso", nx=4, ny=4, dx=1.0, dy=1.0, dt=1.0, steps=1, bc_x=W.BC_PERIODIC,
                      species=[W.Species(-1.0, 1.0, 1, 1.0, 0.0)], tile_nx=4, tile_ny=4)
    sim = oracle.OracleSim.from_config(cfg)
    rng = np.random.default_rng(24)
    n = 16 * 101   # an odd count in most cells: the triple rule runs
    sim.load_particles(0, x=rng.random(n) * 4, y=rng.random(n) * 4, ux=rng.standard_normal(n) * 0.03,
                       uy=rng.standard_normal(n) * 0.01, uz=rng.standard_normal(n) * 0.01, w=np.full(n, 1.0 / 101))
    P = sim.parts[0]
    p0 = np.array([P["ux"].sum(), P["uy"].sum(), P["uz"].sum()])
    e0 = 0.5 * np.sum(P["ux"] ** 2 + P["uy"] ** 2 + P["uz"] ** 2)
    a0 = np.mean(P["ux"] ** 2) / np.mean(0.5 * (P["uy"] ** 2 + P["uz"] ** 2))
    for _ in range(30):
        col.collide(sim, [(0, 0)], seed=9, lnL=10.0, kappa=5e-6)
        sim.step_index += 1
    P = sim.parts[0]
    p1 = np.array([P["ux"].sum(), P["uy"].sum(), P["uz"].sum()])
    e1 = 0.5 * np.sum(P["ux"] ** 2 + P["uy"] ** 2 + P["uz"] ** 2)
    a1 = np.mean(P["ux"] ** 2) / np.mean(0.5 * (P["uy"] ** 2 + P["uz"] ** 2))
    assert np.max(np.abs(p1 - p0)) < 1e-13 and abs(e1 - e0) < 1e-12 * e0
    assert a0 > 5.0 and 1.0 < a1 < 0.5 * a0    # relaxing towards isotropy
