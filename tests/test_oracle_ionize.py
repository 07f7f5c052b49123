"""Pins of the oracle's field ionisation (oracle/ionize.py), -m "not gpu".

The paper's runs gain particles by optical field ionisation (Section 4, Fig. 3)
but state no rate; the oracle takes the static ADK tunnelling rate and draws
its uniform numbers from Philox-4x64-10.  Pinned here: the generator against
numpy's Philox bit generator (an independent implementation of the same
published function); the rate against the textbook hydrogen tunnelling rate
4/F exp(-2/(3F)) (Landau-Lifshitz); the pass against its invariants (counts,
charge, order) and its statistics in a uniform field.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import ionize as ion
from paper_1308_2590_gb300 import workloads as W


def test_philox_matches_numpy():
    rng = np.random.default_rng(3)
    for _ in range(20):
        ctr = [int(v) for v in rng.integers(0, 2 ** 63, size=4)]
        key = [int(v) for v in rng.integers(0, 2 ** 63, size=2)]
        # numpy's Philox(counter=c) produces its first block from c + 1
        c0 = (ctr[0] - 1) % 2 ** 64
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                              counter=np.array([c0] + ctr[1:], dtype=np.uint64))
        want = [int(v) for v in bg.random_raw(4)]
        got = [int(v[()]) for v in ion.philox4x64_10(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1])]
        assert got == want
    u = ion.uniform(np.arange(100000), 3, 17, 1234)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002


def test_adk_rate_of_hydrogen_is_the_textbook_tunnelling_rate():
    """Hydrogen (Z = 1, Ip = 1/2): n* = 1, |C|^2 = 4, so w = 4/F exp(-2/(3F)) below the formula's maximum
    at F = 2/3; above it the rate is held at 6 exp(-1)."""
    F = np.array([0.01, 0.03, 0.05, 0.1, 0.2, 0.5])
    w = ion.adk_rate(F, 0.5, 1.0)
    assert np.max(np.abs(w / (4.0 / F * np.exp(-2.0 / (3.0 * F))) - 1.0)) < 1e-14
    assert ion.adk_rate(np.array([0.0]), 0.5, 1.0)[0] == 0.0
    assert np.max(np.abs(ion.adk_rate(np.array([2.0 / 3.0, 1.0, 40.0]), 0.5, 1.0) / (6.0 * math.exp(-1.0)) - 1)) < 1e-14
    # carbon 1+ -> 2+ (24.38 eV): never decreases with the field
    wc = ion.adk_rate(np.geomspace(1e-3, 100, 80), 24.38 / ion.HARTREE_EV, 2.0)
    assert np.all(np.diff(wc) >= 0) and wc[-1] > 0


def _carbon_run(nx=24, ny=12, ppc=6):
    """Neutral carbon (q = 0) and C1+ with electrons, in a periodic box, chains C0 -> C1+ -> C2+."""
    cfg = W.RunConfig(name="ion", nx=nx, ny=ny, dx=0.2, dy=0.2, dt=0.1, steps=1, bc_x=W.BC_PERIODIC,
                      field_mode=W.FIELD_LITERAL,
                      species=[W.Species(-1.0, 1.0, ppc, 1.0, 1.0), W.Species(0.0, 22032.0, ppc, 1.0, 1.0),
                               W.Species(1.0, 22032.0, ppc, 1.0, 1.0), W.Species(2.0, 22032.0, ppc, 1.0, 1.0)],
                      tile_nx=4, tile_ny=4, seed=77)
    sim = oracle.OracleSim.from_config(cfg)
    parts = W.generate_particles(cfg)
    for s, P in enumerate(parts[:3]):
        sim.load_particles(s, **P)
    chains = [(1, 2, 0, 11.2603), (2, 3, 0, 24.3833)]
    return cfg, sim, chains


def test_ionization_pass_invariants():
    cfg, sim, chains = _carbon_run()
    g = sim.g
    rng = np.random.default_rng(5)
    E = 0.2 + 0.05 * rng.standard_normal((3, g.ny, g.nxn))
    sim.set_fields(E=E)
    before = {s: sim.particles(s) for s in range(4)}
    flags = ion.ionization_flags(sim, chains, 99, 7.8, 17.5)
    n = ion.ionize(sim, chains, 99, 7.8, 17.5)
    assert n == sum(int(f.sum()) for f in flags) and 0 < n
    after = {s: sim.particles(s) for s in range(4)}
    # every transition adds an electron, moves one ion up one charge state, keeps the weights
    assert after[0]["x"].size == before[0]["x"].size + n
    n1, n2 = int(flags[0].sum()), int(flags[1].sum())
    assert after[1]["x"].size == before[1]["x"].size - n1
    assert after[2]["x"].size == before[2]["x"].size - n2 + n1
    assert after[3]["x"].size == n2
    charge = lambda parts: sum(q * parts[s]["w"].sum() for s, (q, _) in enumerate(sim.species))
    assert abs(charge(after) - charge(before)) < 1e-12 * sum(P["w"].sum() for P in before.values())
    # the ions that stay keep their order; the ionised ones are the flagged ones
    for (s_ion, _, _, _), f in zip(chains, flags):
        assert np.array_equal(after[s_ion]["w"], before[s_ion]["w"][~f]) or s_ion == 2
    assert np.array_equal(np.sort(after[3]["w"]), np.sort(before[2]["w"][flags[1]]))
    # appended species are in load order: by (tile, cell)
    for s in (0, 2, 3):
        key = sim.tile_cell_key(after[s]["x"], after[s]["y"])
        assert np.all(np.diff(key) >= 0)
    # moments were redeposited with the new charges: the node charge equals the particles'
    d = sim.diagnostics()
    assert abs(d["charge_grid"] - d["charge_particles"]) < 1e-12 * sum(P["w"].sum() for P in before.values())


def test_ionized_fraction_follows_the_probability():
    """A uniform field: every ion has the same probability P; the count is binomial(n, P)."""
    cfg, sim, chains = _carbon_run(nx=32, ny=32, ppc=16)
    g = sim.g
    for F_norm in (0.05, 0.2):
        E = np.zeros((3, g.ny, g.nxn))
        E[1] = F_norm
        sim.set_fields(E=E)
        flags = ion.ionization_flags(sim, chains[:1], 7, 7.8, 17.5)[0]
        w = ion.adk_rate(np.array([F_norm * 7.8]), 11.2603 / ion.HARTREE_EV, 1.0)[0]
        P = -math.expm1(-w * sim.dt * 17.5)
        n = flags.size
        assert abs(flags.sum() - n * P) <= 5 * math.sqrt(n * P * (1 - P)) + 1
    E = np.zeros((3, g.ny, g.nxn))
    sim.set_fields(E=E)
    assert not ion.ionization_flags(sim, chains, 7, 7.8, 17.5)[0].any()     # no field, no ionisation
