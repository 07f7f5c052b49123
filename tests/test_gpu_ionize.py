"""Field ionisation on the GPU (pic_ionize) against the oracle (oracle/ionize.py).

A neutral carbon foil in the laser box (species: electrons, C0, C1+, C2+;
chains C0 -> C1+ -> C2+).  After every step both sides take an ionisation pass
with the same Philox draws (counter: the particle's index in its species'
order, the species, the step; the orders are the same, bit for bit).  FP64:
every decision, every particle (order exact), every moment and field within
the parity tolerances; FP32: the decisions may differ where u and P agree to
the FP32 field's rounding, so counts are compared to 1 % and charge exactly.
"""
import numpy as np
import pytest

import oracle
from oracle import ionize as ion
from paper_1308_2590_gb300 import pic, workloads as W
from tests.parity import compare_grid, compare_particles, stream

pytestmark = pytest.mark.gpu

FU, TU = W.laser_units_au(0.8)


def _case(precision=W.PREC_FP64, a0=3.0, steps=10):
    cfg = W.carbon_foil("ion-foil", 70, 37, 3, 17, 40.0, 6, steps, a0, seed=321, precision=precision)
    cfg.laser.tau = 6.0
    cfg.laser.t0 = 6.0
    gen = W.generate_particles(cfg.scaled(species=cfg.species[1:2]))[0]
    # distinct weights tag the particles (w never changes, and ionisation keeps it)
    gen["w"] = gen["w"] * (1.0 + 1e-7 * np.arange(1, gen["w"].size + 1))
    empty = {k: v[:0] for k, v in gen.items()}
    return cfg, [empty, gen, empty, empty]


def _load(cfg, parts):
    g = pic.Pic(cfg, stream=stream(), capacity=[parts[1]["x"].size] * len(parts))
    o = oracle.OracleSim.from_config(cfg)
    for s, P in enumerate(parts):
        if P["x"].size:
            g.load(s, P)
            o.load_particles(s, **P)
    return g, o


def test_ionization_matches_oracle_fp64():
    cfg, parts = _case()
    chains = W.carbon_chains(2)
    g, o = _load(cfg, parts)
    total = 0
    for k in range(cfg.steps):
        g.pic_step(1)
        o.step(1)
        ng = g.pic_ionize(chains, 2024, FU, TU)
        no = ion.ionize(o, chains, 2024, FU, TU)
        assert ng == no, (k, ng, no)
        total += ng
        for s in range(4):
            assert g.pic_particle_count(s) == o.parts[s]["x"].size
    assert total > 100                      # the pulse reached the foil and ionised it
    assert o.parts[3]["x"].size > 0         # and ionised some ions twice
    g.pic_step(2)
    o.step(2)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=40.0 / 6.0)
    dg, do = g.pic_diagnostics(), o.diagnostics()
    assert dg["count"] == do["count"]
    for k in ("kinetic", "field"):
        assert abs(dg[k] - do[k]) <= 1e-9 * abs(do[k]) + 1e-15, (k, dg[k], do[k])
    g.close()


def test_ionization_fp32_counts_and_charge():
    cfg, parts = _case(precision=W.PREC_FP32)
    chains = W.carbon_chains(2)
    g, o = _load(cfg, parts)
    charge0 = g.pic_diagnostics()["charge_particles"]
    tg = to = 0
    for _ in range(cfg.steps):
        g.pic_step(1)
        o.step(1)
        tg += g.pic_ionize(chains, 7, FU, TU)
        to += ion.ionize(o, chains, 7, FU, TU)
    assert to > 100 and abs(tg - to) <= 0.01 * to + 2
    d = g.pic_diagnostics()
    assert abs(d["charge_particles"] - charge0) <= 1e-6 * sum(P["w"].sum() for P in parts)
    assert d["count"] == sum(P["x"].size for P in parts) + tg
    g.close()


def test_ionization_rejects_bad_chains():
    cfg, parts = _case()
    g, _ = _load(cfg, parts)
    with pytest.raises(pic.PicError):
        g.pic_ionize([(1, 3, 0, 11.26)], 1, FU, TU)       # target charge is not the ion's plus one
    with pytest.raises(pic.PicError):
        g.pic_ionize([(1, 2, 0, 11.26), (1, 2, 0, 11.26)], 1, FU, TU)   # one ion species twice
    with pytest.raises(pic.PicError):
        g.pic_ionize([(1, 2, 0, 11.26)], 1, 0.0, TU)
    assert g.pic_ionize([(1, 2, 0, 11.26)], 1, FU, TU) == 0   # no field yet: no ionisation
    g.close()
