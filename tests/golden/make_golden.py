"""Writes the stored expected values under tests/golden.

discrete_frequencies.json: closed forms of the implicit scheme (no oracle
call needed): the cold k = 0 plasma oscillation under the time-centred push
and Eq. 4 is the trapezoidal rule for a harmonic oscillator, so
omega dt = 2 atan(omega_pe dt / 2) (Section 2, Eqs. 2-4).

oracle_uniform_8x8.json: diagnostics of the CPU oracle on a small seeded
uniform-plasma run, kept as a regression record of the oracle itself.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def frequencies():
    rows = [{"omega_pe_dt": d, "omega_over_omega_pe": 2 * math.atan(d / 2) / d} for d in (0.5, 0.3)]
    return {"source": "closed form of the implicit scheme (Section 2, Eqs. 2-4): omega dt = 2 atan(omega_pe dt/2); "
                      "the paper prints no worked example", "cold_plasma": rows}


def oracle_regression():
    import oracle
    from paper_1308_2590_gb300 import workloads as W
    cfg = W.config(1).scaled(nx=8, ny=8, tile_nx=4, tile_ny=4)
    sim = oracle.OracleSim.from_config(cfg)
    for s, P in enumerate(W.generate_particles(cfg)):
        sim.load_particles(s, **P)
    out = []
    for _ in range(5):
        sim.step()
        out.append(sim.diagnostics())
    return {"source": "oracle/ on workloads.config(1) scaled to 8x8 cells, seed 1235, 5 steps", "diagnostics": out}


if __name__ == "__main__":
    with open(os.path.join(HERE, "discrete_frequencies.json"), "w") as f:
        json.dump(frequencies(), f, indent=1)
    with open(os.path.join(HERE, "oracle_uniform_8x8.json"), "w") as f:
        json.dump(oracle_regression(), f, indent=1)
