"""Writes the stored expected values under tests/golden.

discrete_frequencies.json: closed forms of the implicit scheme (no oracle
call needed): the cold k = 0 plasma oscillation under the time-centred push
and Eq. 4 is the trapezoidal rule for a harmonic oscillator, so
omega dt = 2 atan(omega_pe dt / 2) (Section 2, Eqs. 2-4).

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


if __name__ == "__main__":
    with open(os.path.join(HERE, "discrete_frequencies.json"), "w") as f:
        json.dump(frequencies(), f, indent=1)
