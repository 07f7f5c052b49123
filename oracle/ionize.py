"""Optical field ionisation on the FP64 oracle (the paper's targets ionise as the
laser arrives, Section 4 and Fig. 3; the paper gives no rate, so the reading
is the static tunnelling rate of Ammosov, Delone and Krainov for s-states).

TEST INFRASTRUCTURE ONLY: the tests may import this module; the product
library never does, and nothing here is shared with the CUDA path.

Per ionisation pass, for every particle of an ion species in a chain
(ion -> ion of the next charge state + electron):
  * F = |E| at the particle (E of the current time level, linear weights),
    in atomic units of field;
  * w = |C|^2 Ip (2 (2 Ip)^{3/2} / F')^{2 n* - 1} exp(-2 (2 Ip)^{3/2} / (3 F')),
    n* = Z / sqrt(2 Ip), |C|^2 = 2^{2 n*} / (n* Gamma(2 n*)), Ip the
    ionisation potential and Z the charge after the transition (atomic units),
    F' = min(F, F_m) with F_m = 2 (2 Ip)^{3/2} / (3 (2 n* - 1)) the field of the
    formula's maximum: above it (beyond the barrier-suppression field, where
    the tunnelling formula no longer holds and would fall) the rate is held at
    its maximum, so that it never decreases with the field;
  * P = 1 - exp(-w dt) with dt in atomic units of time (at most one
    transition per particle and pass);
  * u = the first output of Philox-4x64-10 (Salmon et al., SC 2011) with
    counter (index of the particle in its species' order, species, step, 0)
    and key (seed, 0), as (out >> 11) 2^-53; the particle ionises when u < P.
Ionised particles leave their species (the others keep their order) and are
appended, unchanged, to the target species and, as an electron with the same
position, u and weight, to the electron species -- chain by chain, in chain
order -- each appended species then stably re-ordered by (tile, cell) like a
load; all decisions are taken before any particle moves.
"""
from __future__ import annotations

import math

import numpy as np

HARTREE_EV = 27.211386245988

_M0, _M1 = np.uint64(0xD2E7470EE14C6C93), np.uint64(0xCA5A826395121157)
_W0, _W1 = np.uint64(0x9E3779B97F4A7C15), np.uint64(0xBB67AE8584CAA73B)
_LO = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a: np.uint64, b: np.ndarray):
    """128-bit product of a scalar and an array of uint64: (high, low) words."""
    b = np.asarray(b, dtype=np.uint64)
    a_lo, a_hi = a & _LO, a >> _S32
    b_lo, b_hi = b & _LO, b >> _S32
    ll, lh, hl, hh = a_lo * b_lo, a_lo * b_hi, a_hi * b_lo, a_hi * b_hi
    mid = (ll >> _S32) + (lh & _LO) + (hl & _LO)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    return hi, a * b


def philox4x64_10(c0, c1, c2, c3, k0, k1):
    """Philox-4x64 with 10 rounds for arrays of counters (c0..c3) and a key (k0, k1); returns 4 arrays."""
    with np.errstate(over="ignore"):
        x = [np.asarray(c, dtype=np.uint64).copy() for c in np.broadcast_arrays(c0, c1, c2, c3)]
        k0, k1 = np.uint64(k0), np.uint64(k1)
        for r in range(10):
            if r:
                k0 = k0 + _W0
                k1 = k1 + _W1
            hi0, lo0 = _mulhilo(_M0, x[0])
            hi1, lo1 = _mulhilo(_M1, x[2])
            x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
    return x


def uniform(index, species: int, step: int, seed: int) -> np.ndarray:
    """The method's uniform number of each particle index: (out0 >> 11) 2^-53."""
    out = philox4x64_10(np.asarray(index, dtype=np.uint64), species, step, 0, seed, 0)[0]
    return (out >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def adk_rate(F, ip_au: float, Z: float) -> np.ndarray:
    """Static ADK tunnelling rate (atomic units) of an s-state at field strength F (atomic units), held at
    its maximum above the field of that maximum."""
    F = np.asarray(F, dtype=np.float64)
    n = Z / math.sqrt(2.0 * ip_au)
    c2 = 2.0 ** (2.0 * n) / (n * math.gamma(2.0 * n))
    k = (2.0 * ip_au) ** 1.5
    fmax = 2.0 * k / (3.0 * (2.0 * n - 1.0)) if n > 0.5 else math.inf
    out = np.zeros_like(F)
    pos = F > 0
    Fp = np.minimum(F[pos], fmax)
    out[pos] = c2 * ip_au * (2.0 * k / Fp) ** (2.0 * n - 1.0) * np.exp(-2.0 * k / (3.0 * Fp))
    return out


def ionization_flags(sim, chains, seed: int, field_unit_au: float, time_unit_au: float):
    """Decisions of one pass on an OracleSim: per chain, a boolean array over the ion species' particles."""
    from . import gather
    flags = []
    for (s_ion, s_tgt, s_el, ip_ev) in chains:
        P = sim.parts[s_ion]
        if P["x"].size == 0:
            flags.append(np.zeros(0, bool))
            continue
        Z = sim.species[s_tgt][0]
        E = gather(sim.g, sim.E, P["x"], P["y"])
        F = np.sqrt(np.sum(E * E, axis=1)) * field_unit_au
        w = adk_rate(F, ip_ev / HARTREE_EV, Z)
        prob = -np.expm1(-w * sim.dt * time_unit_au)
        u = uniform(np.arange(P["x"].size), s_ion, sim.step_index, seed)
        flags.append(u < prob)
    return flags


def ionize(sim, chains, seed: int, field_unit_au: float, time_unit_au: float) -> int:
    """One ionisation pass on an OracleSim (moments redeposited afterwards); returns the transitions."""
    flags = ionization_flags(sim, chains, seed, field_unit_au, time_unit_au)
    keys = ("x", "y", "ux", "uy", "uz", "w")
    moved = [{k: sim.parts[s][k][f] for k in keys} for (s, _, _, _), f in zip(chains, flags)]
    for (s_ion, _, _, _), f in zip(chains, flags):
        for k in keys:
            sim.parts[s_ion][k] = np.ascontiguousarray(sim.parts[s_ion][k][~f])
    appends = {}
    for (s_ion, s_tgt, s_el, _), m in zip(chains, moved):
        appends.setdefault(s_tgt, []).append(m)
        appends.setdefault(s_el, []).append(m)
    for s, lst in appends.items():
        P = sim.parts[s]
        for k in keys:
            P[k] = np.concatenate([P[k]] + [m[k] for m in lst])
        order = np.argsort(sim.tile_cell_key(P["x"], P["y"]), kind="stable")
        for k in keys:
            P[k] = np.ascontiguousarray(P[k][order])
    sim.deposit()
    return int(sum(int(f.sum()) for f in flags))
