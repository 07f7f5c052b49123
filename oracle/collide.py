"""Binary Coulomb collisions on the FP64 oracle (the paper names collisions beside ionisation as what
makes its particle counts and runs grow, Section 4 and Section 5; it gives no model).  Reading: the
binary collision model of Takizuka and Abe (J. Comput. Phys. 25, 205, 1977), applied to u = p/(m c)
as the velocity (non-relativistic model: momentum conserved exactly, kinetic energy sum m |u|^2 / 2
conserved exactly by every pair), with the weight rule of Nanbu and Yonemura (1998) for pairs of
unequal weights.

TEST INFRASTRUCTURE ONLY: the tests may import this module; the product library never does, and
nothing here is shared with the CUDA path.

One pass, for each (species a, species b) of the list in turn, cell by cell (the particles of a cell
are consecutive in a species' order):
  * a == b: the cell's N particles pair as (0,1), (2,3), ...; for odd N >= 3 the first three form
    (0,1), (1,2), (2,0) at half the variance, then (3,4), ...;
  * a != b: the species with more particles in the cell (a on a tie) drives: its particle i pairs
    with particle i mod N_other of the other;
  * pairs are processed in that order, each seeing the previous pairs' updates;
  * per pair (1, 2): g = u1 - u2, mu = m1 m2 / (m1 + m2), n_L = the cell density of the species
    (a == b) or the lower of the two (sum of w over the cell's area dx dy), variance
        s2 = q1^2 q2^2 n_L lnL kappa dt / (2 mu^2 |g|^3)
    (kappa = r_e omega / c, the classical electron radius in the code's length unit c / omega; this is
    the SI variance e1^2 e2^2 n lnL dt / (8 pi eps0^2 mu^2 |g|^3) in units c = omega = n_c = 1), halved
    for the odd triple; delta = sqrt(s2) sqrt(-2 ln(1 - v0)) cos(2 pi v1), phi = 2 pi v2; sin T =
    2 delta / (1 + delta^2), 1 - cos T = 2 delta^2 / (1 + delta^2); with g_p = |(gx, gy)|,
        dgx = (gx / g_p) gz sinT cos phi - (gy / g_p) |g| sinT sin phi - gx (1 - cosT)
        dgy = (gy / g_p) gz sinT cos phi + (gx / g_p) |g| sinT sin phi - gy (1 - cosT)
        dgz = -g_p sinT cos phi - gz (1 - cosT)
    (g_p = 0: dg = (|g| sinT cos phi, |g| sinT sin phi, -|g| (1 - cosT))), u1 += m2 / (m1 + m2) dg,
    u2 -= m1 / (m1 + m2) dg -- particle 1 only when v3 < w2 / max(w1, w2), particle 2 only when
    v3 < w1 / max(w1, w2) (both, for equal weights);
  * v0..v3 = the four outputs of Philox-4x64-10 at counter (index of the pair's first particle -- the
    driving species' particle -- in its species' order, 16 + list position, step, 1) and key
    (seed, 0), each as (out >> 11) 2^-53.
Positions do not change; the moments are redeposited afterwards.
"""
from __future__ import annotations

import math

import numpy as np

from .ionize import philox4x64_10


def draws(index: int, spec: int, step: int, seed: int):
    out = philox4x64_10(np.uint64(index), 16 + spec, step, 1, seed, 0)
    return [float((np.uint64(o) >> np.uint64(11))) * 2.0 ** -53 for o in out]


def scatter(u1, u2, m1, m2, q1, q2, w1, w2, nL, dt, lnL, kappa, v, half=False):
    """One Takizuka-Abe pair: returns the new (u1, u2) (3-vectors)."""
    g = u1 - u2
    gm = math.sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2])
    if gm == 0.0 or nL <= 0.0:
        return u1, u2
    mu = m1 * m2 / (m1 + m2)
    s2 = q1 * q1 * q2 * q2 * nL * lnL * kappa * dt / (2.0 * mu * mu * gm ** 3)
    if half:
        s2 *= 0.5
    delta = math.sqrt(s2) * math.sqrt(-2.0 * math.log(1.0 - v[0])) * math.cos(2.0 * math.pi * v[1])
    phi = 2.0 * math.pi * v[2]
    sT = 2.0 * delta / (1.0 + delta * delta)
    cT1 = 2.0 * delta * delta / (1.0 + delta * delta)
    gp = math.sqrt(g[0] * g[0] + g[1] * g[1])
    if gp > 0.0:
        dg = np.array([g[0] / gp * g[2] * sT * math.cos(phi) - g[1] / gp * gm * sT * math.sin(phi) - g[0] * cT1,
                       g[1] / gp * g[2] * sT * math.cos(phi) + g[0] / gp * gm * sT * math.sin(phi) - g[1] * cT1,
                       -gp * sT * math.cos(phi) - g[2] * cT1])
    else:
        dg = np.array([gm * sT * math.cos(phi), gm * sT * math.sin(phi), -gm * cT1])
    wmax = max(w1, w2)
    n1, n2 = u1, u2
    if v[3] < w2 / wmax:
        n1 = u1 + m2 / (m1 + m2) * dg
    if v[3] < w1 / wmax:
        n2 = u2 - m1 / (m1 + m2) * dg
    return n1, n2


def _runs(cells: np.ndarray):
    """(cell, start, end) of the runs of equal cells (the particles of a cell are consecutive)."""
    if cells.size == 0:
        return []
    b = np.flatnonzero(np.diff(cells)) + 1
    starts = np.concatenate([[0], b])
    ends = np.concatenate([b, [cells.size]])
    return [(int(cells[s]), int(s), int(e)) for s, e in zip(starts, ends)]


def collide(sim, specs, seed: int, lnL: float, kappa: float) -> int:
    """One collision pass on an OracleSim (moments redeposited afterwards); returns the pairs processed."""
    from . import locate
    g = sim.g
    area = g.dx * g.dy
    npairs = 0
    for k, (sa, sb) in enumerate(specs):
        A, B = sim.parts[sa], sim.parts[sb]
        (qa, ma), (qb, mb) = sim.species[sa], sim.species[sb]
        if A["x"].size == 0 or B["x"].size == 0:
            continue
        ua = np.stack([A["ux"], A["uy"], A["uz"]], axis=1)
        ub = ua if sa == sb else np.stack([B["ux"], B["uy"], B["uz"]], axis=1)
        cxa, cya, _, _ = locate(g, A["x"], A["y"])
        ca = cya.astype(np.int64) * g.nx + cxa
        runs_a = _runs(ca)
        if sa == sb:
            for (c, s, e) in runs_a:
                n = e - s
                if n < 2:
                    continue
                nL = float(np.sum(A["w"][s:e])) / area
                pairs = []
                if n % 2:
                    pairs += [(s, s + 1, True), (s + 1, s + 2, True), (s + 2, s, True)]
                    first = s + 3
                else:
                    first = s
                pairs += [(i, i + 1, False) for i in range(first, e, 2)]
                for (i, j, half) in pairs:
                    v = draws(i, k, sim.step_index, seed)
                    ua[i], ua[j] = scatter(ua[i], ua[j], ma, ma, qa, qa, A["w"][i], A["w"][j], nL, sim.dt, lnL,
                                           kappa, v, half)
                    npairs += 1
        else:
            cxb, cyb, _, _ = locate(g, B["x"], B["y"])
            cb = cyb.astype(np.int64) * g.nx + cxb
            runs_b = {c: (s, e) for (c, s, e) in _runs(cb)}
            for (c, s, e) in runs_a:
                if c not in runs_b:
                    continue
                sb0, eb0 = runs_b[c]
                na, nb = e - s, eb0 - sb0
                nL = min(float(np.sum(A["w"][s:e])), float(np.sum(B["w"][sb0:eb0]))) / area
                if na >= nb:
                    for t in range(na):
                        i, j = s + t, sb0 + t % nb
                        v = draws(i, k, sim.step_index, seed)
                        ua[i], ub[j] = scatter(ua[i], ub[j], ma, mb, qa, qb, A["w"][i], B["w"][j], nL, sim.dt,
                                               lnL, kappa, v)
                        npairs += 1
                else:
                    for t in range(nb):
                        j, i = sb0 + t, s + t % na
                        v = draws(j, k, sim.step_index, seed)
                        ub[j], ua[i] = scatter(ub[j], ua[i], mb, ma, qb, qa, B["w"][j], A["w"][i], nL, sim.dt,
                                               lnL, kappa, v)
                        npairs += 1
        A["ux"], A["uy"], A["uz"] = [np.ascontiguousarray(ua[:, c]) for c in range(3)]
        if sa != sb:
            B["ux"], B["uy"], B["uz"] = [np.ascontiguousarray(ub[:, c]) for c in range(3)]
    sim.deposit()
    return npairs
