"""Helpers of the GPU-versus-oracle parity tests: run both sides on the same
seeded inputs and compare element by element with the stated tolerances.

Tolerances (FP64 form): particle state 1e-10 relative, moments and fields
1e-9 relative, both normwise per quantity (the error of an element is measured
against the largest magnitude of that quantity over the grid or the species,
so that quantities that cross zero, like rho of a neutral plasma, are not
divided by zero).  Cells and the particle order are compared exactly;
particles whose oracle offset lies within 1e-9 of a cell edge are excluded
from the exact cell comparison and counted.
"""
import numpy as np

import oracle
from paper_1308_2590_gb300 import pic, workloads as W

PART_RTOL_FP64 = 1e-10
GRID_RTOL_FP64 = 1e-9


def stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def normwise(a, b, scale=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.max(np.abs(b)) if scale is None else scale
    if s == 0:
        return float(np.max(np.abs(a - b))) if a.size else 0.0
    return float(np.max(np.abs(a - b)) / s) if a.size else 0.0


def run_pair(cfg, nsteps, parts=None, fields=None, capacity=None):
    """Same inputs on GPU and oracle; returns (gpu Pic, OracleSim) after nsteps."""
    if parts is None:
        parts = W.generate_particles(cfg)
    g = pic.Pic(cfg, stream=stream(), capacity=capacity)
    o = oracle.OracleSim.from_config(cfg)
    if fields is not None:
        g.pic_set_fields(*fields)
        o.set_fields(*fields)
    for s, P in enumerate(parts):
        if P["x"].size:
            g.load(s, P)
            o.load_particles(s, **P)
    if nsteps:
        g.pic_step(nsteps)
        o.step(nsteps)
    return g, o


def compare_particles(g, o, cfg, rtol=PART_RTOL_FP64):
    """Aligned comparison of every species; returns a dict of worst errors."""
    worst = {}
    Lx, Ly = cfg.nx * cfg.dx, cfg.ny * cfg.dy
    for s in range(len(cfg.species)):
        a = g.pic_get_particles(s)
        b = o.particles(s)
        assert a["x"].size == b["x"].size, (s, a["x"].size, b["x"].size)
        if a["x"].size == 0:
            continue
        dxp = np.abs(a["x"] - b["x"])
        if cfg.bc_x == W.BC_PERIODIC:
            dxp = np.minimum(dxp, Lx - dxp)
        dyp = np.abs(a["y"] - b["y"])
        dyp = np.minimum(dyp, Ly - dyp)
        ex = float(np.max(dxp)) / Lx
        ey = float(np.max(dyp)) / Ly
        us = max(np.max(np.abs(b[k])) for k in ("ux", "uy", "uz"))
        eu = max(normwise(a[k], b[k], us) for k in ("ux", "uy", "uz"))
        assert np.array_equal(a["w"], b["w"]), "weights (and so the particle order) differ"
        worst[s] = dict(x=ex, y=ey, u=eu)
        assert ex < rtol and ey < rtol and eu < rtol, (s, worst[s])
        # cells exactly, except within 1e-9 of an edge
        cx, cy, fx, fy = oracle.locate(o.g, b["x"], b["y"])
        cell_o = cy.astype(np.int64) * cfg.nx + cx
        edge = (np.minimum(fx, 1 - fx) < 1e-9) | (np.minimum(fy, 1 - fy) < 1e-9)
        bad = (a["cell"] != cell_o) & ~edge
        assert not np.any(bad), f"species {s}: {int(bad.sum())} cells differ"
    return worst


def compare_grid(g, o, rtol=GRID_RTOL_FP64, rho_scale=None):
    Mg = g.pic_moments()
    Mo = o.M
    errs = {}
    # rho: scaled by the species charge density magnitude (rho of a neutral plasma is ~0)
    rs = rho_scale if rho_scale is not None else max(np.max(np.abs(Mo[0])), 1e-300)
    errs["rho"] = normwise(Mg[0], Mo[0], rs)
    S_scale = np.max(np.abs(Mo[1:10]))
    errs["S"] = normwise(Mg[1:10], Mo[1:10], S_scale if S_scale > 0 else None)
    dj_scale = np.max(np.abs(Mo[10:13]))
    errs["dj"] = normwise(Mg[10:13], Mo[10:13], dj_scale if dj_scale > 0 else None)
    Eg, Hg = g.pic_fields()
    fs = max(np.max(np.abs(o.E)), np.max(np.abs(o.H)), 1e-300)
    errs["E"] = normwise(Eg, o.E, fs)
    errs["H"] = normwise(Hg, o.H, fs)
    for k, v in errs.items():
        assert v < rtol, (k, errs)
    return errs


def density_scale(cfg):
    return max(s.density * abs(s.q) for s in cfg.species)
