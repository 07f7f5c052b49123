"""The paper's strip decomposition (Section 3.1; Section 3.3 steps 1-9) on CPU ranks.

A literal-mode laser-foil run is cut into strips of cell rows, one per gloo
rank; every step the strips exchange the moment row above them (added), the
E and H rows next to them (overwritten) and the particles that crossed
(oracle/strips.py).  The paper's claim -- the multiprocessor run reproduces
the single-processor one -- is checked against the single-domain oracle step
for step: fields, moments, every particle (matched by a distinct weight) and
the FP64 diagnostics, to 1e-12 (the strips move particles in band
coordinates, which round differently by a few ulps).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(hot_kev):
    from paper_1308_2590_gb300 import workloads as W
    cfg = W.laser_foil("strips", 40, 12, 16, 8, 30.0, 3, 10, 4.0, seed=4242, tile=4)
    cfg.laser.tau = 6.0
    cfg.laser.t0 = 6.0
    cfg.species = [W.Species(-1.0, 1.0, 3, 30.0, hot_kev), W.Species(1.0, 1836.0, 3, 30.0, 1.0)]
    parts = W.generate_particles(cfg)
    for s, P in enumerate(parts):
        # distinct weights identify the particles (w never changes in a step)
        P["w"] = P["w"] * (1.0 + 1e-6 * (np.arange(P["w"].size) + 1 + s * 100000))
    return cfg, parts


def _rank(rank, world, port, steps, hot_kev, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from oracle.strips import HALO, StripSim
        cfg, parts = _case(hot_kev)
        las = (cfg.laser.a0, cfg.laser.omega, cfg.laser.tau, cfg.laser.t0, cfg.laser.pol)
        sim = StripSim(cfg.nx, cfg.ny, cfg.dx, cfg.dy, cfg.dt, cfg.bc_x == 0, [(s.q, s.m) for s in cfg.species],
                       las, rank, world, dist)
        for s, P in enumerate(parts):
            sim.load_particles(s, P)
        sim.deposit(tag=1)
        ref = oracle.OracleSim.from_config(cfg) if rank == 0 else None
        if ref is not None:
            for s, P in enumerate(parts):
                ref.load_particles(s, **P)
        worst = {"E": 0.0, "H": 0.0, "M": 0.0, "x": 0.0, "u": 0.0, "diag": 0.0}
        migrants = 0
        for k in range(steps):
            before = [P["y"].size for P in sim.parts]
            sim.step()
            d = sim.diagnostics()
            own = dict(E=sim.own(sim.E), H=sim.own(sim.H), M=sim.own(sim.M), parts=sim.parts, y0=sim.y0, y1=sim.y1)
            got = [None] * world if rank == 0 else None
            dist.gather_object(own, got, dst=0)
            if ref is None:
                continue
            ref.step()
            dr = ref.diagnostics()
            for key in ("kinetic", "field", "charge_grid"):
                worst["diag"] = max(worst["diag"], abs(d[key] - dr[key]) / max(abs(dr[key]), 1e-300))
            assert d["count"] == dr["count"] and d["removed"] == dr["removed"], (d, dr)
            for key, arr in (("E", ref.E), ("H", ref.H), ("M", ref.M)):
                full = np.concatenate([o[key] for o in got], axis=1)
                scale = max(np.max(np.abs(arr)), 1e-300)
                worst[key] = max(worst[key], float(np.max(np.abs(full - arr)) / scale))
            for s in range(len(parts)):
                P = {kk: np.concatenate([o["parts"][s][kk] for o in got]) for kk in ("x", "y", "ux", "uy", "uz", "w")}
                R = ref.particles(s)
                ia, ib = np.argsort(P["w"]), np.argsort(R["w"])
                assert np.array_equal(P["w"][ia], R["w"][ib])
                Lx, Ly = cfg.nx * cfg.dx, cfg.ny * cfg.dy
                dy = np.abs(P["y"][ia] - R["y"][ib]); dy = np.minimum(dy, Ly - dy)
                worst["x"] = max(worst["x"], float(np.max(np.abs(P["x"][ia] - R["x"][ib]))) / Lx,
                                 float(np.max(dy)) / Ly)
                us = max(np.max(np.abs(R[kk])) for kk in ("ux", "uy", "uz"))
                for kk in ("ux", "uy", "uz"):
                    worst["u"] = max(worst["u"], float(np.max(np.abs(P[kk][ia] - R[kk][ib]))) / us)
            # particles that changed strip this step (rows of their strip at the start of the step)
            migrants += sum(abs(a - P["y"].size) for a, P in zip(before, sim.parts))
        q.put((rank, worst, migrants, HALO))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_strips_reproduce_the_single_domain_run(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    steps, hot = 10, 150.0
    procs = [ctx.Process(target=_rank, args=(k, world, port, steps, hot, q)) for k in range(world)]
    for p in procs:
        p.start()
    got = {}
    try:
        for _ in range(world):
            rank, worst, migrants, halo = q.get(timeout=300)
            got[rank] = (worst, migrants)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0] * world
    worst, _ = got[0]
    assert sum(m for _, m in got.values()) > 0     # particles did cross between strips
    for key, v in worst.items():
        assert v < 1e-12, (key, worst)
