"""Run a workload through the C ABI and log its FP64 diagnostics as JSON lines.

    python -m paper_1308_2590_gb300.run --workload 2 --steps 100 --every 10 --log run.jsonl

Every `every` steps one line: step, simulated time, FP64 kinetic / field /
total energy and their drift from the first line, deposited and particle
charge, live and removed particles, the last CN solve's iterations and
residual, and the wall time and particle-steps/s of the interval (the device
is synchronised by the diagnostics read).  --checkpoint writes the exact
checkpoint form (pic_save_particles, pic_fields, the step count) at the end
as an .npz file; --resume starts from one.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import pic
from . import workloads as W

CKEYS = ("cell", "ox", "oy", "ux", "uy", "uz", "w")


def save_checkpoint(g: pic.Pic, path: str) -> None:
    E, H = g.pic_fields()
    arrays = {"E": E, "H": H, "step": np.array([g.pic_diagnostics()["step"]], np.int64)}
    for s in range(g.nsp):
        P = g.pic_save_particles(s)
        for k in CKEYS:
            arrays[f"s{s}_{k}"] = P[k]
    np.savez(path, **arrays)


def load_checkpoint(g: pic.Pic, path: str) -> None:
    z = np.load(path)
    for s in range(g.nsp):
        g.pic_restore_particles(s, {k: z[f"s{s}_{k}"] for k in CKEYS})
    g.pic_set_fields(z["E"], z["H"])
    g.pic_set_step(int(z["step"][0]))


def run(cfg: W.RunConfig, steps: int, every: int, out, resume: str | None = None,
        checkpoint: str | None = None, stream=None) -> dict:
    """Advance cfg by `steps` steps, writing one JSON line to `out` every `every` steps."""
    g = pic.Pic(cfg, stream=stream)
    try:
        if resume:
            load_checkpoint(g, resume)
        else:
            g.pic_load_species(W.generate_particles(cfg))
        d0 = g.pic_diagnostics()
        e0 = d0["total"]
        last = None
        t_prev, n_prev, done = time.perf_counter(), d0["count"], 0
        while done < steps:
            k = min(every, steps - done)
            g.pic_step(k)
            d = g.pic_diagnostics()
            t = time.perf_counter()
            done += k
            line = {"step": d["step"], "time": d["step"] * cfg.dt, "kinetic": d["kinetic"], "field": d["field"],
                    "total": d["total"], "drift": (d["total"] - e0) / abs(e0) if e0 else 0.0,
                    "charge_grid": d["charge_grid"], "charge_particles": d["charge_particles"],
                    "count": d["count"], "removed": d["removed"], "cn_iterations": d["cn_iterations"],
                    "cn_residual": d["cn_residual"], "wall_s": t - t_prev,
                    "particle_steps_per_s": 0.5 * (n_prev + d["count"]) * k / (t - t_prev)}
            out.write(json.dumps(line) + "\n")
            out.flush()
            t_prev, n_prev, last = t, d["count"], line
        if checkpoint:
            save_checkpoint(g, checkpoint)
        return last or {}
    finally:
        g.close()


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", type=int, default=1, help="1..5 (the serving workload's first run for 5)")
    ap.add_argument("--precision", choices=("fp64", "fp32"), default=None)
    ap.add_argument("--deposit", choices=("atomic", "deterministic"), default=None)
    ap.add_argument("--steps", type=int, default=None, help="default: the workload's step count")
    ap.add_argument("--every", type=int, default=10)
    ap.add_argument("--log", default="-", help="JSON-lines file ('-' = stdout)")
    ap.add_argument("--checkpoint", default=None, help=".npz written at the end")
    ap.add_argument("--resume", default=None, help=".npz to start from")
    a = ap.parse_args(argv)
    cfg = W.config(a.workload)
    if a.precision:
        cfg.precision = W.PREC_FP32 if a.precision == "fp32" else W.PREC_FP64
    if a.deposit:
        cfg.deposit = W.DEPOSIT_DETERMINISTIC if a.deposit == "deterministic" else W.DEPOSIT_ATOMIC
    out = sys.stdout if a.log == "-" else open(a.log, "w")
    try:
        run(cfg, a.steps if a.steps is not None else cfg.steps, max(1, a.every), out, a.resume, a.checkpoint)
    finally:
        if out is not sys.stdout:
            out.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
