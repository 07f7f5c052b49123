"""Benchmark of the implicit 2D3V PIC step on GB300.

Workload: the particle-dominated laser-foil run -- 1024 x 512 cells of lambda/40,
absorbing x walls with a 0.8 um, a0 = 5, 30 fs plane wave injected at x = 0,
periodic y, a 100-cell proton-electron foil at 100 n_c with 64 particles per
cell per species (6,553,600 particles), dt = 0.01 lambda/c, literal field
solve (Eqs. 4-5).  Synthetic, seeded inputs; one step = field solve + gather +
push + deposit + regroup of every particle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32] [--impl reference]

Prints one JSON line (rank 0).  value = particle-steps/s over the K timed
steps (inputs resident in HBM), e2e = the same metric through the C ABI with
the step's particles copied from page-locked host arrays (prefetched by the
library up to two steps ahead, the copies inside the timed region) and the
step's 13 moment planes and diagnostics read back every step.  Under torchrun every rank runs an independent replica (the run
does not shard: replicas only); value sums the ranks' particle-steps over the
slowest rank's time.

Besides the headline workload, rank 0 at N = 1 also reports (keys of the same
line): the field-dominated laser foil (4096 x 2048 cells, 20-cell foil at
50 n_c, 4 particles/cell/species) in both forms; the precision form at full
size (2048 x 2048 periodic uniform plasma, 32 particles/cell/species,
268,435,456 particles, FP32 against FP64 on the same seed after 1 and 11
steps); the serving stream (256 Poisson-arriving runs at 20/s under an 8 GB
device-memory budget, plus a burst of 64 runs submitted at once); and a
neutral carbon foil ionising in the laser (particle growth, pass time).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# algorithmic cost of one particle-step of the fused gather + push + deposit:
# bytes of particle state streamed (cell index, in-cell offsets, u and w read
# once; offsets, u and cell index written once; offsets, u and w in the form's
# precision) and FP64 flops (~250: two bilinear gathers, the implicit push of
# Eq. 2, the 13 moments of Eq. 3 and their four-corner deposit; an FMA counts 2)
BYTES_PER_PARTICLE = {"fp32": 52, "fp64": 96}
FLOPS_PER_PARTICLE = 250
# nominal FP64 rate (2 DFMA/clk/SM x 152 SMs x 2070 MHz x 2 flops), used only when the probe cannot run
FP64_NOMINAL_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12

# DRAM bytes (read + write) per particle-step of k_push, from one ncu capture of
# this workload (dram__bytes_read.sum + dram__bytes_write.sum of one launch over
# its particles); they hold for the kernel source whose SHA-256 prefix is
# PUSH_SOURCE_SHA and are reported as null for any other source.  The source is pic_tile.cu and the shared header without
# its host-only sections (the handle struct and the host entry points).
PUSH_TRAFFIC_PER_PARTICLE = {"fp64": 191.2, "fp32": 52.2}
PUSH_SOURCE_SHA = "b80a770c5dbdd5ad"
PUSH_SOURCES = ("paper_1308_2590_gb300/csrc/pic_tile.cu", "paper_1308_2590_gb300/csrc/pic_internal.cuh")
HOST_ONLY_SECTIONS = ("handle", "host entry points")


def kernel_source_text(text: str) -> str:
    """The header text without the sections whose marker line names a host-only section."""
    out, keep = [], True
    for line in text.splitlines(keepends=True):
        if line.startswith("// -----"):
            keep = line.rstrip().split("- ")[-1].strip() not in HOST_ONLY_SECTIONS
        if keep:
            out.append(line)
    return "".join(out)


def push_source_sha() -> str:
    h = hashlib.sha256()
    for rel in PUSH_SOURCES:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            text = f.read()
        h.update((kernel_source_text(text) if rel.endswith(".cuh") else text).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_totals(ms: float, particle_steps: float, e2e: float, world: int, device: str = "cuda"):
    """Whole-job figures of N replicas (one process per GPU, no data exchange):
    the slowest rank's timed region, and the particle-steps and end-to-end
    rates summed over ranks.  world = 1 returns the inputs unchanged."""
    if world <= 1:
        return ms, particle_steps, e2e
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, particle_steps, e2e], dtype=torch.float64, device=device)
    tmax = t[:1].clone()
    tsum = t[1:].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[0]), float(tsum[1])


def workload(precision: str, deposit: str = "atomic"):
    from paper_1308_2590_gb300 import workloads as W
    cfg = W.config(2)
    cfg.precision = W.PREC_FP32 if precision == "fp32" else W.PREC_FP64
    cfg.deposit = W.DEPOSIT_DETERMINISTIC if deposit == "deterministic" else W.DEPOSIT_ATOMIC
    return cfg


def run_gpu(args, rank, world, local):
    import numpy as np
    import torch
    from paper_1308_2590_gb300 import build, pic

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    stream = torch.cuda.current_stream()
    cfg = workload(args.precision, args.deposit)
    from paper_1308_2590_gb300 import workloads as W
    parts = W.generate_particles(cfg, seed=cfg.seed + rank)
    n0 = sum(P["x"].size for P in parts)
    g = pic.Pic(cfg, stream=stream.cuda_stream, capacity=[P["x"].size for P in parts])
    g.pic_load_species(parts)
    g.pic_step(args.warmup)
    g.pic_sync()
    n_before = g.pic_diagnostics()["count"]
    g.pic_set_timing(True)
    g.pic_timings(reset=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.pic_step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    kms, launches = g.pic_timings(reset=True)
    g.pic_set_timing(False)
    n_after = g.pic_diagnostics()["count"]
    particle_steps = 0.5 * (n_before + n_after) * args.steps

    # end to end through the C ABI: host arrays in, diagnostics out, every step
    pinned = []
    for P in parts:
        pinned.append({k: torch.from_numpy(P[k]).pin_memory().numpy() for k in ("x", "y", "ux", "uy", "uz", "w")})
    nxn = cfg.nx if cfg.bc_x == W.BC_PERIODIC else cfg.nx + 1
    moments = torch.empty((13, cfg.ny, nxn), dtype=torch.float64).pin_memory().numpy()
    e2e_steps = max(1, min(args.e2e_steps, args.steps))

    def e2e_loop(prefetch: bool):
        # each step: that step's particles from page-locked host arrays (prefetch: copied by the
        # library's copy stream while the previous steps compute, up to two steps ahead), one
        # step, the 13 moment planes and the diagnostics back to the host
        if prefetch:
            # the two device slots allocated and written once before the timed region, as the direct
            # loads' staging is by the first load
            for _ in range(2):
                g.pic_prefetch_species(pinned)
            for _ in range(2):
                g.pic_clear_particles()
                g.pic_load_prefetched()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = d2h = 0
        if prefetch:
            for _ in range(min(2, e2e_steps)):
                g.pic_prefetch_species(pinned)
        for i in range(e2e_steps):
            g.pic_clear_particles()
            if prefetch:
                g.pic_load_prefetched()
                if i + 2 < e2e_steps:
                    g.pic_prefetch_species(pinned)
            else:
                g.pic_load_species(pinned)
            h2d += sum(6 * 8 * P["x"].size for P in pinned)
            g.pic_step(1)
            g.pic_moments(out=moments)          # the step's result: the moments for the next solve
            d = g.pic_diagnostics()
            d2h += moments.nbytes + 80
        torch.cuda.synchronize()
        return n0 * e2e_steps / (time.perf_counter() - t0), h2d, d2h

    e2e_direct, _, _ = e2e_loop(False)
    e2e_val, h2d, d2h = e2e_loop(True)
    fp64_rate = None
    if args.precision == "fp64" and rank == 0:
        try:
            fp64_rate = pic.probe_fp64_rate(stream.cuda_stream, 5)
        except Exception:
            fp64_rate = None
    g.close()
    ms_job, ps_job, e2e_val = job_totals(ms, particle_steps, e2e_val, world)
    _, _, e2e_direct = job_totals(ms, particle_steps, e2e_direct, world)
    return dict(ms=ms_job, particle_steps=ps_job, kernel_ms=kms.tolist(), launches=launches.tolist(), clocks=clk,
                n0=n0, e2e=dict(value=e2e_val, h2d=h2d / e2e_steps, d2h=d2h / e2e_steps), e2e_direct=e2e_direct,
                n_local=0.5 * (n_before + n_after),
                fp64_rate=fp64_rate)


def roofline(r, precision: str, deposit: str, steps: int, peaks, peak_src):
    """Roofline of k_push from the library's event timers.  Class 0 of the
    timers brackets, per step, the work-list scan and the one persistent
    k_push launch over every species (plus, with the deterministic deposit,
    the fixed-point conversion); its time per step is the push's launch
    duration and the units of one launch are the live particles of all
    species."""
    kms = r["kernel_ms"]
    avg_part_ms = kms[0] / steps
    units_per_launch = r["n_local"]
    tr = PUSH_TRAFFIC_PER_PARTICLE.get(precision)
    traffic = (tr * units_per_launch if tr is not None and PUSH_SOURCE_SHA == push_source_sha()
               and deposit == "atomic" else None)
    kernel = "k_push (persistent: TMA-staged gather, implicit push, deposit, in-place compaction)"
    if precision == "fp64":
        achieved = FLOPS_PER_PARTICLE * units_per_launch / (avg_part_ms * 1e-3) / 1e12
        rate = r.get("fp64_rate")
        peak = rate if rate else FP64_NOMINAL_TFLOPS
        src = ("measured: FP64 FMA probe on this GPU (pic_probe_fp64_rate, best of 5 timed launches, run alone)"
               if rate else "nominal 2 DFMA/clk/SM x 152 SMs x 2070 MHz (the probe did not run)")
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
                "peak_source": src, "flops_per_particle": FLOPS_PER_PARTICLE,
                "hbm_frac": BYTES_PER_PARTICLE["fp64"] * units_per_launch / (avg_part_ms * 1e-3) / 1e9
                / peaks["hbm_gbs"]}
    achieved = BYTES_PER_PARTICLE["fp32"] * units_per_launch / (avg_part_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "kernel": kernel,
            "peak_source": (f"hbm_gbs of MEASURED_PEAKS.json ({peak_src}, burst copy)" if peak_src == "measured"
                            else f"fallback {peaks['hbm_gbs']:.0f} GB/s (no MEASURED_PEAKS.json)")}


def run_serving(n_runs: int, rate: float, steps: int, max_slots: int, batch_min_runs: int = 0,
                mem_budget: int = 0, burst: bool = False):
    """Play the stream of independent laser-foil runs through the server.

    A producer thread draws each run's particles ahead of its arrival time; the
    request is submitted at its scheduled arrival (on the server clock), or all
    at once when burst is set.  Latency = finish (results on the host) -
    scheduled arrival; queue wait = start - arrival; runs on the GPU = the
    overlap of the [start, finish] intervals (mean over the span, and peak)."""
    import queue as _q
    import numpy as np
    from paper_1308_2590_gb300 import pic, workloads as W
    stream = W.serving_stream(n_runs=n_runs, rate_per_s=rate, steps=steps)
    if burst:
        stream = [(0.0, cfg) for _, cfg in stream]
        parts_all = [(t, cfg, W.generate_particles(cfg)) for t, cfg in stream]
    ahead = _q.Queue(maxsize=24)

    def produce():
        for t_arr, cfg in stream:
            ahead.put((t_arr, cfg, W.generate_particles(cfg)))
        ahead.put(None)

    srv = pic.Server(mem_budget=mem_budget, max_slots=max_slots, batch_min_runs=batch_min_runs)
    if not burst:
        th = threading.Thread(target=produce, daemon=True)
        th.start()
        while ahead.qsize() < min(8, n_runs):
            time.sleep(0.01)
    t_base = srv.now()
    ids, arrivals, lags = [], [], []
    items = iter(parts_all) if burst else iter(ahead.get, None)
    for item in items:
        t_arr, cfg, parts = item
        wait = t_base + t_arr - srv.now()
        if wait > 0:
            time.sleep(wait)
        lags.append(max(0.0, srv.now() - (t_base + t_arr)))
        ids.append(srv.submit(cfg, parts, cfg.steps))
        arrivals.append(t_base + t_arr)
    srv.wait_all(3600.0)
    sts = [srv.status(i) for i in ids]
    srv.close()
    done = [s for s in sts if s["state"] == pic.REQ_DONE]
    lat = np.array([s["t_finish"] - a for s, a in zip(sts, arrivals) if s["state"] == pic.REQ_DONE])
    qwait = np.array([s["t_start"] - a for s, a in zip(sts, arrivals) if s["state"] == pic.REQ_DONE])
    ps = sum(s["particle_steps"] for s in done)
    span = max(s["t_finish"] for s in done) - min(arrivals)
    busy = [(s["t_start"], s["t_finish"]) for s in done]
    ev = sorted([(a, 1) for a, _ in busy] + [(b, -1) for _, b in busy], key=lambda e: (e[0], e[1]))
    cur = peak = 0
    for _, d in ev:
        cur += d
        peak = max(peak, cur)
    return {"runs": n_runs, "completed": len(done), "failed": len(sts) - len(done),
            "arrivals": "all at t = 0" if burst else f"Poisson, {rate}/s", "rate_per_s": None if burst else rate,
            "steps_per_run": steps, "max_slots": max_slots, "mem_budget_bytes": mem_budget or None,
            "precision": "fp32", "batched_from_runs": batch_min_runs if batch_min_runs > 0 else None,
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "mean": float(lat.mean()), "max": float(lat.max())},
            "queue_wait_s": {"mean": float(qwait.mean()), "max": float(qwait.max())},
            "particle_steps_per_s": ps / span, "particle_steps": ps, "span_s": span,
            "submit_lag_s_max": float(max(lags)) if lags else 0.0,
            "mean_runs_on_gpu": float(sum(b - a for a, b in busy) / span), "peak_runs_on_gpu": peak}


def run_field_dominated(steps: int, warmup: int):
    """The field-dominated laser foil (4096 x 2048 cells, 20-cell foil at 50 n_c,
    4 particles/cell/species) in both forms: step time, field-solve time and
    particle-steps/s over `steps` steps after `warmup` (inputs resident)."""
    import torch
    from paper_1308_2590_gb300 import pic, workloads as W
    base = W.config(3)
    parts = W.generate_particles(base)
    stream = torch.cuda.current_stream()
    out = {"workload": "laser-foil 4096x2048 cells, 20-cell foil at 50 n_c, 4 particles/cell/species "
                       f"({base.n_particles} particles), literal field solve, walls + a0=5 laser",
           "steps": steps, "warmup": warmup}
    for name, prec in (("fp64", W.PREC_FP64), ("fp32", W.PREC_FP32)):
        cfg = base.scaled(precision=prec)
        g = pic.Pic(cfg, stream=stream.cuda_stream, capacity=[P["x"].size for P in parts])
        g.pic_load_species(parts)
        g.pic_step(warmup)
        g.pic_sync()
        n0 = g.pic_diagnostics()["count"]
        g.pic_set_timing(True)
        g.pic_timings(reset=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.pic_step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kms, _ = g.pic_timings(reset=True)
        g.pic_set_timing(False)
        n1 = g.pic_diagnostics()["count"]
        g.close()
        out[name] = {"ms_per_step": ms / steps, "particle_steps_per_s": 0.5 * (n0 + n1) * steps / (ms * 1e-3),
                     "field_solve_ms_per_step": kms[2] / steps,
                     "kernel_ms_per_step": {"particle": kms[0] / steps, "regroup": kms[1] / steps,
                                            "field_solve": kms[2] / steps, "clear": kms[3] / steps},
                     "field_share_of_kernel_time": kms[2] / max(1e-12, float(sum(kms)))}
    return out


def run_cn_walls(steps: int = 20, warmup: int = 3):
    """The particle-dominated laser foil (1024 x 512, 6,553,600 particles) with the implicit-curl field
    solve instead of Eqs. 4-5: walls with the time-centred Mur rows, mixed-precision BiCGSTAB; both forms
    at c dt/dx = 0.4 (automatic preconditioner: block-Jacobi), and the FP64 form at c dt/dx = 2 (a step
    the leapfrog curls of Eqs. 4-5 cannot take) with the line preconditioner (ny = 512 is a power of two:
    y-FFT, exact block-tridiagonal solves along x per mode; the automatic choice there) and with
    block-Jacobi: step time, field-solve time, iterations per solve."""
    import torch
    from paper_1308_2590_gb300 import pic, workloads as W
    base = W.config(2).scaled(field_mode=W.FIELD_CN)
    parts = W.generate_particles(base)
    stream = torch.cuda.current_stream()
    out = {"workload": "laser-foil 1024x512 cells, 6,553,600 particles, CN field solve with walls (c dt/dx = 0.4; "
                       "fp64_cdt2_*: c dt/dx = 2)", "steps": steps}
    legs = (("fp64", W.PREC_FP64, base.dt, W.CN_PRECOND_AUTO), ("fp32", W.PREC_FP32, base.dt, W.CN_PRECOND_AUTO),
            ("fp64_cdt2_line", W.PREC_FP64, 2.0 * base.dx, W.CN_PRECOND_FFT),
            ("fp64_cdt2_jacobi", W.PREC_FP64, 2.0 * base.dx, W.CN_PRECOND_JACOBI))
    for name, prec, dt, pre in legs:
        g = pic.Pic(base.scaled(precision=prec, dt=dt, cn_precond=pre), stream=stream.cuda_stream,
                    capacity=[P["x"].size for P in parts])
        g.pic_load_species(parts)
        g.pic_step(warmup)
        g.pic_sync()
        g.pic_set_timing(True)
        g.pic_timings(reset=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.pic_step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        kms, _ = g.pic_timings(reset=True)
        g.pic_set_timing(False)
        d = g.pic_diagnostics()
        g.close()
        out[name] = {"ms_per_step": e0.elapsed_time(e1) / steps, "field_solve_ms_per_step": kms[2] / steps,
                     "cn_iterations_last": d["cn_iterations"], "cn_refinements_last": d["cn_refinements"],
                     "cn_residual_last": d["cn_residual"]}
    return out


def run_shapes(steps: int = 20, warmup: int = 3, orders=(2, 3, 4)):
    """The particle-dominated laser foil (1024 x 512, 6,553,600 particles, literal solve) with the spline
    shapes of degree 2, 3, 4 ((n + 1)^2 nodes per particle): both forms, step and push time."""
    import torch
    from paper_1308_2590_gb300 import pic, workloads as W
    parts = W.generate_particles(W.config(2))
    stream = torch.cuda.current_stream()
    n = sum(P["x"].size for P in parts)
    out = {"workload": "laser-foil 1024x512 cells, 6,553,600 particles, literal field solve, spline shapes of "
                       "degree 2, 3, 4 (9, 16, 25 nodes per particle)", "steps": steps}
    for order in orders:
        base = W.config(2).scaled(shape=order)
        out[f"order{order}"] = _shape_leg(base, parts, n, steps, warmup, stream)
    return out


def _shape_leg(base, parts, n, steps, warmup, stream):
    import torch
    from paper_1308_2590_gb300 import pic, workloads as W
    out = {}
    for name, prec in (("fp64", W.PREC_FP64), ("fp32", W.PREC_FP32)):
        g = pic.Pic(base.scaled(precision=prec), stream=stream.cuda_stream, capacity=[P["x"].size for P in parts])
        g.pic_load_species(parts)
        g.pic_step(warmup)
        g.pic_sync()
        g.pic_set_timing(True)
        g.pic_timings(reset=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.pic_step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        kms, _ = g.pic_timings(reset=True)
        g.pic_set_timing(False)
        g.close()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_step": ms, "particle_steps_per_s": n / (ms * 1e-3),
                     "push_ms_per_step": kms[0] / steps, "regroup_ms_per_step": kms[1] / steps,
                     "field_solve_ms_per_step": kms[2] / steps}
    return out


def run_collisions(passes: int = 5, warmup: int = 1):
    """The particle-dominated laser foil (1024 x 512, 6,553,600 particles) after 3 steps: one binary-
    collision pass over the electron-electron, electron-ion and ion-ion entries (kappa of a 0.8 um laser,
    ln_lambda 10), both forms: pass time (host wall clock, the count read back), pairs per pass, and the
    following step (its deposit at rest included)."""
    import time as _time
    import torch
    from paper_1308_2590_gb300 import pic, workloads as W
    cfg = W.config(2)
    parts = W.generate_particles(cfg)
    stream = torch.cuda.current_stream()
    kappa = 2.0 * 3.141592653589793 * 2.8179403262e-15 / 0.8e-6
    pairs = [(0, 0), (0, 1), (1, 1)]
    out = {"workload": "laser-foil 1024x512 cells, 6,553,600 particles; collision entries e-e, e-i, i-i; "
                       "ln_lambda 10, kappa = 2 pi r_e / 0.8 um", "passes": passes}
    for name, prec in (("fp64", W.PREC_FP64), ("fp32", W.PREC_FP32)):
        g = pic.Pic(cfg.scaled(precision=prec), stream=stream.cuda_stream, capacity=[P["x"].size for P in parts])
        g.pic_load_species(parts)
        g.pic_step(3)
        g.pic_sync()
        for _ in range(warmup):
            g.pic_collide(pairs, 1, 10.0, kappa)
        g.pic_sync()
        t0 = _time.perf_counter()
        npairs = 0
        for k in range(passes):
            npairs = g.pic_collide(pairs, 2 + k, 10.0, kappa)
        g.pic_sync()
        t1 = _time.perf_counter()
        g.pic_step(1)
        g.pic_sync()
        t2 = _time.perf_counter()
        g.close()
        out[name] = {"pass_ms": (t1 - t0) / passes * 1e3, "pairs_per_pass": npairs,
                     "next_step_ms": (t2 - t1) * 1e3}
    return out


def run_ionization(steps: int = 80):
    """A neutral carbon foil ionising in the laser (the paper's targets, Section 4, Fig. 3): 1024 x 512
    cells, foil of 100 cells from x = 10 cells, 32 particles/cell, a0 = 5, chains C0 -> C1+ -> ... -> C4+
    (static ADK rate, Philox draws); one ionisation pass after every step.  Reports the particle count's
    growth and the time of a step and of a pass (the pass's count readbacks included)."""
    import torch
    from paper_1308_2590_gb300 import pic, workloads as W
    cfg = W.carbon_foil("carbon-foil-1024x512", 1024, 512, 10, 100, 100.0, 32, steps, 5.0, seed=1234 + 6,
                        charge_states=4)
    chains = W.carbon_chains(4)
    fu, tu = W.laser_units_au(0.8)
    gen = W.generate_particles(cfg.scaled(species=cfg.species[1:2]))[0]
    n0 = gen["x"].size
    empty = {k: v[:0] for k, v in gen.items()}
    parts = [empty, gen] + [empty] * 4
    stream = torch.cuda.current_stream()
    g = pic.Pic(cfg, stream=stream.cuda_stream, capacity=[5 * n0, n0, n0, n0, n0, n0])
    g.pic_load_species(parts)
    step_ms = ion_ms = 0.0
    grown = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    total = 0
    passes = 0
    for k in range(steps):
        torch.cuda.synchronize()
        e0.record(stream)
        g.pic_step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms += e0.elapsed_time(e1)
        t = time.perf_counter()
        n = g.pic_ionize(chains, 99, fu, tu)
        torch.cuda.synchronize()
        ion_ms += 1e3 * (time.perf_counter() - t)
        total += n
        passes += 1
        if (k + 1) % 20 == 0:
            grown.append({"step": k + 1, "particles": int(sum(g.pic_particle_count(s) for s in range(6))),
                          "per_species": [int(g.pic_particle_count(s)) for s in range(6)]})
    g.close()
    return {"workload": f"carbon foil 1024x512, 100 cells from x = 10 at 100 n_c (fully ionised), 32 particles/cell, "
                        f"a0 = 5, chains C0 -> C4+, {steps} steps with a pass after each",
            "initial_particles": n0, "transitions": total, "growth": grown,
            "step_ms_mean": step_ms / steps, "pass_ms_mean": ion_ms / passes}


def _moment_errors(Ma, Mb, density: float):
    """Normwise FP32-vs-FP64 moment errors: rho over the species' charge density,
    S and dj over their largest magnitude."""
    import numpy as np
    err = lambda a, b, s: float(np.max(np.abs(a - b)) / s) if s > 0 else float(np.max(np.abs(a - b)))
    return {"rho": err(Ma[0], Mb[0], density), "S": err(Ma[1:10], Mb[1:10], float(np.max(np.abs(Mb[1:10])))),
            "dj": err(Ma[10:13], Mb[10:13], float(np.max(np.abs(Mb[10:13]))))}


def run_precision_form(more_steps: int = 10):
    """The precision form at full size: 2048 x 2048 periodic uniform plasma,
    32 particles/cell/species (268,435,456 particles), CN field solve; the FP32
    form against the FP64 form on the GPU from the same seeded particles,
    compared after 1 and after 1 + more_steps steps; both forms timed."""
    import gc
    import numpy as np
    import torch
    from paper_1308_2590_gb300 import pic, workloads as W
    cfg32 = W.config(4)
    cfg64 = cfg32.scaled(precision=W.PREC_FP64)
    t_gen = time.perf_counter()
    parts = W.generate_particles(cfg32)
    t_gen = time.perf_counter() - t_gen
    n = sum(P["x"].size for P in parts)
    stream = torch.cuda.current_stream()
    runs = {}
    for name, cfg in (("fp64", cfg64), ("fp32", cfg32)):
        g = pic.Pic(cfg, stream=stream.cuda_stream, capacity=[P["x"].size for P in parts])
        g.pic_load_species(parts)
        runs[name] = g
    del parts
    gc.collect()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    res = {"workload": f"uniform 2048x2048 periodic, 32 particles/cell/species ({n} particles), CN field solve, "
                       "same seeded particles in both forms", "particles": n, "generation_s": t_gen}
    diag0 = {k: g.pic_diagnostics() for k, g in runs.items()}
    ms = {}
    for k, g in runs.items():
        torch.cuda.synchronize()
        e0.record(stream)
        g.pic_step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms[k] = [e0.elapsed_time(e1)]
    dens = 1.0
    res["after_1_step"] = _moment_errors(runs["fp32"].pic_moments(), runs["fp64"].pic_moments(), dens)
    for k, g in runs.items():
        torch.cuda.synchronize()
        e0.record(stream)
        g.pic_step(more_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms[k].append(e0.elapsed_time(e1) / more_steps)
    res[f"after_{1 + more_steps}_steps"] = _moment_errors(runs["fp32"].pic_moments(), runs["fp64"].pic_moments(), dens)
    d = {k: g.pic_diagnostics() for k, g in runs.items()}
    e64_0 = diag0["fp64"]["total"]
    res["energy"] = {"fp64_total": d["fp64"]["total"], "fp32_total": d["fp32"]["total"],
                     "relative_difference": abs(d["fp32"]["total"] - d["fp64"]["total"]) / abs(e64_0),
                     "fp64_drift": (d["fp64"]["total"] - e64_0) / abs(e64_0),
                     "fp32_drift": (d["fp32"]["total"] - diag0["fp32"]["total"]) / abs(diag0["fp32"]["total"])}
    res["targets"] = {"moments": 1e-5, "energy": 1e-3}
    for k, g in runs.items():
        res[k] = {"ms_per_step": ms[k][1], "first_step_ms": ms[k][0],
                  "particle_steps_per_s": n / (ms[k][1] * 1e-3), "cn_iterations_last": d[k]["cn_iterations"]}
        g.close()
    res["fp32_speedup"] = ms["fp64"][1] / ms["fp32"][1]
    return res


def oracle_sample(cfg, budget_s: float, nsteps_hint: int):
    """A slice of the workload (the first `rows` cell rows, all columns) sized so
    that one oracle step takes about budget_s seconds."""
    import oracle
    from paper_1308_2590_gb300 import workloads as W
    probe = cfg.scaled(ny=8)
    sim = oracle.OracleSim.from_config(probe)
    for s, P in enumerate(W.generate_particles(probe)):
        sim.load_particles(s, **P)
    t = time.perf_counter()
    sim.step(1)
    per_row = (time.perf_counter() - t) / 8
    rows = int(max(8, min(cfg.ny, budget_s / max(per_row, 1e-6))))
    rows -= rows % 8
    rows = max(rows, 8)
    return cfg.scaled(ny=rows), rows


def run_oracle(cfg, steps: int, warmup: int, budget_total_s: float):
    import oracle
    from paper_1308_2590_gb300 import workloads as W
    oracle.build()
    per_step = budget_total_s / max(1, steps + warmup)
    scfg, rows = oracle_sample(cfg, per_step, steps)
    sim = oracle.OracleSim.from_config(scfg)
    for s, P in enumerate(W.generate_particles(scfg)):
        sim.load_particles(s, **P)
    sim.step(warmup)
    n = sim.diagnostics()["count"]
    t = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t
    n2 = sim.diagnostics()["count"]
    value = 0.5 * (n + n2) * steps / dt
    sample = (f"first {rows} of {cfg.ny} cell rows of the workload ({scfg.n_particles} particles), "
              f"{steps} oracle steps after {warmup} warm-up steps, single-threaded C + numpy")
    return value, sample, dt


def _oracle_replica(job):
    """One spawned process: the oracle on the given slice, timed over `steps`."""
    cfg, steps, warmup = job
    import oracle
    from paper_1308_2590_gb300 import workloads as W
    sim = oracle.OracleSim.from_config(cfg)
    for s, P in enumerate(W.generate_particles(cfg)):
        sim.load_particles(s, **P)
    sim.step(warmup)
    n = sim.diagnostics()["count"]
    t0 = time.time()
    sim.step(steps)
    t1 = time.time()
    n2 = sim.diagnostics()["count"]
    return 0.5 * (n + n2) * steps, t0, t1


def run_oracle_all_cores(cfg, rows: int, steps: int, warmup: int):
    """The oracle as it stands, one replica per host core on the same slice
    (processes started with spawn, before any CUDA context): aggregate
    particle-steps over the span from the first start to the last finish."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    ncores = os.cpu_count() or 1
    scfg = cfg.scaled(ny=rows)
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ["OMP_NUM_THREADS"] = os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        with mp.get_context("spawn").Pool(ncores) as pool:
            res = pool.map(_oracle_replica, [(scfg, steps, warmup)] * ncores)
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    work = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    sample = (f"{ncores} replicas of the first {rows} of {cfg.ny} cell rows ({scfg.n_particles} particles each), "
              f"{steps} oracle steps after {warmup} warm-up steps, one process per core")
    return work / span, sample, ncores


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--precision", choices=("fp64", "fp32"), default="fp64")
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--deposit", choices=("atomic", "deterministic"), default="atomic")
    ap.add_argument("--serve-runs", type=int, default=256)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-steps", type=int, default=200)
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-budget-gb", type=float, default=8.0, help="device-memory budget of the serving legs")
    ap.add_argument("--serve-burst-runs", type=int, default=64, help="runs of the submitted-at-once serving leg")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the field-dominated and full-size precision-form legs")
    ap.add_argument("--precision-steps", type=int, default=10)
    ap.add_argument("--single-form", action="store_true", help="time only the --precision form")
    args = ap.parse_args()
    rank, world, local = dist_env()
    metric = "particle-steps/s (gather+push+deposit)"
    cfg = workload(args.precision, args.deposit)
    config = {"workload": "laser-foil 1024x512 cells, 100-cell foil at 100 n_c, 64 particles/cell/species "
                          "(6,553,600 particles), literal field solve, absorbing x walls + a0=5 laser, periodic y",
              "run_steps": cfg.steps, "particles": cfg.n_particles, "grid": [cfg.nx, cfg.ny],
              "form": args.precision, "deposit": args.deposit, "l2": "particle state (>=340 MB) exceeds the 129 MB L2; no flush needed",
              "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}

    if args.impl == "reference":
        if rank != 0:
            return
        budget = 150.0
        value, sample, dt = run_oracle(cfg, args.steps, args.warmup, budget)
        line = {"impl": "reference", "metric": metric, "value": value, "unit": "particle-steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic (seeded)", "config": config,
                "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    # CPU baseline first (before any CUDA context), rank 0 at N = 1 only
    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        value, sample, dt = run_oracle(cfg, 4, 1, 20.0)
        cpu = {"value": value, "unit": "particle-steps/s", "cores": 1, "kind": "oracle", "sample": sample}
        v_all, s_all, ncores = run_oracle_all_cores(cfg, 64, 12, 1)
        cpu_all = {"value": v_all, "unit": "particle-steps/s", "cores": ncores, "kind": "oracle", "sample": s_all}

    r = run_gpu(args, rank, world, local)
    if rank != 0 and args.precision != "fp64":
        return
    r32 = None
    if args.precision == "fp64" and not args.single_form:
        # the FP32 form on the same workload, for the FP32-vs-FP64 comparison
        import copy
        a32 = copy.copy(args)
        a32.precision = "fp32"
        r32 = run_gpu(a32, rank, world, local)
    if rank != 0:
        return
    peaks, peak_src = measured_peaks()
    value = r["particle_steps"] / (r["ms"] * 1e-3)
    kms = r["kernel_ms"]
    la = r["launches"]
    roof = roofline(r, args.precision, args.deposit, args.steps, peaks, peak_src)
    serving = burst = field_dom = precision = ionization = cn_walls = shape2 = collisions = None
    if world == 1 and not args.no_serving:
        budget = int(args.serve_budget_gb * (1 << 30))
        serving = run_serving(args.serve_runs, args.serve_rate, args.serve_steps, args.serve_slots,
                              mem_budget=budget)
        if args.serve_burst_runs > 0:
            burst = run_serving(args.serve_burst_runs, args.serve_rate, args.serve_steps, args.serve_slots,
                                mem_budget=budget, burst=True)
    if world == 1 and not args.no_other_workloads:
        field_dom = run_field_dominated(min(args.steps, 200), max(3, args.warmup))
        precision = run_precision_form(args.precision_steps)
        ionization = run_ionization()
        cn_walls = run_cn_walls()
        shape2 = run_shapes()
        collisions = run_collisions()
    steps = args.steps
    line = {
        "metric": metric, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": r["ms"] / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic (seeded)",
        "config": config,
        "e2e": {"value": r["e2e"]["value"], "unit": "particle-steps/s", "h2d_bytes_per_step": int(r["e2e"]["h2d"]),
                "d2h_bytes_per_step": int(r["e2e"]["d2h"]),
                "loads": "prefetched (pic_prefetch_species / pic_load_prefetched, up to two steps ahead)"},
        "e2e_without_prefetch": {"value": r["e2e_direct"], "unit": "particle-steps/s",
                                 "loads": "pic_load_species from the page-locked arrays, in the step"},
        "gpu_launches": int(la[4]),
        "clocks": r["clocks"],
        "roofline": roof,
        "kernel_ms_per_step": {"particle": kms[0] / steps, "regroup": kms[1] / steps, "field_solve": kms[2] / steps,
                               "clear": kms[3] / steps},
        "field_solve_ms_per_step": kms[2] / steps,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
    }
    if r32 is not None:
        k32 = r32["kernel_ms"]
        line["fp32_form"] = {
            "value": r32["particle_steps"] / (r32["ms"] * 1e-3), "unit": "particle-steps/s",
            "ms_per_step": r32["ms"] / steps, "dtype": "f32", "clocks": r32["clocks"],
            "e2e": {"value": r32["e2e"]["value"], "unit": "particle-steps/s",
                    "h2d_bytes_per_step": int(r32["e2e"]["h2d"]), "d2h_bytes_per_step": int(r32["e2e"]["d2h"])},
            "e2e_without_prefetch": {"value": r32["e2e_direct"], "unit": "particle-steps/s"},
            "roofline": roofline(r32, "fp32", args.deposit, steps, peaks, peak_src),
            "kernel_ms_per_step": {"particle": k32[0] / steps, "regroup": k32[1] / steps,
                                   "field_solve": k32[2] / steps, "clear": k32[3] / steps},
            "speedup_vs_fp64": (r32["particle_steps"] / r32["ms"]) / (r["particle_steps"] / r["ms"])}
        line["gpu_launches"] = int(la[4] + r32["launches"][4])
    if serving is not None:
        line["serving"] = serving
    if burst is not None:
        line["serving_burst"] = burst
    if field_dom is not None:
        line["field_dominated"] = field_dom
    if precision is not None:
        line["precision_form"] = precision
    if ionization is not None:
        line["ionization"] = ionization
    if cn_walls is not None:
        line["cn_walls"] = cn_walls
    if shape2 is not None:
        line["shapes"] = shape2
    if collisions is not None:
        line["collisions"] = collisions
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
