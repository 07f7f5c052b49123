"""Serving on the GPU: independent laser-foil runs admitted by device memory
and slots, stepped together on their own streams (or, optionally, by batched
steps: one push and one regroup launch for all admitted runs of one form).

Each served result must be the same alone and in the mix: with the
deterministic deposit bitwise (moments, fields, diagnostics); with the atomic
deposit within the FP32 form's moment tolerance (1e-5 relative, normwise).
"""
import time

import numpy as np
import pytest

from paper_1308_2590_gb300 import pic, workloads as W
from tests.parity import normwise, stream
from tests.test_gpu_parity import hot, small_uniform

pytestmark = pytest.mark.gpu


def _runs(deposit, n=5):
    """Small laser-foil runs of different sizes (the serving workload's shape)."""
    out = []
    shapes = [(64, 48, 6, 60.0, 3.0), (96, 32, 4, 120.0, 8.0), (48, 64, 8, 30.0, 15.0), (80, 40, 5, 200.0, 1.5),
              (64, 64, 3, 10.0, 20.0), (40, 40, 7, 90.0, 5.0)]
    for k, (nx, ny, ppc, dens, a0) in enumerate(shapes[:n]):
        thick = max(1, round(nx / 10))
        cfg = W.laser_foil(f"serve-test-{k}", nx, ny, (nx - thick) // 2, thick, dens, ppc, 12, a0,
                           seed=500 + k, precision=W.PREC_FP32, tile=8)
        cfg.laser.tau = 6.0
        cfg.laser.t0 = 6.0
        cfg.deposit = deposit
        out.append(cfg)
    return out


def _alone(cfg, parts, steps):
    g = pic.Pic(cfg, stream=stream())
    for s, P in enumerate(parts):
        g.load(s, P)
    g.pic_step(steps)
    d = g.pic_diagnostics()
    M = g.pic_moments()
    E, H = g.pic_fields()
    g.close()
    return d, M, E, H


def _serve(cfgs, parts, steps, max_slots, stagger_s=0.0, batch_min_runs=0):
    with pic.Server(max_slots=max_slots, batch_min_runs=batch_min_runs) as srv:
        ids = []
        for cfg, P in zip(cfgs, parts):
            ids.append(srv.submit(cfg, P, steps, keep_grids=True))
            if stagger_s:
                time.sleep(stagger_s)
        srv.wait_all(300.0)
        out = []
        for rid in ids:
            st = srv.status(rid)
            assert st["state"] == pic.REQ_DONE, st
            d, (M, E, H) = srv.result(rid, grids=True)
            out.append((d, M, E, H, st))
            srv.release(rid)
    return out


@pytest.mark.parametrize("max_slots,stagger,batch", [(8, 0.0, 0), (2, 0.002, 0), (8, 0.0, 2)])
def test_served_runs_same_alone_and_in_mix_bitwise(max_slots, stagger, batch):
    """Per-run streams, a two-slot server with staggered arrivals, and batched
    steps (one push and one regroup launch for all admitted runs)."""
    cfgs = _runs(W.DEPOSIT_DETERMINISTIC)
    parts = [W.generate_particles(c) for c in cfgs]
    steps = 12
    alone = [_alone(c, P, steps) for c, P in zip(cfgs, parts)]
    served = _serve(cfgs, parts, steps, max_slots, stagger, batch)
    for (da, Ma, Ea, Ha), (ds, Ms, Es, Hs, st) in zip(alone, served):
        assert np.array_equal(Ma, Ms)
        assert np.array_equal(Ea, Es)
        assert np.array_equal(Ha, Hs)
        for k in ("kinetic", "field", "charge_grid", "count", "removed", "step"):
            assert da[k] == ds[k], k
        assert st["steps_done"] == steps
        assert st["t_submit"] <= st["t_start"] <= st["t_finish"]


def test_served_runs_same_alone_and_in_mix_atomic_within_tolerance():
    cfgs = _runs(W.DEPOSIT_ATOMIC)
    parts = [W.generate_particles(c) for c in cfgs]
    steps = 12
    alone = [_alone(c, P, steps) for c, P in zip(cfgs, parts)]
    served = _serve(cfgs, parts, steps, 8)
    for (da, Ma, Ea, Ha), (ds, Ms, Es, Hs, st) in zip(alone, served):
        assert normwise(Ms[0], Ma[0], max(np.max(np.abs(Ma[0])), 1e-30)) < 1e-5
        assert normwise(Ms[1:10], Ma[1:10]) < 1e-5
        assert normwise(Ms[10:13], Ma[10:13]) < 1e-5
        assert da["count"] == ds["count"]
        assert abs(da["kinetic"] - ds["kinetic"]) <= 1e-5 * abs(da["kinetic"])


def test_admission_respects_memory_budget_and_slots():
    cfgs = _runs(W.DEPOSIT_ATOMIC, n=6)
    parts = [W.generate_particles(c) for c in cfgs]
    est = [pic.estimate_bytes(c, [P["x"].size for P in ps]) for c, ps in zip(cfgs, parts)]
    budget = sorted(est)[-1] + sorted(est)[-2]     # any two runs fit, not always three
    with pic.Server(mem_budget=budget, max_slots=8) as srv:
        ids = [srv.submit(c, P, 12) for c, P in zip(cfgs, parts)]
        # a run that can never fit fails at once with PIC_ERR_OOM
        big = cfgs[0].scaled(nx=2048, ny=2048)
        big_id = srv.submit(big, [{k: v[:0] for k, v in P.items()} for P in parts[0]], 1)
        st_big = srv.status(big_id)
        assert st_big["state"] == pic.REQ_FAILED and st_big["error"] == pic.PIC_ERR_OOM
        srv.wait_all(300.0)
        sts = [srv.status(i) for i in ids]
    assert all(s["state"] == pic.REQ_DONE for s in sts)
    # at every admission, the admitted runs' estimates fit the budget
    for s in sts:
        t = s["t_start"]
        live = [o for o in sts if o["t_start"] <= t < o["t_finish"]]
        assert sum(o["device_bytes"] for o in live) <= budget
    # arrival order is kept
    starts = [s["t_start"] for s in sts]
    assert starts == sorted(starts)


def test_slot_limit_and_invalid_requests():
    cfgs = _runs(W.DEPOSIT_ATOMIC, n=4)
    parts = [W.generate_particles(c) for c in cfgs]
    with pic.Server(max_slots=1) as srv:
        ids = [srv.submit(c, P, 6) for c, P in zip(cfgs, parts)]
        with pytest.raises(pic.PicError):
            srv.submit(cfgs[0].scaled(nx=1), parts[0], 6)
        srv.wait_all(300.0)
        sts = [srv.status(i) for i in ids]
        with pytest.raises(pic.PicError):
            srv.result(ids[0], grids=True)     # grids were not kept
        d, _ = srv.result(ids[0])
        assert d["step"] == 6
    # one slot: the runs never overlap
    for a, b in zip(sts, sts[1:]):
        assert a["t_finish"] <= b["t_start"]


def _state(g):
    out = [g.pic_moments(), *g.pic_fields()]
    for s in range(g.nsp):
        P = g.pic_get_particles(s)
        out += [P[k] for k in ("x", "y", "ux", "uy", "uz", "w", "cell")]
    return out


@pytest.mark.parametrize("precision", [W.PREC_FP32, W.PREC_FP64])
def test_batched_step_equals_single_runs_bitwise(precision):
    """One push and one regroup launch over several runs (laser foils of
    different sizes and a CN uniform plasma) give bitwise the same state as
    stepping each run alone (deterministic deposit)."""
    cfgs = _runs(W.DEPOSIT_DETERMINISTIC, n=4)
    uni = hot(small_uniform(tile=8), 20.0)
    uni.nx, uni.ny = 32, 16
    cfgs.append(uni)
    for c in cfgs:
        c.precision = precision
        c.deposit = W.DEPOSIT_DETERMINISTIC
    parts = [W.generate_particles(c) for c in cfgs]

    def make(c, P):
        g = pic.Pic(c, stream=stream())
        for s, Q in enumerate(P):
            g.load(s, Q)
        return g

    alone = []
    for c, P in zip(cfgs, parts):
        g = make(c, P)
        g.pic_step(7)
        alone.append(_state(g))
        g.close()
    runs = [make(c, P) for c, P in zip(cfgs, parts)]
    b = pic.Batch(8, stream=stream())
    b.step(runs, 3)
    b.step(runs[1:], 2)        # a smaller batch in between
    runs[0].pic_step(2)        # and a run stepped on its own
    b.step(runs, 2)
    for g, ref in zip(runs, alone):
        got = _state(g)
        for x, y in zip(ref, got):
            assert x.shape == y.shape and np.array_equal(x.view(np.uint8), y.view(np.uint8))
        g.close()
    b.close()


def test_batched_step_rejects_mixed_forms():
    c32 = _runs(W.DEPOSIT_ATOMIC, n=1)[0]
    c64 = c32.scaled(precision=W.PREC_FP64)
    g1, g2 = pic.Pic(c32, stream=stream()), pic.Pic(c64, stream=stream())
    b = pic.Batch(4, stream=stream())
    with pytest.raises(pic.PicError):
        b.step([g1, g2], 1)
    b.close()
    g1.close()
    g2.close()


def test_cancel_queued_and_running_requests():
    """A queued request leaves the queue at once; a running one stops after a
    few steps and frees its slot; the other runs finish with bitwise the
    results they have alone."""
    cfgs = _runs(W.DEPOSIT_DETERMINISTIC, n=4)
    parts = [W.generate_particles(c) for c in cfgs]
    long_steps, steps = 4000, 12
    alone = [_alone(c, P, steps) for c, P in zip(cfgs[2:], parts[2:])]
    with pic.Server(max_slots=1) as srv:
        victim = srv.submit(cfgs[0], parts[0], long_steps)            # runs first, cancelled mid-run
        queued = srv.submit(cfgs[1], parts[1], long_steps)            # cancelled while queued
        ids = [srv.submit(c, P, steps, keep_grids=True) for c, P in zip(cfgs[2:], parts[2:])]
        srv.cancel(queued)
        assert srv.status(queued)["state"] == pic.REQ_CANCELLED
        deadline = time.time() + 120.0
        while srv.status(victim)["steps_done"] < 3 and time.time() < deadline:
            time.sleep(0.001)
        srv.cancel(victim)
        with pytest.raises(pic.PicError):
            srv.cancel(victim)                                        # already cancelled
        srv.wait_all(300.0)
        sv, sq = srv.status(victim), srv.status(queued)
        assert sv["state"] == pic.REQ_CANCELLED and 3 <= sv["steps_done"] < long_steps
        assert sv["t_start"] <= sv["t_finish"]
        assert sq["state"] == pic.REQ_CANCELLED and sq["steps_done"] == 0
        with pytest.raises(pic.PicError):
            srv.result(victim)
        for rid, (da, Ma, Ea, Ha) in zip(ids, alone):
            st = srv.status(rid)
            assert st["state"] == pic.REQ_DONE
            ds, (Ms, Es, Hs) = srv.result(rid, grids=True)
            assert np.array_equal(Ma, Ms) and np.array_equal(Ea, Es) and np.array_equal(Ha, Hs)
            assert da["kinetic"] == ds["kinetic"]
        with pytest.raises(pic.PicError):
            srv.cancel(ids[0])                                        # finished
        with pytest.raises(pic.PicError):
            srv.cancel(123456789)                                     # unknown
        srv.release(victim)
        srv.release(queued)


def test_admitted_run_whose_allocation_fails():
    """A run the budget admits but the device cannot hold fails with
    PIC_ERR_OOM when it is started (its partial allocations freed); the server
    keeps serving."""
    cfgs = _runs(W.DEPOSIT_ATOMIC, n=2)
    parts = [W.generate_particles(c) for c in cfgs]
    huge = cfgs[0].scaled(nx=32768, ny=32768, precision=W.PREC_FP64)   # ~0.4 TB of grid arrays
    with pic.Server(mem_budget=1 << 50, max_slots=4) as srv:
        bad = srv.submit(huge, [{k: v[:0] for k, v in P.items()} for P in parts[0]], 1)
        good = srv.submit(cfgs[1], parts[1], 6)
        srv.wait_all(300.0)
        sb, sg = srv.status(bad), srv.status(good)
    assert sb["state"] == pic.REQ_FAILED and sb["error"] == pic.PIC_ERR_OOM
    assert sg["state"] == pic.REQ_DONE and sg["steps_done"] == 6
