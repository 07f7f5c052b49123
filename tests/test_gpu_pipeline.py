"""Steps queued ahead of the regroup decision.

Within one pic_step call every step's particle kernels are queued before the
host has read the previous step's regroup flags; they do nothing if that
regroup failed (a bin overflow or a move farther than a neighbour tile), and
the host then regroups with the full sort and queues the step again.  Between
calls the flags are resolved before anything else runs.  With the exact
(deterministic) deposit the two schedules must give bitwise the same moments,
fields and particles, also when full regroups happen on the way; with the
L2-reduction deposit they must agree with the oracle as any step does.
Batched steps of several runs are queued the same way: a run whose regroup
failed takes no part in the next batched push and regroup and is redone alone.
"""
import numpy as np
import pytest

from paper_1308_2590_gb300 import pic, workloads as W
from tests.parity import compare_grid, compare_particles, run_pair, stream
from tests.test_gpu_parity import small_uniform

pytestmark = pytest.mark.gpu

STEPS = 4


def _beam_config(precision, field_mode):
    """A dense beam leaving its tile for an empty neighbour (bin overflow) and a few
    particles crossing more than one tile per step (far moves)."""
    cfg = small_uniform(n=32, ppc=1, tile=4, field_mode=field_mode, dt=0.01, precision=precision)
    cfg.ny = 32
    cfg.dx = cfg.dy = 0.02
    if precision == W.PREC_FP32:
        cfg.cn_tol = 1e-10
    n = 400
    rng = np.random.default_rng(11)
    x = (1.0 + 2.0 * rng.random(n)) * cfg.dx          # all in cells 1..2 of tile (0, 0)
    y = (0.5 + 3.0 * rng.random(n)) * cfg.dy
    ux = np.full(n, 3.0)                               # ~2.8 cells per step: into tile (1, 0)
    ux[:5] = 40.0                                      # ~5 cells per step: two tiles away
    P = dict(x=x, y=y, ux=ux, uy=0.01 * rng.standard_normal(n), uz=np.zeros(n), w=np.full(n, 0.01))
    empty = dict((k, v[:0]) for k, v in P.items())
    return cfg, [P, empty]


def _state(g, nsp):
    out = [g.pic_moments(), *g.pic_fields()]
    for s in range(nsp):
        P = g.pic_get_particles(s)
        out += [P[k] for k in ("x", "y", "ux", "uy", "uz", "w", "cell")]
    return out


def _run(cfg, parts, calls, sync=False):
    g = pic.Pic(cfg, stream=stream())
    for s, P in enumerate(parts):
        g.load(s, P)
    for n in calls:
        g.pic_step(n)
        if sync:
            g.pic_sync()   # the step's regroup resolved (and a failed one redone) before the next call
    full = g.pic_diagnostics()["full_regroups"]
    st = _state(g, len(cfg.species))
    g.close()
    return st, full


@pytest.mark.parametrize("field_mode", [W.FIELD_LITERAL, W.FIELD_CN])
@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32])
def test_queued_steps_equal_single_step_calls_bitwise_with_full_regroups(precision, field_mode):
    cfg, parts = _beam_config(precision, field_mode)
    cfg.deposit = W.DEPOSIT_DETERMINISTIC
    queued, full_q = _run(cfg, parts, [STEPS])                    # one call: every step queued ahead
    single, full_s = _run(cfg, parts, [1] * STEPS, sync=True)      # each step resolved before the next
    mixed, full_m = _run(cfg, parts, [1, STEPS - 1])
    assert full_q >= 1 and full_q == full_s == full_m           # the fallbacks happened, in every schedule
    for other in (single, mixed):
        for a, b in zip(queued, other):
            assert a.dtype == b.dtype and a.shape == b.shape
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8))


@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32])
def test_queued_steps_with_full_regroups_match_the_oracle(precision):
    cfg, parts = _beam_config(precision, W.FIELD_LITERAL)
    g, o = run_pair(cfg, STEPS, parts=parts)
    assert g.pic_diagnostics()["full_regroups"] >= 1
    if precision == W.PREC_FP64:
        compare_particles(g, o, cfg)
        compare_grid(g, o, rho_scale=1.0)
    else:
        Mg, Mo = g.pic_moments(), o.M
        err = np.max(np.abs(Mg - Mo)) / np.max(np.abs(Mo))
        assert err < 1e-4, err
    g.close()


def _loaded(cfg, parts):
    g = pic.Pic(cfg, stream=stream())
    for s, P in enumerate(parts):
        g.load(s, P)
    return g


@pytest.mark.parametrize("field_mode", [W.FIELD_LITERAL, W.FIELD_CN])
@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32])
def test_batched_steps_with_full_regroups_equal_runs_alone_bitwise(precision, field_mode):
    beam, beam_parts = _beam_config(precision, field_mode)
    plain = small_uniform(n=32, ppc=3, tile=4, field_mode=field_mode, dt=0.01, precision=precision)
    if precision == W.PREC_FP32:
        plain.cn_tol = 1e-10
    cfgs = [(beam, beam_parts), (plain, W.generate_particles(plain)), (beam, beam_parts)]
    for c, _ in cfgs:
        c.deposit = W.DEPOSIT_DETERMINISTIC
    alone, full_alone = [], []
    for c, P in cfgs:
        st, full = _run(c, P, [STEPS])
        alone.append(st)
        full_alone.append(full)
    assert full_alone[0] >= 1
    runs = [_loaded(c, P) for c, P in cfgs]
    b = pic.Batch(4, stream=stream())
    b.step(runs, 1)
    b.step(runs, STEPS - 2)    # queued ahead of the first call's regroup decisions
    b.step(runs[1:], 1)        # a smaller batch: run 0 goes on alone
    runs[0].pic_step(1)
    for g, (c, _), ref, full in zip(runs, cfgs, alone, full_alone):
        assert g.pic_diagnostics()["full_regroups"] == full
        got = _state(g, len(c.species))
        for x, y in zip(ref, got):
            assert x.dtype == y.dtype and x.shape == y.shape
            assert np.array_equal(x.view(np.uint8), y.view(np.uint8))
        g.close()
    b.close()
