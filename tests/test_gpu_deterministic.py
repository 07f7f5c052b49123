"""Deterministic deposit (PIC_DEPOSIT_DETERMINISTIC) on the GPU.

Every corner contribution is rounded once to 64-bit fixed point and summed
with integer additions, so repeated runs on the same inputs give bitwise the
same moments, fields and particles, whatever order the atomics land in.  The
run must also stay within the oracle tolerances of its form: FP64 1e-9 on
moments and fields, 1e-10 on particles; FP32 1e-5 on moments.
"""
import numpy as np
import pytest

from paper_1308_2590_gb300 import pic, workloads as W
from tests.parity import (compare_grid, compare_particles, density_scale, normwise, run_pair, stream)
from tests.test_gpu_parity import small_foil, small_uniform, hot

pytestmark = pytest.mark.gpu


def _state(g, nsp):
    out = [g.pic_moments(), *g.pic_fields()]
    for s in range(nsp):
        P = g.pic_get_particles(s)
        out += [P[k] for k in ("x", "y", "ux", "uy", "uz", "w", "cell")]
    return out


def _run(cfg, steps, parts):
    g = pic.Pic(cfg, stream=stream())
    for s, P in enumerate(parts):
        g.load(s, P)
    g.pic_step(steps)
    st = _state(g, len(cfg.species))
    g.close()
    return st


def _bitwise_equal(a, b):
    for x, y in zip(a, b):
        assert x.dtype == y.dtype and x.shape == y.shape
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))


@pytest.mark.parametrize("maker", ["foil", "uniform"])
@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32])
def test_deterministic_deposit_is_bitwise_reproducible(maker, precision):
    if maker == "foil":
        cfg = small_foil(precision=precision)
        steps = cfg.steps
    else:
        cfg = hot(small_uniform(precision=precision), 20.0)
        cfg.cn_tol = 1e-10 if precision == W.PREC_FP32 else 1e-14
        steps = 6
    cfg.deposit = W.DEPOSIT_DETERMINISTIC
    parts = W.generate_particles(cfg)
    ref = _run(cfg, steps, parts)
    for _ in range(2):
        _bitwise_equal(ref, _run(cfg, steps, parts))


def test_deterministic_deposit_bitwise_with_other_work_interleaved():
    """Two handles stepped alternately on the same stream: the one under test
    gives the same bits as when it runs alone."""
    cfg = small_foil()
    cfg.deposit = W.DEPOSIT_DETERMINISTIC
    parts = W.generate_particles(cfg)
    alone = _run(cfg, 8, parts)
    other_cfg = hot(small_uniform(), 30.0)
    other = pic.Pic(other_cfg, stream=stream())
    for s, P in enumerate(W.generate_particles(other_cfg)):
        other.load(s, P)
    g = pic.Pic(cfg, stream=stream())
    for s, P in enumerate(parts):
        g.load(s, P)
    for _ in range(8):
        other.pic_step(1)
        g.pic_step(1)
    mixed = _state(g, len(cfg.species))
    g.close()
    other.close()
    _bitwise_equal(alone, mixed)


@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32])
def test_overlapped_steps_equal_serialised_steps(precision):
    """pic_step(n) runs each literal field solve on the handle's second stream
    beside the previous step's regroup, ordered by events; with the exact
    deposit it must give the bits of n single steps each followed by a full
    synchronisation, where no two steps' kernels run at once."""
    cfg = small_foil(nx=256, ny=128, ppc=16, precision=precision)
    cfg.laser.t0 = 2.0
    cfg.deposit = W.DEPOSIT_DETERMINISTIC
    parts = W.generate_particles(cfg)
    steps = 12
    overlapped = _run(cfg, steps, parts)
    g = pic.Pic(cfg, stream=stream())
    for s, P in enumerate(parts):
        g.load(s, P)
    for _ in range(steps):
        g.pic_step(1)
        g.pic_sync()
    serial = _state(g, len(cfg.species))
    g.close()
    _bitwise_equal(overlapped, serial)


@pytest.mark.parametrize("maker,tile", [("foil", 8), ("uniform", 4), ("uniform", 8)])
def test_deterministic_deposit_matches_oracle_fp64(maker, tile):
    if maker == "foil":
        cfg = small_foil(tile=tile)
        steps = cfg.steps
    else:
        cfg = hot(small_uniform(tile=tile), 20.0)
        steps = 6
    cfg.deposit = W.DEPOSIT_DETERMINISTIC
    g, o = run_pair(cfg, steps)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    g.close()


def test_deterministic_deposit_matches_oracle_fp32():
    cfg = small_foil(precision=W.PREC_FP32)
    cfg.deposit = W.DEPOSIT_DETERMINISTIC
    g, o = run_pair(cfg, cfg.steps)
    Mg, Mo = g.pic_moments(), o.M
    assert normwise(Mg[0], Mo[0], density_scale(cfg)) < 1e-5
    assert normwise(Mg[1:10], Mo[1:10]) < 1e-5
    assert normwise(Mg[10:13], Mo[10:13]) < 1e-5
    g.close()


def test_deterministic_and_atomic_deposits_agree_fp64():
    """Same run, both deposits: the sums differ only by rounding order."""
    cfg = small_foil()
    parts = W.generate_particles(cfg)
    a = _run(cfg, cfg.steps, parts)
    cfg.deposit = W.DEPOSIT_DETERMINISTIC
    d = _run(cfg, cfg.steps, parts)
    for k in (0,):
        Ma, Md = a[k], d[k]
        for lo, hi in ((0, 1), (1, 10), (10, 13)):
            assert normwise(Md[lo:hi], Ma[lo:hi]) < 1e-12
