"""Checkpoint and resume through the C ABI: a run saved after k steps
(pic_save_particles, pic_fields, the step count) and restored into a fresh
handle (pic_restore_particles, pic_set_fields, pic_set_step) continues like
the uninterrupted run -- the laser foil with walls and the source (literal
mode) and the hot periodic plasma (CN mode), with the deterministic deposit.
FP64 form: bitwise (every corner contribution is rounded to fixed point on
its own, so the moments the new handle deposits at rest are exactly the ones
the step deposited).  FP32 form: within its tolerance (its push sums a warp's
contributions in FP32 registers before the rounding, the deposit at rest
groups them differently).  Also: the checkpoint form round-trips exactly, and
an invalid checkpoint particle is refused."""
import numpy as np
import pytest

from paper_1308_2590_gb300 import pic, workloads as W
from tests.parity import density_scale, normwise, stream
from tests.test_gpu_parity import hot, small_foil, small_uniform

pytestmark = pytest.mark.gpu

CKEYS = ("cell", "ox", "oy", "ux", "uy", "uz", "w")


def _state(g, nsp):
    out = [g.pic_moments(), *g.pic_fields()]
    for s in range(nsp):
        P = g.pic_save_particles(s)
        out += [P[k] for k in CKEYS]
    return out


def _equal(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x.shape == y.shape and np.array_equal(x.view(np.uint8), y.view(np.uint8))


def _cfg(kind, precision):
    if kind == "foil":
        cfg = small_foil(precision=precision)
        cfg.laser.t0 = 2.0       # the pulse is on while the run is split
    else:
        cfg = hot(small_uniform(tile=4, precision=precision), 20.0)
        cfg.cn_tol = 1e-12
    cfg.deposit = W.DEPOSIT_DETERMINISTIC
    return cfg


@pytest.mark.parametrize("kind", ["foil", "uniform"])
@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32])
def test_resume_from_checkpoint_is_bitwise(kind, precision):
    cfg = _cfg(kind, precision)
    parts = W.generate_particles(cfg)
    nsp = len(parts)
    k, total = 5, 10
    whole = pic.Pic(cfg, stream=stream())
    whole.pic_load_species(parts)
    whole.pic_step(total)
    ref = _state(whole, nsp)
    whole.close()

    first = pic.Pic(cfg, stream=stream())
    first.pic_load_species(parts)
    first.pic_step(k)
    E, H = first.pic_fields()
    saved = [first.pic_save_particles(s) for s in range(nsp)]
    step = first.pic_diagnostics()["step"]
    first.close()
    assert step == k

    resumed = pic.Pic(cfg, stream=stream())
    for s, P in enumerate(saved):
        resumed.pic_restore_particles(s, P)
    resumed.pic_set_fields(E, H)
    resumed.pic_set_step(step)
    _equal(saved_flat(saved), saved_flat([resumed.pic_save_particles(s) for s in range(nsp)]))   # exact round trip
    resumed.pic_step(total - k)
    got = _state(resumed, nsp)
    if precision == W.PREC_FP64:
        _equal(ref, got)
    else:
        Mr, Mg = ref[0], got[0]
        assert normwise(Mg[0], Mr[0], density_scale(cfg)) < 1e-5
        assert normwise(Mg[1:10], Mr[1:10]) < 1e-5 and normwise(Mg[10:13], Mr[10:13]) < 1e-5
        for a, b in zip(ref[1:3], got[1:3]):
            assert normwise(b, a) < 1e-5
        for s in range(nsp):
            u_ref = np.stack([ref[3 + 7 * s + j] for j in (3, 4, 5)])
            u_got = np.stack([got[3 + 7 * s + j] for j in (3, 4, 5)])
            assert u_ref.shape == u_got.shape and normwise(u_got, u_ref) < 1e-5
    assert resumed.pic_diagnostics()["step"] == total
    resumed.close()


def saved_flat(saved):
    return [P[k] for P in saved for k in CKEYS]


def test_checkpoint_form_round_trips_and_is_checked():
    cfg = _cfg("foil", W.PREC_FP64)
    parts = W.generate_particles(cfg)
    g = pic.Pic(cfg, stream=stream())
    g.pic_load_species(parts)
    g.pic_step(3)
    saved = [g.pic_save_particles(s) for s in range(2)]
    h = pic.Pic(cfg, stream=stream())
    for s, P in enumerate(saved):
        h.pic_restore_particles(s, P)
    _equal(saved_flat(saved), saved_flat([h.pic_save_particles(s) for s in range(2)]))
    for key, value in (("cell", cfg.nx * cfg.ny), ("ox", 1.0), ("oy", -1e-3), ("uz", np.inf)):
        bad = {k: v.copy() for k, v in saved[0].items()}
        bad[key][7] = value
        e = pic.Pic(cfg, stream=stream())
        with pytest.raises(pic.PicError, match="particle 7"):
            e.pic_restore_particles(0, bad)
        assert e.pic_particle_count(0) == 0
        e.close()
    with pytest.raises(pic.PicError):
        h.pic_set_step(-1)
    g.close()
    h.close()
