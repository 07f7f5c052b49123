"""Bounded device waits, tested without a GPU fault: a kernel waits on an
mbarrier that nothing completes, gives up after the push's poll bound and
returns the timeout status after about a second; the context stays usable
afterwards."""
import numpy as np
import pytest

from paper_1308_2590_gb300 import pic, workloads as W
from tests.parity import stream
from tests.test_gpu_parity import small_foil

pytestmark = pytest.mark.gpu


def _run(cfg, parts, steps):
    g = pic.Pic(cfg, stream=stream())
    g.pic_load_species(parts)
    g.pic_step(steps)
    M = g.pic_moments()
    d = g.pic_diagnostics()
    g.close()
    return M, d


def test_bounded_wait_times_out_and_context_stays_usable():
    cfg = small_foil()
    cfg.deposit = W.DEPOSIT_DETERMINISTIC
    parts = W.generate_particles(cfg)
    before = _run(cfg, parts, 4)
    rc, seconds = pic.selftest_wait(stream())
    assert rc == pic.PIC_ERR_TIMEOUT
    assert 0.5 < seconds < 10.0   # the wait gives up after about one second
    after = _run(cfg, parts, 4)   # same inputs, same bits: nothing left behind
    assert np.array_equal(before[0], after[0])
    assert before[1]["kinetic"] == after[1]["kinetic"] and before[1]["flags"] == after[1]["flags"] == 0
