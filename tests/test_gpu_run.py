"""The run driver (python -m paper_1308_2590_gb300.run): JSON lines of FP64
diagnostics every k steps, and a checkpoint it writes and resumes from
continues bitwise like the uninterrupted run (FP64, deterministic deposit)."""
import io
import json
import math

import pytest

from paper_1308_2590_gb300 import run as R, workloads as W
from tests.parity import stream

pytestmark = pytest.mark.gpu


def test_run_logs_and_resumes_from_its_checkpoint(tmp_path):
    cfg = W.config(1)
    cfg.deposit = W.DEPOSIT_DETERMINISTIC
    ckpt = str(tmp_path / "ckpt.npz")
    buf = io.StringIO()
    R.run(cfg, 12, 4, buf, checkpoint=ckpt, stream=stream())
    lines = [json.loads(s) for s in buf.getvalue().splitlines()]
    assert [d["step"] for d in lines] == [4, 8, 12]
    for d in lines:
        assert math.isfinite(d["total"]) and d["count"] == cfg.n_particles and d["cn_iterations"] > 0
        assert abs(d["drift"]) < 1e-2 and d["particle_steps_per_s"] > 0
    resumed = R.run(cfg, 6, 6, io.StringIO(), resume=ckpt, stream=stream())
    whole = R.run(cfg, 18, 18, io.StringIO(), stream=stream())
    assert resumed["step"] == whole["step"] == 18
    for k in ("kinetic", "field", "charge_grid", "count"):
        assert resumed[k] == whole[k], k
