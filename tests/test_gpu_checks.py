"""The checks build (PIC_CHECKS: indices in range, offsets in [0, 1),
regroup destinations inside their bin, the push's shared-memory canary) runs
the small cases -- laser foil, hot CN plasma and particles just inside the far
wall in both forms, and a beam that forces the fallback regroup -- without
reporting a broken invariant, and gives bitwise the normal build's results."""
import json
import os
import subprocess
import sys

import pytest

from paper_1308_2590_gb300 import build as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(lib):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checks_run.py"), lib], capture_output=True,
                       text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout + r.stderr
    return [json.loads(line) for line in r.stdout.splitlines() if line.startswith("{")]


def test_checks_build_reports_nothing_and_matches_normal_build():
    lib, lib_checks = B.build(), B.build(checks=True)
    with open(lib, "rb") as f, open(lib_checks, "rb") as fc:
        assert lib != lib_checks and f.read() != fc.read()   # the checks are compiled in
    normal = _run(lib)
    checked = _run(lib_checks)
    assert len(normal) == len(checked) == 7
    for a, b in zip(normal, checked):
        assert a["case"] == b["case"]
        # bit 0 only records a move farther than one tile (the hot plasma makes some); the
        # checks build's own bit is 32
        assert not (b["flags"] & 32) and a["flags"] == b["flags"], (a, b)
        assert a["digest"] == b["digest"], (a, b)
        assert a["count"] == b["count"]
