"""Run a set of small cases with one build of the library and print, per
case, SHA-256 digests of the final state and the sticky flags (JSON, one line
per case).  Used by tests/test_gpu_checks.py to compare the checks build
(PIC_CHECKS) with the normal build.  Usage: python tests/checks_run.py LIB"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1308_2590_gb300 import pic, workloads as W  # noqa: E402
from tests.test_gpu_parity import hot, small_foil, small_uniform, wall_edge_particles  # noqa: E402


def _beam():
    """Dense beam that overflows its neighbour tile, a few particles crossing two tiles."""
    cfg = small_uniform(n=32, ppc=1, tile=4, field_mode=W.FIELD_LITERAL, dt=0.01)
    cfg.ny = 32
    rng = np.random.default_rng(3)
    n = 400
    x = (1.0 + 2.0 * rng.random(n)) * cfg.dx
    y = (0.5 + 3.0 * rng.random(n)) * cfg.dy
    ux = np.full(n, 3.0)
    ux[:5] = 40.0
    P = dict(x=x, y=y, ux=ux, uy=0.01 * rng.standard_normal(n), uz=np.zeros(n), w=np.full(n, 0.01))
    return cfg, [P, {k: v[:0] for k, v in P.items()}], 4


def cases():
    out = []
    for prec in (W.PREC_FP64, W.PREC_FP32):
        c = small_foil(precision=prec)
        out.append((f"foil-{prec}", c, None, c.steps))
        u = hot(small_uniform(tile=4, precision=prec), 20.0)
        out.append((f"uniform-cn-{prec}", u, None, 6))
        e = small_foil(nx=20, ny=8, ppc=1, steps=3, a0=0.0, precision=prec)
        out.append((f"wall-edge-{prec}", e, wall_edge_particles(e), 3))
    b, parts, steps = _beam()
    out.append(("beam-fallback", b, parts, steps))
    return out


def main():
    pic.lib(sys.argv[1])
    for name, cfg, parts, steps in cases():
        cfg.deposit = W.DEPOSIT_DETERMINISTIC
        if parts is None:
            parts = W.generate_particles(cfg)
        g = pic.Pic(cfg)
        g.pic_load_species(parts)
        g.pic_step(steps)
        d = g.pic_diagnostics()
        h = hashlib.sha256()
        h.update(g.pic_moments().tobytes())
        for a in g.pic_fields():
            h.update(a.tobytes())
        for s in range(len(parts)):
            P = g.pic_get_particles(s)
            for k in ("x", "y", "ux", "uy", "uz", "w", "cell"):
                h.update(P[k].tobytes())
        g.close()
        print(json.dumps({"case": name, "digest": h.hexdigest(), "flags": d["flags"], "count": d["count"]}), flush=True)


if __name__ == "__main__":
    main()
