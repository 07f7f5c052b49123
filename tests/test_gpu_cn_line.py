"""The line preconditioner of the implicit-curl (CN) field solve in boxes with walls (ny a power of
two): y-FFT, then per y-mode an exact block-tridiagonal solve along x with the column means of S and
the walls' Mur rows.  The solution must be the oracle's (the preconditioner changes only how fast
the FP32 inner solve converges): the laser foil at c dt/dx = 0.4 and 2, every particle, node and cell
within the FP64 tolerances.  In vacuum (no plasma) it is the exact inverse of the operator up to FP32
rounding, so each refinement's inner solve takes about one iteration."""
import numpy as np
import pytest

from paper_1308_2590_gb300 import pic, workloads as W
from tests.parity import compare_grid, compare_particles, density_scale, run_pair, stream
from tests.test_gpu_parity import small_foil

pytestmark = pytest.mark.gpu


def _foil(cdt, ny):
    cfg = small_foil(ny=ny, a0=4.0)
    cfg.field_mode = W.FIELD_CN
    cfg.cn_precond = W.CN_PRECOND_FFT
    cfg.dt = cdt * cfg.dx
    cfg.cn_tol = 1e-13
    cfg.cn_max_iter = 4000
    return cfg


@pytest.mark.parametrize("cdt", [0.4, 2.0])
def test_line_preconditioned_cn_foil_matches(cdt):
    cfg = _foil(cdt, 32)
    g, o = run_pair(cfg, cfg.steps)
    compare_particles(g, o, cfg)
    compare_grid(g, o, rho_scale=density_scale(cfg))
    dg, do = g.pic_diagnostics(), o.diagnostics()
    assert dg["count"] == do["count"] and dg["removed"] == do["removed"]
    for k in ("kinetic", "field"):
        assert abs(dg[k] - do[k]) <= 1e-9 * abs(do[k]) + 1e-15, (k, dg[k], do[k])
    assert dg["cn_residual"] < 1e-12, dg
    print("line", cdt, dg["cn_iterations"], dg["cn_refinements"])
    g.close()


@pytest.mark.parametrize("cdt", [0.4, 2.0])
def test_line_preconditioner_needs_fewer_iterations_than_block_jacobi(cdt):
    """The same foil with the line preconditioner and with block-Jacobi: the last solve's inner iterations."""
    its = {}
    for pre in (W.CN_PRECOND_FFT, W.CN_PRECOND_JACOBI):
        cfg = _foil(cdt, 32)
        cfg.cn_precond = pre
        g = pic.Pic(cfg, stream=stream())
        g.pic_load_species(W.generate_particles(cfg))
        g.pic_step(cfg.steps)
        its[pre] = g.pic_diagnostics()["cn_iterations"]
        g.close()
    print("iterations line / block-Jacobi", cdt, its)
    assert its[W.CN_PRECOND_FFT] < its[W.CN_PRECOND_JACOBI], its


def test_line_preconditioner_inverts_the_vacuum_operator():
    """No plasma: about one FP32 iteration per FP64 refinement."""
    cfg = small_foil(ny=64, a0=4.0)
    cfg.field_mode = W.FIELD_CN
    cfg.cn_precond = W.CN_PRECOND_FFT
    cfg.dt = 2.0 * cfg.dx
    cfg.cn_tol = 1e-13
    g = pic.Pic(cfg, stream=stream())
    for _ in range(6):
        g.pic_step(1)
        d = g.pic_diagnostics()
        assert d["cn_residual"] < 1e-12
        assert d["cn_iterations"] <= 2 * max(d["cn_refinements"], 1), d
    E, H = g.pic_fields()
    assert np.max(np.abs(E)) > 0.1          # the laser came in
    g.close()
