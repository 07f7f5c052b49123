"""FP32 form on the GPU: particles, offsets and moments in FP32 with a TwoSum-
compensated flush of the moment sums; checked against the FP64 oracle and the
FP64 GPU form on the same seeded inputs.

Targets: moments within 1e-5 relative (normwise), total energy within 0.1 %
of the FP64 run; particle state within 1e-5 (positions relative to the box,
momenta relative to the largest momentum) over the short runs below."""
import numpy as np
import pytest

from paper_1308_2590_gb300 import pic, workloads as W
from tests.parity import density_scale, normwise, run_pair, stream
from tests.test_gpu_parity import small_foil, small_uniform, hot

pytestmark = pytest.mark.gpu

MOM_RTOL = 1e-5
PART_RTOL = 1e-5


def _errors(g, o, cfg):
    errs = {}
    Mg, Mo = g.pic_moments(), o.M
    errs["rho"] = normwise(Mg[0], Mo[0], density_scale(cfg))
    errs["S"] = normwise(Mg[1:10], Mo[1:10])
    errs["dj"] = normwise(Mg[10:13], Mo[10:13])
    Lx, Ly = cfg.nx * cfg.dx, cfg.ny * cfg.dy
    ex = eu = 0.0
    for s in range(len(cfg.species)):
        a, b = g.pic_get_particles(s), o.particles(s)
        assert a["x"].size == b["x"].size
        if a["x"].size == 0:
            continue
        dxp = np.abs(a["x"] - b["x"])
        if cfg.bc_x == W.BC_PERIODIC:
            dxp = np.minimum(dxp, Lx - dxp)
        dyp = np.abs(a["y"] - b["y"])
        dyp = np.minimum(dyp, Ly - dyp)
        ex = max(ex, float(np.max(dxp)) / Lx, float(np.max(dyp)) / Ly)
        us = max(np.max(np.abs(b[k])) for k in ("ux", "uy", "uz"))
        eu = max(eu, max(normwise(a[k], b[k], us) for k in ("ux", "uy", "uz")))
    errs["x"] = ex
    errs["u"] = eu
    return errs


@pytest.mark.parametrize("maker,mom_rtol", [("foil", MOM_RTOL), ("uniform-1keV", MOM_RTOL), ("uniform-30keV", 5e-5)])
def test_fp32_form_within_targets_of_fp64_oracle(maker, mom_rtol):
    """Workload conditions (the laser foil, the 1 keV uniform plasma) meet 1e-5 on the
    moments.  A 30 keV plasma moving ~6 cells per step is held to 5e-5: there the FP32
    position error (~1e-5 cell per step from the FP32 velocity) dominates the moments."""
    if maker == "foil":
        cfg = small_foil(precision=W.PREC_FP32)
        steps = cfg.steps
    elif maker == "uniform-1keV":
        cfg = small_uniform(precision=W.PREC_FP32)
        cfg.cn_tol = 1e-10
        steps = 10
    else:
        cfg = hot(small_uniform(precision=W.PREC_FP32), 30.0)
        cfg.cn_tol = 1e-10
        steps = 6
    g, o = run_pair(cfg, steps)
    errs = _errors(g, o, cfg)
    print(maker, errs)
    for k in ("rho", "S", "dj"):
        assert errs[k] < mom_rtol, (k, errs)
    assert errs["x"] < PART_RTOL and errs["u"] < PART_RTOL, errs
    dg, do = g.pic_diagnostics(), o.diagnostics()
    assert dg["count"] == do["count"]
    assert abs(dg["total"] - do["total"]) <= 1e-3 * abs(do["total"])
    g.close()


def test_fp32_and_fp64_gpu_forms_agree():
    cfg64 = small_foil()
    cfg32 = small_foil(precision=W.PREC_FP32)
    parts = W.generate_particles(cfg64)
    with pic.Pic(cfg64, stream=stream()) as a, pic.Pic(cfg32, stream=stream()) as b:
        for s, P in enumerate(parts):
            a.load(s, P)
            b.load(s, P)
        a.pic_step(cfg64.steps)
        b.pic_step(cfg32.steps)
        Ma, Mb = a.pic_moments(), b.pic_moments()
        assert normwise(Mb[1:10], Ma[1:10]) < MOM_RTOL
        assert normwise(Mb[10:13], Ma[10:13]) < MOM_RTOL
        assert normwise(Mb[0], Ma[0], density_scale(cfg64)) < MOM_RTOL
        da, db = a.pic_diagnostics(), b.pic_diagnostics()
        assert abs(db["total"] - da["total"]) <= 1e-3 * abs(da["total"])


def _snapshot(g, nsp):
    E, H = g.pic_fields()
    return E, H, [g.pic_get_particles(s) for s in range(nsp)]


def _from_snapshot(cfg, snap, precision):
    E, H, parts = snap
    c = cfg.scaled(precision=precision)
    h = pic.Pic(c, stream=stream(), capacity=[P["x"].size for P in parts])
    for s, P in enumerate(parts):
        h.load(s, P)
    h.pic_set_fields(E, H)
    return h


@pytest.mark.slow
def test_precision_form_step_by_step_against_fp64_gpu():
    """Precision form on a uniform CN plasma (256x256, 16 particles/cell/species,
    2.1M particles): from the same FP64 GPU state, one FP32 step and one FP64
    step give moments within 1e-5 (checked at several points of an FP64 run);
    run side by side from the same seed for 20 steps, the FP32 total energy
    stays within 0.1 % of the FP64 run's."""
    cfg = W.uniform_plasma("uniform-256-cn", 256, 16, 20, seed=1234 + 4, precision=W.PREC_FP64, tile=16)
    cfg.cn_tol = 1e-12
    parts = W.generate_particles(cfg)
    g64 = pic.Pic(cfg, stream=stream(), capacity=[P["x"].size for P in parts])
    g32 = pic.Pic(cfg.scaled(precision=W.PREC_FP32), stream=stream(), capacity=[P["x"].size for P in parts])
    for s, P in enumerate(parts):
        g64.load(s, P)
        g32.load(s, P)
    e64 = [g64.pic_diagnostics()["total"]]
    e32 = [g32.pic_diagnostics()["total"]]
    worst = 0.0
    for k in range(20):
        if k % 5 == 0:
            snap = _snapshot(g64, len(cfg.species))
            a = _from_snapshot(cfg, snap, W.PREC_FP64)
            b = _from_snapshot(cfg, snap, W.PREC_FP32)
            a.pic_step(1)
            b.pic_step(1)
            Ma, Mb = a.pic_moments(), b.pic_moments()
            errs = [normwise(Mb[0], Ma[0], density_scale(cfg)), normwise(Mb[1:10], Ma[1:10]),
                    normwise(Mb[10:13], Ma[10:13])]
            worst = max(worst, max(errs))
            assert max(errs) < MOM_RTOL, (k, errs)
            a.close()
            b.close()
        g64.pic_step(1)
        g32.pic_step(1)
        e64.append(g64.pic_diagnostics()["total"])
        e32.append(g32.pic_diagnostics()["total"])
    e64, e32 = np.array(e64), np.array(e32)
    assert np.max(np.abs(e32 - e64)) <= 1e-3 * abs(e64[0]), (e32, e64)
    g64.close()
    g32.close()


@pytest.mark.slow
def test_precision_form_at_1024_squared_with_16x16_tiles():
    """The precision form's code paths at a size close to its workload: uniform CN plasma on 1024x1024
    periodic cells (the spectral preconditioner's power-of-two grid), 16x16 tiles, 4 particles/cell/species
    (8.4M particles) from one seed in both forms.  After one step the FP32 moments are within 1e-5 of the
    FP64 GPU path's; over 5 steps the total energies stay within 0.1 % of each other."""
    cfg = W.uniform_plasma("uniform-1024-cn", 1024, 4, 5, seed=1234 + 4, precision=W.PREC_FP64, tile=16)
    cfg.cn_tol = 1e-12
    parts = W.generate_particles(cfg)
    cap = [P["x"].size for P in parts]
    with pic.Pic(cfg, stream=stream(), capacity=cap) as a, \
            pic.Pic(cfg.scaled(precision=W.PREC_FP32), stream=stream(), capacity=cap) as b:
        a.pic_load_species(parts)
        b.pic_load_species(parts)
        e0 = a.pic_diagnostics()["total"]
        a.pic_step(1)
        b.pic_step(1)
        Ma, Mb = a.pic_moments(), b.pic_moments()
        errs = [normwise(Mb[0], Ma[0], density_scale(cfg)), normwise(Mb[1:10], Ma[1:10]),
                normwise(Mb[10:13], Ma[10:13])]
        assert max(errs) < MOM_RTOL, errs
        a.pic_step(4)
        b.pic_step(4)
        da, db = a.pic_diagnostics(), b.pic_diagnostics()
        assert da["count"] == db["count"] == sum(cap)
        assert abs(db["total"] - da["total"]) <= 1e-3 * abs(e0), (da["total"], db["total"], e0)
        assert da["cn_residual"] < 1e-11 and db["cn_residual"] < 1e-11
