"""Pins of the CPU oracle against what the physics and the mathematics fix.

These run without a GPU.  Each test names the passage it checks:
P1 magnetic rotation, P2 pure electric push, P3 charge sum, P4 cold-plasma
k = 0 oscillation, P5 vacuum dispersion, P6 lumped versus actual current,
P7 dense brute force on 4x4 grids, P8 invariances; plus the ordering rule,
the wall/laser readings and energy conservation of the implicit-curl mode.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_1308_2590_gb300 import workloads as W


def _rand_particles(rng, n, Lx, Ly, u_scale=0.3):
    return dict(x=rng.random(n) * Lx, y=rng.random(n) * Ly,
                ux=rng.standard_normal(n) * u_scale, uy=rng.standard_normal(n) * u_scale,
                uz=rng.standard_normal(n) * u_scale, w=0.5 + rng.random(n))


def _uniform_field(g, vec):
    F = np.zeros((3, g.ny, g.nxn))
    for c in range(3):
        F[c] = vec[c]
    return F


# ----------------------------------------------------------------------------- P1
@pytest.mark.parametrize("q,m", [(-1.0, 1.0), (1.0, 1836.0), (2.0, 3.0)])
def test_p1_magnetic_rotation_closed_form(q, m):
    """E = 0, uniform B: u^{n+1} = (2R - I) u^n is a rotation about B by
    -sign(q) * 2 atan(|q| dt |B| / (2 m gamma)) per step (Eq. 2a, Section 2)."""
    g = oracle.Grid(4, 4, 1.0, 1.0, True)
    dt, Bz = 0.7, 1.3
    E = np.zeros((3, 4, 4))
    B = _uniform_field(g, (0.0, 0.0, Bz))
    P = dict(x=np.array([1.3]), y=np.array([2.2]), ux=np.array([0.8]), uy=np.array([0.0]),
             uz=np.array([0.35]), w=np.array([1.0]))
    u0 = np.array([0.8, 0.0, 0.35])
    gam = math.sqrt(1 + u0 @ u0)
    theta = 2.0 * math.atan(abs(q) * dt * Bz / (2 * m * gam))
    for n in range(1, 41):
        oracle.push(g, dt, q, m, E, B, P)
        u = np.array([P["ux"][0], P["uy"][0], P["uz"][0]])
        assert abs(np.linalg.norm(u) - np.linalg.norm(u0)) < 1e-14
        assert abs(u[2] - 0.35) < 1e-14
        ang = -math.copysign(1.0, q) * n * theta
        expect = 0.8 * np.array([math.cos(ang), math.sin(ang)])
        assert np.max(np.abs(u[:2] - expect)) < 1e-13


def test_p1_rotation_matrix_is_inverse_of_cross():
    """R(b) solves ubar = w + ubar x b (Section 2: Eq. 2a inverted for momentum)."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        b = rng.standard_normal(3)
        w = rng.standard_normal(3)
        ub = oracle.rotate(b, w)
        assert np.max(np.abs(ub - np.cross(ub, b) - w)) < 1e-13
        assert np.max(np.abs(brute.r_matrix(b) @ w - ub)) < 1e-13


# ----------------------------------------------------------------------------- P2
def test_p2_pure_electric_push():
    """B = 0: R = I, so u^{n+1} = u^n + q dt E / m and r^{n+1} = r^n + dt (u^n + k E)/gamma^n."""
    g = oracle.Grid(8, 8, 0.5, 0.5, True)
    rng = np.random.default_rng(1)
    P = _rand_particles(rng, 50, g.Lx, g.Ly)
    P0 = {k: v.copy() for k, v in P.items()}
    Evec = np.array([0.3, -0.2, 0.7])
    E = _uniform_field(g, Evec)
    B = np.zeros_like(E)
    q, m, dt = -1.0, 1.0, 0.4
    oracle.push(g, dt, q, m, E, B, P)
    u0 = np.stack([P0["ux"], P0["uy"], P0["uz"]], 1)
    u1 = np.stack([P["ux"], P["uy"], P["uz"]], 1)
    assert np.max(np.abs(u1 - (u0 + q * dt * Evec / m))) < 1e-14
    gam = np.sqrt(1 + np.sum(u0 ** 2, 1))
    ub = u0 + q * dt / (2 * m) * Evec
    xe = np.mod(P0["x"] + dt * ub[:, 0] / gam, g.Lx)
    ye = np.mod(P0["y"] + dt * ub[:, 1] / gam, g.Ly)
    assert np.max(np.abs(P["x"] - xe)) < 1e-13
    assert np.max(np.abs(P["y"] - ye)) < 1e-13


# ----------------------------------------------------------------------------- P3
@pytest.mark.parametrize("periodic", [True, False])
def test_p3_charge_sum(periodic):
    """Linear weights sum to one, so the raw node charge equals sum(q w) to 1e-12."""
    g = oracle.Grid(13, 9, 0.3, 0.7, periodic)
    rng = np.random.default_rng(2)
    P = _rand_particles(rng, 4000, g.Lx * (1 - 1e-12), g.Ly)
    B = np.zeros((3, g.ny, g.nxn))
    M = oracle.deposit_raw(g, 0.5, -1.0, 1.0, B, P)
    tot = -np.sum(P["w"])
    assert abs(M[0].sum() - tot) <= 1e-12 * abs(tot)
    Mn = oracle.normalize(g, M)
    assert abs(np.sum(Mn[0] * g.node_area()) - tot) <= 1e-12 * abs(tot)


def test_p3_single_particle_weights():
    """A single particle's charge splits as (1-fx)(1-fy), fx(1-fy), (1-fx)fy, fx fy onto its cell corners."""
    g = oracle.Grid(5, 4, 1.0, 2.0, True)
    P = dict(x=np.array([2.25]), y=np.array([5.0]), ux=np.zeros(1), uy=np.zeros(1), uz=np.zeros(1), w=np.array([1.0]))
    M = oracle.deposit_raw(g, 1.0, 1.0, 1.0, np.zeros((3, 4, 5)), P)
    expect = np.zeros((4, 5))
    fx, fy = 0.25, 0.5
    expect[2, 2] = (1 - fx) * (1 - fy); expect[2, 3] = fx * (1 - fy)
    expect[3, 2] = (1 - fx) * fy; expect[3, 3] = fx * fy
    assert np.array_equal(M[0], expect)


# ----------------------------------------------------------------------------- P4
def _cold_plasma_run(dt, field_mode, nsteps, u0=1e-5, n=1.0):
    # dt <= min(dx, dy) keeps the literal (leapfrog-curl) mode stable (the curls of Eqs. 4-5 are explicit)
    cfg = W.RunConfig(name="cold", nx=6, ny=5, dx=0.6, dy=0.8, dt=dt, steps=nsteps, bc_x=W.BC_PERIODIC,
                      field_mode=field_mode, species=[W.Species(-1.0, 1.0, 1, n, 0.0)], tile_nx=3, tile_ny=5)
    sim = oracle.OracleSim.from_config(cfg)
    P = W.lattice_particles(cfg, 0, offsets=((0.25, 0.6),), drift=(u0, 0.0, 0.0), density=n)
    sim.load_particles(0, **P)
    Ex, ux = [sim.E[0, 0, 0]], [sim.parts[0]["ux"][0]]
    for _ in range(nsteps):
        sim.step()
        Ex.append(sim.E[0, 2, 3]); ux.append(sim.parts[0]["ux"][7])
        assert np.ptp(sim.E[0]) < 1e-15 + 1e-9 * np.max(np.abs(sim.E[0]))  # stays uniform
    return sim, np.array(Ex), np.array(ux)


def test_p4_lattice_response_tensor_is_exact():
    """Uniform lattice, B = 0: S = (omega_pe dt / 2)^2 I at every node (S from the linearised
    time-centred push, Eq. 3 with B = 0)."""
    cfg = W.RunConfig(name="cold", nx=6, ny=5, dx=0.3, dy=0.4, dt=0.5, steps=1,
                      species=[W.Species(-1.0, 1.0, 1, 1.0, 0.0)], tile_nx=3, tile_ny=5)
    sim = oracle.OracleSim.from_config(cfg)
    u0 = 0.01
    sim.load_particles(0, **W.lattice_particles(cfg, 0, offsets=((0.25, 0.6), (0.7, 0.1)), drift=(u0, 0, 0)))
    gam = math.sqrt(1 + u0 * u0)
    s = (0.5 / 2) ** 2 / gam
    for k in range(9):
        target = s if k in (0, 4, 8) else 0.0
        assert np.max(np.abs(sim.M[1 + k] - target)) < 1e-15
    assert np.max(np.abs(sim.M[10] - (-u0 / gam))) < 1e-15


@pytest.mark.parametrize("field_mode", [W.FIELD_LITERAL, W.FIELD_CN])
@pytest.mark.parametrize("dt", [0.5, 0.3])
def test_p4_cold_plasma_discrete_frequency(dt, field_mode):
    """k = 0 cold oscillation: E and u obey the trapezoidal recurrence, so
    x^{n+1} + x^{n-1} = 2 cos(w dt) x^n with w dt = 2 atan(omega_pe dt / 2) (the discrete cold-plasma
    frequency of the implicit scheme)."""
    sim, Ex, ux = _cold_plasma_run(dt, field_mode, 40)
    wdt = 2 * math.atan(dt / 2)
    for series in (Ex, ux):
        n = np.arange(1, len(series) - 1)
        big = np.abs(series[n]) > 0.2 * np.max(np.abs(series))
        c = (series[n + 1] + series[n - 1])[big] / series[n][big]
        assert np.max(np.abs(c - 2 * math.cos(wdt))) < 1e-8
    if dt <= 0.3:
        assert abs(wdt / dt - 1.0) < 0.01   # within 1 % of omega_pe


def test_p4_golden_frequencies():
    """Closed-form discrete frequencies stored in tests/golden (derived, cited there)."""
    import json, os
    with open(os.path.join(os.path.dirname(__file__), "golden", "discrete_frequencies.json")) as f:
        gold = json.load(f)
    for row in gold["cold_plasma"]:
        assert abs(2 * math.atan(row["omega_pe_dt"] / 2) / row["omega_pe_dt"] - row["omega_over_omega_pe"]) < 1e-12
    sim, Ex, _ = _cold_plasma_run(0.5, W.FIELD_CN, 40)
    n = np.arange(1, len(Ex) - 1)
    big = np.abs(Ex[n]) > 0.2 * np.max(np.abs(Ex))
    c = np.median((Ex[n + 1] + Ex[n - 1])[big] / Ex[n][big])
    w = math.acos(c / 2) / 0.5
    assert abs(w - gold["cold_plasma"][0]["omega_over_omega_pe"]) < 1e-7


# ----------------------------------------------------------------------------- P5
def _mode(g, kx_i, ky_i, comp):
    E = np.zeros((3, g.ny, g.nxn))
    jj, ii = np.meshgrid(np.arange(g.ny), np.arange(g.nxn), indexing="ij")
    E[comp] = np.cos(2 * np.pi * (kx_i * ii / g.nx + ky_i * jj / g.ny))
    return E


@pytest.mark.parametrize("field_mode,dt", [(W.FIELD_LITERAL, 0.5), (W.FIELD_CN, 0.5), (W.FIELD_CN, 3.0)])
@pytest.mark.parametrize("kx_i,ky_i,comp", [(2, 3, 2), (3, 0, 1), (1, 5, 2)])
def test_p5_vacuum_dispersion(field_mode, dt, kx_i, ky_i, comp):
    """One discrete eigenmode stays one, with phase per step from
    sin(w dt/2) = (dt/2) k_eff (literal, Eqs. 4-5) or tan(w dt/2) = (dt/2) k_eff (implicit curls),
    k_eff^2 = 4[sin^2 a cos^2 b / dx^2 + cos^2 a sin^2 b / dy^2] (the symbol of the transversely averaged
    centred curls between nodes and cell centres)."""
    nx, ny, dx, dy = 16, 12, 1.0, 0.8
    g = oracle.Grid(nx, ny, dx, dy, True)
    sim = oracle.OracleSim(nx, ny, dx, dy, dt, True, field_mode, [(-1.0, 1.0)], 4, 4)
    E0 = _mode(g, kx_i, ky_i, comp)
    sim.set_fields(E=E0)
    a = math.pi * kx_i / nx
    b = math.pi * ky_i / ny
    keff = math.sqrt(4 * (math.sin(a) ** 2 * math.cos(b) ** 2 / dx ** 2 + math.cos(a) ** 2 * math.sin(b) ** 2 / dy ** 2))
    if field_mode == W.FIELD_LITERAL:
        cos_wdt = 1 - 2 * (dt * keff / 2) ** 2
    else:
        th = dt * keff / 2
        cos_wdt = (1 - th * th) / (1 + th * th)
    amps = [1.0]
    for _ in range(30):
        sim.step()
        F = sim.E[comp]
        amp = np.sum(F * E0[comp]) / np.sum(E0[comp] ** 2)
        assert np.max(np.abs(F - amp * E0[comp])) < 1e-12     # still the same mode
        amps.append(amp)
    a_ = np.array(amps)
    n = np.arange(1, len(a_) - 1)
    big = np.abs(a_[n]) > 0.2
    c = (a_[n + 1] + a_[n - 1])[big] / a_[n][big]
    assert np.max(np.abs(c - 2 * cos_wdt)) < 1e-11


def test_p5_checkerboard_is_static():
    """a = b = pi/2 gives k_eff = 0: the checkerboard is a static mode of this grid (excluded above)."""
    g = oracle.Grid(8, 8, 1.0, 1.0, True)
    E0 = _mode(g, 4, 4, 2)
    assert np.max(np.abs(oracle.curl_e(g, E0))) < 1e-14


def test_p5_cn_conserves_vacuum_energy():
    """With curl_h the adjoint of curl_e, the time-centred scheme keeps sum E^2 dA + sum H^2 dA exactly."""
    nx, ny = 10, 8
    g = oracle.Grid(nx, ny, 0.7, 0.9, True)
    rng = np.random.default_rng(3)
    sim = oracle.OracleSim(nx, ny, 0.7, 0.9, 2.5, True, W.FIELD_CN, [(-1.0, 1.0)], 5, 4)
    sim.set_fields(E=rng.standard_normal((3, ny, nx)), H=rng.standard_normal((3, ny, nx)))
    e0 = sim.diagnostics()["field"]
    for _ in range(10):
        sim.step()
    assert abs(sim.diagnostics()["field"] - e0) < 1e-11 * e0
    Ce, Ch = oracle.curl_matrices(g)
    assert abs(Ch - Ce.T).max() < 1e-15


# ----------------------------------------------------------------------------- P6
def test_p6_lumped_current_matches_pushed_particles():
    """For uniform E, B: (2/dt) S_node E + dj_node = sum W w q ubar/gamma / dA exactly (Eq. 3)."""
    g = oracle.Grid(7, 6, 0.4, 0.3, True)
    rng = np.random.default_rng(4)
    P = _rand_particles(rng, 3000, g.Lx, g.Ly, u_scale=0.8)
    q, m, dt = -1.0, 1.0, 0.6
    Evec = np.array([0.4, -0.9, 0.25])
    Bvec = np.array([1.1, 0.3, -2.0])
    E = _uniform_field(g, Evec)
    B = _uniform_field(g, Bvec)
    M = oracle.normalize(g, oracle.deposit_raw(g, dt, q, m, B, P))
    S = M[1:10].reshape(3, 3, g.ny, g.nxn)
    jpred = (2 / dt) * np.einsum("rcyx,c->ryx", S, Evec) + M[10:13]
    P0 = {k: v.copy() for k, v in P.items()}
    oracle.push(g, dt, q, m, E, B, P)
    u0 = np.stack([P0["ux"], P0["uy"], P0["uz"]])
    u1 = np.stack([P["ux"], P["uy"], P["uz"]])
    vbar = 0.5 * (u0 + u1) / np.sqrt(1 + np.sum(u0 ** 2, 0))
    cx, cy, fx, fy = oracle.locate(g, P0["x"], P0["y"])
    jact = np.zeros((3, g.ny, g.nxn))
    for di in (0, 1):
        for dj in (0, 1):
            wgt = (fx if di else 1 - fx) * (fy if dj else 1 - fy)
            for c in range(3):
                np.add.at(jact[c], ((cy + dj) % g.ny, (cx + di) % g.nx), wgt * P0["w"] * q * vbar[c])
    jact /= g.dx * g.dy
    assert np.max(np.abs(jpred - jact)) < 1e-12 * np.max(np.abs(jact))


# ----------------------------------------------------------------------------- P7
def test_p7_brute_force_deposit_4x4():
    g = oracle.Grid(4, 4, 0.5, 0.25, True)
    rng = np.random.default_rng(5)
    P = _rand_particles(rng, 64, g.Lx, g.Ly, u_scale=0.7)
    B = rng.standard_normal((3, 4, 4))
    for (q, m) in ((-1.0, 1.0), (1.0, 1836.0)):
        Ms = oracle.deposit_raw(g, 0.8, q, m, B, P)
        Mb = brute.brute_deposit(4, 4, 0.5, 0.25, 0.8, q, m, B, P)
        assert np.max(np.abs(Ms - Mb)) < 1e-13 * max(1.0, np.max(np.abs(Mb)))


def test_p7_brute_force_curls_and_literal_solve_4x4():
    g = oracle.Grid(4, 4, 0.5, 0.25, True)
    rng = np.random.default_rng(6)
    E = rng.standard_normal((3, 4, 4)); H = rng.standard_normal((3, 4, 4))
    assert np.max(np.abs(oracle.curl_e(g, E).ravel() - brute.dense_curl_e(4, 4, 0.5, 0.25) @ E.ravel())) < 1e-13
    assert np.max(np.abs(oracle.curl_h(g, H).ravel() - brute.dense_curl_h(4, 4, 0.5, 0.25) @ H.ravel())) < 1e-13
    Ce, Ch = oracle.curl_matrices(g)
    assert np.max(np.abs(Ce.toarray() - brute.dense_curl_e(4, 4, 0.5, 0.25))) == 0.0
    assert np.max(np.abs(Ch.toarray() - brute.dense_curl_h(4, 4, 0.5, 0.25))) == 0.0
    M = np.zeros((13, 4, 4))
    M[1:10] = 0.3 * rng.standard_normal((9, 4, 4)) + np.eye(3).ravel()[:, None, None] * 0.5
    M[10:13] = rng.standard_normal((3, 4, 4))
    dt = 0.1
    En, Hn = oracle.field_literal(g, dt, dt, (0, 1, 0, 0, 0), E, H, M)
    Eb = brute.brute_literal_E(4, 4, 0.5, 0.25, dt, E, H, M)
    assert np.max(np.abs(En - Eb)) < 1e-13
    Hb = H.ravel() - dt * brute.dense_curl_e(4, 4, 0.5, 0.25) @ Eb.ravel()
    assert np.max(np.abs(Hn.ravel() - Hb)) < 1e-13


def test_p7_brute_force_cn_solve_4x4():
    g = oracle.Grid(4, 4, 0.5, 0.25, True)
    rng = np.random.default_rng(7)
    E = rng.standard_normal((3, 4, 4)); H = rng.standard_normal((3, 4, 4))
    M = np.zeros((13, 4, 4))
    M[1:10] = 0.2 * rng.standard_normal((9, 4, 4)) + np.eye(3).ravel()[:, None, None] * 0.3
    M[10:13] = rng.standard_normal((3, 4, 4))
    dt = 1.7
    En, Hn, X = oracle.field_cn(g, dt, E, H, M)
    Xb = brute.brute_cn_X(4, 4, 0.5, 0.25, dt, E, H, M)
    assert np.max(np.abs(X - Xb)) < 1e-12 * np.max(np.abs(Xb))
    assert np.max(np.abs(En - (2 * Xb - E))) < 1e-12 * np.max(np.abs(En))


def test_p7_brute_force_cn_solve_with_walls_4x4():
    """The implicit-curl system of a box with walls (vacuum wall nodes: one-sided curl_h in the x row,
    the time-centred first-order Mur condition in the y and z rows, the incident wave subtracted at
    x = 0) against an independently written dense assembly, incident values from the closed-form wave."""
    nx, ny, dx, dy, dt = 4, 4, 0.5, 0.25, 0.3
    g = oracle.Grid(nx, ny, dx, dy, False)
    rng = np.random.default_rng(21)
    E = rng.standard_normal((3, ny, nx + 1)); H = rng.standard_normal((3, ny, nx))
    M = np.zeros((13, ny, nx + 1))
    M[1:10] = 0.2 * rng.standard_normal((9, ny, nx + 1)) + np.eye(3).ravel()[:, None, None] * 0.3
    M[10:13] = rng.standard_normal((3, ny, nx + 1))
    Ce, Ch = oracle.curl_matrices(g)
    assert np.max(np.abs(Ce.toarray() - brute.dense_curl_e_walls(nx, ny, dx, dy))) == 0.0
    assert np.max(np.abs(Ch.toarray() - brute.dense_curl_h_walls(nx, ny, dx, dy))) == 0.0
    assert np.max(np.abs(oracle.curl_h(g, H).ravel() - Ch @ H.ravel())) < 1e-13
    a0, om, tau, t0 = 1.3, 2.0, 5.0, 4.0
    t_new = 2.7
    inc = lambda x, t: (a0 * math.sin(om * (t - x)) * math.exp(-2 * math.log(2) * ((t - x) - t0) ** 2 / tau ** 2)
                        if t - x >= 0 else 0.0)
    for pol, pc in ((0, 1), (1, 2)):
        io = np.array([inc(0, t_new - dt), inc(dx, t_new - dt)])
        iN = np.array([inc(0, t_new), inc(dx, t_new)])
        Xb = brute.brute_cn_walls_X(nx, ny, dx, dy, dt, E, H, M, io, iN, pc)
        En, Hn, X = oracle.field_cn(g, dt, E, H, M, t_new, (a0, om, tau, t0, pol))
        assert np.max(np.abs(X - Xb)) < 1e-12 * np.max(np.abs(Xb))
        assert np.max(np.abs(En - (2 * Xb - E))) < 1e-12 * np.max(np.abs(En))


# ----------------------------------------------------------------------------- P8
def test_p8_integer_cell_translation_and_weight_doubling():
    """Translation by whole cells shifts every moment exactly; doubling w doubles them exactly."""
    nx, ny, dx, dy = 8, 8, 0.25, 0.5
    g = oracle.Grid(nx, ny, dx, dy, True)
    rng = np.random.default_rng(8)
    n = 300
    # dyadic positions so x/dx is exact and the shift is exact
    P = dict(x=np.floor(rng.random(n) * nx * 2 ** 20) / 2 ** 20 * dx,
             y=np.floor(rng.random(n) * ny * 2 ** 20) / 2 ** 20 * dy,
             ux=rng.standard_normal(n) * 0.3, uy=rng.standard_normal(n) * 0.3, uz=rng.standard_normal(n) * 0.3,
             w=0.5 + rng.random(n))
    B = np.zeros((3, ny, nx)); B[2] = 0.7
    M0 = oracle.deposit_raw(g, 0.5, -1.0, 1.0, B, P)
    sx, sy = 3, 5
    P2 = dict(P); P2["x"] = np.mod(P["x"] + sx * dx, g.Lx); P2["y"] = np.mod(P["y"] + sy * dy, g.Ly)
    M1 = oracle.deposit_raw(g, 0.5, -1.0, 1.0, B, P2)
    assert np.array_equal(np.roll(M0, (sy, sx), axis=(1, 2)), M1)
    P3 = dict(P); P3["w"] = 2 * P["w"]
    assert np.array_equal(oracle.deposit_raw(g, 0.5, -1.0, 1.0, B, P3), 2 * M0)


def test_p8_mirror_symmetry_in_y():
    """y -> Ly - y, uy -> -uy (B = 0): rho, dj_x, dj_z mirror; dj_y and the xy/yz entries of S flip sign."""
    nx, ny, dx, dy = 6, 8, 0.25, 0.5
    g = oracle.Grid(nx, ny, dx, dy, True)
    rng = np.random.default_rng(9)
    P = _rand_particles(rng, 200, g.Lx, g.Ly)
    B = np.zeros((3, ny, nx)); B[1] = 0.9   # By is unchanged by the reflection (axial vector)
    M0 = oracle.deposit_raw(g, 0.5, -1.0, 1.0, B, P)
    P2 = dict(P); P2["y"] = np.mod(g.Ly - P["y"], g.Ly); P2["uy"] = -P["uy"]
    M1 = oracle.deposit_raw(g, 0.5, -1.0, 1.0, B, P2)
    mirror = lambda A: np.roll(A[::-1], 1, axis=0)   # node j -> (ny - j) mod ny
    sign = np.ones(13)
    for k, (r, c) in enumerate([(r, c) for r in range(3) for c in range(3)]):
        if (r == 1) != (c == 1):
            sign[1 + k] = -1.0
    sign[11] = -1.0
    for k in range(13):
        assert np.max(np.abs(sign[k] * mirror(M0[k]) - M1[k])) < 1e-13 * max(1.0, np.max(np.abs(M0[k])))


# ----------------------------------------------------------------------------- ordering rule
def test_ordering_rule_tile_then_cell_stayers_then_arrivals():
    cfg = W.config(1).scaled(nx=16, ny=16, tile_nx=4, tile_ny=4, field_mode=W.FIELD_CN)
    sim = oracle.OracleSim.from_config(cfg)
    parts = W.generate_particles(cfg.scaled(species=[W.Species(-1.0, 1.0, 4, 1.0, 400.0)]))
    sim.species = sim.species[:1]; sim.parts = sim.parts[:1]; sim.removed = [0]
    ids = np.arange(parts[0]["x"].size, dtype=float)
    P = parts[0]
    sim.load_particles(0, **P)
    # identify particles by their exact initial uz (distinct floats)
    order_ids = lambda: np.searchsorted(np.sort(P["uz"]), sim.parts[0]["uz"]) if False else None
    before = sim.particles(0)
    tiles_before = sim.tile_of(before["x"], before["y"])
    assert np.all(np.diff(tiles_before) >= 0)
    # after a load: by tile, inside a tile by cell (row-major), ties in load order
    cx, cy, _, _ = oracle.locate(sim.g, before["x"], before["y"])
    local = (cy % 4) * 4 + cx % 4
    for tile in np.unique(tiles_before):
        assert np.all(np.diff(local[tiles_before == tile]) >= 0)
    # track identity with a tag hidden in w (w is never changed by a step)
    sim.parts[0]["w"] = np.arange(before["x"].size, dtype=float) + 1.0
    sim.deposit()
    tags_before = sim.parts[0]["w"].copy()
    sim.step()
    after = sim.particles(0)
    t_new = sim.tile_of(after["x"], after["y"])
    assert np.all(np.diff(t_new) >= 0)
    pos_before = {t: i for i, t in enumerate(tags_before)}
    old_tile = {t: tiles_before[i] for i, t in enumerate(tags_before)}
    cxa, cya, _, _ = oracle.locate(sim.g, after["x"], after["y"])
    local_after = (cya % 4) * 4 + cxa % 4
    n_cells_seen = 0
    for tile in np.unique(t_new):
        sel = t_new == tile
        tags = after["w"][sel]
        loc = local_after[sel]
        assert np.all(np.diff(loc) >= 0)          # cells of a tile in row-major order
        for c in np.unique(loc):
            ct = tags[loc == c]
            moved = np.array([old_tile[t] != tile for t in ct])
            # inside a cell: stayers first, then arrivals, each in previous order
            assert not np.any(moved[:-1] & ~moved[1:])
            prev_pos = np.array([pos_before[t] for t in ct])
            assert np.all(np.diff(prev_pos[~moved]) > 0)
            assert np.all(np.diff(prev_pos[moved]) > 0)
            n_cells_seen += int(moved.any() and (~moved).any())
    assert n_cells_seen > 0   # the case of stayers and arrivals sharing a cell occurred
    assert sim.tile_of(after["x"], after["y"]).size == before["x"].size  # periodic: nobody lost


# ----------------------------------------------------------------------------- walls + laser readings
def test_wall_absorbs_and_source_injects():
    """Readings of Eq. 14/15: the source reproduces the incident waveform at x = 0,
    and a pulse crossing the box leaves through the far wall with < 1 % of its energy left."""
    nx, ny = 120, 4
    dx = 2 * math.pi / 40
    dt = 0.8 * dx                  # c dt / dx = 0.8
    tau = 8.0
    las = (1.0, 1.0, tau, 2 * tau, 0)
    sim = oracle.OracleSim(nx, ny, dx, dx, dt, False, W.FIELD_LITERAL, [(-1.0, 1.0)], 8, 4, las)
    peak = 0.0
    for n in range(1, 520):
        sim.step()
        inc = oracle.laser(n * dt, *las[:4])
        assert abs(sim.E[1, 0, 0] - inc) < 2e-3
        peak = max(peak, sim.diagnostics()["field"])
    assert peak > 1.0
    assert sim.diagnostics()["field"] < 0.01 * peak


@pytest.mark.parametrize("cdt,src_tol", [(0.8, 2e-3), (2.0, 6e-3)])
def test_cn_walls_absorb_and_source_injects(cdt, src_tol):
    """Implicit-curl mode in a box with walls (reading 11 for this mode): the field at x = 0 follows the
    incident waveform, and the pulse leaves through the far wall with less than 1e-6 of its peak energy
    left; also at c dt / dx = 2, where the leapfrog curls of Eqs. 4-5 would be unstable."""
    nx, ny = 120, 4
    dx = 2 * math.pi / 40
    dt = cdt * dx
    tau = 8.0
    las = (1.0, 1.0, tau, 2 * tau, 0)
    sim = oracle.OracleSim(nx, ny, dx, dx, dt, False, W.FIELD_CN, [(-1.0, 1.0)], 8, 4, las)
    peak = 0.0
    for n in range(1, int(416 / cdt)):
        sim.step()
        inc = oracle.laser(n * dt, *las[:4])
        assert abs(sim.E[1, 0, 0] - inc) < src_tol
        peak = max(peak, sim.diagnostics()["field"])
    assert peak > 1.0
    assert sim.diagnostics()["field"] < 1e-6 * peak


def test_cn_walls_keep_the_energy_of_an_interior_pulse():
    """Away from the walls the implicit-curl scheme is the periodic one (curl_h the adjoint of curl_e):
    a pulse whose tails at the walls are below 1e-20 keeps its field energy to 1e-12 while it moves."""
    nx, ny, dx = 200, 4, 0.1
    for dt in (0.1, 0.5):
        sim = oracle.OracleSim(nx, ny, dx, dx, dt, False, W.FIELD_CN, [(-1.0, 1.0)], 8, 4)
        x = np.arange(sim.g.nxn) * dx
        E = np.zeros((3, ny, sim.g.nxn))
        E[2] = np.exp(-0.5 * ((x - 10.0) / 1.0) ** 2)[None, :]
        E[1] = 0.5 * np.exp(-0.5 * ((x - 9.5) / 0.8) ** 2)[None, :]
        sim.set_fields(E=E)
        e0 = sim.diagnostics()["field"]
        sim.step(int(round(2.0 / dt)))
        assert abs(sim.diagnostics()["field"] - e0) < 1e-12 * e0


# ----------------------------------------------------------------------------- node average (reading 9)
def _linear_cells(g, coef):
    """H_c = a_c + b_c x + c_c y sampled at the cell centres ((i+1/2) dx, (j+1/2) dy)."""
    jj, ii = np.meshgrid(np.arange(g.ny), np.arange(g.nx), indexing="ij")
    xc, yc = (ii + 0.5) * g.dx, (jj + 0.5) * g.dy
    return np.stack([a + b * xc + c * yc for a, b, c in coef])


@pytest.mark.parametrize("periodic", [True, False])
def test_node_average_reproduces_linear_field(periodic):
    """B at a node is the mean of the cells around it (reading 9 of Section 3.3's 'within a cell'
    weighting, H cell-centred per Fig. 1): for H linear in x and y the mean of the 4 cells around an
    interior node is the field at the node itself, and on a wall column the 2 cells inside the box give
    the field half a cell inside the wall at the node's y.  A swapped neighbour (i+1 for i-1, j+1 for j-1)
    or the wrong pair on a wall column moves the result by a whole cell and fails."""
    nx, ny, dx, dy = 9, 7, 0.3, 0.45
    g = oracle.Grid(nx, ny, dx, dy, periodic)
    coef = [(0.4, 1.3, -0.7), (-1.1, 0.25, 2.2), (0.05, -3.1, 0.6)]
    Bn = oracle.node_average(g, _linear_cells(g, coef))
    for c, (a, b, cc) in enumerate(coef):
        for j in range(1, ny):            # j = 0 averages across the periodic seam in y
            for i in range(1, nx):        # i = 0 is a wall column or the periodic seam in x
                assert abs(Bn[c, j, i] - (a + b * i * dx + cc * j * dy)) < 1e-14
            if not periodic:
                assert abs(Bn[c, j, 0] - (a + b * 0.5 * dx + cc * j * dy)) < 1e-14
                assert abs(Bn[c, j, nx] - (a + b * (nx - 0.5) * dx + cc * j * dy)) < 1e-14


def test_node_average_of_a_periodic_mode():
    """Across the periodic seams: cos(k (i+1/2)) cos(l (j+1/2)) on the cells averages to
    cos(k i) cos(k/2) cos(l j) cos(l/2) at node (i, j) (cos(A - d) + cos(A + d) = 2 cos A cos d),
    at every node, the seam nodes included."""
    nx, ny = 10, 6
    g = oracle.Grid(nx, ny, 0.5, 0.5, True)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    k, l = 2 * np.pi * 3 / nx, 2 * np.pi * 1 / ny
    H = np.zeros((3, ny, nx))
    H[0] = np.cos(k * (ii + 0.5)) * np.cos(l * (jj + 0.5))
    H[1] = np.sin(k * (ii + 0.5)) * np.cos(l * (jj + 0.5))
    H[2] = np.cos(k * (ii + 0.5)) * np.sin(l * (jj + 0.5))
    Bn = oracle.node_average(g, H)
    f = math.cos(k / 2) * math.cos(l / 2)
    assert np.max(np.abs(Bn[0] - f * np.cos(k * ii) * np.cos(l * jj))) < 1e-14
    assert np.max(np.abs(Bn[1] - f * np.sin(k * ii) * np.cos(l * jj))) < 1e-14
    assert np.max(np.abs(Bn[2] - f * np.cos(k * ii) * np.sin(l * jj))) < 1e-14


# ----------------------------------------------------------------------------- gather of a linear field (a2)
@pytest.mark.parametrize("periodic", [True, False])
def test_gather_and_push_reproduce_linear_field(periodic):
    """Linear (area) weighting within a cell (Section 3.3, last paragraph) reproduces any field linear
    in x and y exactly, so the gathered E at a particle is E(x, y); with B = 0 the push then adds
    q dt E(x^n, y^n)/m to u (Eq. 2a, R = I).  A transposed pair of weights or a corner taken from the
    wrong row fails by a sizable fraction of the gradient."""
    nx, ny, dx, dy = 8, 6, 0.4, 0.3
    g = oracle.Grid(nx, ny, dx, dy, periodic)
    coef = [(0.3, 0.9, -0.4), (-0.2, -1.7, 0.35), (0.8, 0.15, 2.1)]
    jj, ii = np.meshgrid(np.arange(ny), np.arange(g.nxn), indexing="ij")
    E = np.stack([a + b * ii * dx + c * jj * dy for a, b, c in coef])
    rng = np.random.default_rng(11)
    n = 400
    # inside cells 0..nx-2 / 0..ny-2, so no corner lies across a periodic seam
    x = rng.random(n) * (nx - 1) * dx
    y = rng.random(n) * (ny - 1) * dy
    out = oracle.gather(g, E, x, y)
    for c, (a, b, cc) in enumerate(coef):
        assert np.max(np.abs(out[:, c] - (a + b * x + cc * y))) < 1e-14
    P = dict(x=x.copy(), y=y.copy(), ux=rng.standard_normal(n) * 0.2, uy=rng.standard_normal(n) * 0.2,
             uz=rng.standard_normal(n) * 0.2, w=np.ones(n))
    u0 = np.stack([P["ux"], P["uy"], P["uz"]], 1)
    q, m, dt = -1.0, 1.0, 0.25
    oracle.push(g, dt, q, m, E, np.zeros_like(E), P)
    Eat = np.stack([a + b * x + cc * y for a, b, cc in coef], 1)
    u1 = np.stack([P["ux"], P["uy"], P["uz"]], 1)
    assert np.max(np.abs(u1 - (u0 + q * dt / m * Eat))) < 1e-14


# ----------------------------------------------------------------------------- diagnostics (reading 21)
def test_kinetic_energy_closed_forms():
    """Kinetic energy sum w m (gamma - 1), gamma = sqrt(1 + |u|^2), u = p/(m c) (Section 2's units):
    |u|^2 = 3 and 8 give gamma = 2 and 3, so those particles carry exactly w m and 2 w m whichever axis
    u points along; small |u| tends to the classical w m |u|^2 / 2, large |u| to w m (|u| - 1).  A particle
    starting at rest and pushed by a uniform E with q dt E / m = (1, 1, 1) (Eq. 2a, B = 0) reaches
    gamma = 2 in one push."""
    sim = oracle.OracleSim(4, 4, 1.0, 1.0, 0.5, True, W.FIELD_LITERAL, [(-1.0, 1.0), (1.0, 1836.0)], 4, 4)
    r3, r8 = math.sqrt(3.0), math.sqrt(8.0)
    ux = np.array([r3, 0.0, 0.0, 1.0, 2.0])
    uy = np.array([0.0, r3, 0.0, 1.0, 2.0])
    uz = np.array([0.0, 0.0, r3, 1.0, 0.0])
    w = np.array([1.0, 0.5, 2.0, 0.25, 3.0])
    n = ux.size
    xy = dict(x=np.linspace(0.1, 3.9, n), y=np.linspace(0.2, 3.3, n))
    sim.load_particles(0, ux=ux, uy=uy, uz=uz, w=w, **xy)
    # species 1 (m = 1836): gamma = 3 along x, y and diagonally
    sim.load_particles(1, ux=np.array([r8, 0.0, 2.0]), uy=np.array([0.0, r8, 2.0]), uz=np.zeros(3),
                       w=np.array([1.0, 2.0, 0.5]), x=np.array([0.5, 1.5, 2.5]), y=np.array([0.5, 0.5, 0.5]))
    # electrons: gamma = 2 for the first four (|u|^2 = 3), 3 for the last (|u|^2 = 8)
    expect = 1.0 * (w[:4].sum() * 1.0 + w[4] * 2.0) + 1836.0 * 2.0 * (1.0 + 2.0 + 0.5)
    d = sim.diagnostics()
    assert abs(d["kinetic"] - expect) <= 1e-15 * expect   # sqrt(3)^2, sqrt(8)^2 round by an ulp
    # classical and ultra-relativistic limits
    for u, lim, tol in ((1e-3, 0.5e-6, 1e-6), (1e6, 1e6 - 1.0, 1e-12)):
        s2 = oracle.OracleSim(4, 4, 1.0, 1.0, 0.5, True, W.FIELD_LITERAL, [(-1.0, 1.0)], 4, 4)
        s2.load_particles(0, x=np.array([1.0]), y=np.array([1.0]), ux=np.array([0.0]), uy=np.array([0.0]),
                          uz=np.array([u]), w=np.array([1.0]))
        assert abs(s2.diagnostics()["kinetic"] - lim) <= tol * lim
    # pushed from rest by a uniform E (through the oracle's push), then measured
    g = oracle.Grid(4, 4, 1.0, 1.0, True)
    q, m, dt = -1.0, 1.0, 0.5
    Evec = np.array([1.0, 1.0, 1.0]) * m / (q * dt)
    P = dict(x=np.array([1.3]), y=np.array([2.6]), ux=np.zeros(1), uy=np.zeros(1), uz=np.zeros(1), w=np.array([0.75]))
    oracle.push(g, dt, q, m, _uniform_field(g, Evec), np.zeros((3, 4, 4)), P)
    s3 = oracle.OracleSim(4, 4, 1.0, 1.0, dt, True, W.FIELD_LITERAL, [(q, m)], 4, 4)
    s3.load_particles(0, **P)
    assert s3.diagnostics()["kinetic"] == 0.75 * m * 1.0


@pytest.mark.parametrize("periodic", [True, False])
def test_field_energy_closed_forms(periodic):
    """Field energy 1/2 sum E^2 dA + 1/2 sum H^2 dA (reading 21; E on nodes, H on cells, Fig. 1): a
    uniform E or H carries |E|^2 Lx Ly / 2 -- on a walled box only because the two wall columns count
    half a node area each (nx + 1 node columns, nx cells); in the literal mode H at the integer time is the
    mean of the two stored half-step values (Eqs. 4-5 stagger H by half a step); a cosine mode of
    amplitude A carries A^2 Lx Ly / 4."""
    nx, ny, dx, dy = 12, 5, 0.7, 0.4
    Lx, Ly = nx * dx, ny * dy
    sim = oracle.OracleSim(nx, ny, dx, dy, 0.2, periodic, W.FIELD_LITERAL, [(-1.0, 1.0)], 4, 5)
    g = sim.g
    Ev = np.array([0.3, -1.2, 0.5])
    sim.set_fields(E=_uniform_field(g, Ev))
    assert abs(sim.diagnostics()["field"] - 0.5 * (Ev @ Ev) * Lx * Ly) < 1e-13 * Lx * Ly
    Hv, Hp = np.array([0.9, 0.1, -0.4]), np.array([-0.3, 0.7, 1.4])
    sim.set_fields(E=np.zeros((3, ny, g.nxn)), H=np.broadcast_to(Hv[:, None, None], (3, ny, nx)))
    assert abs(sim.diagnostics()["field"] - 0.5 * (Hv @ Hv) * Lx * Ly) < 1e-13 * Lx * Ly
    sim.H_prev = np.broadcast_to(Hp[:, None, None], (3, ny, nx)).copy()
    Hm = 0.5 * (Hv + Hp)
    assert abs(sim.diagnostics()["field"] - 0.5 * (Hm @ Hm) * Lx * Ly) < 1e-13 * Lx * Ly
    if periodic:
        A = 1.7
        Ez = np.zeros((3, ny, nx))
        Ez[2] = A * np.cos(2 * np.pi * 5 * np.arange(nx) / nx)[None, :]
        sim.set_fields(E=Ez, H=np.zeros((3, ny, nx)))
        assert abs(sim.diagnostics()["field"] - 0.25 * A * A * Lx * Ly) < 1e-13 * Lx * Ly
        cn = oracle.OracleSim(nx, ny, dx, dy, 0.2, True, W.FIELD_CN, [(-1.0, 1.0)], 4, 5)
        cn.set_fields(H=np.broadcast_to(Hv[:, None, None], (3, ny, nx)))
        cn.H_prev = np.zeros((3, ny, nx))       # the implicit-curl mode keeps H at integer times
        assert abs(cn.diagnostics()["field"] - 0.5 * (Hv @ Hv) * Lx * Ly) < 1e-13 * Lx * Ly


# ----------------------------------------------------------------------------- laser reading (reading 12)
def test_laser_envelope_closed_form():
    """Reading of the missing Eq. 15: a0 sin(omega t) under a Gaussian envelope whose intensity has
    full width tau at half maximum and peaks at t0: the envelope is 1 at t0, its square is 1/2 at
    t0 +- tau/2, and nothing is emitted before t = 0."""
    a0, omega, tau, t0 = 5.0, 1.0, 70.0, 70.0
    env = lambda t: oracle.laser(t, a0, omega, tau, t0) / (a0 * math.sin(omega * t))
    assert abs(env(t0) - 1.0) < 1e-15
    for t in (t0 - tau / 2, t0 + tau / 2):
        assert abs(env(t) ** 2 - 0.5) < 1e-14
    assert oracle.laser(-1e-9, a0, omega, tau, t0) == 0.0
    assert abs(oracle.laser(t0 + 0.3, a0, omega, 0.0, t0) - a0 * math.sin(omega * (t0 + 0.3))) < 1e-15


# ----------------------------------------------------------------------------- CN operator symbol
def test_curl_curl_fourier_symbol():
    """On a periodic grid curl_h curl_e maps the node mode e^{i(a i + b j)} e_c to
    M(a, b) e_c with p = (e^{ia}-1)(1+e^{ib})/(2dx), q = (1+e^{ia})(e^{ib}-1)/(2dy):
    M = [[|q|^2, -q* p, 0], [-p* q, |p|^2, 0], [0, 0, |p|^2 + |q|^2]] (closed form of
    the stencils' Fourier symbols; the GPU's spectral preconditioner inverts it)."""
    nx, ny, dx, dy = 12, 8, 0.3, 0.5
    g = oracle.Grid(nx, ny, dx, dy, True)
    Ce, Ch = oracle.curl_matrices(g)
    K = Ch @ Ce
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for kx in range(nx):
        for ky in range(ny):
            a, b = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
            ph = np.exp(1j * (a * ii + b * jj)).ravel()
            p = (np.exp(1j * a) - 1) * (1 + np.exp(1j * b)) / (2 * dx)
            q = (1 + np.exp(1j * a)) * (np.exp(1j * b) - 1) / (2 * dy)
            M = np.array([[abs(q) ** 2, -np.conj(q) * p, 0], [-np.conj(p) * q, abs(p) ** 2, 0],
                          [0, 0, abs(p) ** 2 + abs(q) ** 2]])
            for c in range(3):
                e = np.zeros(3 * nx * ny, complex)
                e[c * nx * ny:(c + 1) * nx * ny] = ph
                r = (K @ e).reshape(3, -1)
                for rr in range(3):
                    assert np.max(np.abs(r[rr] - M[rr, c] * ph)) < 1e-12 * (1 + abs(M[rr, c]))
