"""Pins of the oracle's shape orders 2-4 (the centred B-spline of that degree over the nearest
(n + 1) x (n + 1) nodes), the higher-order weighting up to fourth order the paper mentions beside
its own linear one (Section 3.3, last paragraph).

Each pin checks the oracle against something fixed independently of its code: the spline built by
the Cox-de Boor recursion from the unit box (the oracle evaluates closed piecewise forms) at every
node, partition of unity and the spline's constant second moment ((n + 1)/12 cell^2), exact
reproduction of linear fields, charge conservation (with the wall reading: a node beyond a wall
gives its weight to the wall node), and the k = 0 pins of the linear scheme (uniform lattice
response, discrete cold-plasma frequency), which hold for any shape whose weights sum to one.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1308_2590_gb300 import workloads as W


def bspline(n, x):
    """Centred cardinal B-spline of degree n by the Cox-de Boor recursion from the unit box."""
    x = np.asarray(x, dtype=float)
    if n == 0:
        return np.where((x >= -0.5) & (x < 0.5), 1.0, 0.0)
    h = (n + 1) / 2.0
    return ((x + h) * bspline(n - 1, x + 0.5) + (h - x) * bspline(n - 1, x - 0.5)) / n


def b2(t):
    return bspline(2, t)


def _dense_weights(g, x, y, order=2):
    node, W_ = oracle.shape_nodes(g, x, y, order)
    D = np.zeros((x.size, g.ny * g.nxn))
    for p in range(x.size):
        for k in range(node.shape[1]):
            if node[p, k] >= 0:
                D[p, node[p, k]] += W_[p, k]
    return D


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("periodic", [True, False])
def test_spline_weights_match_the_recursive_definition(periodic, order):
    """Every node's weight equals B_n of its distance (cells) along x times along y; periodic images
    wrap; on a walled box a node beyond a wall adds its weight to the wall node."""
    rng = np.random.default_rng(11)
    g = oracle.Grid(7, 6, 0.4, 0.3, periodic, shape=order)
    x = rng.random(200) * g.Lx
    y = rng.random(200) * g.Ly
    x[:4] = [0.0, 0.3 * g.dx, g.Lx - 0.2 * g.dx, 0.5 * g.dx]     # wall and half-cell cases
    D = _dense_weights(g, x, y, order)
    for p in range(x.size):
        sx, sy = x[p] / g.dx, y[p] / g.dy
        wx = np.zeros(g.nxn)
        for i in range(-4, g.nx + 5):
            wgt = bspline(order, i - sx)
            if wgt == 0.0:
                continue
            if periodic:
                wx[i % g.nx] += wgt
            else:
                wx[min(max(i, 0), g.nx)] += wgt
        wy = np.zeros(g.ny)
        for j in range(-4, g.ny + 5):
            wy[j % g.ny] += bspline(order, j - sy)
        assert np.max(np.abs(D[p].reshape(g.ny, g.nxn) - np.outer(wy, wx))) < 1e-14


@pytest.mark.parametrize("order", [2, 3, 4])
def test_spline_partition_of_unity_and_second_moment(order):
    """Weights sum to 1; along each axis sum w (i - s)^2 = (n + 1)/12 for every position (the B_n
    variance), where the linear weights give f (1 - f) instead."""
    rng = np.random.default_rng(12)
    g = oracle.Grid(13, 12, 1.0, 1.0, True, shape=order)
    x = 4.0 + rng.random(300) * 4.0
    y = 4.0 + rng.random(300) * 4.0
    node, W_ = oracle.shape_nodes(g, x, y)
    assert np.max(np.abs(W_.sum(axis=1) - 1.0)) < 1e-14
    ix, iy = node % g.nxn, node // g.nxn
    mx = np.sum(W_ * (ix - x[:, None]) ** 2, axis=1)
    my = np.sum(W_ * (iy - y[:, None]) ** 2, axis=1)
    v = (order + 1) / 12.0
    assert np.max(np.abs(mx - v)) < 1e-13 and np.max(np.abs(my - v)) < 1e-13
    # the linear shape, for contrast: variance f (1 - f)
    n1, w1 = oracle.shape_nodes(g, x, y, order=1)
    v1 = np.sum(w1[:, :4] * ((n1[:, :4] % g.nxn) - x[:, None]) ** 2, axis=1)
    f = x - np.floor(x)
    assert np.max(np.abs(v1 - f * (1 - f))) < 1e-13


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("periodic", [True, False])
def test_spline_gather_reproduces_linear_fields(periodic, order):
    """A field linear in x and y is gathered exactly (the spline reproduces degree-1 polynomials), away
    from a periodic seam and from the walls (where a folded node changes the sum)."""
    rng = np.random.default_rng(13)
    g = oracle.Grid(14, 12, 0.5, 0.25, periodic, shape=order)
    jj, ii = np.meshgrid(np.arange(g.ny), np.arange(g.nxn), indexing="ij")
    F = np.zeros((3, g.ny, g.nxn))
    a = np.array([[0.3, -1.2, 0.7], [2.0, 0.5, -0.4], [-0.6, 1.1, 0.9]])
    for c in range(3):
        F[c] = a[c, 0] + a[c, 1] * ii * g.dx + a[c, 2] * jj * g.dy
    x = (3.0 + rng.random(100) * (g.nx - 6.0)) * g.dx
    y = (3.0 + rng.random(100) * (g.ny - 6.0)) * g.dy
    got = oracle.gather(g, F, x, y)
    want = np.stack([a[c, 0] + a[c, 1] * x + a[c, 2] * y for c in range(3)], axis=1)
    assert np.max(np.abs(got - want)) < 1e-13


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("periodic", [True, False])
def test_spline_deposit_conserves_charge(periodic, order):
    rng = np.random.default_rng(14)
    g = oracle.Grid(11, 7, 0.6, 0.8, periodic, shape=order)
    n = 500
    P = dict(x=rng.random(n) * g.Lx, y=rng.random(n) * g.Ly, ux=rng.standard_normal(n) * 0.3,
             uy=rng.standard_normal(n) * 0.3, uz=rng.standard_normal(n) * 0.3, w=0.5 + rng.random(n))
    P["x"][:3] = [0.0, 0.1 * g.dx, g.Lx - 0.1 * g.dx]
    M = oracle.deposit_raw(g, 0.4, -1.0, 1.0, np.zeros((3, g.ny, g.nxn)), P)
    assert abs(M[0].sum() - (-1.0) * P["w"].sum()) < 1e-12 * P["w"].sum()


@pytest.mark.parametrize("order", [2, 3, 4])
def test_spline_wall_node_takes_the_folded_weight(order):
    """A particle in the first cell: node 0 holds B_n(0 - s) plus the weights of every node beyond the
    wall, nodes 1.. their own B_n(i - s)."""
    g = oracle.Grid(8, 8, 1.0, 1.0, False, shape=order)
    s = 0.2
    node, W_ = oracle.shape_nodes(g, np.array([s]), np.array([3.0]))
    col = np.zeros(g.nxn)
    for k in range(node.shape[1]):
        if node[0, k] >= 0:
            col[node[0, k] % g.nxn] += W_[0, k]
    outside = sum(bspline(order, i - s) for i in range(-4, 0))
    assert abs(col[0] - (bspline(order, -s) + outside)) < 1e-15
    for i in range(1, 4):
        assert abs(col[i] - bspline(order, i - s)) < 1e-15
    assert abs(col.sum() - 1.0) < 1e-15


@pytest.mark.parametrize("order", [2, 3, 4])
def test_spline_push_in_uniform_fields_equals_the_linear_push(order):
    """Uniform E and B: gathered values do not depend on the shape (weights sum to one), so both
    orders push every particle the same to rounding."""
    rng = np.random.default_rng(15)
    g1 = oracle.Grid(8, 8, 0.5, 0.5, False, shape=1)
    g2 = oracle.Grid(8, 8, 0.5, 0.5, False, shape=order)
    E = np.zeros((3, 8, 9)); B = np.zeros((3, 8, 9))
    for c, (e, b) in enumerate(zip((0.3, -0.2, 0.1), (0.5, 1.5, -0.7))):
        E[c] = e; B[c] = b
    n = 64
    P = dict(x=0.5 + rng.random(n) * 3.0, y=rng.random(n) * 4.0, ux=rng.standard_normal(n),
             uy=rng.standard_normal(n), uz=rng.standard_normal(n), w=np.ones(n))
    P2 = {k: v.copy() for k, v in P.items()}
    oracle.push(g1, 0.2, -1.0, 1.0, E, B, P)
    oracle.push(g2, 0.2, -1.0, 1.0, E, B, P2)
    for k in ("x", "y", "ux", "uy", "uz"):
        assert np.max(np.abs(P[k] - P2[k])) < 1e-14 * (1 + np.max(np.abs(P[k])))


@pytest.mark.parametrize("order", [2, 3, 4])
def test_spline_lattice_response_tensor_is_exact(order):
    """The k = 0 lattice pin with the spline shapes: a uniform lattice deposits the same uniform
    S = (omega_pe dt / 2)^2 I / gamma and dj = -u / gamma."""
    cfg = W.RunConfig(name="cold", nx=6, ny=5, dx=0.3, dy=0.4, dt=0.5, steps=1,
                      species=[W.Species(-1.0, 1.0, 1, 1.0, 0.0)], tile_nx=3, tile_ny=5, shape=order)
    sim = oracle.OracleSim.from_config(cfg)
    u0 = 0.01
    sim.load_particles(0, **W.lattice_particles(cfg, 0, offsets=((0.25, 0.6), (0.7, 0.1)), drift=(u0, 0, 0)))
    gam = math.sqrt(1 + u0 * u0)
    s = (0.5 / 2) ** 2 / gam
    for k in range(9):
        target = s if k in (0, 4, 8) else 0.0
        assert np.max(np.abs(sim.M[1 + k] - target)) < 1e-15
    assert np.max(np.abs(sim.M[10] - (-u0 / gam))) < 1e-15


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("field_mode", [W.FIELD_LITERAL, W.FIELD_CN])
def test_spline_cold_plasma_discrete_frequency(field_mode, order):
    """k = 0 cold oscillation with the spline shape: the same discrete frequency 2 atan(omega_pe dt / 2)."""
    dt = 0.5
    cfg = W.RunConfig(name="cold", nx=6, ny=5, dx=0.6, dy=0.8, dt=dt, steps=40, bc_x=W.BC_PERIODIC,
                      field_mode=field_mode, species=[W.Species(-1.0, 1.0, 1, 1.0, 0.0)], tile_nx=3, tile_ny=5,
                      shape=order)
    sim = oracle.OracleSim.from_config(cfg)
    sim.load_particles(0, **W.lattice_particles(cfg, 0, offsets=((0.25, 0.6),), drift=(1e-5, 0.0, 0.0)))
    ux = [sim.parts[0]["ux"][0]]
    for _ in range(40):
        sim.step()
        assert np.ptp(sim.E[0]) < 1e-15 + 1e-9 * np.max(np.abs(sim.E[0]))
        ux.append(sim.parts[0]["ux"][7])
    ux = np.array(ux)
    n = np.arange(1, len(ux) - 1)
    big = np.abs(ux[n]) > 0.2 * np.max(np.abs(ux))
    c = (ux[n + 1] + ux[n - 1])[big] / ux[n][big]
    assert np.max(np.abs(c - 2 * math.cos(2 * math.atan(dt / 2)))) < 1e-6
