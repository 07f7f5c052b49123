"""FP64 CPU oracle of the implicit 2D3V PIC particle loop and field solve.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product library
never does, and nothing here is shared with the CUDA path.

What it computes (Petrov & Davis, Section 2 and Section 3.3):
  * gather of E and B at each particle with linear (area) weights -- Section 3.3
    (or, shape orders 2-4, the centred B-spline of that degree over the nearest
    (n + 1) x (n + 1) nodes, the higher orders the same paragraph mentions);
  * the implicit push, Eq. 2a-c with E factored out -- Section 2;
  * deposit of rho, the 9-component tensor S and the 3-component residual
    current dj on the nodes -- Eq. 3, Section 3.3 step 1;
  * the field advance, Eqs. 4-5 (``literal`` mode), or its time-centred
    variant with implicit curls (``cn`` mode, solved by sparse LU; in a box
    with walls the wall nodes take a time-centred first-order Mur condition,
    see ``cn_system``);
  * the order in which particles are kept (grouped by tile);
  * FP64 diagnostics: charge, kinetic and field energy, particle count.

The per-particle and per-node loops are plain C (``pic_oracle.c``); the
sparse CN system is assembled here from the same stencil definitions and
solved with ``scipy.sparse.linalg.splu`` (a library LU, used as one step).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

NMOM = 13


def build(force: bool = False) -> str:
    """Compile pic_oracle.c into a shared library (plain C, no FP contraction)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.c_double
        i = ctypes.c_int
        i64 = ctypes.c_int64
        p = ctypes.c_void_p
        _lib.orc_locate.argtypes = [i, i, i, d, d, i64, p, p, p, p, p, p]
        _lib.orc_shape_nodes.argtypes = [i, i, i, d, d, i, i64, p, p, p, p]
        _lib.orc_gather.argtypes = [i, i, i, d, d, p, i64, p, p, p, i]
        _lib.orc_rotate.argtypes = [p, p, p]
        _lib.orc_push.argtypes = [i, i, i, d, d, d, d, d, p, p, i64, p, p, p, p, p, p, i]
        _lib.orc_deposit.argtypes = [i, i, i, d, d, d, d, d, p, i64, p, p, p, p, p, p, p, i]
        _lib.orc_normalize.argtypes = [i, i, i, d, d, p, p]
        _lib.orc_curl_h.argtypes = [i, i, i, d, d, p, p]
        _lib.orc_curl_e.argtypes = [i, i, i, d, d, p, p]
        _lib.orc_node_average.argtypes = [i, i, i, p, p]
        _lib.orc_laser.argtypes = [d, d, d, d, d]
        _lib.orc_laser.restype = d
        _lib.orc_field_literal.argtypes = [i, i, i, d, d, d, d, d, d, d, d, i, p, p, p, p, p, p]
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------- grid helpers

class Grid:
    """nx x ny cells; E/moments on nodes, H at cell centres (Section 3.2, Fig. 1); shape order 1 (the
    paper's area weighting) or 2-4 (B-splines of that degree) for gather and deposit (Section 3.3)."""

    def __init__(self, nx: int, ny: int, dx: float, dy: float, periodic_x: bool, shape: int = 1):
        self.nx, self.ny, self.dx, self.dy = int(nx), int(ny), float(dx), float(dy)
        self.periodic_x = bool(periodic_x)
        assert shape in (1, 2, 3, 4)
        self.shape = int(shape)
        self.nxn = self.nx if self.periodic_x else self.nx + 1
        self.nnode = self.ny * self.nxn
        self.ncell = self.ny * self.nx
        self.Lx = self.nx * self.dx
        self.Ly = self.ny * self.dy

    def args(self):
        return (self.nx, self.ny, int(self.periodic_x), self.dx, self.dy)

    def node_area(self) -> np.ndarray:
        a = np.full((self.ny, self.nxn), self.dx * self.dy)
        if not self.periodic_x:
            a[:, 0] *= 0.5
            a[:, -1] *= 0.5
        return a


def locate(g: Grid, x, y):
    x = _f64(x); y = _f64(y)
    n = x.size
    cx = np.empty(n, np.int32); cy = np.empty(n, np.int32)
    fx = np.empty(n); fy = np.empty(n)
    lib().orc_locate(*g.args(), n, _p(x), _p(y), _p(cx), _p(cy), _p(fx), _p(fy))
    return cx, cy, fx, fy


MAX_SHAPE_NODES = 25


def shape_nodes(g: Grid, x, y, order: Optional[int] = None):
    """Node indices (-1: unused entry) and weights, MAX_SHAPE_NODES per particle, of the grid's shape."""
    x = _f64(x); y = _f64(y)
    node = np.empty((x.size, MAX_SHAPE_NODES), np.int64); W = np.empty((x.size, MAX_SHAPE_NODES))
    lib().orc_shape_nodes(*g.args(), g.shape if order is None else int(order), x.size, _p(x), _p(y), _p(node), _p(W))
    return node, W


def gather(g: Grid, F, x, y) -> np.ndarray:
    F = _f64(F); x = _f64(x); y = _f64(y)
    out = np.empty((x.size, 3))
    lib().orc_gather(*g.args(), _p(F), x.size, _p(x), _p(y), _p(out), g.shape)
    return out


def rotate(b, v) -> np.ndarray:
    b = _f64(b); v = _f64(v); o = np.empty(3)
    lib().orc_rotate(_p(b), _p(v), _p(o))
    return o


def push(g: Grid, dt: float, q: float, m: float, Ehalf, Bold, P: dict) -> np.ndarray:
    """Advance the particle dict P in place; returns the alive mask."""
    n = P["x"].size
    alive = np.ones(n, np.uint8)
    lib().orc_push(*g.args(), dt, q, m, _p(_f64(Ehalf)), _p(_f64(Bold)), n,
                   _p(P["x"]), _p(P["y"]), _p(P["ux"]), _p(P["uy"]), _p(P["uz"]), _p(alive), g.shape)
    return alive.astype(bool)


def deposit_raw(g: Grid, dt: float, q: float, m: float, Bn, P: dict, Mraw: Optional[np.ndarray] = None) -> np.ndarray:
    if Mraw is None:
        Mraw = np.zeros((NMOM, g.ny, g.nxn))
    n = P["x"].size
    lib().orc_deposit(*g.args(), dt, q, m, _p(_f64(Bn)), n, _p(P["x"]), _p(P["y"]),
                      _p(P["ux"]), _p(P["uy"]), _p(P["uz"]), _p(P["w"]), _p(Mraw), g.shape)
    return Mraw


def normalize(g: Grid, Mraw) -> np.ndarray:
    out = np.empty((NMOM, g.ny, g.nxn))
    lib().orc_normalize(*g.args(), _p(_f64(Mraw)), _p(out))
    return out


def curl_h(g: Grid, H) -> np.ndarray:
    out = np.empty((3, g.ny, g.nxn))
    lib().orc_curl_h(*g.args(), _p(_f64(H)), _p(out))
    return out


def curl_e(g: Grid, E) -> np.ndarray:
    out = np.empty((3, g.ny, g.nx))
    lib().orc_curl_e(*g.args(), _p(_f64(E)), _p(out))
    return out


def node_average(g: Grid, Hc) -> np.ndarray:
    out = np.empty((3, g.ny, g.nxn))
    lib().orc_node_average(g.nx, g.ny, int(g.periodic_x), _p(_f64(Hc)), _p(out))
    return out


def laser(t: float, a0: float, omega: float, tau: float, t0: float) -> float:
    return lib().orc_laser(t, a0, omega, tau, t0)


def field_literal(g: Grid, dt: float, t_new: float, las, E, H, M):
    """Eqs. 4-5 with the wall/laser readings; returns (E^{n+1}, H^{n+3/2})."""
    Enew = np.empty((3, g.ny, g.nxn))
    Hnew = np.empty((3, g.ny, g.nx))
    work = np.empty((3, g.ny, g.nxn))
    a0, omega, tau, t0, pol = las
    lib().orc_field_literal(*g.args(), dt, t_new, a0, omega, tau, t0, int(pol),
                            _p(_f64(E)), _p(_f64(H)), _p(_f64(M)), _p(Enew), _p(Hnew), _p(work))
    return Enew, Hnew


# ----------------------------------------------------------------------------- CN system

def curl_matrices(g: Grid):
    """Sparse curl_e (nodes -> cells) and curl_h (nodes <- cells).

    Unknowns are ordered component-major, as the planar arrays flatten:
    index c * nnode + j * nxn + i.  Same stencils as the C routines: in a box
    with walls a cell's corners are never wrapped in x, and on a wall column
    curl_h keeps only the y-differences of the two cells inside the box.
    """
    import scipy.sparse as sp
    nx, ny, nxn, NN, NC = g.nx, g.ny, g.nxn, g.nnode, g.ncell
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    jj = jj.ravel(); ii = ii.ravel()
    ip = (ii + 1) % nx if g.periodic_x else ii + 1
    jp = (jj + 1) % ny; jm = (jj - 1) % ny
    cell = jj * nx + ii
    # curl_e: cell (i,j) from corners p00=(i,j) p10=(i+1,j) p01=(i,j+1) p11=(i+1,j+1)
    p00 = jj * nxn + ii; p10 = jj * nxn + ip; p01 = jp * nxn + ii; p11 = jp * nxn + ip
    rows, cols, vals = [], [], []

    def add(r, c, v):
        rows.append(r); cols.append(c); vals.append(np.broadcast_to(v, r.shape))

    hy = 1.0 / (2 * g.dy); hx = 1.0 / (2 * g.dx)
    # x: dEz/dy
    for pnt, s in ((p01, 1), (p11, 1), (p00, -1), (p10, -1)):
        add(0 * NC + cell, 2 * NN + pnt, s * hy)
    # y: -dEz/dx
    for pnt, s in ((p10, 1), (p11, 1), (p00, -1), (p01, -1)):
        add(1 * NC + cell, 2 * NN + pnt, -s * hx)
    # z: dEy/dx - dEx/dy
    for pnt, s in ((p10, 1), (p11, 1), (p00, -1), (p01, -1)):
        add(2 * NC + cell, 1 * NN + pnt, s * hx)
    for pnt, s in ((p01, 1), (p11, 1), (p00, -1), (p10, -1)):
        add(2 * NC + cell, 0 * NN + pnt, -s * hy)
    Ce = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(3 * NC, 3 * NN))
    # curl_h: node (i,j) from cells a=(i,j) b=(i-1,j) c=(i,j-1) d=(i-1,j-1)
    jn, inn = np.meshgrid(np.arange(ny), np.arange(nxn), indexing="ij")
    jn = jn.ravel(); inn = inn.ravel()
    node = jn * nxn + inn
    jnm = (jn - 1) % ny
    rows, cols, vals = [], [], []
    if g.periodic_x:
        inside = np.ones(node.size, bool)
    else:
        inside = (inn > 0) & (inn < nx)
    n_in, i_in, j_in, jm_in = node[inside], inn[inside], jn[inside], jnm[inside]
    im_in = (i_in - 1) % nx
    a = j_in * nx + i_in; b = j_in * nx + im_in; c = jm_in * nx + i_in; d = jm_in * nx + im_in
    for cl, s in ((a, 1), (b, 1), (c, -1), (d, -1)):      # x: dHz/dy
        add(0 * NN + n_in, 2 * NC + cl, s * hy)
    for cl, s in ((a, 1), (c, 1), (b, -1), (d, -1)):      # y: -dHz/dx
        add(1 * NN + n_in, 2 * NC + cl, -s * hx)
    for cl, s in ((a, 1), (c, 1), (b, -1), (d, -1)):      # z: dHy/dx
        add(2 * NN + n_in, 1 * NC + cl, s * hx)
    for cl, s in ((a, 1), (b, 1), (c, -1), (d, -1)):      # z: -dHx/dy
        add(2 * NN + n_in, 0 * NC + cl, -s * hy)
    if not g.periodic_x:
        wall = ~inside
        n_w, i_w, j_w, jm_w = node[wall], inn[wall], jn[wall], jnm[wall]
        ic = np.where(i_w == 0, 0, nx - 1)
        up = j_w * nx + ic; dn = jm_w * nx + ic
        for cl, s in ((up, 1), (dn, -1)):                 # x: dHz/dy of the inside cells
            add(0 * NN + n_w, 2 * NC + cl, s * 2 * hy)
        for cl, s in ((up, 1), (dn, -1)):                 # z: -dHx/dy of the inside cells
            add(2 * NN + n_w, 0 * NC + cl, -s * 2 * hy)
    Ch = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(3 * NN, 3 * NC))
    return Ce, Ch


def wall_mask(g: Grid) -> np.ndarray:
    """True at the node columns on a wall (none in a periodic box), shape (ny, nxn)."""
    m = np.zeros((g.ny, g.nxn), bool)
    if not g.periodic_x:
        m[:, 0] = m[:, -1] = True
    return m


def cn_operator(g: Grid, dt: float, M):
    """A = I + S + (dt/2)^2 curl_h curl_e acting on E^{n+1/2} (component-major); in a box with walls
    the wall nodes are vacuum (S left out there) and their y and z rows are replaced by cn_system."""
    import scipy.sparse as sp
    NN = g.nnode
    Ce, Ch = curl_matrices(g)
    keep = (~wall_mask(g)).ravel().astype(float)
    rows, cols, vals = [], [], []
    idx = np.arange(NN)
    for r in range(3):
        for c in range(3):
            rows.append(r * NN + idx); cols.append(c * NN + idx)
            vals.append(M[1 + 3 * r + c].ravel() * keep)
    S = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(3 * NN, 3 * NN))
    A = sp.identity(3 * NN, format="csr") + S + (0.25 * dt * dt) * (Ch @ Ce)
    return A.tocsc()


def cn_rhs(g: Grid, dt: float, E, H, M) -> np.ndarray:
    """E^n + (dt/2)(curl_h H^n - dj) (dj left out on wall nodes)."""
    dj = M[10:13] * (~wall_mask(g))[None]
    return (E + 0.5 * dt * (curl_h(g, H) - dj)).ravel()


def cn_system(g: Grid, dt: float, E, H, M, t_new: float = 0.0, las=(0.0, 1.0, 0.0, 0.0, 0)):
    """The implicit-curl system for X = E^{n+1/2}: (A, rhs) with A X = rhs.

    Interior nodes: (I + S) X + (dt/2)^2 curl_h curl_e X = E^n + (dt/2)(curl_h H^n - dj).
    Walls (reading of the missing Eq. 14 for this mode): the wall node is vacuum; its x row is the same
    equation with the one-sided curl_h of the wall column; its y and z rows are the first-order Mur
    condition (d/dt -+ d/dx) E = 0 at x = 0 / Lx written time-centred between the wall node w and its
    neighbour v (E^{n+1} = 2 X - E^n):  (1/dt + 1/dx) X_w + (1/dt - 1/dx) X_v = (E_w^n + E_v^n)/dt,
    at x = 0 for the field minus the incident plane wave (reading 12: E_inc(x, t) = laser(t - x) in the
    polarised component), whose centred values (E_inc^n + E_inc^{n+1})/2 move to the right-hand side.
    """
    import scipy.sparse as sp
    A = cn_operator(g, dt, M)
    rhs = cn_rhs(g, dt, E, H, M)
    if g.periodic_x:
        return A, rhs
    NN, nxn, ny = g.nnode, g.nxn, g.ny
    a0, omega, tau, t0, pol = las
    pc = 1 if int(pol) == 0 else 2
    t_old = t_new - dt
    cw, cv = 1.0 / dt + 1.0 / g.dx, 1.0 / dt - 1.0 / g.dx
    A = A.tolil()
    for comp in (1, 2):
        for j in range(ny):
            for (w, v, left) in ((0, 1, True), (nxn - 1, nxn - 2, False)):
                row = comp * NN + j * nxn + w
                A.rows[row] = []
                A.data[row] = []
                A[row, comp * NN + j * nxn + w] = cw
                A[row, comp * NN + j * nxn + v] = cv
                r = (E[comp, j, w] + E[comp, j, v]) / dt
                if left and comp == pc:
                    inc = lambda x, t: laser(t - x, a0, omega, tau, t0)
                    iw = 0.5 * (inc(0.0, t_old) + inc(0.0, t_new))
                    iv = 0.5 * (inc(g.dx, t_old) + inc(g.dx, t_new))
                    r += -(inc(0.0, t_old) + inc(g.dx, t_old)) / dt + cw * iw + cv * iv
                rhs[row] = r
    return A.tocsc(), rhs


def field_cn(g: Grid, dt: float, E, H, M, t_new: float = 0.0, las=(0.0, 1.0, 0.0, 0.0, 0)):
    """Time-centred field advance with implicit curls:
    solve cn_system for X = E^{n+1/2}, then E^{n+1} = 2 X - E^n,  H^{n+1} = H^n - dt curl_e X.
    Returns (E^{n+1}, H^{n+1}, X)."""
    import scipy.sparse.linalg as spl
    A, rhs = cn_system(g, dt, E, H, M, t_new, las)
    X = spl.splu(A).solve(rhs).reshape(3, g.ny, g.nxn)
    Enew = 2.0 * X - E
    Hnew = H - dt * curl_e(g, X)
    return Enew, Hnew, X


# ----------------------------------------------------------------------------- simulation

class OracleSim:
    """Whole-step oracle: state, ordering rule, diagnostics.

    Order of one step (Section 3.3: field solver, forces, pusher, moments):
      1. field advance from the moments deposited at the end of the last step;
      2. B at the nodes from the new H;
      3. per particle: gather (E^{n+1/2}, and the B the moments were made with)
         at r^n, push, move; particles leaving a wall are dropped;
      4. particles re-ordered: grouped by tile in ascending tile order, inside
         a tile by cell (row by row, x fastest); inside a cell, particles that
         were already in the tile keep their order, then the particles that
         arrived from other tiles, in their previous order (a stable sort of
         the previous order by (tile, cell, arrived));
      5. moments deposited at r^{n+1} with u^{n+1} and the new B.
    A load appends the new particles after the old ones and stably sorts all
    of them by (tile, cell).
    """

    def __init__(self, nx, ny, dx, dy, dt, periodic_x, field_mode, species, tile_nx, tile_ny,
                 laser_params=(0.0, 1.0, 0.0, 0.0, 0), shape: int = 1):
        self.g = Grid(nx, ny, dx, dy, periodic_x, shape)
        self.dt = float(dt)
        self.field_mode = int(field_mode)   # 0 literal, 1 cn
        self.species = [(float(q), float(m)) for (q, m) in species]
        self.tile_nx, self.tile_ny = int(min(tile_nx, nx)), int(min(tile_ny, ny))
        self.ntx = -(-self.g.nx // self.tile_nx)
        self.laser = tuple(laser_params)
        g = self.g
        self.E = np.zeros((3, g.ny, g.nxn))
        self.H = np.zeros((3, g.ny, g.nx))
        self.H_prev = np.zeros((3, g.ny, g.nx))
        self.B = np.zeros((3, g.ny, g.nxn))
        self.parts: List[dict] = [self._empty() for _ in self.species]
        self.step_index = 0
        self.removed = [0 for _ in self.species]
        self.M = np.zeros((NMOM, g.ny, g.nxn))

    @staticmethod
    def _empty():
        return {k: np.zeros(0) for k in ("x", "y", "ux", "uy", "uz", "w")}

    @classmethod
    def from_config(cls, cfg):
        las = (cfg.laser.a0, cfg.laser.omega, cfg.laser.tau, cfg.laser.t0, cfg.laser.pol)
        return cls(cfg.nx, cfg.ny, cfg.dx, cfg.dy, cfg.dt, cfg.bc_x == 0, cfg.field_mode,
                   [(s.q, s.m) for s in cfg.species], cfg.tile_nx, cfg.tile_ny, las, getattr(cfg, "shape", 1))

    def tile_of(self, x, y) -> np.ndarray:
        cx, cy, _, _ = locate(self.g, x, y)
        return (cy // self.tile_ny).astype(np.int64) * self.ntx + (cx // self.tile_nx)

    def tile_cell_key(self, x, y) -> np.ndarray:
        """(tile, cell inside the tile) as one integer: tile * tile_nx * tile_ny + ly * tile_nx + lx."""
        cx, cy, _, _ = locate(self.g, x, y)
        cx = cx.astype(np.int64); cy = cy.astype(np.int64)
        tile = (cy // self.tile_ny) * self.ntx + cx // self.tile_nx
        return tile * (self.tile_nx * self.tile_ny) + (cy % self.tile_ny) * self.tile_nx + cx % self.tile_nx

    def load_particles(self, s: int, x, y, ux, uy, uz, w):
        """Append particles; the species is then stably ordered by (tile, cell)."""
        P = self.parts[s]
        new = dict(x=_f64(x), y=_f64(y), ux=_f64(ux), uy=_f64(uy), uz=_f64(uz), w=_f64(w))
        for k in P:
            P[k] = np.concatenate([P[k], new[k]])
        order = np.argsort(self.tile_cell_key(P["x"], P["y"]), kind="stable")
        for k in P:
            P[k] = np.ascontiguousarray(P[k][order])
        self.deposit()

    def set_fields(self, E=None, H=None):
        if E is not None:
            self.E = _f64(E).reshape(3, self.g.ny, self.g.nxn).copy()
        if H is not None:
            self.H = _f64(H).reshape(3, self.g.ny, self.g.nx).copy()
            self.H_prev = self.H.copy()
        self.B = node_average(self.g, self.H)
        self.deposit()

    def deposit(self):
        raw = np.zeros((NMOM, self.g.ny, self.g.nxn))
        for (q, m), P in zip(self.species, self.parts):
            deposit_raw(self.g, self.dt, q, m, self.B, P, raw)
        self.M_raw = raw
        self.M = normalize(self.g, raw)

    def step(self, nsteps: int = 1):
        for _ in range(nsteps):
            self._step()

    def _step(self):
        g, dt = self.g, self.dt
        t_new = (self.step_index + 1) * dt
        if self.field_mode == 0:
            Enew, Hnew = field_literal(g, dt, t_new, self.laser, self.E, self.H, self.M)
            Ehalf = 0.5 * (self.E + Enew)
        else:
            Enew, Hnew, Ehalf = field_cn(g, dt, self.E, self.H, self.M, t_new, self.laser)
        Bnew = node_average(g, Hnew)
        for s, ((q, m), P) in enumerate(zip(self.species, self.parts)):
            if P["x"].size == 0:
                continue
            old_tile = self.tile_of(P["x"], P["y"])
            alive = push(g, dt, q, m, Ehalf, self.B, P)
            self.removed[s] += int((~alive).sum())
            for k in P:
                P[k] = P[k][alive]
            old_tile = old_tile[alive]
            new_tile = self.tile_of(P["x"], P["y"])
            key = 2 * self.tile_cell_key(P["x"], P["y"]) + (new_tile != old_tile)
            order = np.argsort(key, kind="stable")
            for k in P:
                P[k] = np.ascontiguousarray(P[k][order])
        self.H_prev = self.H
        self.E, self.H, self.B = Enew, Hnew, Bnew
        self.deposit()
        self.step_index += 1

    def diagnostics(self) -> dict:
        g = self.g
        ke = 0.0
        qw = 0.0
        count = 0
        for (q, m), P in zip(self.species, self.parts):
            u2 = P["ux"] ** 2 + P["uy"] ** 2 + P["uz"] ** 2
            ke += float(np.sum(P["w"] * m * (np.sqrt(1.0 + u2) - 1.0)))
            qw += float(np.sum(q * P["w"]))
            count += P["x"].size
        area = g.node_area()
        if self.field_mode == 0:
            Hc = 0.5 * (self.H + self.H_prev)
        else:
            Hc = self.H
        fe = 0.5 * float(np.sum(self.E ** 2 * area[None])) + 0.5 * float(np.sum(Hc ** 2)) * g.dx * g.dy
        charge = float(np.sum(self.M_raw[0]))
        return dict(kinetic=ke, field=fe, total=ke + fe, charge_grid=charge, charge_particles=qw,
                    count=count, removed=sum(self.removed))

    def particles(self, s: int) -> dict:
        return {k: v.copy() for k, v in self.parts[s].items()}
