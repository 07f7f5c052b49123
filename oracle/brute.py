"""Dense brute-force cross-check of the oracle on tiny periodic grids.

TEST INFRASTRUCTURE ONLY.  Written separately from ``pic_oracle.c`` and from
the sparse CN assembly: every operator is built as a dense matrix by
enumerating, for each node or cell, its neighbours one by one with explicit
offsets, and the implicit-response matrix R(b) is written out entry by entry
(rather than applied as the vector formula).  Used for the 4x4 comparisons of
the structured oracle (deposit, Eq. 4 per-node solve, the implicit-curl
system).
"""
from __future__ import annotations

import numpy as np


def _node(i, j, nx, ny):
    return (j % ny) * nx + (i % nx)


def dense_curl_e(nx, ny, dx, dy):
    """(3*cells) x (3*nodes) matrix of curl E at cell centres (periodic box)."""
    NN = NC = nx * ny
    C = np.zeros((3 * NC, 3 * NN))
    for j in range(ny):
        for i in range(nx):
            cell = j * nx + i
            for di in (0, 1):
                for dj in (0, 1):
                    nd = _node(i + di, j + dj, nx, ny)
                    sx = (1.0 if di == 1 else -1.0) / (2.0 * dx)   # d/dx weight of this corner
                    sy = (1.0 if dj == 1 else -1.0) / (2.0 * dy)   # d/dy weight of this corner
                    C[0 * NC + cell, 2 * NN + nd] += sy            # (curl E)_x =  dEz/dy
                    C[1 * NC + cell, 2 * NN + nd] += -sx           # (curl E)_y = -dEz/dx
                    C[2 * NC + cell, 1 * NN + nd] += sx            # (curl E)_z =  dEy/dx
                    C[2 * NC + cell, 0 * NN + nd] += -sy           #            -  dEx/dy
    return C


def dense_curl_h(nx, ny, dx, dy):
    """(3*nodes) x (3*cells) matrix of curl H at the nodes (periodic box)."""
    NN = NC = nx * ny
    C = np.zeros((3 * NN, 3 * NC))
    for j in range(ny):
        for i in range(nx):
            nd = j * nx + i
            for ci in (-1, 0):
                for cj in (-1, 0):
                    cell = ((j + cj) % ny) * nx + ((i + ci) % nx)
                    sx = (1.0 if ci == 0 else -1.0) / (2.0 * dx)
                    sy = (1.0 if cj == 0 else -1.0) / (2.0 * dy)
                    C[0 * NN + nd, 2 * NC + cell] += sy
                    C[1 * NN + nd, 2 * NC + cell] += -sx
                    C[2 * NN + nd, 1 * NC + cell] += sx
                    C[2 * NN + nd, 0 * NC + cell] += -sy
    return C


def r_matrix(b):
    """R(b) written out: ((1 + b b^T) + skew part) / (1 + |b|^2), the inverse of (I - [. x b])."""
    bx, by, bz = b
    den = 1.0 + bx * bx + by * by + bz * bz
    return np.array([[1 + bx * bx, bz + bx * by, -by + bx * bz],
                     [-bz + by * bx, 1 + by * by, bx + by * bz],
                     [by + bz * bx, -bx + bz * by, 1 + bz * bz]]) / den


def brute_deposit(nx, ny, dx, dy, dt, q, m, Bn, P):
    """Raw node sums (13, ny, nx) of rho, S (row-major) and dj, with explicit corner loops."""
    M = np.zeros((13, ny, nx))
    for p in range(P["x"].size):
        sx = P["x"][p] / dx
        sy = P["y"][p] / dy
        ci = int(np.floor(sx)); cj = int(np.floor(sy))
        fx = sx - ci; fy = sy - cj
        u = np.array([P["ux"][p], P["uy"][p], P["uz"][p]])
        g = np.sqrt(1.0 + u @ u)
        corners = []
        for di in (0, 1):
            for dj in (0, 1):
                wgt = (fx if di else 1.0 - fx) * (fy if dj else 1.0 - fy)
                corners.append(((ci + di) % nx, (cj + dj) % ny, wgt))
        B = np.zeros(3)
        for (a, bb, wgt) in corners:
            B += wgt * Bn[:, bb, a]
        R = r_matrix(q * dt * B / (2.0 * m * g))
        vals = np.concatenate([[P["w"][p] * q],
                               (P["w"][p] * q * q * dt * dt / (4.0 * m * g) * R).ravel(),
                               P["w"][p] * q * (R @ u) / g])
        for (a, bb, wgt) in corners:
            M[:, bb, a] += wgt * vals
    return M


def brute_literal_E(nx, ny, dx, dy, dt, E, H, M):
    """Eq. 4 as one dense (3 nodes) x (3 nodes) block system: (I + S) E' = (I - S) E + dt (curl H - dj)."""
    NN = nx * ny
    S = np.zeros((3 * NN, 3 * NN))
    for r in range(3):
        for c in range(3):
            S[r * NN:(r + 1) * NN, c * NN:(c + 1) * NN] = np.diag(M[1 + 3 * r + c].ravel())
    I = np.eye(3 * NN)
    rhs = (I - S) @ E.ravel() + dt * (dense_curl_h(nx, ny, dx, dy) @ H.ravel() - M[10:13].ravel())
    return np.linalg.solve(I + S, rhs).reshape(3, ny, nx)


def brute_cn_X(nx, ny, dx, dy, dt, E, H, M):
    """Dense solve of (I + S) X + (dt/2)^2 curl_h curl_e X = E + (dt/2)(curl_h H - dj)."""
    NN = nx * ny
    S = np.zeros((3 * NN, 3 * NN))
    for r in range(3):
        for c in range(3):
            S[r * NN:(r + 1) * NN, c * NN:(c + 1) * NN] = np.diag(M[1 + 3 * r + c].ravel())
    Ch = dense_curl_h(nx, ny, dx, dy)
    Ce = dense_curl_e(nx, ny, dx, dy)
    A = np.eye(3 * NN) + S + (dt / 2.0) ** 2 * (Ch @ Ce)
    rhs = E.ravel() + 0.5 * dt * (Ch @ H.ravel() - M[10:13].ravel())
    return np.linalg.solve(A, rhs).reshape(3, ny, nx)


# ----------------------------------------------------------------------------- boxes with walls in x

def _wnode(i, j, nx, ny):
    """Node (i, j) of a box with walls at x = 0 and x = Lx: nx + 1 node columns, y periodic."""
    assert 0 <= i <= nx
    return (j % ny) * (nx + 1) + i


def dense_curl_e_walls(nx, ny, dx, dy):
    """(3*cells) x (3*nodes): curl E at each cell from its four corners (never wrapped in x)."""
    NN, NC = (nx + 1) * ny, nx * ny
    C = np.zeros((3 * NC, 3 * NN))
    for j in range(ny):
        for i in range(nx):
            cell = j * nx + i
            for di in (0, 1):
                for dj in (0, 1):
                    nd = _wnode(i + di, j + dj, nx, ny)
                    sx = (1.0 if di else -1.0) / (2.0 * dx)
                    sy = (1.0 if dj else -1.0) / (2.0 * dy)
                    C[0 * NC + cell, 2 * NN + nd] += sy
                    C[1 * NC + cell, 2 * NN + nd] += -sx
                    C[2 * NC + cell, 1 * NN + nd] += sx
                    C[2 * NC + cell, 0 * NN + nd] += -sy
    return C


def dense_curl_h_walls(nx, ny, dx, dy):
    """(3*nodes) x (3*cells): curl H at interior nodes from the four cells around them; on a wall column
    only the y-differences of the one cell column inside the box (dHz/dy for x, -dHx/dy for z)."""
    NN, NC = (nx + 1) * ny, nx * ny
    C = np.zeros((3 * NN, 3 * NC))
    for j in range(ny):
        for i in range(nx + 1):
            nd = _wnode(i, j, nx, ny)
            if i == 0 or i == nx:
                col = 0 if i == 0 else nx - 1
                for cj, sgn in ((0, 1.0), (-1, -1.0)):
                    cell = ((j + cj) % ny) * nx + col
                    C[0 * NN + nd, 2 * NC + cell] += sgn / dy
                    C[2 * NN + nd, 0 * NC + cell] += -sgn / dy
                continue
            for ci in (-1, 0):
                for cj in (-1, 0):
                    cell = ((j + cj) % ny) * nx + (i + ci)
                    sx = (1.0 if ci == 0 else -1.0) / (2.0 * dx)
                    sy = (1.0 if cj == 0 else -1.0) / (2.0 * dy)
                    C[0 * NN + nd, 2 * NC + cell] += sy
                    C[1 * NN + nd, 2 * NC + cell] += -sx
                    C[2 * NN + nd, 1 * NC + cell] += sx
                    C[2 * NN + nd, 0 * NC + cell] += -sy
    return C


def brute_cn_walls_X(nx, ny, dx, dy, dt, E, H, M, inc_old, inc_new, pc):
    """Dense solve for X = E^{n+1/2} in a box with walls: interior rows as brute_cn_X (S and dj left out
    on the wall columns); on each wall row j the y and z equations are the time-centred first-order Mur
    condition between the wall node and its neighbour, written out as the two-point difference
    [(X_w + X_v) - (E_w + E_v)]/dt + s (X_w - X_v)/dx = 0 with s = +1 on both walls (outward normal
    derivative), at x = 0 for the scattered field.  inc_old / inc_new: incident field in component pc at
    node columns 0 and 1 (arrays of 2) at t^n and t^{n+1}."""
    NN = (nx + 1) * ny
    E = np.asarray(E); H = np.asarray(H); M = np.asarray(M)
    Ch = dense_curl_h_walls(nx, ny, dx, dy)
    Ce = dense_curl_e_walls(nx, ny, dx, dy)
    A = np.eye(3 * NN) + (dt / 2.0) ** 2 * (Ch @ Ce)
    rhs = E.ravel() + 0.5 * dt * (Ch @ H.ravel())
    for j in range(ny):
        for i in range(1, nx):
            nd = _wnode(i, j, nx, ny)
            for r in range(3):
                rhs[r * NN + nd] -= 0.5 * dt * M[10 + r, j, i]
                for c in range(3):
                    A[r * NN + nd, c * NN + nd] += M[1 + 3 * r + c, j, i]
    for j in range(ny):
        for (w, v) in ((0, 1), (nx, nx - 1)):
            for comp in (1, 2):
                row = comp * NN + _wnode(w, j, nx, ny)
                A[row, :] = 0.0
                A[row, comp * NN + _wnode(w, j, nx, ny)] = 1.0 / dt + 1.0 / dx
                A[row, comp * NN + _wnode(v, j, nx, ny)] = 1.0 / dt - 1.0 / dx
                ew, ev = E[comp, j, w], E[comp, j, v]
                if w == 0 and comp == pc:
                    # scattered field: subtract the incident wave at both times
                    ew_s, ev_s = ew - inc_old[0], ev - inc_old[1]
                    xw_inc = 0.5 * (inc_old[0] + inc_new[0])
                    xv_inc = 0.5 * (inc_old[1] + inc_new[1])
                    rhs[row] = (ew_s + ev_s) / dt + (1.0 / dt + 1.0 / dx) * xw_inc + (1.0 / dt - 1.0 / dx) * xv_inc
                else:
                    rhs[row] = (ew + ev) / dt
    return np.linalg.solve(A, rhs).reshape(3, ny, nx + 1)
