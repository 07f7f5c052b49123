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
