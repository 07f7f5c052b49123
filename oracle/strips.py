"""The paper's strip decomposition of the literal-mode step, on the FP64 oracle.

TEST INFRASTRUCTURE ONLY: the tests may import this module; the product
library never does.  It shows, on CPU ranks of ``torch.distributed`` (gloo),
that cutting the box into strips of cell rows (Section 3.1) and exchanging,
every step, the rows the paper exchanges (Section 3.3 steps 1-9) reproduces
the single-domain step:

  * the moment row a strip deposits into above its last cell row (its
    particles' upper corner nodes), sent to the strip above and added there
    (13 values per node: rho, S, dj -- the paper's twelve plus rho);
  * E^{n+1} rows, sent after the E solve (Eq. 4) and overwritten in the
    neighbours' halo rows, before the H update (Eq. 5) needs them;
  * H rows, sent after the H update and overwritten in the halo rows, before
    the node average of B and the next E solve need them;
  * the particles that left the strip in the push (migrants), sent to the
    strip that now holds them.

Each rank keeps its strip's rows [y0, y1) plus HALO rows below and above in
local arrays, runs the oracle's routines on that band (the routines' own
periodic wrap in y only touches halo rows, which the exchanges overwrite),
and holds its particles in global coordinates.  Particles are moved in the
band's coordinates (y - (y0 - HALO) dy), which rounds differently from the
single-domain run by a few ulps, so the comparison is to ~1e-13, not bitwise.
Only the literal field mode; x may be periodic or walled (not decomposed).
"""
from __future__ import annotations

import numpy as np

from . import (NMOM, Grid, curl_e, deposit_raw, field_literal, node_average, normalize, push)

HALO = 2   # halo rows on each side (a particle moves less than HALO - 1 cells a step)


def strip_rows(ny: int, size: int, rank: int):
    """Cell rows [y0, y1) of strip `rank` of `size` (as equal as possible, lower strips first)."""
    base, extra = divmod(ny, size)
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


class StripSim:
    """One rank's strip of an OracleSim-like literal-mode run."""

    def __init__(self, nx, ny, dx, dy, dt, periodic_x, species, laser_params, rank, size, dist):
        self.dist = dist
        self.rank, self.size = rank, size
        self.nx, self.ny, self.dx, self.dy, self.dt = nx, ny, float(dx), float(dy), float(dt)
        self.y0, self.y1 = strip_rows(ny, size, rank)
        self.nown = self.y1 - self.y0
        assert self.nown >= HALO, "every strip needs at least HALO rows"
        self.L = self.nown + 2 * HALO
        self.g = Grid(nx, self.L, dx, dy, periodic_x)
        self.Ly = ny * self.dy
        self.off = (self.y0 - HALO) * self.dy          # global y of the band's row 0
        self.up = (rank + 1) % size
        self.down = (rank - 1) % size
        self.species = [(float(q), float(m)) for (q, m) in species]
        self.laser = tuple(laser_params)
        g = self.g
        self.E = np.zeros((3, self.L, g.nxn))
        self.H = np.zeros((3, self.L, nx))
        self.H_prev = np.zeros((3, self.L, nx))
        self.B = np.zeros((3, self.L, g.nxn))
        self.M_raw = np.zeros((NMOM, self.L, g.nxn))
        self.M = np.zeros((NMOM, self.L, g.nxn))
        self.parts = [{k: np.zeros(0) for k in ("x", "y", "ux", "uy", "uz", "w")} for _ in species]
        self.removed = [0 for _ in species]
        self.step_index = 0

    # ------------------------------------------------------------------ rows and exchange
    def own(self, a):
        """The strip's own rows of a band array (axis 1)."""
        return a[:, HALO:HALO + self.nown]

    def _exchange_rows(self, a, tag):
        """Overwrite the halo rows of band array a (axis 1) with the neighbours' own boundary rows."""
        import torch
        d = self.dist
        send_up = torch.from_numpy(np.ascontiguousarray(a[:, HALO + self.nown - HALO:HALO + self.nown]))
        send_dn = torch.from_numpy(np.ascontiguousarray(a[:, HALO:2 * HALO]))
        recv_dn = torch.empty_like(send_up)      # the lower strip's top rows -> my lower halo
        recv_up = torch.empty_like(send_dn)      # the upper strip's bottom rows -> my upper halo
        reqs = [d.isend(send_up, self.up, tag=2 * tag), d.isend(send_dn, self.down, tag=2 * tag + 1),
                d.irecv(recv_dn, self.down, tag=2 * tag), d.irecv(recv_up, self.up, tag=2 * tag + 1)]
        for r in reqs:
            r.wait()
        a[:, :HALO] = recv_dn.numpy()
        a[:, HALO + self.nown:] = recv_up.numpy()

    def _add_moment_row(self, raw, tag):
        """The node row above the strip (its first upper halo row) holds deposits that belong to the strip
        above: send it there and add the row received from below to the strip's first row."""
        import torch
        d = self.dist
        send = torch.from_numpy(np.ascontiguousarray(raw[:, HALO + self.nown]))
        recv = torch.empty_like(send)
        reqs = [d.isend(send, self.up, tag=2 * tag), d.irecv(recv, self.down, tag=2 * tag)]
        for r in reqs:
            r.wait()
        raw[:, HALO] += recv.numpy()

    def _migrate(self, s, tag):
        """Particles of species s outside the strip's rows go to the strip above or below."""
        import torch
        d = self.dist
        P = self.parts[s]
        row = np.floor(P["y"] / self.dy).astype(np.int64)
        row = np.where(row >= self.ny, row - self.ny, row)
        rel = (row - self.y0) % self.ny                      # rows above y0 (mod ny)
        stay = rel < self.nown
        go_up = ~stay & (rel < self.nown + HALO)
        go_dn = ~stay & ~go_up
        assert np.all(~go_dn | (rel >= self.ny - HALO)), "a particle moved farther than HALO rows"
        keys = ("x", "y", "ux", "uy", "uz", "w")
        out_up = np.stack([P[k][go_up] for k in keys]) if go_up.any() else np.zeros((6, 0))
        out_dn = np.stack([P[k][go_dn] for k in keys]) if go_dn.any() else np.zeros((6, 0))
        n_send = [torch.tensor([out_up.shape[1]], dtype=torch.int64), torch.tensor([out_dn.shape[1]], dtype=torch.int64)]
        n_recv = [torch.zeros(1, dtype=torch.int64), torch.zeros(1, dtype=torch.int64)]
        reqs = [d.isend(n_send[0], self.up, tag=4 * tag), d.isend(n_send[1], self.down, tag=4 * tag + 1),
                d.irecv(n_recv[0], self.down, tag=4 * tag), d.irecv(n_recv[1], self.up, tag=4 * tag + 1)]
        for r in reqs:
            r.wait()
        buf_from_dn = torch.empty((6, int(n_recv[0])), dtype=torch.float64)
        buf_from_up = torch.empty((6, int(n_recv[1])), dtype=torch.float64)
        reqs = []
        if out_up.shape[1]:
            reqs.append(d.isend(torch.from_numpy(np.ascontiguousarray(out_up)), self.up, tag=4 * tag + 2))
        if out_dn.shape[1]:
            reqs.append(d.isend(torch.from_numpy(np.ascontiguousarray(out_dn)), self.down, tag=4 * tag + 3))
        if buf_from_dn.shape[1]:
            reqs.append(d.irecv(buf_from_dn, self.down, tag=4 * tag + 2))
        if buf_from_up.shape[1]:
            reqs.append(d.irecv(buf_from_up, self.up, tag=4 * tag + 3))
        for r in reqs:
            r.wait()
        for k, key in enumerate(keys):
            P[key] = np.concatenate([P[key][stay], buf_from_dn[k].numpy(), buf_from_up[k].numpy()])

    # ------------------------------------------------------------------ state
    def to_band(self, y):
        return np.mod(y - self.off, self.Ly)

    def from_band(self, yb):
        return np.mod(yb + self.off, self.Ly)

    def load_particles(self, s, P):
        """Take, of a species' full particle list, the particles in this strip's rows."""
        row = np.floor(np.asarray(P["y"]) / self.dy).astype(np.int64) % self.ny
        mine = (row >= self.y0) & (row < self.y1)
        for k in self.parts[s]:
            self.parts[s][k] = np.ascontiguousarray(np.asarray(P[k], dtype=np.float64)[mine])

    def deposit(self, tag):
        raw = np.zeros((NMOM, self.L, self.g.nxn))
        for (q, m), P in zip(self.species, self.parts):
            if P["x"].size == 0:
                continue
            Pb = dict(P)
            Pb["y"] = np.ascontiguousarray(self.to_band(P["y"]))
            deposit_raw(self.g, self.dt, q, m, self.B, Pb, raw)
        self._add_moment_row(raw, tag)
        self.M_raw = raw
        self.M = normalize(self.g, raw)

    def step(self, nsteps=1):
        for _ in range(nsteps):
            self._step()

    def _step(self):
        g, dt = self.g, self.dt
        tag = 16 * (self.step_index + 1)
        t_new = (self.step_index + 1) * dt
        # Eq. 4 on the band; the own rows are right (the H halo below is current), then the E rows
        Enew, _ = field_literal(g, dt, t_new, self.laser, self.E, self.H, self.M)
        self._exchange_rows(Enew, tag + 1)
        # Eq. 5 with the exchanged E rows above, then the H rows
        Hnew = self.H - dt * curl_e(g, Enew)
        self._exchange_rows(Hnew, tag + 2)
        Bnew = node_average(g, Hnew)
        Ehalf = 0.5 * (self.E + Enew)
        for s, ((q, m), P) in enumerate(zip(self.species, self.parts)):
            if P["x"].size:
                Pb = {k: v.copy() for k, v in P.items()}
                Pb["y"] = np.ascontiguousarray(self.to_band(P["y"]))
                alive = push(g, dt, q, m, Ehalf, self.B, Pb)
                self.removed[s] += int((~alive).sum())
                Pb["y"] = self.from_band(Pb["y"])
                for k in P:
                    P[k] = np.ascontiguousarray(Pb[k][alive])
            self._migrate(s, tag + 3 + s)
        self.H_prev = self.H
        self.E, self.H, self.B = Enew, Hnew, Bnew
        self.deposit(tag + 12)
        self.step_index += 1

    def set_fields(self, E_global, H_global):
        """Band rows of full-grid fields (y0 - HALO ... y1 + HALO - 1, periodic)."""
        rows = (np.arange(self.L) + self.y0 - HALO) % self.ny
        self.E = np.ascontiguousarray(E_global[:, rows])
        self.H = np.ascontiguousarray(H_global[:, rows])
        self.H_prev = self.H.copy()
        self.B = node_average(self.g, self.H)

    # ------------------------------------------------------------------ diagnostics
    def diagnostics(self):
        """FP64 sums over the strip's own rows and particles, summed over the ranks."""
        import torch
        ke = qw = 0.0
        count = 0
        for (q, m), P in zip(self.species, self.parts):
            u2 = P["ux"] ** 2 + P["uy"] ** 2 + P["uz"] ** 2
            ke += float(np.sum(P["w"] * m * (np.sqrt(1.0 + u2) - 1.0)))
            qw += float(np.sum(q * P["w"]))
            count += P["x"].size
        area = self.g.node_area()[:self.nown]
        Hc = 0.5 * (self.own(self.H) + self.own(self.H_prev))
        fe = 0.5 * float(np.sum(self.own(self.E) ** 2 * area[None])) + 0.5 * float(np.sum(Hc ** 2)) * self.dx * self.dy
        t = torch.tensor([ke, fe, float(np.sum(self.own(self.M_raw)[0])), qw, count, sum(self.removed)],
                         dtype=torch.float64)
        self.dist.all_reduce(t)
        ke, fe, ch, qw, count, removed = t.tolist()
        return dict(kinetic=ke, field=fe, total=ke + fe, charge_grid=ch, charge_particles=qw, count=int(count),
                    removed=int(removed))
