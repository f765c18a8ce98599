"""Spatial decomposition of one periodic system over ranks (one process per
GPU): the multi-device counterpart of the paper's ghost model for many
wafers (Section "Weak Scaling to Many Wafers"), where each node keeps copies
of the atoms near its edge that its neighbours own.

Each rank owns the atoms of a slab along one axis (z by default) and, per
timestep:

  1. kicks and drifts its own atoms (velocity Verlet, FP64);
  2. position halo: sends the current positions of its atoms within r_list of
     each shared face to the rank across it, and receives the same from both
     neighbours -- the ghosts;
  3. density pass over owned + ghost atoms: owned atoms' densities are
     complete (every neighbour within r_cut is owned or a ghost), ghosts' are
     not;
  4. F' halo: sends F'(rho) of the atoms it sent in 2 and sets its ghosts'
     F' from what it receives, so that every F' the force pass reads is its
     owner's;
  5. force pass for its own atoms, closing kick.

The ghost sets are chosen at a list rebuild (every `rebuild_every` steps, or
once an atom anywhere has moved more than skin/2: the largest displacement is
reduced over ranks) with width r_list = r_cut + skin, the Verlet-list
argument: until the next rebuild no pair can close from beyond r_list to
within r_cut.  At a rebuild, atoms whose position left the slab migrate to
the rank that owns their new position (their id, type, position and
velocity), and the ghost sets are chosen again.

The per-rank arithmetic is injected (`backend`: density and force passes
over a local system whose decomposition axis is open), so this module holds
only the bookkeeping and the exchanges.  Messages use torch.distributed
point-to-point sends (gloo between CPU processes; NCCL send/recv between
GPUs, after which the ghosts are ordinary device memory of the receiving
GPU).  Slabs must be at least 2 r_list thick, so ghosts come from the two
adjacent ranks only and no atom is sent to a rank twice.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import inputs as I

_TAG_COUNT, _TAG_DATA = 0, 1


@dataclass
class Slab:
    lo: float
    hi: float
    down: int
    up: int


class SlabDecomposition:
    """Bookkeeping of the slab decomposition along `axis` of a periodic box."""

    def __init__(self, box, r_list: float, skin: float, rank: int, world: int, axis: int = 2):
        self.box = np.asarray(box, dtype=np.float64)
        self.r_list = float(r_list)
        self.skin = float(skin)
        self.rank, self.world, self.axis = int(rank), int(world), int(axis)
        L = self.box[axis]
        self.width = L / world
        if world > 1 and self.width < 2.0 * r_list:
            raise ValueError("slabs must be at least 2 r_list thick")
        self.slab = Slab(rank * self.width, (rank + 1) * self.width, (rank - 1) % world, (rank + 1) % world)

    def owner(self, pos) -> np.ndarray:
        """Rank owning each (global) position: the slab of its periodic image
        along the axis."""
        z = np.mod(np.asarray(pos, dtype=np.float64)[:, self.axis], self.box[self.axis])
        return np.minimum((z / self.width).astype(np.int64), self.world - 1)

    def wrap_into_slab(self, pos) -> np.ndarray:
        """Periodic image of each owned position closest to the slab (the
        image whose axis coordinate lies in [lo - L/2, lo + L/2))."""
        p = np.array(pos, dtype=np.float64, copy=True)
        L = self.box[self.axis]
        c = 0.5 * (self.slab.lo + self.slab.hi)
        p[:, self.axis] -= L * np.round((p[:, self.axis] - c) / L)
        return p

    def halo_selection(self, pos_owned):
        """Indices of owned atoms within r_list of the lower and the upper
        face: the ghosts of the rank below and of the rank above."""
        z = np.asarray(pos_owned, dtype=np.float64)[:, self.axis]
        return np.flatnonzero(z - self.slab.lo < self.r_list), np.flatnonzero(self.slab.hi - z < self.r_list)

    def ghost_shift(self, from_up: bool) -> float:
        """Axis shift that places ghosts received from below (above) just
        under (over) this slab: across the periodic seam for the first and
        the last rank."""
        L = self.box[self.axis]
        if from_up:
            return L if self.rank == self.world - 1 else 0.0
        return -L if self.rank == 0 else 0.0

    def local_frame(self):
        """Origin shift and box of the local system (owned + ghosts): the
        axis open, spanning [lo - r_list - skin/2, hi + r_list + skin/2);
        the other axes periodic as in the global box."""
        pad = self.r_list + 0.5 * self.skin
        box = self.box.copy()
        box[self.axis] = self.width + 2.0 * pad
        shift = np.zeros(3)
        shift[self.axis] = self.slab.lo - pad
        return shift, box


def _exchange(dec: SlabDecomposition, send_down, send_up, dtype):
    """Send one array to each neighbour and receive one from each (sizes
    first).  Returns (from_down, from_up)."""
    import torch
    import torch.distributed as dist

    def t(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype))

    s = dec.slab
    counts_out = [torch.tensor([len(send_down)], dtype=torch.int64), torch.tensor([len(send_up)], dtype=torch.int64)]
    counts_in = [torch.zeros(1, dtype=torch.int64), torch.zeros(1, dtype=torch.int64)]
    # tag = 2 x direction (0: sent down, 1: sent up) + kind: the two messages
    # between the same pair of ranks (two ranks) stay apart
    reqs = [dist.irecv(counts_in[0], s.down, tag=2 * 1 + _TAG_COUNT),   # from below: its "up" message
            dist.irecv(counts_in[1], s.up, tag=2 * 0 + _TAG_COUNT),     # from above: its "down" message
            dist.isend(counts_out[0], s.down, tag=2 * 0 + _TAG_COUNT),
            dist.isend(counts_out[1], s.up, tag=2 * 1 + _TAG_COUNT)]
    for r in reqs:
        r.wait()
    tail = send_down.shape[1:] if np.ndim(send_down) > 1 else ()
    n_down, n_up = int(counts_in[0].item()), int(counts_in[1].item())
    buf_down = torch.zeros((n_down,) + tuple(tail), dtype=t(send_down).dtype)
    buf_up = torch.zeros((n_up,) + tuple(tail), dtype=t(send_up).dtype)
    reqs = []
    if n_down:
        reqs.append(dist.irecv(buf_down, s.down, tag=2 * 1 + _TAG_DATA))
    if n_up:
        reqs.append(dist.irecv(buf_up, s.up, tag=2 * 0 + _TAG_DATA))
    if len(send_down):
        reqs.append(dist.isend(t(send_down), s.down, tag=2 * 0 + _TAG_DATA))
    if len(send_up):
        reqs.append(dist.isend(t(send_up), s.up, tag=2 * 1 + _TAG_DATA))
    for r in reqs:
        r.wait()
    return buf_down.numpy(), buf_up.numpy()


def _max_over_ranks(v: float) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class HaloMD:
    """One rank's part of a slab-decomposed velocity-Verlet run.

    `ids, pos, vel, types`: the atoms this rank owns at the start (global
    ids, global positions).  `backend`: object with
      density(pos, types, box, open_axes) -> (rho, Fp)   every atom
      forces(pos, types, box, open_axes, Fp) -> (n, 3)   every atom
    over a local system (positions in the local frame)."""

    def __init__(self, dec: SlabDecomposition, mass, ids, pos, vel, types, backend, rebuild_every: int = 10):
        self.dec = dec
        self.mass = np.asarray(mass, dtype=np.float64)
        self.ids = np.asarray(ids, dtype=np.int64)
        self.pos = dec.wrap_into_slab(pos)
        self.vel = np.array(vel, dtype=np.float64, copy=True)
        self.types = np.asarray(types, dtype=np.int32)
        self.backend = backend
        self.rebuild_every = int(rebuild_every)
        self.since = 0
        self.rebuilds = 0
        self.migrated_in = 0
        self._rebuild()
        self.force = self._forces()

    # ---- rebuild: migration and ghost selection ----
    def _rebuild(self):
        dec = self.dec
        own = dec.owner(self.pos)
        go_down = np.flatnonzero(own == dec.slab.down) if dec.world > 1 else np.zeros(0, np.int64)
        go_up = np.flatnonzero((own == dec.slab.up) & (own != dec.slab.down)) if dec.world > 1 else np.zeros(0, np.int64)
        if dec.world > 1:
            stray = np.flatnonzero((own != dec.rank) & (own != dec.slab.down) & (own != dec.slab.up))
            if len(stray):
                raise RuntimeError("an atom crossed a whole slab between rebuilds")

            def pack(idx):
                return np.hstack([self.ids[idx, None].astype(np.float64), self.types[idx, None].astype(np.float64),
                                  self.pos[idx], self.vel[idx]]) if len(idx) else np.zeros((0, 8))

            in_down, in_up = _exchange(dec, pack(go_down), pack(go_up), np.float64)
            self.migrated_in += len(in_down) + len(in_up)
            keep = np.setdiff1d(np.arange(len(self.ids)), np.concatenate([go_down, go_up]))
            rows = [np.hstack([self.ids[keep, None].astype(np.float64), self.types[keep, None].astype(np.float64),
                               self.pos[keep], self.vel[keep]]), in_down.reshape(-1, 8), in_up.reshape(-1, 8)]
            allr = np.vstack(rows)
            order = np.argsort(allr[:, 0], kind="stable")
            allr = allr[order]
            self.ids = allr[:, 0].astype(np.int64)
            self.types = allr[:, 1].astype(np.int32)
            self.pos = dec.wrap_into_slab(allr[:, 2:5])
            self.vel = allr[:, 5:8].copy()
            if hasattr(self, "force"):
                del self.force
        self.ref = self.pos.copy()
        self.send_down, self.send_up = dec.halo_selection(self.pos) if dec.world > 1 else (None, None)
        if dec.world > 1:
            tdown = self.types[self.send_down].astype(np.float64)
            tup = self.types[self.send_up].astype(np.float64)
            gt_down, gt_up = _exchange(dec, tdown, tup, np.float64)
            self.ghost_types = np.concatenate([gt_down, gt_up]).astype(np.int32)
            self.n_ghost_down = len(gt_down)
        self.since = 0
        self.rebuilds += 1

    # ---- one evaluation: position halo, density, F' halo, forces ----
    def _forces(self):
        dec = self.dec
        if dec.world == 1:
            w = np.mod(self.pos, dec.box)
            rho, Fp = self.backend.density(w, self.types, dec.box, 0)
            self.Fp = Fp
            return self.backend.forces(w, self.types, dec.box, 0, Fp)
        g_down, g_up = _exchange(dec, self.pos[self.send_down], self.pos[self.send_up], np.float64)
        g_down = g_down.reshape(-1, 3).copy()
        g_up = g_up.reshape(-1, 3).copy()
        g_down[:, dec.axis] += dec.ghost_shift(False)
        g_up[:, dec.axis] += dec.ghost_shift(True)
        shift, lbox = dec.local_frame()
        open_axes = 1 << dec.axis
        local = np.vstack([self.pos, g_down, g_up]) - shift
        # the periodic axes of the local frame: positions wrapped as in the
        # global box
        for a in range(3):
            if a != dec.axis:
                local[:, a] = np.mod(local[:, a], lbox[a])
        types = np.concatenate([self.types, self.ghost_types])
        n = len(self.ids)
        rho, Fp = self.backend.density(local, types, lbox, open_axes)
        # F' halo: the owners' values for every ghost
        f_down, f_up = _exchange(dec, Fp[self.send_down], Fp[self.send_up], np.float64)
        Fp = Fp.copy()
        Fp[n:n + len(f_down)] = f_down
        Fp[n + len(f_down):] = f_up
        self.Fp = Fp[:n]
        return self.backend.forces(local, types, lbox, open_axes, Fp)[:n]

    def step(self, nsteps: int, dt: float):
        acc = I.ACCEL_EV_A_AMU
        half_skin2 = 0.25 * self.dec.skin ** 2
        for _ in range(nsteps):
            m = self.mass[self.types][:, None]
            self.vel += self.force / m * acc * (0.5 * dt)
            self.pos += self.vel * dt
            self.since += 1
            d = self.pos - self.ref
            worst = float((d * d).sum(1).max()) if len(d) else 0.0
            if self.dec.world > 1:
                worst = _max_over_ranks(worst)
            if self.since >= self.rebuild_every or worst > half_skin2:
                self._rebuild()
            self.force = self._forces()
            m = self.mass[self.types][:, None]
            self.vel += self.force / m * acc * (0.5 * dt)

    def state(self):
        """(ids, positions wrapped into the global box, velocities, forces)."""
        return self.ids.copy(), np.mod(self.pos, self.dec.box), self.vel.copy(), self.force.copy()
