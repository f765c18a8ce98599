"""The spatial slab decomposition of one system (paper_2405_07898_gb300/halo.py)
on CPU: its bookkeeping, and two gloo ranks against the single-system serial
FP64 oracle.  Each rank owns a slab along z, receives r_list-wide ghosts,
exchanges F' of the ghosts between the density and force passes and migrates
atoms at list rebuilds; the per-rank density and force passes here are the
oracle's own (the decomposition is host-side bookkeeping and exchanges), so
forces and trajectories must match the undecomposed oracle to FP64 rounding
(the neighbour summation order differs)."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as O
from paper_2405_07898_gb300 import halo, inputs as I
from bars import assert_forces

CELLS = (8, 8, 12)
TEMP = 1500.0
STEPS = 30


class OracleBackend:
    def __init__(self, pot):
        self.pot = O.Potential(pot)

    def density(self, pos, types, box, open_axes):
        return O.density_pass(self.pot, pos, box, types, open_axes)

    def forces(self, pos, types, box, open_axes, Fp):
        return O.force_pass(self.pot, pos, box, types, Fp, open_axes)


def system():
    return I.thermal_system(I.BCC_TA_LIKE, CELLS, 0.02, TEMP, I.SEED_BASE + 880)


def test_slab_bookkeeping():
    s = system()
    p = s.pot
    box = s.box
    dec = halo.SlabDecomposition(box, p.r_list, p.skin, 0, 2)
    assert dec.width == pytest.approx(box[2] / 2)
    z = np.array([[0, 0, 0.0], [0, 0, box[2] / 2 - 1e-9], [0, 0, box[2] / 2], [0, 0, box[2] - 1e-12],
                  [0, 0, -0.1], [0, 0, box[2] + 0.1]])
    assert dec.owner(z).tolist() == [0, 0, 1, 1, 1, 0]
    pos = np.array([[1.0, 1.0, 0.5], [1.0, 1.0, 4.7], [1.0, 1.0, 10.0], [1.0, 1.0, dec.slab.hi - 4.0]])
    down, up = dec.halo_selection(pos)
    assert down.tolist() == [0, 1] and up.tolist() == [3]
    assert dec.ghost_shift(False) == -box[2] and dec.ghost_shift(True) == 0.0
    top = halo.SlabDecomposition(box, p.r_list, p.skin, 1, 2)
    assert top.ghost_shift(True) == box[2] and top.ghost_shift(False) == 0.0
    shift, lbox = dec.local_frame()
    assert shift[2] == pytest.approx(-(p.r_list + 0.5 * p.skin)) and lbox[2] == pytest.approx(dec.width + 2 * p.r_list + p.skin)
    with pytest.raises(ValueError):
        halo.SlabDecomposition(box, p.r_list, p.skin, 0, 5)  # slabs thinner than 2 r_list


def test_one_rank_is_the_oracle():
    s = system()
    md = halo.HaloMD(halo.SlabDecomposition(s.box, s.pot.r_list, s.pot.skin, 0, 1), s.pot.mass,
                     np.arange(s.n), s.pos, s.vel, s.types, OracleBackend(s.pot))
    ref = O.System(O.Potential(s.pot), s.box, s.pos, s.vel, s.types)
    md.step(10, 2.0)
    ref.step(10, 2.0)
    ids, pos, vel, f = md.state()
    st = ref.state()
    d = pos - st["pos"][ids]
    d -= s.box * np.round(d / s.box)
    assert np.abs(d).max() < 1e-9
    assert_forces(f, st["force"][ids], "fp64")


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        s = system()
        dec = halo.SlabDecomposition(s.box, s.pot.r_list, s.pot.skin, rank, world)
        mine = np.flatnonzero(dec.owner(O.wrap(s.pos, s.box)) == rank)
        md = halo.HaloMD(dec, s.pot.mass, mine, s.pos[mine], s.vel[mine], s.types[mine], OracleBackend(s.pot))
        f0 = md.state()
        md.step(STEPS, 2.0)
        out.put((rank, f0, md.state(), md.rebuilds, md.migrated_in))
    finally:
        dist.destroy_process_group()


def test_two_ranks_match_the_single_system_oracle():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    s = system()
    pot = O.Potential(s.pot)
    F0 = O.eam_eval(pot, O.wrap(s.pos, s.box), s.box, s.types)[2]
    ref = O.System(pot, s.box, s.pos, s.vel, s.types)
    ref.step(STEPS, 2.0)
    st = ref.state()
    seen0, seen1 = [], []
    migrated = 0
    for rank, (ids0, _, _, f0), (ids, pos, vel, f), rebuilds, mig in res:
        assert rebuilds == 1 + STEPS // 10
        migrated += mig
        seen0 += ids0.tolist()
        seen1 += ids.tolist()
        assert_forces(f0, F0[ids0], "fp64", f"rank {rank} step 0")
        d = pos - st["pos"][ids]
        d -= s.box * np.round(d / s.box)
        assert np.abs(d).max() < 1e-9, rank
        assert np.abs(vel - st["vel"][ids]).max() < 1e-11, rank
        assert_forces(f, st["force"][ids], "fp64", f"rank {rank} step {STEPS}")
    # every atom owned by exactly one rank, before and after migration
    assert sorted(seen0) == list(range(s.n)) and sorted(seen1) == list(range(s.n))
    assert migrated > 0  # atoms near the slab faces changed owners at rebuilds
