"""The schedules of the density and force passes (lanes per atom, threads per
block, the autotuner's choice) against one another and the serial FP64
oracle.

Lanes per atom change the order in which an atom's pair terms are summed, so
different lane counts agree within the oracle bars (tests/bars.py); threads
per block change only the block partition of the energy sums, so forces and
trajectories are bitwise equal across block sizes.  The tuner's choice is
kept for the process, so two contexts of one shape give bitwise equal
trajectories.
"""
import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import binding, inputs as I
from bars import assert_forces

pytestmark = pytest.mark.gpu


def oracle_eval(system, pos=None):
    pot = O.Potential(system.pot)
    p = system.pos if pos is None else pos
    return O.eam_eval(pot, O.wrap(p, system.box), system.box, system.types)


def random_gas(seed=2405, n=3333, box=(33.0, 29.0, 41.0)):
    """Uniform random positions thinned to a 1.6 A minimum distance: uneven
    cells and uneven neighbour counts."""
    rng = np.random.default_rng(seed)
    box = np.array(box)
    pos = rng.random((n, 3)) * box
    keep = [0]
    for i in range(1, len(pos)):
        d = pos[keep] - pos[i]
        d -= box * np.round(d / box)
        if (d * d).sum(1).min() > 1.6**2:
            keep.append(i)
    pos = pos[keep]
    vel = rng.normal(scale=0.003, size=pos.shape)
    return I.System(box=box, pos=pos, vel=vel, types=np.zeros(len(pos), np.int32),
                    pot=I.johnson_potential(I.BCC_TA_LIKE))


@pytest.fixture(scope="module")
def c1():
    return I.bcc_2000_fp64()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_lanes_per_atom_meet_the_oracle(c1, precision, lanes):
    """Every lane count, graph path, at step 0 and after 37 steps (with list
    rebuilds) at the run's own positions."""
    _, _, F, E, W = oracle_eval(c1)
    with binding.MD(c1, precision=precision, lanes_per_atom=lanes, persistent="off") as md:
        st = md.stats()
        assert st["lanes_density"] == st["lanes_force"] == lanes
        assert_forces(md.forces(), F, precision, f"{lanes} lanes")
        pe, _ = md.energy()
        assert abs(pe - E.sum()) / abs(E.sum()) < (1e-10 if precision == "fp64" else 2e-5)
        md.step(37, 2.0)
        pos, _, _ = md.get_state()
        _, _, F2, _, _ = oracle_eval(c1, pos)
        assert_forces(md.forces(), F2, precision, f"{lanes} lanes, step 37")


def test_uneven_cells_and_ragged_tail():
    """The random gas (uneven neighbour counts; atom count not a multiple of
    any block width) for 1 and 4 lanes per atom, against the oracle after 25
    steps."""
    s = random_gas()
    for precision in ("fp64", "mixed"):
        for lanes in (1, 4):
            with binding.MD(s, precision=precision, lanes_per_atom=lanes, persistent="off") as a:
                assert a.n % (256 // lanes) != 0
                a.step(25, 1.0)
                pos, _, _ = a.get_state()
                _, _, F, _, _ = oracle_eval(s, pos)
                assert_forces(a.forces(), F, precision, f"gas {lanes} lanes")


def test_autotuned_schedule_is_deterministic():
    """Whatever the tuner picks for the 128,000-atom lattice is kept for the
    process: two contexts give bitwise equal trajectories."""
    s = I.bcc_cube(40)
    out = []
    for _ in range(2):
        with binding.MD(s, precision="mixed") as md:
            md.step(20, 2.0)
            out.append((md.get_state()[0], md.stats()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    for k in ("lanes_density", "lanes_force", "threads_density", "threads_force"):
        assert out[0][1][k] == out[1][1][k]


@pytest.mark.parametrize("block", [96, 160, 224])
def test_block_sizes_give_the_same_forces(c1, block):
    """Threads per block change only the block partition of the energy sums:
    forces and trajectories are bitwise those of 256-thread blocks."""
    for precision in ("fp64", "mixed"):
        kw = dict(precision=precision, lanes_per_atom=2, persistent="off")
        with binding.MD(c1, block_size=block, **kw) as a, binding.MD(c1, block_size=256, **kw) as b:
            assert a.stats()["threads_force"] == block
            np.testing.assert_array_equal(a.forces(), b.forces())
            a.step(23, 2.0)
            b.step(23, 2.0)
            np.testing.assert_array_equal(a.get_state()[0], b.get_state()[0])
            ea, eb = sum(a.energy()), sum(b.energy())
            assert abs(ea - eb) / abs(eb) < (1e-13 if precision == "fp64" else 1e-9)


def _offset_allocator(offset=256):
    """Device memory from torch's caching allocator, handed out `offset` bytes
    past a 512-byte boundary: still 256-byte aligned as the C ABI requires,
    but off the texture alignment of the device."""
    import torch
    bases = {}

    def alloc(nbytes):
        try:
            base = torch.cuda.caching_allocator_alloc(nbytes + 512)
        except Exception:
            return None
        p = base + offset
        bases[p] = base
        return p

    def free(p):
        torch.cuda.caching_allocator_delete(bases.pop(p))

    return alloc, free


def test_record_gathers_through_textures_or_loads_give_the_same_results():
    """The density pass gathers neighbour records through texture objects
    where the record buffers allow it, through ordinary loads otherwise:
    the same words either way, so trajectories, forces and energies are
    bitwise equal."""
    s = I.thermal_system(I.BCC_TA_LIKE, (20, 20, 20), 0.02, 600.0, 31)
    kw = dict(precision="mixed", persistent="off", lanes_per_atom=1)
    with binding.MD(s, **kw) as a, binding.MD(s, allocator=_offset_allocator(), **kw) as b:
        assert a.stats()["record_textures"] == 1
        if b.stats()["record_textures"] == 1:
            pytest.skip("this device takes textures on 256-byte aligned buffers")
        for m in (a, b):
            m.step(57, 2.0)
        for x, y in zip(a.get_state(), b.get_state()):
            np.testing.assert_array_equal(np.asarray(x), np.asarray(y))
        np.testing.assert_array_equal(a.forces(), b.forces())
        assert a.energy() == b.energy()
        assert a.stats()["rebuilds"] == b.stats()["rebuilds"] > 0
    with binding.MD(s, precision="fp64", persistent="off") as c:
        assert c.stats()["record_textures"] == 0
