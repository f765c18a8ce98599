"""The row-staged and list-tiled schedules of the density and force passes
against the atom-parallel one and the serial FP64 oracle.

A row-staged block copies the neighbour records of the 3 x 3 rows of cells
around its row into shared memory and gathers from there; a list-tiled block
bulk-copies its atoms' list columns into shared memory first.  The per-atom
sums run in the same order as in the atom-parallel passes with the same lanes
per atom, so forces and trajectories must agree bitwise, and all must meet
the oracle bars (FP64 1e-10, mixed 2e-5, relative 2-norm over all 3N
components).
"""
import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import binding, inputs as I
from bars import assert_forces

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 2e-5}
FLAGS = ("rows_density", "rows_force", "tiles_density", "tiles_force", "table_density", "table_force")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_eval(system, pos=None):
    pot = O.Potential(system.pot)
    p = system.pos if pos is None else pos
    return O.eam_eval(pot, O.wrap(p, system.box), system.box, system.types)


def row_block_sums(ncell, start):
    """Records a row-staged block of each row (cy, cz) would stage."""
    nx, ny, nz = (int(v) for v in ncell)
    rows = np.array([start[(r + 1) * nx] - start[r * nx] for r in range(ny * nz)]).reshape(nz, ny)
    out = np.zeros_like(rows)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            out += np.roll(np.roll(rows, -dz, axis=0), -dy, axis=1)
    return out.ravel()


def random_gas(seed=2405, n=3333, box=(33.0, 29.0, 41.0)):
    """Uniform random positions thinned to a 1.6 A minimum distance: uneven
    cells, so rows differ in how many records they stage."""
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


@pytest.mark.parametrize("schedule", ["rows", "tiles", "table"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_schedule_equals_atoms_and_oracle(c1, schedule, precision, lanes):
    _, _, F, E, W = oracle_eval(c1)
    kw = dict(precision=precision, lanes_per_atom=lanes)
    with binding.MD(c1, schedule=schedule, **kw) as a, binding.MD(c1, schedule="atoms", **kw) as b:
        sa, sb = a.stats(), b.stats()
        if schedule == "rows":
            assert sa["rows_density"] == sa["rows_force"] == 1 and sa["stage_capacity"] > 0
        elif schedule == "tiles":
            assert sa["tiles_density"] == sa["tiles_force"] == 1
        else:  # FP32 only; the FP64 path falls back to the atom-parallel passes
            assert sa["table_density"] == sa["table_force"] == (1 if precision == "mixed" else 0)
        for k in FLAGS:
            assert sb[k] == 0
        np.testing.assert_array_equal(a.forces(), b.forces())
        assert_forces(a.forces(), F, precision)
        pe, _ = a.energy()
        assert abs(pe - E.sum()) / abs(E.sum()) < TOL[precision]
        assert rel(a.virial(), W) < TOL[precision]
        a.step(37, 2.0)
        b.step(37, 2.0)
        pa, va, _ = a.get_state()
        pb, vb, _ = b.get_state()
        np.testing.assert_array_equal(pa, pb)
        np.testing.assert_array_equal(va, vb)
        np.testing.assert_array_equal(a.forces(), b.forces())
        assert a.stats()["rebuilds"] == b.stats()["rebuilds"]
        # energy sums: same terms, other block partition (FP32 pair sums in
        # the mixed path, compensated)
        ea, eb = sum(a.energy()), sum(b.energy())
        assert abs(ea - eb) / abs(eb) < (1e-13 if precision == "fp64" else 1e-9)
    _, _, F2, _, _ = oracle_eval(c1, pa)
    with binding.MD(c1, schedule=schedule, **kw) as c:
        c.set_state(pa, va, 37)
        assert_forces(c.forces(), F2, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rows_with_blocks_past_the_stage(precision):
    """A stage smaller than some rows' neighbourhoods: those blocks gather
    from device memory, the others from shared memory; forces are the same
    either way and meet the oracle bar, before and after 40 steps."""
    s = random_gas()
    with binding.MD(s, precision=precision, schedule="atoms", lanes_per_atom=2) as b:
        ncell, start, _ = b.cells()
        sums = np.sort(row_block_sums(ncell, start))
        cap = int(sums[len(sums) // 2])
        assert sums[0] <= cap < sums[-1]
        with binding.MD(s, precision=precision, schedule="rows", lanes_per_atom=2,
                        stage_capacity=cap) as a:
            assert a.stats()["stage_capacity"] == cap
            _, _, F, _, _ = oracle_eval(s)
            np.testing.assert_array_equal(a.forces(), b.forces())
            assert_forces(a.forces(), F, precision)
            a.step(40, 1.0)
            b.step(40, 1.0)
            pa, _, _ = a.get_state()
            pb, _, _ = b.get_state()
            np.testing.assert_array_equal(pa, pb)
            np.testing.assert_array_equal(a.forces(), b.forces())
            _, _, F2, _, _ = oracle_eval(s, pa)
            assert_forces(a.forces(), F2, precision)


@pytest.mark.parametrize("schedule", ["tiles", "table"])
def test_uneven_cells_and_ragged_tail(schedule):
    """List tiles and shared-table passes on the random gas (uneven neighbour
    counts; the last tile holds a ragged tail of atoms): bitwise equal to the
    atom-parallel passes."""
    s = random_gas()
    for precision in ("fp64", "mixed"):
        for lanes in (1, 4):
            kw = dict(precision=precision, lanes_per_atom=lanes)
            with binding.MD(s, schedule=schedule, **kw) as a, binding.MD(s, schedule="atoms", **kw) as b:
                assert a.n % (256 // lanes) != 0
                np.testing.assert_array_equal(a.forces(), b.forces())
                a.step(25, 1.0)
                b.step(25, 1.0)
                np.testing.assert_array_equal(a.get_state()[0], b.get_state()[0])
                np.testing.assert_array_equal(a.forces(), b.forces())


def test_rows_rejections_and_multi_type_fallback():
    s = I.bcc_2000_fp64()
    for sched in ("rows", "tiles", "table"):
        with pytest.raises(binding.MDError) as e:
            binding.MD(s, schedule=sched, lanes_per_atom=8)
        assert e.value.status == -1
    with pytest.raises(binding.MDError) as e:
        binding.MD(s, schedule="rows", precision="fp64", stage_capacity=1 << 20)
    assert e.value.status == -1
    # two atom types: the type-dependent path has no row-staged form
    m = I.multi_type_system()
    _, _, F, _, _ = oracle_eval(m)
    for sched in ("rows", "tiles", "table"):
        for precision in ("fp64", "mixed"):
            with binding.MD(m, precision=precision, schedule=sched, lanes_per_atom=2) as md:
                st = md.stats()
                for k in FLAGS:
                    assert st[k] == 0
                assert_forces(md.forces(), F, precision)


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
    for k in ("lanes_density", "lanes_force", "threads_density", "threads_force") + FLAGS:
        assert out[0][1][k] == out[1][1][k]


@pytest.mark.parametrize("block", [96, 160, 224])
def test_block_sizes_give_the_same_forces(c1, block):
    """Threads per block change only the block partition of the energy sums:
    forces and trajectories are bitwise those of 256-thread blocks."""
    for precision in ("fp64", "mixed"):
        kw = dict(precision=precision, lanes_per_atom=2, schedule="atoms")
        with binding.MD(c1, block_size=block, **kw) as a, binding.MD(c1, block_size=256, **kw) as b:
            assert a.stats()["threads_force"] == block
            np.testing.assert_array_equal(a.forces(), b.forces())
            a.step(23, 2.0)
            b.step(23, 2.0)
            np.testing.assert_array_equal(a.get_state()[0], b.get_state()[0])
            ea, eb = sum(a.energy()), sum(b.energy())
            assert abs(ea - eb) / abs(eb) < (1e-13 if precision == "fp64" else 1e-9)
