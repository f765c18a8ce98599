"""The row-staged schedule of the density and force passes against the
atom-parallel one and the serial FP64 oracle.

A row-staged block copies the neighbour records of the 3 x 3 rows of cells
around its row into shared memory and gathers from there; the per-atom sums
run in the same order as in the atom-parallel passes with the same lanes per
atom, so forces and trajectories must agree bitwise, and both must meet the
oracle bars (FP64 1e-10, mixed 2e-5, relative 2-norm over all 3N components).
"""
import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import binding, inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 2e-5}


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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_rows_equal_atoms_and_oracle(c1, precision, lanes):
    _, _, F, E, W = oracle_eval(c1)
    kw = dict(precision=precision, lanes_per_atom=lanes)
    with binding.MD(c1, schedule="rows", **kw) as a, binding.MD(c1, schedule="atoms", **kw) as b:
        sa, sb = a.stats(), b.stats()
        assert sa["rows_density"] == sa["rows_force"] == 1 and sa["stage_capacity"] > 0
        assert sb["rows_density"] == sb["rows_force"] == 0
        np.testing.assert_array_equal(a.forces(), b.forces())
        assert rel(a.forces(), F) < TOL[precision]
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
    with binding.MD(c1, schedule="rows", **kw) as c:
        c.set_state(pa, va, 37)
        assert rel(c.forces(), F2) < TOL[precision]


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
            assert rel(a.forces(), F) < TOL[precision]
            a.step(40, 1.0)
            b.step(40, 1.0)
            pa, _, _ = a.get_state()
            pb, _, _ = b.get_state()
            np.testing.assert_array_equal(pa, pb)
            np.testing.assert_array_equal(a.forces(), b.forces())
            _, _, F2, _, _ = oracle_eval(s, pa)
            assert rel(a.forces(), F2) < TOL[precision]


def test_rows_rejections_and_multi_type_fallback():
    s = I.bcc_2000_fp64()
    with pytest.raises(binding.MDError) as e:
        binding.MD(s, schedule="rows", lanes_per_atom=8)
    assert e.value.status == -1
    with pytest.raises(binding.MDError) as e:
        binding.MD(s, schedule="rows", precision="fp64", stage_capacity=1 << 20)
    assert e.value.status == -1
    # two atom types: the type-dependent path has no row-staged form
    m = I.multi_type_system()
    _, _, F, _, _ = oracle_eval(m)
    with binding.MD(m, precision="fp64", schedule="rows", lanes_per_atom=2) as md:
        st = md.stats()
        assert st["rows_density"] == st["rows_force"] == 0
        assert rel(md.forces(), F) < TOL["fp64"]


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
    for k in ("lanes_density", "lanes_force", "rows_density", "rows_force"):
        assert out[0][1][k] == out[1][1][k]
