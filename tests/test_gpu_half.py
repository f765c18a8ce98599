"""The force-symmetry form (half lists) against the serial FP64 oracle.

Each pair is listed once (by the atom that sees the other in the upper half
space, decided exactly) and evaluated once;
the other atom's density and force terms reach it through fixed-point
accumulators.  The summation order differs from the full-list passes, so the
results are held to the oracle bars (tests/bars.py), not to bitwise equality
with the full-list form; the exported lists are still every atom's full list
in the oracle's order, bit for bit; runs are bitwise reproducible.
"""
import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import binding, inputs as I
from bars import assert_forces

pytestmark = pytest.mark.gpu

MIXED_TOL = 2e-5


def oracle_eval(system, pos=None, open_axes=0):
    pot = O.Potential(system.pot)
    p = system.pos if pos is None else pos
    return O.eam_eval(pot, O.wrap(p, system.box, open_axes), system.box, system.types, open_axes=open_axes)


@pytest.fixture(scope="module")
def c1():
    return I.bcc_2000_fp64()


def test_initial_forces_energy_virial_and_full_list_export(c1):
    _, _, F, E, W = oracle_eval(c1)
    with binding.MD(c1, precision="mixed", half_list=True) as md:
        st = md.stats()
        assert st["half_list"] == 1 and st["lanes_force"] == 1 and st["persistent_blocks"] == 0
        # 26 neighbours, each pair once, the upper half space of each atom's
        # nearly symmetric neighbourhood: about 13 for every atom (a few more
        # where thermal motion moves third-shell pairs across r_list)
        assert 13 <= st["max_neighbors"] <= 20
        assert_forces(md.forces(), F, "mixed")
        pe, _ = md.energy()
        assert abs(pe - E.sum()) / abs(E.sum()) < MIXED_TOL
        w = md.virial()
        assert np.linalg.norm(w - W) / np.linalg.norm(W) < MIXED_TOL
        off, js = md.neighbors()
        ooff, ojs = O.neighbors_cells(O.wrap(c1.pos, c1.box), c1.box, c1.pot.r_list)
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(js, ojs)


def test_trajectory_tracks_the_full_list_form_and_meets_the_oracle(c1):
    """100 steps (10 list builds): positions within 1e-5 A of the full-list
    mixed run, forces at the run's own positions against the oracle, total
    energy conserved to the full-list run's level."""
    with binding.MD(c1, precision="mixed", half_list=True) as a, \
            binding.MD(c1, precision="mixed", persistent="off") as b:
        e0 = sum(a.energy())
        a.step(100, 2.0)
        b.step(100, 2.0)
        pa, _, sa = a.get_state()
        pb, _, _ = b.get_state()
        assert sa == 100 and a.stats()["rebuilds"] == 10
        d = pa - pb
        d -= c1.box * np.round(d / c1.box)
        assert np.abs(d).max() < 1e-5
        ea, eb = sum(a.energy()), sum(b.energy())
        assert abs(ea - eb) / abs(eb) < 1e-6
        assert abs(ea - e0) / c1.n < 1e-4
        _, _, F, _, _ = oracle_eval(c1, pa)
        assert_forces(a.forces(), F, "mixed")


def test_runs_are_bitwise_reproducible(c1):
    out = []
    for use_graphs in (True, False, True):
        with binding.MD(c1, precision="mixed", half_list=True, use_graphs=use_graphs) as md:
            md.step(37, 2.0)
            pos, vel, _ = md.get_state()
            out.append((pos, vel, md.energy(), md.forces(), md.virial()))
    for other in out[1:]:
        for x, y in zip(out[0], other):
            np.testing.assert_array_equal(np.asarray(x), np.asarray(y))


def test_uneven_lists_open_slab_and_displacement_rebuilds():
    """A random gas (uneven list lengths, ragged tail), a slab open on every
    axis, and a hot lattice whose builds are triggered by displacement."""
    rng = np.random.default_rng(77)
    box = np.array([31.0, 28.0, 36.0])
    pos = rng.random((3000, 3)) * box
    keep = [0]
    for i in range(1, len(pos)):
        d = pos[keep] - pos[i]
        d -= box * np.round(d / box)
        if (d * d).sum(1).min() > 1.6**2:
            keep.append(i)
    gas = I.System(box=box, pos=pos[keep], vel=np.zeros((len(keep), 3)), types=np.zeros(len(keep), np.int32),
                   pot=I.johnson_potential(I.BCC_TA_LIKE))
    _, _, F, _, _ = oracle_eval(gas)
    with binding.MD(gas, precision="mixed", half_list=True) as md:
        assert_forces(md.forces(), F, "mixed", "gas")
        off, js = md.neighbors()
        ooff, ojs = O.neighbors_cells(O.wrap(gas.pos, gas.box), gas.box, gas.pot.r_list)
        np.testing.assert_array_equal(js, ojs)
    slab = I.bcc_slab_small(7)
    _, _, F, E, _ = oracle_eval(slab, open_axes=7)
    with binding.MD(slab, precision="mixed", half_list=True) as md:
        assert_forces(md.forces(), F, "mixed", "slab")
        md.step(30, 2.0)
        p, _, _ = md.get_state()
    _, _, F2, _, _ = oracle_eval(slab, p, open_axes=7)
    with binding.MD(I.System(slab.box, p, slab.vel, slab.types, slab.pot, open_axes=7), precision="mixed",
                    half_list=True) as md:
        assert_forces(md.forces(), F2, "mixed", "slab after 30 steps")
    hot = I.thermal_system(I.BCC_TA_LIKE, (10, 10, 10), 0.02, 3000.0, 99)
    with binding.MD(hot, precision="mixed", half_list=True, rebuild_every=1000) as md:
        md.step(60, 4.0)
        assert md.stats()["rebuilds"] > 0
        p, _, _ = md.get_state()
        _, _, F, _, _ = oracle_eval(hot, p)
        assert_forces(md.forces(), F, "mixed", "hot")


def test_full_size_800k_forces():
    """The 799,496-atom benchmark system in the half-list form: all forces
    against the oracle at step 0 and after 10 steps (one list build)."""
    s = I.bcc_799496()
    _, _, F, E, W = oracle_eval(s)
    with binding.MD(s, precision="mixed", half_list=True) as md:
        assert_forces(md.forces(), F, "mixed", "800k step 0")
        pe, _ = md.energy()
        assert abs(pe - E.sum()) / abs(E.sum()) < MIXED_TOL
        md.step(10, 2.0)
        pos, _, _ = md.get_state()
        f10 = md.forces()
    _, _, F10, _, _ = oracle_eval(s, pos)
    assert_forces(f10, F10, "mixed", "800k step 10")


def test_rejections():
    s = I.bcc_2000_fp64()
    for kw in (dict(precision="fp64"), dict(persistent="on"), dict(lanes_per_atom=4)):
        with pytest.raises(binding.MDError) as e:
            binding.MD(s, half_list=True, **kw)
        assert e.value.status == -1, kw
    with pytest.raises(binding.MDError) as e:
        binding.MD(I.multi_type_system(), precision="mixed", half_list=True)
    assert e.value.status == -1
