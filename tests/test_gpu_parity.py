"""Parity of the CUDA path (through the C ABI) with the serial FP64 oracle on
the same seeded inputs.

Bars: cell bins and neighbour lists bit-exact; FP64 forces within 1e-10 and
mixed-precision forces within 2e-5 of the oracle, relative in the 2-norm over
all 3N components, and every atom's force within 1e-9 (FP64) or 1e-4
(mixed) of the RMS atomic force (tests/bars.py); energies and virial within
the norm bars.  Sizes span many thread
blocks with a ragged tail (2,000 atoms = 7 full blocks of 256 + 208).
"""
import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import binding, inputs as I
from bars import assert_forces

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 2e-5


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_eval(system, pos=None):
    pot = O.Potential(system.pot)
    p = system.pos if pos is None else pos
    return O.eam_eval(pot, O.wrap(p, system.box), system.box, system.types)


@pytest.fixture(scope="module")
def c1():
    return I.bcc_2000_fp64()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cells_and_neighbor_list_bit_exact(c1, precision):
    with binding.MD(c1, precision=precision) as md:
        nc, start, atoms = md.cells()
        onc, ostart, oatoms = O.cells(O.wrap(c1.pos, c1.box), c1.box, c1.pot.r_list)
        np.testing.assert_array_equal(nc, onc)
        np.testing.assert_array_equal(start, ostart)
        np.testing.assert_array_equal(atoms, oatoms)
        off, js = md.neighbors()
        ooff, ojs = O.neighbors_cells(O.wrap(c1.pos, c1.box), c1.box, c1.pot.r_list)
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(js, ojs)  # same stencil order, same order in a cell


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cells_on_cell_boundaries_bit_exact(c1, precision):
    """Coordinates on cell boundaries k L/n, one ulp either side of them, at
    -0, just below 0 and just below L: the binning's FP32 estimate must hand
    every case it cannot settle to the FP64 product, so the bins stay those of
    the definition."""
    r_list = c1.pot.r_list
    nc = O.cell_dims(c1.box, r_list)
    pos = O.wrap(c1.pos, c1.box).copy()
    moved = 0
    for a in range(3):
        h = c1.box[a] / nc[a]
        k = np.rint(pos[:, a] / h)
        near = np.abs(pos[:, a] - k * h) < 0.05
        for m, i in enumerate(np.flatnonzero(near)):
            b = k[i] * h
            pos[i, a] = (b, np.nextafter(b, -np.inf), np.nextafter(b, np.inf))[m % 3]
            moved += 1
    i0 = np.argsort(pos[:, 0])[:4]
    pos[i0, 0] = (0.0, -0.0, -1e-300, -5e-324)
    i1 = np.argsort(pos[:, 1])[-2:]
    pos[i1, 1] = (np.nextafter(c1.box[1], 0), c1.box[1])
    assert moved > 100
    s = I.System(box=c1.box, pos=pos, vel=c1.vel, types=c1.types, pot=c1.pot)
    w = O.wrap(s.pos, s.box)
    with binding.MD(s, precision=precision) as md:
        got = md.cells()
        off, js = md.neighbors()
    for g, o in zip(got, O.cells(w, s.box, r_list)):
        np.testing.assert_array_equal(g, o)
    ooff, ojs = O.neighbors_cells(w, s.box, r_list)
    np.testing.assert_array_equal(off, ooff)
    np.testing.assert_array_equal(js, ojs)


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("mixed", MIXED_TOL)])
def test_initial_forces_energy_virial(c1, precision, tol):
    rho, Fp, F, E, W = oracle_eval(c1)
    with binding.MD(c1, precision=precision) as md:
        f = md.forces()
        pe, ke = md.energy()
        w = md.virial()
    assert_forces(f, F, precision)
    assert abs(pe - E.sum()) / abs(E.sum()) < tol
    assert rel(w, W) < tol
    m = c1.pot.mass[c1.types]
    ke_ref = 0.5 * (m[:, None] * c1.vel**2).sum() / I.ACCEL_EV_A_AMU
    assert abs(ke - ke_ref) / ke_ref < 1e-12


def test_random_gas_lists_and_forces_fp64():
    """Non-lattice input: uniform random positions (close pairs, uneven cells,
    atoms near cell and box faces), 3,333 atoms."""
    rng = np.random.default_rng(2405)
    box = np.array([33.0, 29.0, 41.0])
    pos = rng.random((3333, 3)) * box
    # keep pairs at least 1.6 A apart so the tables stay well inside their range
    keep = [0]
    for i in range(1, len(pos)):
        d = pos[keep] - pos[i]
        d -= box * np.round(d / box)
        if (d * d).sum(1).min() > 1.6**2:
            keep.append(i)
    pos = pos[keep]
    s = I.System(box=box, pos=pos, vel=np.zeros_like(pos), types=np.zeros(len(pos), np.int32),
                 pot=I.johnson_potential(I.BCC_TA_LIKE))
    with binding.MD(s, precision="fp64") as md:
        off, js = md.neighbors()
        ooff, ojs = O.neighbors_brute(pos, box, s.pot.r_list)
        np.testing.assert_array_equal(off, ooff)
        for i in range(0, len(pos), 7):
            assert sorted(js[off[i]:off[i + 1]]) == list(ojs[ooff[i]:ooff[i + 1]])
        _, _, F, E, W = oracle_eval(s)
        assert_forces(md.forces(), F, "fp64")
        pe, _ = md.energy()
        assert abs(pe - E.sum()) / abs(E.sum()) < FP64_TOL


def test_two_types_fp64_and_mixed():
    s = I.multi_type_system(cells=(8, 8, 8), n_knots=600)
    _, _, F, E, W = oracle_eval(s)
    for precision, tol in (("fp64", FP64_TOL), ("mixed", MIXED_TOL)):
        with binding.MD(s, precision=precision) as md:
            assert_forces(md.forces(), F, precision)
            pe, _ = md.energy()
            assert abs(pe - E.sum()) / abs(E.sum()) < tol
            assert rel(md.virial(), W) < tol


LAUNCH = {"graphs": dict(use_graphs=True, persistent="off"), "eager": dict(use_graphs=False, persistent="off"),
          "single_launch": dict(persistent="on")}


@pytest.mark.parametrize("launch", ["graphs", "eager", "single_launch"])
def test_trajectory_fp64_matches_oracle(c1, launch):
    """100 velocity-Verlet steps at dt = 2 fs, compared every 10 steps; the
    forces are also re-checked at the GPU's own positions (same input)."""
    pot = O.Potential(c1.pot)
    ref = O.System(pot, c1.box, c1.pos, c1.vel, c1.types)
    with binding.MD(c1, precision="fp64", **LAUNCH[launch]) as md:
        for block in range(10):
            md.step(10, 2.0)
            ref.step(10, 2.0)
            pos, vel, step = md.get_state()
            st = ref.state()
            assert step == st["step"] == 10 * (block + 1)
            d = pos - st["pos"]
            d -= c1.box * np.round(d / c1.box)
            assert np.abs(d).max() < 1e-9
            assert np.abs(vel - st["vel"]).max() < 1e-11
            pe, ke = md.energy()
            ope, oke = ref.energy()
            assert abs(pe - ope) / abs(ope) < 1e-11 and abs(ke - oke) / oke < 1e-9
            _, _, F, _, _ = oracle_eval(c1, pos)
            assert_forces(md.forces(), F, "fp64")
        assert md.stats()["rebuilds"] == ref.state()["rebuilds"] == 10


def test_mixed_trajectory_tracks_fp64(c1):
    with binding.MD(c1, precision="mixed") as a, binding.MD(c1, precision="fp64") as b:
        a.step(100, 2.0)
        b.step(100, 2.0)
        pa, va, _ = a.get_state()
        pb, vb, _ = b.get_state()
        d = pa - pb
        d -= c1.box * np.round(d / c1.box)
        assert np.abs(d).max() < 1e-5
        ea, eb = sum(a.energy()), sum(b.energy())
        assert abs(ea - eb) / abs(eb) < 1e-6
        # forces at the mixed run's own positions against the oracle
        _, _, F, _, _ = oracle_eval(c1, pa)
        assert_forces(a.forces(), F, "mixed")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graphs_equal_eager_and_runs_are_deterministic(c1, precision):
    out = []
    for use_graphs in (True, False, True):
        with binding.MD(c1, precision=precision, use_graphs=use_graphs, persistent="off") as md:
            md.step(37, 2.0)
            pos, vel, _ = md.get_state()
            out.append((pos, vel, md.energy(), md.forces()))
    for other in out[1:]:
        np.testing.assert_array_equal(out[0][0], other[0])
        np.testing.assert_array_equal(out[0][1], other[1])
        assert out[0][2] == other[2]
        np.testing.assert_array_equal(out[0][3], other[3])


def test_set_state_roundtrip_and_resume(c1):
    """n steps == k steps, save, restore into a fresh context, n - k steps."""
    with binding.MD(c1, precision="fp64") as a:
        a.step(30, 2.0)
        pos, vel, step = a.get_state()
        a.step(20, 2.0)
        ref_pos, ref_vel, _ = a.get_state()
    with binding.MD(c1, precision="fp64") as b:
        b.set_state(pos, vel, step)
        _, _, st = b.get_state()
        assert st == 30
        b.step(20, 2.0)
        p2, v2, st2 = b.get_state()
    assert st2 == 50
    d = p2 - ref_pos
    d -= c1.box * np.round(d / c1.box)
    assert np.abs(d).max() < 1e-12
    assert np.abs(v2 - ref_vel).max() < 1e-13


def test_set_state_rejects_non_finite_and_recovers(c1):
    """Non-finite positions or velocities are caught on the device while the
    state loads (MD_ERR_NONFINITE); the next valid md_set_state recovers."""
    with binding.MD(c1, precision="mixed") as md:
        pos, vel, step = md.get_state()
        bad = pos.copy()
        bad[7, 2] = np.nan
        with pytest.raises(binding.MDError) as e:
            md.set_state(bad, vel, step)
        assert e.value.status == -5
        badv = vel.copy()
        badv[3, 0] = np.inf
        with pytest.raises(binding.MDError) as e:
            md.set_state(pos, badv, step)
        assert e.value.status == -5
        md.set_state(pos, vel, step)
        md.step(10, 2.0)
        p2, _, _ = md.get_state()
        _, _, F, _, _ = oracle_eval(c1, p2)
        assert_forces(md.forces(), F, "mixed")


def test_displacement_triggers_rebuild():
    """At high temperature atoms cross skin/2 before 10 steps: the list is
    rebuilt on the device as in the oracle, and forces stay exact."""
    s = I.thermal_system(I.BCC_TA_LIKE, (10, 10, 10), 0.02, 3000.0, 99)
    pot = O.Potential(s.pot)
    ref = O.System(pot, s.box, s.pos, s.vel, s.types)
    with binding.MD(s, precision="fp64", rebuild_every=1000, persistent="off") as md:
        md.step(60, 4.0)
        ref.step(60, 4.0, rebuild_every=1000)
        assert md.stats()["rebuilds"] == ref.state()["rebuilds"] > 0
        pos, _, _ = md.get_state()
        _, _, F, _, _ = oracle_eval(s, pos)
        assert_forces(md.forces(), F, "fp64")


def test_edge_cases():
    s = I.bcc_2000_fp64()
    # empty system
    empty = I.System(box=s.box, pos=np.zeros((0, 3)), vel=np.zeros((0, 3)),
                     types=np.zeros(0, np.int32), pot=s.pot)
    with binding.MD(empty) as md:
        md.step(5, 2.0)
        assert md.energy() == (0.0, 0.0)
        assert md.get_state()[2] == 5
    # one atom: no neighbours, no force, energy F(0)
    one = I.System(box=s.box, pos=np.array([[1.0, 2.0, 3.0]]), vel=np.zeros((1, 3)),
                   types=np.zeros(1, np.int32), pot=s.pot)
    with binding.MD(one, precision="fp64") as md:
        md.step(3, 2.0)
        np.testing.assert_array_equal(md.forces(), np.zeros((1, 3)))
        off, js = md.neighbors()
        assert off.tolist() == [0, 0] and len(js) == 0
        pe, _ = md.energy()
        assert abs(pe - I.johnson_F(I.BCC_TA_LIKE, 0.0)) < 1e-12
    # smallest legal box (3 cells per axis) and a list that must overflow
    small = I.thermal_system(I.BCC_TA_LIKE, (5, 5, 5), 0.02, 300.0, 5)
    _, _, F, _, _ = oracle_eval(small)
    with binding.MD(small, precision="fp64") as md:
        assert_forces(md.forces(), F, "fp64")
    with pytest.raises(binding.MDError) as e:
        binding.MD(small, precision="mixed", list_capacity=8)
    assert e.value.status == -7


def test_list_overflow_during_a_run_is_reported_and_recovered():
    """A list capacity equal to the initial longest list and a hot lattice
    rebuilt every step: a later build finds an atom with more neighbours, the
    run reports MD_ERR_LIST_OVERFLOW at its next synchronising call (a sticky
    device flag; the entries past the capacity are dropped, never written
    out of bounds), and md_set_state of a state that fits restores a context
    whose forces meet the oracle."""
    hot = I.thermal_system(I.BCC_TA_LIKE, (6, 6, 6), 0.01, 3000.0, 17)
    with binding.MD(hot, precision="mixed", persistent="off") as probe:
        cap0 = probe.stats()["max_neighbors"]
    with binding.MD(hot, precision="mixed", persistent="off", list_capacity=cap0, rebuild_every=1) as md:
        assert md.stats()["list_capacity"] == cap0
        with pytest.raises(binding.MDError) as e:
            for _ in range(100):
                md.step(5, 2.0)
                md.energy()
        assert e.value.status == -7
        md.set_state(hot.pos, hot.vel, 0)
        _, _, F, _, _ = oracle_eval(hot)
        assert_forces(md.forces(), F, "mixed", "after recovery")


def test_full_size_800k_mixed_forces():
    """799,496 atoms in the configuration the benchmark times: all forces
    against the oracle (which finishes this O(N) evaluation in seconds)."""
    s = I.bcc_799496()
    _, _, F, E, W = oracle_eval(s)
    with binding.MD(s, precision="mixed") as md:
        assert_forces(md.forces(), F, "mixed")
        pe, _ = md.energy()
        assert abs(pe - E.sum()) / abs(E.sum()) < MIXED_TOL
        assert rel(md.virial(), W) < MIXED_TOL
        md.step(10, 2.0)
        pos, _, _ = md.get_state()
    _, _, F2, _, _ = oracle_eval(s, pos)
    with binding.MD(I.System(s.box, pos, s.vel, s.types, s.pot), precision="mixed") as md2:
        assert_forces(md2.forces(), F2, "mixed")


@pytest.mark.parametrize("every", [1, 10, 1000])
def test_profile_counts_the_list_builds(every):
    """md_profile's per-kernel timing counts a step's rebuild span as a build
    exactly when the device built a list in that step (its own counter), so
    the average build time is over real builds: rebuild every step, every 10
    steps, and (with dt = 0) never."""
    s = I.thermal_system(I.BCC_TA_LIKE, (20, 20, 20), 0.02, 300.0, 23)
    dt = 0.0 if every == 1000 else 2.0
    with binding.MD(s, precision="mixed", persistent="off", rebuild_every=every) as md:
        before = md.stats()["rebuilds"]
        prof = md.profile(20, dt)
        built = md.stats()["rebuilds"] - before
        assert prof["rebuilds"] == built == {1: 20, 10: 2, 1000: 0}[every]
        if built:
            assert prof["rebuild_ms"] > 0.0
        else:
            assert prof["rebuild_ms"] == 0.0
        assert prof["density_ms"] > 0.0 and prof["force_ms"] > 0.0
