"""md_step as one cooperative launch (all phases of all steps, blocks meeting
at grid barriers) against the graph path and the serial FP64 oracle.

The single launch runs the same per-atom device code with the same lanes per
atom, so positions, velocities and forces must equal the graph path's bitwise
over trajectories that include list rebuilds (scheduled and triggered by
displacement); energy sums come from another block partition and agree to
rounding.
"""
import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import binding, inputs as I
from bars import assert_forces

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 2e-5}
ETOL = {"fp64": 1e-13, "mixed": 1e-9}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_forces(system, pos):
    pot = O.Potential(system.pot)
    return O.eam_eval(pot, O.wrap(pos, system.box), system.box, system.types)[2]


def run_pair(system, precision, lanes, calls, dt, **kw):
    """The same md_step calls on a single-launch and a graph context."""
    out = []
    for persistent in ("on", "off"):
        with binding.MD(system, precision=precision, lanes_per_atom=lanes, persistent=persistent, **kw) as md:
            st = md.stats()
            assert (st["persistent_blocks"] > 0) == (persistent == "on")
            if persistent == "on":
                assert st["persistent_lanes"] == lanes
            for nsteps in calls:
                md.step(nsteps, dt)
            pos, vel, step = md.get_state()
            out.append(dict(pos=pos, vel=vel, step=step, forces=md.forces(), energy=md.energy(),
                            virial=md.virial(), stats=md.stats()))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("lanes", [1, 2, 8])
def test_single_launch_equals_graphs(precision, lanes):
    s = I.bcc_2000_fp64()
    a, b = run_pair(s, precision, lanes, [37, 1, 12], 2.0)
    np.testing.assert_array_equal(a["pos"], b["pos"])
    np.testing.assert_array_equal(a["vel"], b["vel"])
    np.testing.assert_array_equal(a["forces"], b["forces"])
    assert a["step"] == b["step"] == 50
    assert a["stats"]["rebuilds"] == b["stats"]["rebuilds"] >= 4
    for x, y in zip(a["energy"], b["energy"]):
        assert abs(x - y) <= ETOL[precision] * abs(y)
    np.testing.assert_allclose(a["virial"], b["virial"], rtol=ETOL[precision] * 100, atol=1e-12)
    assert_forces(a["forces"], oracle_forces(s, a["pos"]), precision)


def test_single_launch_displacement_rebuilds():
    """Hot system, rebuild_every 1000: every build is triggered by an atom
    moving more than skin/2, decided inside the launch."""
    s = I.thermal_system(I.BCC_TA_LIKE, (10, 10, 10), 0.02, 3000.0, 99)
    a, b = run_pair(s, "fp64", 2, [60], 4.0, rebuild_every=1000)
    np.testing.assert_array_equal(a["pos"], b["pos"])
    assert a["stats"]["rebuilds"] == b["stats"]["rebuilds"] > 0
    ref = O.System(O.Potential(s.pot), s.box, s.pos, s.vel, s.types)
    ref.step(60, 4.0, rebuild_every=1000)
    assert a["stats"]["rebuilds"] == ref.state()["rebuilds"]
    d = a["pos"] - ref.state()["pos"]
    d -= s.box * np.round(d / s.box)
    assert np.abs(d).max() < 1e-9


def test_single_launch_two_types_and_uneven_cells():
    m = I.multi_type_system()
    a, b = run_pair(m, "mixed", 4, [25], 2.0)
    np.testing.assert_array_equal(a["pos"], b["pos"])
    np.testing.assert_array_equal(a["forces"], b["forces"])
    rng = np.random.default_rng(11)
    box = np.array([31.0, 27.0, 35.0])
    pos = rng.random((2600, 3)) * box
    keep = [0]
    for i in range(1, len(pos)):
        d = pos[keep] - pos[i]
        d -= box * np.round(d / box)
        if (d * d).sum(1).min() > 1.7**2:
            keep.append(i)
    pos = pos[keep]
    gas = I.System(box=box, pos=pos, vel=rng.normal(scale=0.004, size=pos.shape),
                   types=np.zeros(len(pos), np.int32), pot=I.johnson_potential(I.BCC_TA_LIKE))
    a, b = run_pair(gas, "fp64", 1, [30], 1.0)
    np.testing.assert_array_equal(a["pos"], b["pos"])
    assert_forces(a["forces"], oracle_forces(gas, a["pos"]), "fp64")


def test_single_launch_after_set_state_and_auto_threshold():
    s = I.bcc_2000_fp64()
    with binding.MD(s, precision="fp64") as md:  # auto: 2,000 atoms take the single launch
        assert md.stats()["persistent_blocks"] > 0
        md.step(20, 2.0)
        pos, vel, step = md.get_state()
        md.step(15, 2.0)
        p1, v1, _ = md.get_state()
    with binding.MD(s, precision="fp64", persistent="on") as md:
        md.set_state(pos, vel, step)
        md.step(15, 2.0)
        p2, v2, st2 = md.get_state()
    assert st2 == 35
    d = p2 - p1
    d -= s.box * np.round(d / s.box)
    assert np.abs(d).max() < 1e-12
    big = I.bcc_cube(33)  # 71,874 atoms: above the automatic threshold
    with binding.MD(big, precision="mixed") as md:
        assert md.stats()["persistent_blocks"] == 0


def test_wait_limit_raises_timeout_and_the_context_recovers():
    """A barrier wait longer than the configured limit (1 us here, so the
    barriers of the single launch run out) ends the launch with
    MD_ERR_TIMEOUT; md_set_state clears it and the context answers again."""
    s = I.bcc_2000_fp64()
    with binding.MD(s, precision="mixed", persistent="on", lanes_per_atom=2, wait_limit_us=1) as md:
        md.step(200, 2.0)
        with pytest.raises(binding.MDError) as e:
            md.sync()
        assert e.value.status == -6  # MD_ERR_TIMEOUT
        md.set_state(s.pos, s.vel, 0)
        assert_forces(md.forces(), oracle_forces(s, s.pos), "mixed")
    with pytest.raises(binding.MDError) as e:
        binding.MD(s, wait_limit_us=-1)
    assert e.value.status == -1


def test_single_launch_list_build_with_crowded_cells():
    """More than 64 atoms in a cell.  The single launch builds lists with a
    warp per atom, a lane per stencil cell, keeping the decisions of a
    cell's first 64 candidates as a bit mask and recomputing the rest: the
    lists built inside the launch (a rebuild every step) must equal the
    oracle's at the launch's own positions, and the graph path's (same lanes
    per atom, so the same positions bit for bit)."""
    rng = np.random.default_rng(64)
    box = np.array([15.0, 15.0, 15.0])  # 3 x 3 x 3 cells of 5 A
    cand = rng.random((8000, 3)) * box
    keep = [cand[0]]
    for x in cand[1:]:
        d = np.asarray(keep) - x
        d -= box * np.round(d / box)
        if (d * d).sum(1).min() > 0.8**2:
            keep.append(x)
        if len(keep) == 2500:
            break
    pos = np.asarray(keep)
    gas = I.System(box=box, pos=pos, vel=np.zeros_like(pos), types=np.zeros(len(pos), np.int32),
                   pot=I.johnson_potential(I.BCC_TA_LIKE))
    _, start, _ = O.cells(O.wrap(pos, box), box, gas.pot.r_list)
    assert np.diff(start).max() > 64
    for precision in ("mixed", "fp64"):
        lists = []
        for persistent in ("on", "off"):
            with binding.MD(gas, precision=precision, persistent=persistent, rebuild_every=1,
                            lanes_per_atom=1) as md:
                assert (md.stats()["persistent_blocks"] > 0) == (persistent == "on")
                md.step(3, 0.001)
                assert md.stats()["rebuilds"] == 3
                p, _, _ = md.get_state()
                off, js = md.neighbors()
            ooff, ojs = O.neighbors_cells(O.wrap(p, box), box, gas.pot.r_list)
            np.testing.assert_array_equal(off, ooff)
            np.testing.assert_array_equal(js, ojs)
            lists.append((p, js))
        np.testing.assert_array_equal(lists[0][0], lists[1][0])
        np.testing.assert_array_equal(lists[0][1], lists[1][1])
