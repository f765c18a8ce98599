"""The 799,496-atom benchmark system (74 x 74 x 73 BCC cells, 300 K) at full
size: the FP64 path's forces at step 0; the mixed path's running state
after 100 steps (ten list builds) against the oracle -- cell bins and
neighbour lists bit for bit, forces, energies; and the mixed path's NVE
drift over 10,000 steps (the stability bar of the mixed-precision form:
below 1e-4 eV/atom per 1e5 steps)."""
import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import binding, inputs as I
from bars import assert_forces

pytestmark = pytest.mark.gpu

DRIFT_BAR = 1e-4  # eV/atom per 1e5 steps


@pytest.fixture(scope="module")
def c2():
    return I.bcc_799496()


def oracle_eval(system, pos):
    pot = O.Potential(system.pot)
    return O.eam_eval(pot, O.wrap(pos, system.box), system.box, system.types)


def test_fp64_path_at_step_0(c2):
    _, _, F, E, W = oracle_eval(c2, c2.pos)
    with binding.MD(c2, precision="fp64") as md:
        assert_forces(md.forces(), F, "fp64", "800k fp64")
        pe, _ = md.energy()
        assert abs(pe - E.sum()) / abs(E.sum()) < 1e-10
        w = md.virial()
        assert np.linalg.norm(w - W) / np.linalg.norm(W) < 1e-10


def test_mixed_running_state_after_100_steps(c2):
    """The context's own state after 100 steps: the list in use was built at
    step 100 (builds every 10 steps, none triggered early at 300 K), so its
    cells and lists are those of the positions it reports."""
    with binding.MD(c2, precision="mixed") as md:
        md.step(100, 2.0)
        pos, vel, step = md.get_state()
        assert step == 100 and md.stats()["rebuilds"] == 10
        f = md.forces()
        pe, ke = md.energy()
        nc, start, atoms = md.cells()
        off, js = md.neighbors()
    wpos = O.wrap(pos, c2.box)
    onc, ostart, oatoms = O.cells(wpos, c2.box, c2.pot.r_list)
    np.testing.assert_array_equal(nc, onc)
    np.testing.assert_array_equal(start, ostart)
    np.testing.assert_array_equal(atoms, oatoms)
    ooff, ojs = O.neighbors_cells(wpos, c2.box, c2.pot.r_list)
    np.testing.assert_array_equal(off, ooff)
    np.testing.assert_array_equal(js, ojs)
    _, _, F, E, _ = oracle_eval(c2, pos)
    assert_forces(f, F, "mixed", "800k step 100")
    assert abs(pe - E.sum()) / abs(E.sum()) < 2e-5
    m = c2.pot.mass[0]
    ke_ref = 0.5 * m * (vel ** 2).sum() / I.ACCEL_EV_A_AMU
    assert abs(ke - ke_ref) / ke_ref < 1e-12


def test_mixed_drift_10000_steps(c2):
    e = []
    with binding.MD(c2, precision="mixed") as md:
        pe, ke = md.energy()
        e.append((pe + ke) / c2.n)
        for _ in range(100):
            md.step(100, 2.0)
            pe, ke = md.energy()
            e.append((pe + ke) / c2.n)
        assert md.get_state()[2] == 10_000
    t = np.arange(len(e)) * 100.0
    e = np.array(e)
    drift = abs(np.polyfit(t, e - e[0], 1)[0]) * 1e5
    assert drift < DRIFT_BAR, f"drift {drift:.3e} eV/atom per 1e5 steps"
    assert np.abs(e - e[0]).max() < 1e-4
