"""Open (non-periodic) axes on the GPU against the serial FP64 oracle: the
free-surface slabs of the paper's benchmark systems.

Bars as for periodic systems: cell bins and neighbour lists bit-exact (same
order), FP64 forces within 1e-10 and mixed-precision forces within 2e-5 of
the oracle (relative 2-norm over all 3N components), trajectories within
1e-9 A in FP64; the single launch bitwise equal to the
atom-parallel graph path.
"""
import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import binding, inputs as I
from bars import assert_forces

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 2e-5}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_eval(s, pos=None):
    pot = O.Potential(s.pot)
    p = s.pos if pos is None else pos
    return O.eam_eval(pot, O.wrap(p, s.box, s.open_axes), s.box, s.types, open_axes=s.open_axes)


def periodic_delta(d, s):
    d = d.copy()
    for a in range(3):
        if not (s.open_axes >> a) & 1:
            d[:, a] -= s.box[a] * np.round(d[:, a] / s.box[a])
    return d


@pytest.mark.parametrize("open_axes", [4, 3, 7])
def test_open_cells_and_lists_bit_exact(open_axes):
    s = I.bcc_slab_small(open_axes)
    # a few atoms outside the box along the open axes go to the edge cells
    rng = np.random.default_rng(3)
    pos = s.pos.copy()
    for a in range(3):
        if (open_axes >> a) & 1:
            k = rng.choice(s.n, size=4, replace=False)
            pos[k[:2], a] = -0.3 - 0.5 * rng.random(2)
            pos[k[2:], a] = s.box[a] + 0.3 + 0.5 * rng.random(2)
    s = I.System(box=s.box, pos=pos, vel=s.vel, types=s.types, pot=s.pot, open_axes=open_axes)
    r_list = s.pot.r_cut + s.pot.skin
    w = O.wrap(s.pos, s.box, open_axes)
    for precision in ("fp64", "mixed"):
        with binding.MD(s, precision=precision) as md:
            nc, start, atoms = md.cells()
            onc, ostart, oatoms = O.cells(w, s.box, r_list, open_axes)
            np.testing.assert_array_equal(nc, onc)
            np.testing.assert_array_equal(start, ostart)
            np.testing.assert_array_equal(atoms, oatoms)
            off, js = md.neighbors()
            ooff, ojs = O.neighbors_cells(w, s.box, r_list, open_axes)
            np.testing.assert_array_equal(off, ooff)
            np.testing.assert_array_equal(js, ojs)


@pytest.mark.parametrize("open_axes", [4, 7])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_open_forces_energy_virial(open_axes, precision):
    s = I.bcc_slab_small(open_axes)
    _, _, F, E, W = oracle_eval(s)
    with binding.MD(s, precision=precision) as md:
        assert_forces(md.forces(), F, precision)
        pe, _ = md.energy()
        assert abs(pe - E.sum()) / abs(E.sum()) < TOL[precision]
        assert rel(md.virial(), W) < TOL[precision]


def test_open_trajectory_fp64_matches_oracle():
    s = I.bcc_slab_small(4)
    pot = O.Potential(s.pot)
    ref = O.System(pot, s.box, s.pos, s.vel, s.types, open_axes=4)
    with binding.MD(s, precision="fp64", persistent="off") as md:
        for block in range(10):
            md.step(10, 2.0)
            ref.step(10, 2.0)
            pos, vel, step = md.get_state()
            st = ref.state()
            assert np.abs(periodic_delta(pos - st["pos"], s)).max() < 1e-9
            assert np.abs(vel - st["vel"]).max() < 1e-11
        assert md.stats()["rebuilds"] == ref.state()["rebuilds"] == 10
        _, _, F, _, _ = oracle_eval(s, pos)
        assert_forces(md.forces(), F, "fp64")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_open_single_launch_bitwise(precision):
    """The single launch follows the same lists across open edges as the
    graph path: forces and positions bitwise equal after 30 steps."""
    s = I.bcc_slab_small(7)
    out = {}
    for name, kw in (("graphs", dict(persistent="off")), ("single", dict(persistent="on"))):
        with binding.MD(s, precision=precision, lanes_per_atom=2, **kw) as md:
            f0 = md.forces()
            md.step(30, 2.0)
            out[name] = (f0, md.get_state()[0], md.forces())
    for a, b in zip(out["single"], out["graphs"]):
        np.testing.assert_array_equal(a, b)
    _, _, F, _, _ = oracle_eval(s, out["graphs"][1])
    assert_forces(out["graphs"][2], F, precision)


def test_paper_size_ta_slab_forces():
    """The 801,792-atom open slab (256 x 261 x 6 BCC cells): all forces
    against the oracle, before and after 10 steps."""
    s = I.ta_slab_801792()
    _, _, F, E, _ = oracle_eval(s)
    with binding.MD(s, precision="mixed") as md:
        assert_forces(md.forces(), F, "mixed")
        pe, _ = md.energy()
        assert abs(pe - E.sum()) / abs(E.sum()) < TOL["mixed"]
        md.step(10, 2.0)
        pos, _, _ = md.get_state()
        f10 = md.forces()
    _, _, F10, _, _ = oracle_eval(s, pos)
    assert_forces(f10, F10, "mixed")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_open_fcc_slab_forces(precision):
    """FCC stand-in (r_cut 5.0, 42 interactions per atom) in a slab open
    along z: 54 list entries per bulk atom."""
    s = I.slab_system(I.FCC_CU_LIKE, (8, 8, 5), 4, 5.0, 0.03, 350.0, I.SEED_BASE + 603, n_knots=2000)
    _, _, F, E, _ = oracle_eval(s)
    with binding.MD(s, precision=precision) as md:
        assert md.stats()["max_neighbors"] >= 54
        assert_forces(md.forces(), F, precision)
        pe, _ = md.energy()
        assert abs(pe - E.sum()) / abs(E.sum()) < TOL[precision]
