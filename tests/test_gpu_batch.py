"""The batching form: many independent replicas (BCC and FCC, uneven sizes,
different temperatures) advanced in one persistent launch, through the C ABI,
against the oracle replica by replica."""
import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import binding, inputs as I
from bars import assert_forces

pytestmark = pytest.mark.gpu

MIXED_TOL = 2e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def small_batch():
    return [
        I.thermal_system(I.BCC_TA_LIKE, (5, 5, 5), 0.02, 300.0, 101),
        I.thermal_system(I.FCC_CU_LIKE, (5, 5, 5), 0.02, 900.0, 102),
        I.thermal_system(I.BCC_TA_LIKE, (9, 7, 6), 0.03, 1200.0, 103),
        I.thermal_system(I.FCC_CU_LIKE, (7, 6, 5), 0.02, 200.0, 104),
        I.thermal_system(I.BCC_TA_LIKE, (12, 12, 12), 0.02, 600.0, 105),
        I.thermal_system(I.FCC_CU_LIKE, (10, 9, 8), 0.02, 450.0, 106),
        I.thermal_system(I.BCC_TA_LIKE, (6, 5, 5), 0.02, 300.0, 107),
    ]


def oracle_state(s, pos=None):
    pot = O.Potential(s.pot)
    p = s.pos if pos is None else pos
    return O.eam_eval(pot, O.wrap(p, s.box), s.box, s.types)


def test_initial_forces_and_energies_per_replica():
    systems = small_batch()
    with binding.MDBatch(systems) as b:
        pe, ke = b.energy()
        for r, s in enumerate(systems):
            _, _, F, E, _ = oracle_state(s)
            _, _, f = b.get_state(r)
            assert_forces(f, F, "mixed", f"replica {r}")
            assert abs(pe[r] - E.sum()) / abs(E.sum()) < MIXED_TOL
            m = s.pot.mass[0]
            ke_ref = 0.5 * m * (s.vel**2).sum() / I.ACCEL_EV_A_AMU
            assert abs(ke[r] - ke_ref) / ke_ref < 1e-9


def test_trajectories_against_oracle():
    systems = small_batch()
    with binding.MDBatch(systems) as b:
        b.step(40, 2.0)
        pe, ke = b.energy()
        info = b.info()
        assert info["steps"] == 40 and info["rebuilds"] >= 4 * len(systems)
        for r, s in enumerate(systems):
            ref = O.System(O.Potential(s.pot), s.box, s.pos, s.vel, s.types)
            ref.step(40, 2.0)
            st = ref.state()
            pos, vel, f = b.get_state(r)
            d = pos - st["pos"]
            d -= s.box * np.round(d / s.box)
            assert np.abs(d).max() < 1e-4, r
            ope, oke = ref.energy()
            assert abs((pe[r] + ke[r]) - (ope + oke)) / abs(ope + oke) < 1e-5, r
            # forces at the batch's own positions
            _, _, F, _, _ = oracle_state(s, pos)
            assert_forces(f, F, "mixed", f"replica {r}")


def test_batch_equals_itself_and_graphs_equal_plain_launches():
    systems = small_batch()[:4]
    runs = []
    for use_graphs in (True, False):
        with binding.MDBatch(systems, use_graphs=use_graphs) as b:
            b.step(25, 2.0)
            b.step(25, 2.0)
            runs.append([b.get_state(r) for r in range(len(systems))] + [b.energy()])
    for (a, c) in zip(runs[0][:-1], runs[1][:-1]):
        for x, y in zip(a, c):
            np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(runs[0][-1][0], runs[1][-1][0])


def test_rejects_bad_replicas():
    s = I.bcc_2000_fp64()
    tiny = I.System(box=s.box / 3, pos=s.pos / 3, vel=s.vel, types=s.types, pot=s.pot)
    with pytest.raises(binding.MDError) as e:
        binding.MDBatch([s, tiny])
    assert e.value.status == -2
    with pytest.raises(binding.MDError) as e:
        binding.MDBatch([s], schedule=6)
    assert e.value.status == -1


def test_every_block_shape_gives_the_same_trajectories():
    """Each threads-per-block x blocks-per-SM shape of the batch launch, on a
    replica whose cell scan spans several 1,024-cell chunks (so every warp of
    a 1,024-thread block holds cells): forces meet the oracle bar, and
    positions after 20 steps are bitwise those of every other shape."""
    systems = [I.thermal_system(I.BCC_TA_LIKE, (28, 28, 28), 0.02, 600.0, 111),
               I.thermal_system(I.FCC_CU_LIKE, (6, 6, 6), 0.02, 500.0, 112)]
    refs = [oracle_state(s)[2] for s in systems]
    out = []
    for sched in range(1, 6):
        with binding.MDBatch(systems, schedule=sched) as b:
            for r in range(len(systems)):
                assert_forces(b.get_state(r)[2], refs[r], "mixed", f"schedule {sched} replica {r}")
            b.step(20, 2.0)
            out.append([b.get_state(r)[0] for r in range(len(systems))])
    for o in out[1:]:
        for a, c in zip(o, out[0]):
            np.testing.assert_array_equal(a, c)


def test_full_512_replica_batch_sample_against_oracle():
    """The batched workload the benchmark times: 512 replicas (about 3.0 M
    atoms; BCC and FCC; 1,024 to 16,384 atoms; 200 to 1,200 K) in one launch
    with its largest-first queue and the timed block shape.  A seeded sample
    of 16 replicas, always including the largest BCC and the largest FCC
    replica, is checked against the oracle at step 0 and after 100 steps:
    every atom's force at the batch's own positions (both bars), the
    potential energy, and the kinetic energy from the batch's velocities."""
    systems = I.replica_batch()
    n = np.array([s.n for s in systems])
    half = len(systems) // 2
    big_bcc = int(np.argmax(n[:half]))
    big_fcc = half + int(np.argmax(n[half:]))
    rng = np.random.Generator(np.random.PCG64(I.SEED_BASE + 512))
    rest = [r for r in range(len(systems)) if r not in (big_bcc, big_fcc)]
    sample = [big_bcc, big_fcc] + sorted(int(r) for r in rng.choice(rest, 14, replace=False))
    assert n[big_bcc] > 14000 and n[big_fcc] > 14000
    with binding.MDBatch(systems) as b:
        for r in sample:
            _, _, F, _, _ = oracle_state(systems[r])
            assert_forces(b.get_state(r)[2], F, "mixed", f"step 0 replica {r}")
        b.step(100, 2.0)
        pe, ke = b.energy()
        for r in sample:
            s = systems[r]
            pos, vel, f = b.get_state(r)
            _, _, F, E, _ = oracle_state(s, pos)
            assert_forces(f, F, "mixed", f"step 100 replica {r} ({s.n} atoms)")
            assert abs(pe[r] - E.sum()) / abs(E.sum()) < MIXED_TOL, r
            m = s.pot.mass[0]
            ke_ref = 0.5 * m * (vel**2).sum() / I.ACCEL_EV_A_AMU
            assert abs(ke[r] - ke_ref) / ke_ref < 1e-9, r
