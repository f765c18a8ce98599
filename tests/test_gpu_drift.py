"""NVE energy drift of the GPU path (the stability requirement on the mixed
precision form: drift below 1e-4 eV/atom per 1e5 steps).

Drift is the magnitude of the least-squares slope of E_tot/N, sampled every
100 steps, times 1e5 steps.  The FP64 path runs beside the mixed path on the
same input, so that a drift that the integrator itself shows is not charged
to the FP32 pair arithmetic.  Systems are small enough for the single-launch
path to run 1e5 steps in seconds."""
import numpy as np
import pytest

from paper_2405_07898_gb300 import binding, inputs as I

pytestmark = pytest.mark.gpu

DRIFT_BAR = 1e-4  # eV/atom per 1e5 steps


def energy_series(system, precision, nsteps, every=100, dt=2.0):
    e = []
    with binding.MD(system, precision=precision) as md:
        pe, ke = md.energy()
        e.append((pe + ke) / system.n)
        for _ in range(nsteps // every):
            md.step(every, dt)
            pe, ke = md.energy()
            e.append((pe + ke) / system.n)
        assert md.get_state()[2] == nsteps
    return np.arange(len(e)) * every, np.array(e)


def drift_per_1e5(t, e):
    slope = np.polyfit(t.astype(np.float64), e - e[0], 1)[0]
    return abs(slope) * 1e5


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_drift_2000_atoms_300K_1e5_steps(precision):
    s = I.bcc_2000_fp64()
    t, e = energy_series(s, precision, 100_000)
    d = drift_per_1e5(t, e)
    excursion = np.abs(e - e[0]).max()
    print(f"{precision}: drift {d:.2e} eV/atom per 1e5 steps, max |E(t)-E(0)|/N {excursion:.2e}")
    assert d < DRIFT_BAR
    assert excursion < 1e-3


def test_drift_mixed_16000_atoms_1000K_tracks_fp64():
    """A hotter, larger system (16,000 atoms at 1,000 K, 2e4 steps): both
    paths meet the bar from the same start."""
    s = I.bcc_cube(20, temperature=1000.0, seed=I.SEED_BASE + 720)
    tm, em = energy_series(s, "mixed", 20_000)
    tf, ef = energy_series(s, "fp64", 20_000)
    dm, df = drift_per_1e5(tm, em), drift_per_1e5(tf, ef)
    print(f"16,000 atoms 1000 K: drift mixed {dm:.2e}, fp64 {df:.2e} eV/atom per 1e5 steps")
    assert dm < DRIFT_BAR and df < DRIFT_BAR
    # same start: the energies agree within the mixed path's energy bar
    assert abs(em[0] - ef[0]) < 2e-5 * abs(ef[0])
