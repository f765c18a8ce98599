"""CPU pins of two host-side pieces that feed measurements: the least-squares
fit of the linear time model (the paper's Eq. 6 form) and the Sigma-5 tilt
bicrystal generator of the drift and sweep workloads."""
import math

import numpy as np
import pytest

from paper_2405_07898_gb300 import inputs as I
from paper_2405_07898_gb300 import timemodel


# ---- the linear time model fit --------------------------------------------

def test_fit_recovers_known_coefficients_exactly():
    rng = np.random.default_rng(6)
    X = rng.uniform(10, 60, size=(12, 2))
    c_true = np.array([4.2e-3, 1.9e-3, 0.05])  # per list entry, per interaction, fixed (ns)
    y = X @ c_true[:2] + c_true[2]
    c, r2 = timemodel.fit_linear(X, y)
    np.testing.assert_allclose(c, c_true, rtol=1e-10, atol=1e-13)
    assert r2 == pytest.approx(1.0, abs=1e-12)


def test_fit_with_noise_and_the_four_model_fits():
    rng = np.random.default_rng(7)
    pts = []
    for _ in range(40):
        nl, ni, nc = rng.uniform(14, 64), rng.uniform(14, 58), rng.uniform(84, 566)
        pts.append({"n_list": nl, "n_inter": ni, "n_cand": nc,
                    "pair_ns_per_atom": 0.004 * nl + 0.002 * ni + 0.046 + rng.normal(0, 1e-4),
                    "density_ns_per_atom": 0.0022 * nl + 0.0006 * ni + 0.012 + rng.normal(0, 1e-4),
                    "force_ns_per_atom": 0.0020 * nl + 0.0014 * ni + 0.034 + rng.normal(0, 1e-4),
                    "build_ns_per_atom": 0.0011 * nc + 0.0022 * nl + 0.18 + rng.normal(0, 1e-3)})
    f = timemodel.fit_points(pts)
    assert f["pair_passes"]["per_list_entry"] == pytest.approx(0.004, abs=2e-5)
    assert f["pair_passes"]["per_interaction"] == pytest.approx(0.002, abs=2e-5)
    assert f["pair_passes"]["fixed"] == pytest.approx(0.046, abs=2e-3)
    assert f["list_build"]["per_candidate"] == pytest.approx(0.0011, abs=1e-5)
    assert f["list_build"]["per_list_entry"] == pytest.approx(0.0022, abs=1e-4)
    for k in ("pair_passes", "density", "force", "list_build"):
        assert f[k]["r2"] > 0.99


def test_fit_rejects_too_few_points():
    with pytest.raises(ValueError):
        timemodel.fit_linear([[1.0, 2.0], [2.0, 1.0]], [1.0, 2.0])


# ---- the Sigma-5 (310)[001] tilt bicrystal ---------------------------------

def _on_lattice(pos, a, sign):
    """Whether each atom sits on the BCC lattice of constant a rotated by
    sign * atan(1/3) about z (counterclockwise for sign +1): its in-plane lattice coordinates (positions
    rotated back) and z/a are all integers or all half-integers."""
    th = sign * math.atan(1.0 / 3.0)
    c, s = math.cos(th), math.sin(th)
    u = (c * pos[:, 0] + s * pos[:, 1]) / a
    v = (-s * pos[:, 0] + c * pos[:, 1]) / a
    w = pos[:, 2] / a
    twice = np.stack([2 * u, 2 * v, 2 * w], 1)
    near = np.abs(twice - np.rint(twice)).max(1) < 1e-6
    parity = np.rint(twice).astype(np.int64) % 2
    return near & (parity[:, 0] == parity[:, 1]) & (parity[:, 1] == parity[:, 2])


@pytest.fixture(scope="module")
def bicrystals():
    full = I.sigma5_bicrystal(temperature=10.0, min_sep=0.0, sigma=0.0)
    cut = I.sigma5_bicrystal(temperature=10.0, sigma=0.0)
    return full, cut


def test_bicrystal_grains_and_counts(bicrystals):
    full, cut = bicrystals
    a = I.BCC_TA_LIKE.a
    s10 = math.sqrt(10.0)
    np.testing.assert_allclose(full.box, [25 * a * s10, 20 * a * s10, 25 * a], rtol=1e-14)
    # 25 x (2 x 10) x 25 grain periods of 20 atoms before any removal
    assert full.n == 250000
    plus, minus = _on_lattice(full.pos, a, 1), _on_lattice(full.pos, a, -1)
    y = full.pos[:, 1]
    Ly = full.box[1]

    def lower_grain(yy):
        # [0, Ly/2), periodic: the grain's bottom plane may wrap to y ~ Ly
        return (yy < Ly / 2 - 1e-6) | (yy > Ly - 1e-6)

    lower = lower_grain(y)
    # grains stacked along y: the lower half on the lattice rotated by
    # -atan(1/3), the upper half on the one rotated by +atan(1/3)
    assert minus[lower].all() and plus[~lower].all()
    assert lower.sum() == 125000  # equal grains
    # Sigma 5: one site in five of either lattice lies on the other too
    assert plus[lower].sum() * 5 == lower.sum()
    assert minus[~lower].sum() * 5 == (~lower).sum()
    # removal: upper-grain atoms closer than min_sep a to a lower-grain atom,
    # counted here with a periodic KD-tree on the unremoved crystal.  The
    # closest cross-boundary pairs of this boundary are a sqrt(2/5) apart,
    # so the default 0.3 a removes none (250,000 atoms); 0.75 a removes some.
    from scipy.spatial import cKDTree
    tree = cKDTree(np.mod(full.pos[lower], full.box), boxsize=full.box)
    dist, _ = tree.query(np.mod(full.pos[~lower], full.box), k=1)
    assert dist.min() == pytest.approx(a * math.sqrt(0.4), rel=1e-9)
    assert cut.n == full.n - int((dist < 0.3 * a).sum()) == 250000
    wide = I.sigma5_bicrystal(temperature=10.0, sigma=0.0, min_sep=0.75)
    removed = int((dist < 0.75 * a).sum())
    assert removed > 0 and wide.n == full.n - removed
    wl = lower_grain(wide.pos[:, 1])
    tl = cKDTree(np.mod(wide.pos[wl], wide.box), boxsize=wide.box)
    d2, _ = tl.query(np.mod(wide.pos[~wl], wide.box), k=1)
    assert d2.min() >= 0.75 * a


def test_bicrystal_thermal_state(bicrystals):
    """The default (thermal) generator removes the same atoms and gives
    zero momentum at the requested temperature."""
    _, cut = bicrystals
    hot = I.sigma5_bicrystal(temperature=1000.0)
    assert hot.n == cut.n
    m = I.BCC_TA_LIKE.mass
    p = (m * hot.vel).sum(0)
    assert np.abs(p).max() < 1e-9 * m * np.abs(hot.vel).sum()
    ke = 0.5 * m * (hot.vel ** 2).sum() / I.ACCEL_EV_A_AMU
    t = 2 * ke / ((3 * hot.n - 3) * I.KB_EV)
    assert t == pytest.approx(1000.0, rel=1e-9)
