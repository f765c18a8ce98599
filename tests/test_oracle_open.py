"""Pins of the oracle's open (non-periodic) axes: the free-surface thin-slab
geometry of the paper's benchmark systems (Section "How Performance Was
Measured": open boundaries).  On an open axis positions are not wrapped,
displacements are plain differences, cells beyond the edge do not exist and
atoms outside the box fall into the edge cells.  Each pin ties that code to
something independent of it: the all-pairs list, the same cluster evaluated
in a periodic box too large for any image to interact, finite differences of
the energy, and translation invariance.
"""
import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import inputs as I


def pot():
    return O.Potential(I.johnson_potential(I.BCC_TA_LIKE))


def cluster(n=150, seed=5, radius=11.0):
    """A random dense cluster (minimum separation 2.2 A) around the origin."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        x = rng.uniform(-radius, radius, size=3)
        if np.linalg.norm(x) > radius:
            continue
        if pts and np.min(np.linalg.norm(np.array(pts) - x, axis=1)) < 2.2:
            continue
        pts.append(x)
    return np.array(pts)


@pytest.mark.parametrize("open_axes", [4, 3, 7])
def test_open_lists_equal_all_pairs(open_axes):
    s = I.bcc_slab_small(open_axes)
    pos = s.pos.copy()
    # a few atoms just outside the box along the open axes: edge cells
    rng = np.random.default_rng(3)
    for a in range(3):
        if (open_axes >> a) & 1:
            k = rng.choice(s.n, size=4, replace=False)
            pos[k[:2], a] = -0.4 - rng.random(2)
            pos[k[2:], a] = s.box[a] + 0.4 + rng.random(2)
    r_list = s.pot.r_cut + s.pot.skin
    w = O.wrap(pos, s.box, open_axes)
    for a in range(3):
        if (open_axes >> a) & 1:
            np.testing.assert_array_equal(w[:, a], pos[:, a])  # no wrap on open axes
    oc, jc = O.neighbors_cells(w, s.box, r_list, open_axes)
    ob, jb = O.neighbors_brute(w, s.box, r_list, open_axes)
    np.testing.assert_array_equal(oc, ob)
    for i in range(s.n):
        assert sorted(jc[oc[i]:oc[i + 1]]) == sorted(jb[ob[i]:ob[i + 1]])
    # atoms near an open face have fewer neighbours than bulk atoms
    counts = np.diff(oc)
    assert counts.min() < 20 and counts.max() == 26


def test_isolated_cluster_open_equals_periodic():
    """A cluster in a fully open box and in a periodic box whose images lie
    beyond the list radius: same energy, forces and virial (the periodic
    route uses the minimum image and the wrapped stencil instead)."""
    P = pot()
    x = cluster()
    types = np.zeros(len(x), dtype=np.int32)
    box_open = np.array([28.0, 28.0, 28.0])
    box_per = np.array([44.0, 44.0, 44.0])
    _, _, Fo, Eo, Wo = O.eam_eval(P, x + 14.0, box_open, types, open_axes=7)
    _, _, Fp, Ep, Wp = O.eam_eval(P, x + 22.0, box_per, types, open_axes=0)
    assert abs(Eo.sum() - Ep.sum()) < 1e-11 * abs(Ep.sum())
    np.testing.assert_allclose(Fo, Fp, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Wo, Wp, rtol=1e-12, atol=1e-12)
    assert np.abs(Fo.sum(0)).max() < 1e-10


def test_open_slab_forces_are_the_energy_gradient():
    P = pot()
    s = I.bcc_slab_small(4)
    types = s.types
    _, _, F, _, _ = O.eam_eval(P, s.pos, s.box, types, open_axes=4)
    rng = np.random.default_rng(8)
    h = 1e-5
    # surface atoms (largest and smallest z) and bulk atoms
    z = s.pos[:, 2]
    picks = list(np.argsort(z)[:3]) + list(np.argsort(z)[-3:]) + list(rng.choice(s.n, 3, replace=False))
    got, want = [], []
    for i in picks:
        for a in range(3):
            p1 = s.pos.copy()
            p1[i, a] += h
            p2 = s.pos.copy()
            p2[i, a] -= h
            e1 = O.eam_eval(P, p1, s.box, types, open_axes=4)[3].sum()
            e2 = O.eam_eval(P, p2, s.box, types, open_axes=4)[3].sum()
            got.append(F[i, a])
            want.append(-(e1 - e2) / (2 * h))
    got, want = np.array(got), np.array(want)
    # relative 2-norm; the central difference's own error at |E| ~ 9,000 eV
    # is ~1e-7 per component
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-6
    # the surface atoms feel the free surface: their z forces are not small
    assert np.abs(F[np.argsort(z)[:3], 2]).max() > 1e-3


def test_open_slab_translation_invariance_and_momentum():
    P = pot()
    s = I.bcc_slab_small(4)
    _, _, F0, E0, _ = O.eam_eval(P, s.pos, s.box, s.types, open_axes=4)
    shifted = s.pos + np.array([0.0, 0.0, -0.83])  # still inside the box
    _, _, F1, E1, _ = O.eam_eval(P, shifted, s.box, s.types, open_axes=4)
    assert abs(E1.sum() - E0.sum()) < 1e-10 * abs(E0.sum())
    np.testing.assert_allclose(F1, F0, rtol=0, atol=1e-10)
    assert np.abs(F0.sum(0)).max() < 1e-9
    ref = O.System(P, s.box, s.pos, s.vel, s.types, open_axes=4)
    m = P.src.mass[s.types]
    p0 = (m[:, None] * s.vel).sum(0)
    e0 = sum(ref.energy())
    ref.step(50, 2.0)
    st = ref.state()
    p1 = (m[:, None] * st["vel"]).sum(0)
    assert np.abs(p1 - p0).max() < 1e-10
    assert abs(sum(ref.energy()) - e0) / s.n < 5e-5
    # time reversibility with free surfaces: 50 steps back
    back = O.System(P, s.box, st["pos"], -st["vel"], s.types, open_axes=4)
    back.step(50, 2.0)
    d = back.state()["pos"] - s.pos
    d[:, :2] -= s.box[:2] * np.round(d[:, :2] / s.box[:2])  # x, y periodic
    assert np.abs(d).max() < 1e-9
