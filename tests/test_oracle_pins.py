"""Pins of the CPU oracle against facts fixed outside it: a library spline,
exact polynomial reproduction, brute-force pair search, closed-form lattice
sums, finite differences of the energy, symmetries and the integrator's
exact properties.  No GPU is used.

Each test names the passage of arXiv 2405.07898 it pins: Eq. 2 (density),
Eq. 3 (energy), Eq. 4 (force), Eq. 5 (leap-frog / velocity Verlet), Section
"Neighbor list" (r^2 filter), Section "Periodic Boundary Conditions", and the
interaction counts of Table "Results for 800,000 atom models".
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# splines (per-type arbitrary splines, Section "Computational Molecular Dynamics")


def _scipy_cs():
    return pytest.importorskip("scipy.interpolate").CubicSpline


@pytest.mark.parametrize("bc", [("clamped", "natural"), ("natural", "natural"), ("clamped", "clamped")])
def test_spline_matches_scipy(bc):
    CubicSpline = _scipy_cs()
    rng = np.random.default_rng(1)
    n, h = 37, 0.125
    y = np.cumsum(rng.normal(size=n))
    s0, s1 = 0.7, -1.3
    k = I.Knots(0.0, h, y, I.BC_CLAMPED if bc[0] == "clamped" else I.BC_NATURAL,
                I.BC_CLAMPED if bc[1] == "clamped" else I.BC_NATURAL, s0, s1)
    coef = O.spline_coeffs(k)
    bct = ((1, s0) if bc[0] == "clamped" else (2, 0.0), (1, s1) if bc[1] == "clamped" else (2, 0.0))
    cs = CubicSpline(k.x, y, bc_type=bct)
    # scipy stores the highest power first
    np.testing.assert_allclose(coef[:, 0], cs.c[3], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(coef[:, 1], cs.c[2], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(coef[:, 2], cs.c[1], rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(coef[:, 3], cs.c[0], rtol=1e-9, atol=1e-8)


def test_spline_reproduces_cubic_and_linear():
    h = 0.3
    x = h * np.arange(12)
    cubic = lambda t: 1.5 - 2.0 * t + 0.25 * t**2 - 0.125 * t**3
    dcubic = lambda t: -2.0 + 0.5 * t - 0.375 * t**2
    k = I.Knots(0.0, h, cubic(x), I.BC_CLAMPED, I.BC_CLAMPED, dcubic(0.0), dcubic(x[-1]))
    coef = O.spline_coeffs(k)
    xs = np.linspace(0.0, x[-1], 301)
    val, der, der2 = O.spline_eval(k, coef, xs)
    np.testing.assert_allclose(val, cubic(xs), atol=1e-12)
    np.testing.assert_allclose(der, dcubic(xs), atol=1e-11)
    np.testing.assert_allclose(der2, 0.5 - 0.75 * xs, atol=1e-10)
    # natural ends reproduce any straight line
    k2 = I.Knots(0.0, h, 3.0 - 0.5 * x, I.BC_NATURAL, I.BC_NATURAL)
    val, der, _ = O.spline_eval(k2, O.spline_coeffs(k2), xs)
    np.testing.assert_allclose(val, 3.0 - 0.5 * xs, atol=1e-13)
    np.testing.assert_allclose(der, -0.5, atol=1e-13)


def test_spline_interpolates_is_c2_and_extrapolates_linearly():
    rng = np.random.default_rng(2)
    k = I.Knots(0.5, 0.2, rng.normal(size=25), I.BC_NATURAL, I.BC_NATURAL)
    coef = O.spline_coeffs(k)
    v, _, _ = O.spline_eval(k, coef, k.x[:-1])
    np.testing.assert_allclose(v, k.y[:-1], atol=1e-13)
    # value, slope and curvature of interval k at its right end equal those
    # of interval k+1 at its left end (C2 continuity)
    h = k.dx
    a, b, c, d = coef[:-1].T
    np.testing.assert_allclose(a + h * (b + h * (c + h * d)), coef[1:, 0], atol=1e-12)
    np.testing.assert_allclose(b + h * (2 * c + 3 * h * d), coef[1:, 1], atol=1e-10)
    np.testing.assert_allclose(2 * c + 6 * h * d, 2 * coef[1:, 2], atol=1e-9)
    # beyond the last knot: straight line with the end slope
    xe = k.x[-1]
    ve, se, _ = O.spline_eval(k, coef, np.array([xe]))
    vo, so, s2 = O.spline_eval(k, coef, np.array([xe + 0.7, xe + 1.4]))
    np.testing.assert_allclose(vo, ve + se * np.array([0.7, 1.4]), atol=1e-12)
    np.testing.assert_allclose(so, se[0], atol=1e-12)
    np.testing.assert_allclose(s2, 0.0)


def test_johnson_tables_close_to_analytic():
    p = I.BCC_TA_LIKE
    pot = I.johnson_potential(p)
    r = np.linspace(1.5, p.r_cut - 1e-9, 2001)
    v, _, _ = O.spline_eval(pot.f[0], O.spline_coeffs(pot.f[0]), r)
    np.testing.assert_allclose(v, I.johnson_f(p, r), rtol=0, atol=5e-9)
    v, _, _ = O.spline_eval(pot.phi[0], O.spline_coeffs(pot.phi[0]), r)
    np.testing.assert_allclose(v, I.johnson_phi(p, r), rtol=0, atol=5e-9)


# --------------------------------------------------------------------------
# cells and neighbour lists (Section "Neighbor list"; Section "Periodic Boundary Conditions")


def _random_system(n, box, seed):
    rng = np.random.default_rng(seed)
    return rng.random((n, 3)) * box


def test_wrap_and_cells_stable_counting_sort():
    box = np.array([15.0, 16.1, 21.3])
    pos = _random_system(300, box, 3) + np.array([-15.0, 16.1, 0.0]) * (np.arange(300) % 2)[:, None]
    w = O.wrap(pos, box)
    assert (w >= 0).all() and (w < box).all()
    np.testing.assert_allclose(np.mod(pos, box), w, atol=1e-12)
    inside = (pos >= 0) & (pos < box)
    assert inside.any() and (~inside).any()
    np.testing.assert_array_equal(w[inside], pos[inside])  # in-box coordinates are kept bit for bit
    # one ulp below the box edge stays (x / L may round up to 1: the image
    # formula alone would give a negative coordinate there)
    edge = np.tile(np.nextafter(box, 0), (1, 1))
    np.testing.assert_array_equal(O.wrap(edge, box), edge)
    nc, start, atoms = O.cells(w, box, 4.8)
    assert tuple(nc) == (3, 3, 4)
    c = np.minimum(np.floor(w * (nc / box)).astype(int), nc - 1)
    cell = (c[:, 2] * nc[1] + c[:, 1]) * nc[0] + c[:, 0]
    expected = np.lexsort((np.arange(300), cell))  # by cell, ascending index inside a cell
    np.testing.assert_array_equal(atoms, expected)
    np.testing.assert_array_equal(np.diff(start), np.bincount(cell, minlength=int(np.prod(nc))))


@pytest.mark.parametrize("boxv,n,seed", [((14.5, 14.5, 14.5), 200, 4), ((20.0, 15.0, 33.0), 500, 5),
                                         ((40.0, 40.0, 40.0), 900, 6)])
def test_cell_list_equals_all_pairs(boxv, n, seed):
    box = np.array(boxv)
    pos = _random_system(n, box, seed)
    off_c, js_c = O.neighbors_cells(pos, box, 4.8)
    off_b, js_b = O.neighbors_brute(pos, box, 4.8)
    np.testing.assert_array_equal(off_c, off_b)
    for i in range(n):
        assert sorted(js_c[off_c[i]:off_c[i + 1]]) == list(js_b[off_b[i]:off_b[i + 1]])
    # every pair is symmetric and really closer than r_list (numpy minimum image)
    i_idx = np.repeat(np.arange(n), np.diff(off_b))
    d = pos[js_b] - pos[i_idx]
    d -= box * np.round(d / box)
    assert ((d**2).sum(1) < 4.8**2).all()
    pairs = set(zip(i_idx.tolist(), js_b.tolist()))
    assert all((j, i) in pairs for i, j in pairs)


def test_interaction_counts_match_paper_table():
    """Ta (BCC) has 14 interactions per atom and Cu (FCC) 42 in the paper's
    800k-atom table; the stand-in potentials reproduce both, and the lists
    with the 0.3 A skin hold 26 and 54 entries."""
    with open(os.path.join(GOLDEN, "paper_table_800k.json")) as fh:
        table = json.load(fh)["systems"]
    for p, paper_key, n_list in ((I.BCC_TA_LIKE, "Ta", 26), (I.FCC_CU_LIKE, "Cu", 54)):
        pos, box = I.lattice(p, 6, 6, 6)
        off, js = O.neighbors_cells(O.wrap(pos, box), box, p.r_cut + p.skin)
        assert set(np.diff(off).tolist()) == {n_list}
        off2, _ = O.neighbors_brute(pos, box, p.r_cut)
        assert set(np.diff(off2).tolist()) == {table[paper_key]["interactions"]}


# --------------------------------------------------------------------------
# closed-form lattice sums (Eqs. 2 and 3)


def _shells(p, nmax=4):
    base = np.array([[0, 0, 0], [0.5, 0.5, 0.5]]) if p.lattice == "bcc" else \
        np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.arange(-nmax, nmax + 1)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pts = (cells[:, None, :] + base[None]).reshape(-1, 3) * p.a
    r = np.sqrt((pts**2).sum(1))
    r = r[(r > 1e-9) & (r < p.r_cut)]
    keys, inv, counts = np.unique(np.round(r, 9), return_inverse=True, return_counts=True)
    vals = np.array([r[inv == k].mean() for k in range(len(keys))])  # exact radii, not rounded keys
    return vals, counts


def _dfdr(fun, r, h=1e-6):
    return (fun(r + h) - fun(r - h)) / (2 * h)


@pytest.mark.parametrize("p", [I.BCC_TA_LIKE, I.FCC_CU_LIKE])
def test_cohesive_energy_and_virial_closed_form(p):
    rs, ns = _shells(p)
    rho = (ns * I.johnson_f(p, rs)).sum()
    e_coh = I.johnson_F(p, rho) + 0.5 * (ns * I.johnson_phi(p, rs)).sum()
    pos, box = I.lattice(p, 5, 5, 5) if p.lattice == "fcc" else I.lattice(p, 6, 6, 6)
    n = pos.shape[0]
    pot = O.Potential(I.johnson_potential(p))
    rho_o, Fp_o, F, E, W = O.eam_eval(pot, pos, box, np.zeros(n, np.int32))
    np.testing.assert_allclose(rho_o, rho, rtol=1e-10)
    np.testing.assert_allclose(E.sum() / n, e_coh, rtol=1e-10)
    assert np.abs(F).max() < 1e-11
    # virial of a cubic lattice: W_aa = -(N/6) sum_s n_s s(r_s) r_s, off-diagonals 0,
    # with s = phi'(r) + 2 F'(rho) f'(r)
    Fp = _dfdr(lambda x: I.johnson_F(p, x), rho)
    s = _dfdr(lambda x: I.johnson_phi(p, x), rs) + 2 * Fp * _dfdr(lambda x: I.johnson_f(p, x), rs)
    w_aa = -(n / 6.0) * (ns * s * rs).sum()
    np.testing.assert_allclose(W[:3], w_aa, rtol=1e-6)
    assert np.abs(W[3:]).max() < 1e-8 * abs(w_aa)


# --------------------------------------------------------------------------
# forces (Eq. 4) against finite differences of the energy (Eq. 3)


def _energy(pot, pos, box, types):
    return O.eam_eval(pot, pos, box, types)[3].sum()


def _fd_check(system, atoms, h=1e-5, tol=1e-7):
    pot = O.Potential(system.pot)
    _, _, F, _, _ = O.eam_eval(pot, system.pos, system.box, system.types)
    got, want = [], []
    for i in atoms:
        for a in range(3):
            xp = system.pos.copy(); xp[i, a] += h
            xm = system.pos.copy(); xm[i, a] -= h
            fd = -(_energy(pot, xp, system.box, system.types) -
                   _energy(pot, xm, system.box, system.types)) / (2 * h)
            got.append(F[i, a]); want.append(fd)
    got, want = np.array(got), np.array(want)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol
    return F


def test_forces_are_minus_energy_gradient_single_type():
    s = I.thermal_system(I.BCC_TA_LIKE, (5, 5, 5), 0.08, 300.0, 11, n_knots=2000)
    F = _fd_check(s, atoms=range(0, 250, 13))
    assert np.abs(F.sum(0)).max() < 1e-11 * np.abs(F).max() * len(F)


def test_forces_are_minus_energy_gradient_two_types():
    """Type-dependent terms F'_i f'_{t_j} + F'_j f'_{t_i} + phi'_{t_i t_j} of Eq. 4:
    a swapped type index fails this finite-difference check."""
    s = I.multi_type_system(cells=(5, 5, 5), n_knots=600)
    assert 0 < s.types.sum() < len(s.types)
    _fd_check(s, atoms=range(0, 250, 11), tol=2e-7)


def test_fcc_forces_fd():
    s = I.thermal_system(I.FCC_CU_LIKE, (5, 5, 5), 0.05, 300.0, 12, n_knots=2000)
    _fd_check(s, atoms=range(0, 500, 29))


def test_virial_is_minus_strain_derivative():
    """W_aa = -dU/d(eps_aa) under the homogeneous strain x_a -> (1 + eps) x_a."""
    s = I.thermal_system(I.BCC_TA_LIKE, (5, 5, 5), 0.05, 300.0, 13, n_knots=2000)
    pot = O.Potential(s.pot)
    W = O.eam_eval(pot, s.pos, s.box, s.types)[4]
    h = 1e-6
    for a in range(3):
        scale = np.ones(3); scale[a] = 1 + h
        ep = _energy(pot, s.pos * scale, s.box * scale, s.types)
        scale[a] = 1 - h
        em = _energy(pot, s.pos * scale, s.box * scale, s.types)
        np.testing.assert_allclose(W[a], -(ep - em) / (2 * h), rtol=1e-6)


def test_translation_and_cubic_rotation_invariance():
    s = I.thermal_system(I.BCC_TA_LIKE, (5, 5, 5), 0.08, 300.0, 14, n_knots=2000)
    pot = O.Potential(s.pot)
    _, _, F, E, _ = O.eam_eval(pot, s.pos, s.box, s.types)
    shifted = O.wrap(s.pos + np.array([3.21, -7.7, 11.05]), s.box)
    _, _, F2, E2, _ = O.eam_eval(pot, shifted, s.box, s.types)
    np.testing.assert_allclose(F2, F, atol=1e-11)
    np.testing.assert_allclose(E2.sum(), E.sum(), rtol=1e-13)
    # 90 degree rotation about z of a cubic periodic box: (x, y) -> (L - y, x)
    L = s.box[0]
    rot = np.stack([L - s.pos[:, 1], s.pos[:, 0], s.pos[:, 2]], 1)
    _, _, F3, E3, _ = O.eam_eval(pot, O.wrap(rot, s.box), s.box, s.types)
    np.testing.assert_allclose(F3, np.stack([-F[:, 1], F[:, 0], F[:, 2]], 1), atol=1e-11)
    np.testing.assert_allclose(E3.sum(), E.sum(), rtol=1e-13)


def test_arbitrary_rotation_of_isolated_cluster():
    p = I.BCC_TA_LIKE
    rng = np.random.default_rng(15)
    pos, _ = I.bcc_lattice(3, 3, 3, p.a)
    pos = pos + rng.normal(0, 0.05, pos.shape)
    box = np.full(3, 40.0)
    pos = pos + 12.0
    pot = O.Potential(I.johnson_potential(p))
    types = np.zeros(len(pos), np.int32)
    _, _, F, E, W = O.eam_eval(pot, pos, box, types)
    q = rng.normal(size=4); q /= np.linalg.norm(q)
    a, b, c, d = q
    R = np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                  [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                  [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])
    ctr = pos.mean(0)
    pr = (pos - ctr) @ R.T + 20.0
    _, _, Fr, Er, Wr = O.eam_eval(pot, pr, box, types)
    np.testing.assert_allclose(Fr, F @ R.T, atol=1e-10)
    np.testing.assert_allclose(Er.sum(), E.sum(), rtol=1e-12)
    Wm = lambda w: np.array([[w[0], w[3], w[4]], [w[3], w[1], w[5]], [w[4], w[5], w[2]]])
    np.testing.assert_allclose(Wm(Wr), R @ Wm(W) @ R.T, atol=1e-9)
    # shear derivative on the isolated cluster: dU/d(eps) for x_a += eps x_b is -W_ab
    h = 1e-6
    for k, (ia, ib) in zip((3, 4, 5), ((0, 1), (0, 2), (1, 2))):
        def sheared(e):
            out = pos.copy(); out[:, ia] += e * (pos[:, ib] - ctr[ib])
            return out
        ep = _energy(pot, sheared(h), box, types)
        em = _energy(pot, sheared(-h), box, types)
        np.testing.assert_allclose(W[k], -(ep - em) / (2 * h), rtol=1e-5, atol=1e-8)


# --------------------------------------------------------------------------
# integrator (Eq. 5)


def _run(system, nsteps, dt):
    pot = O.Potential(system.pot)
    sysm = O.System(pot, system.box, system.pos, system.vel, system.types)
    return pot, sysm


def test_time_reversibility_and_momentum():
    s = I.thermal_system(I.BCC_TA_LIKE, (5, 5, 5), 0.02, 300.0, 16, n_knots=2000)
    pot = O.Potential(s.pot)
    fwd = O.System(pot, s.box, s.pos, s.vel, s.types)
    m = s.pot.mass[s.types]
    p0 = (m[:, None] * s.vel).sum(0)
    fwd.step(100, 2.0)
    st = fwd.state()
    assert st["rebuilds"] >= 10
    np.testing.assert_allclose((m[:, None] * st["vel"]).sum(0), p0, atol=1e-12)
    back = O.System(pot, s.box, st["pos"], -st["vel"], s.types)
    back.step(100, 2.0)
    end = back.state()
    d = end["pos"] - s.pos
    d -= s.box * np.round(d / s.box)
    assert np.abs(d).max() < 1e-9
    np.testing.assert_allclose(-end["vel"], s.vel, atol=1e-11)


def test_energy_error_scales_as_dt_squared():
    s = I.thermal_system(I.BCC_TA_LIKE, (5, 5, 5), 0.02, 600.0, 17, n_knots=2000)
    pot = O.Potential(s.pot)
    amp = []
    for dt, nsub in ((4.0, 1), (2.0, 2)):
        sysm = O.System(pot, s.box, s.pos, s.vel, s.types)
        e = []
        for _ in range(100):
            sysm.step(nsub, dt)
            pe, ke = sysm.energy()
            e.append(pe + ke)
        amp.append(np.ptp(e))
    ratio = amp[0] / amp[1]
    assert 3.0 < ratio < 5.0, ratio


def test_kinetic_energy_and_maxwell_temperature():
    s = I.bcc_2000_fp64()
    pot = O.Potential(s.pot)
    sysm = O.System(pot, s.box, s.pos, s.vel, s.types)
    _, ke = sysm.energy()
    t = 2 * ke / ((3 * s.n - 3) * I.KB_EV)
    np.testing.assert_allclose(t, 300.0, rtol=1e-12)
