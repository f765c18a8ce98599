"""Pins of the oracle's force-matching gradient (the differentiation form):
the exact adjoint against central finite differences of the oracle's own
loss, and a special case with a closed route.  No GPU."""
import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import inputs as I


def small_problem(n_configs=3, n_knots=24, w=0.1, seed=11):
    prob = I.fit_problem(n_configs=n_configs, cells=(5, 5, 5), n_knots=n_knots, w=w, seed=seed)
    ref = O.Potential(I.johnson_potential(I.BCC_TA_LIKE))
    configs = []
    for pos, box in prob.configs:
        _, _, F, E, _ = O.eam_eval(ref, O.wrap(pos, box), box, np.zeros(len(pos), np.int32))
        configs.append((pos, box, E.sum(), F))
    return prob, configs


def loss_at(prob, configs, theta):
    pot = O.Potential(prob.potential(theta))
    return O.force_match_knot_grad(pot, configs, prob.w)[0]


def test_adjoint_matches_finite_differences():
    prob, configs = small_problem()
    theta = prob.theta0.copy()
    L, g = O.force_match_knot_grad(O.Potential(prob.potential(theta)), configs, prob.w)
    n = prob.n_knots
    fd = np.zeros_like(theta)
    # the clamped end slope is fixed; every knot value is a parameter except
    # the knots where a function is pinned to zero (the r_cut knots) -- those
    # are still parameters, checked like the others
    for k in range(theta.size):
        h = 1e-5 * max(abs(theta[k]), 1e-3)
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (loss_at(prob, configs, tp) - loss_at(prob, configs, tm)) / (2 * h)
    for q, name in enumerate(("phi", "f", "F")):
        sl = slice(q * n, (q + 1) * n)
        err = np.linalg.norm(g[sl] - fd[sl]) / np.linalg.norm(fd[sl])
        assert err < 1e-6, (name, err)
    assert np.linalg.norm(g - fd) / np.linalg.norm(fd) < 1e-6


def test_energy_only_gradient_for_embedding_knots_closed_route():
    """w = 0: E is affine in the F knots, so dL/dtheta^F_k =
    sum_c 2 (E_c - E_ref,c)/N_c sum_i S_k(rho_i), S_k the spline through the
    unit knot vector e_k (evaluated here with the oracle's own spline
    evaluation, not through the coefficient adjoint)."""
    prob, configs = small_problem(w=0.0)
    theta = prob.theta0
    pot = O.Potential(prob.potential(theta))
    _, g = O.force_match_knot_grad(pot, configs, 0.0)
    n = prob.n_knots
    Fk = prob.potential(theta).F[0]
    expect = np.zeros(n)
    for pos, box, e_ref, f_ref in configs:
        rho, _, _, E, _ = O.eam_eval(pot, O.wrap(pos, box), box, np.zeros(len(pos), np.int32))
        A = 2 * (E.sum() - e_ref) / len(pos)
        for k in range(n):
            unit = I.Knots(Fk.x0, Fk.dx, np.eye(n)[k], Fk.bc_lo, Fk.bc_hi)
            val, _, _ = O.spline_eval(unit, O.spline_coeffs(unit), rho)
            expect[k] += A * val.sum()
    np.testing.assert_allclose(g[2 * n:], expect, rtol=1e-10, atol=1e-12 * np.abs(expect).max())


def test_loss_is_zero_at_the_reference_potential_tables():
    """With theta = the reference knots on the reference grid the loss and the
    gradient vanish (same tables produce the same energies and forces)."""
    prob = I.fit_problem(n_configs=2, cells=(5, 5, 5), n_knots=2000, seed=5)
    ref = O.Potential(I.johnson_potential(I.BCC_TA_LIKE))
    configs = []
    for pos, box in prob.configs:
        _, _, F, E, _ = O.eam_eval(ref, O.wrap(pos, box), box, np.zeros(len(pos), np.int32))
        configs.append((pos, box, E.sum(), F))
    F, f, phi = I.johnson_knots(I.BCC_TA_LIKE, 2000)
    theta = np.concatenate([phi.y, f.y, F.y])
    L, g = O.force_match_knot_grad(O.Potential(prob.potential(theta)), configs, 0.1)
    assert L < 1e-24
    assert np.abs(g).max() < 1e-10
