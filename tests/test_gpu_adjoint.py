"""The differentiation form on the GPU: md_force_match (through the C ABI)
against the oracle's exact adjoint, against finite differences of the GPU
loss, bitwise reproducibility, and the torch.autograd.Function."""
import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import autodiff, binding, inputs as I
from bars import assert_forces

pytestmark = pytest.mark.gpu


def oracle_loss_grad(prob, theta, refs):
    pot = O.Potential(prob.potential(theta))
    configs = [(pos, box, e, f) for (pos, box), (e, f) in zip(prob.configs, refs)]
    return O.force_match_knot_grad(pot, configs, prob.w)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def small():
    prob = I.fit_problem(n_configs=4, cells=(6, 6, 6), n_knots=24, w=0.1, seed=21)
    fm = autodiff.ForceMatch(prob)
    yield prob, fm
    fm.close()


def test_references_match_oracle(small):
    prob, fm = small
    ref = O.Potential(I.johnson_potential(I.BCC_TA_LIKE))
    for (pos, box), (e, f) in zip(prob.configs, fm.refs):
        _, _, F, E, _ = O.eam_eval(ref, O.wrap(pos, box), box, np.zeros(len(pos), np.int32))
        assert abs(e - E.sum()) / abs(E.sum()) < 1e-10
        assert_forces(f, F, "fp64")


def test_gradient_matches_oracle_adjoint(small):
    prob, fm = small
    L, g = fm.evaluate(prob.theta0)
    Lo, go = oracle_loss_grad(prob, prob.theta0, fm.refs)
    assert abs(L - Lo) / abs(Lo) < 1e-9
    n = prob.n_knots
    for q in range(3):
        assert rel(g[q * n:(q + 1) * n], go[q * n:(q + 1) * n]) < 1e-9


def test_gradient_matches_finite_differences(small):
    prob, fm = small
    theta = prob.theta0.copy()
    _, g = fm.evaluate(theta)
    rng = np.random.default_rng(3)
    ks = rng.choice(theta.size, size=18, replace=False)
    fd = []
    for k in ks:
        h = 1e-5 * max(abs(theta[k]), 1e-3)
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd.append((fm.evaluate(tp, grad=False)[0] - fm.evaluate(tm, grad=False)[0]) / (2 * h))
    fd = np.array(fd)
    assert np.linalg.norm(g[ks] - fd) / np.linalg.norm(fd) < 1e-6


def test_gradient_is_bitwise_reproducible(small):
    prob, fm = small
    theta = prob.theta0 * 1.001
    a = fm.evaluate(theta)
    b = fm.evaluate(theta.copy() * 1.0)
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1], b[1])


def test_autograd_function(small):
    torch = pytest.importorskip("torch")
    prob, fm = small
    n = prob.n_knots
    t = torch.tensor(prob.theta0, dtype=torch.float64)
    tp, tf, tF = (t[:n].clone().requires_grad_(), t[n:2 * n].clone().requires_grad_(),
                  t[2 * n:].clone().requires_grad_())
    loss = autodiff.EAMKnotLoss.apply(tp, tf, tF, fm)
    (3.0 * loss).backward()
    L, g = fm.evaluate(prob.theta0)
    assert abs(loss.item() - L) <= 1e-12 * abs(L)
    got = torch.cat([tp.grad, tf.grad, tF.grad]).numpy()
    np.testing.assert_allclose(got, 3.0 * g, rtol=1e-12, atol=0)


def test_full_size_64_configs_against_oracle():
    """The benchmarked size: 64 BCC configurations of 2,000 atoms (three with
    a vacancy), 3 x 64 knots, w = 0.1."""
    prob = I.fit_problem()
    assert sorted({len(p) for p, _ in prob.configs}) == [1999, 2000]
    fm = autodiff.ForceMatch(prob)
    try:
        L, g = fm.evaluate(prob.theta0)
        Lo, go = oracle_loss_grad(prob, prob.theta0, fm.refs)
        assert abs(L - Lo) / abs(Lo) < 1e-9
        assert rel(g, go) < 1e-9
    finally:
        fm.close()


def test_set_potential_keeps_grids():
    s = I.bcc_2000_fp64()
    with binding.MD(s, precision="fp64") as md:
        other = I.johnson_potential(I.BCC_TA_LIKE, n_knots=1000)
        with pytest.raises(binding.MDError):
            md.set_potential(other)
        # same grids, scaled values: forces scale with phi and change with f
        p2 = I.johnson_potential(I.BCC_TA_LIKE)
        p2.phi[0].y = p2.phi[0].y * 1.1
        md.set_potential(p2)
        _, _, F, _, _ = O.eam_eval(O.Potential(p2), O.wrap(s.pos, s.box), s.box, s.types)
        assert_forces(md.forces(), F, "fp64")


def test_worker_threads_give_the_same_loss_and_gradient():
    """Configurations spread over worker contexts (own streams, host
    threads) and summed in configuration order: loss and gradient bitwise
    those of one context."""
    prob = I.fit_problem(n_configs=7, cells=(6, 6, 6), n_knots=24, w=0.1, seed=23)
    theta = prob.theta0 * (1.0 + 0.01 * np.sin(np.arange(len(prob.theta0))))
    out = []
    for workers in (1, 3):
        fm = autodiff.ForceMatch(prob, workers=workers)
        out.append(fm.evaluate(theta, grad=True))
        out.append(fm.evaluate(prob.theta0, grad=True))
        fm.close()
    assert out[0][0] == out[2][0] and out[1][0] == out[3][0]
    np.testing.assert_array_equal(out[0][1], out[2][1])
    np.testing.assert_array_equal(out[1][1], out[3][1])
