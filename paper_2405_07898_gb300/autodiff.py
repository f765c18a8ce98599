"""The differentiation form: gradients of a force-matching loss with respect
to the spline knots of phi, f and F, behind a torch.autograd.Function.

    L(theta) = sum_c [ (E_c - E_ref,c)^2 / N_c + w sum_i |F_c,i - F_ref,c,i|^2 ]

theta = (phi knots, f knots, F knots) on fixed grids.  E_c, F_c are the EAM
energy (Eq. 3) and forces (Eq. 4) of configuration c under the splines
through theta; the references come from the same library evaluated with the
reference potential.  Every number is computed by the CUDA library
(md_set_state, md_set_potential, md_force_match); this module only loops over
configurations and moves arrays.  The forward pass evaluates the loss; the
backward pass runs the adjoint kernels, which recompute the densities rather
than keep per-pair terms from the forward pass.
"""
from __future__ import annotations

import numpy as np

from . import binding
from . import inputs as I


class ForceMatch:
    """Loss and knot gradient over a set of single-type configurations.

    workers: contexts per configuration size, each on its own stream and
    host thread, so that the small kernels of several configurations share
    the GPU; per-configuration results are summed in configuration order, so
    the loss and gradient do not depend on the number of workers."""

    def __init__(self, problem: I.FitProblem, reference: I.Potential | None = None, workers: int = 4):
        self.problem = problem
        self.w = problem.w
        n = problem.n_knots
        self.sizes = (n, n, n)
        self.workers = max(1, int(workers))
        ref_pot = reference if reference is not None else I.johnson_potential(problem.params)
        self._ref_ctx = {}
        self._ctx = {}
        self.refs = []
        theta0 = problem.theta0
        pot0 = problem.potential(theta0)
        for pos, box in problem.configs:
            m = pos.shape[0]
            if m not in self._ref_ctx:
                self._ref_ctx[m] = binding.MD(self._system(pos, box, ref_pot), precision="fp64")
                self._ctx[m] = [binding.MD(self._system(pos, box, pot0), precision="fp64")
                                for _ in range(self.workers)]
            ref = self._ref_ctx[m]
            ref.set_state(pos, None, 0)
            e_ref = ref.energy()[0]  # potential energy
            self.refs.append((e_ref, ref.forces().copy()))
        for c in self._ref_ctx.values():
            c.close()
        self._ref_ctx = {}
        self._pool = None
        if self.workers > 1:
            from concurrent.futures import ThreadPoolExecutor
            self._pool = ThreadPoolExecutor(max_workers=self.workers)
        self._theta = theta0.copy()

    @staticmethod
    def _system(pos, box, pot):
        m = pos.shape[0]
        return I.System(box=np.asarray(box, dtype=np.float64), pos=pos, vel=np.zeros_like(pos),
                        types=np.zeros(m, np.int32), pot=pot)

    def _set_theta(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        if np.array_equal(theta, self._theta):
            return
        pot = self.problem.potential(theta)
        for cs in self._ctx.values():
            for c in cs:
                c.set_potential(pot)
        self._theta = theta.copy()

    def _run(self, worker: int, grad: bool):
        """Configurations worker, worker + workers, ... on that worker's
        contexts: {index: (loss, gradient)}."""
        out = {}
        for k in range(worker, len(self.refs), self.workers):
            pos, _ = self.problem.configs[k]
            e_ref, f_ref = self.refs[k]
            ctx = self._ctx[pos.shape[0]][worker]
            ctx.set_state(pos, None, 0)
            out[k] = ctx.force_match(f_ref, e_ref, self.w, grad=grad)
        return out

    def evaluate(self, theta, grad: bool = True):
        """(L, dL/dtheta or None)."""
        self._set_theta(theta)
        if self._pool is None:
            parts = [self._run(0, grad)]
        else:
            parts = list(self._pool.map(lambda wk: self._run(wk, grad), range(self.workers)))
        results = {}
        for p in parts:
            results.update(p)
        total = 0.0
        g = np.zeros(sum(self.sizes)) if grad else None
        for k in range(len(self.refs)):  # configuration order
            loss, gc = results[k]
            total += loss
            if grad:
                g += gc
        return total, g

    def close(self):
        if self._pool is not None:
            self._pool.shutdown()
            self._pool = None
        for cs in self._ctx.values():
            for c in cs:
                c.close()
        self._ctx = {}


def _torch():
    import torch
    return torch


class EAMKnotLoss:
    """torch.autograd.Function factory: EAMKnotLoss.apply(theta_phi, theta_f,
    theta_F, force_match) -> scalar loss tensor (float64, CPU)."""

    _fn = None

    @classmethod
    def function(cls):
        if cls._fn is None:
            torch = _torch()

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, theta_phi, theta_f, theta_F, fm: ForceMatch):
                    theta = torch.cat([theta_phi, theta_f, theta_F]).detach().cpu().double().numpy()
                    loss, _ = fm.evaluate(theta, grad=False)
                    ctx.fm = fm
                    ctx.save_for_backward(theta_phi, theta_f, theta_F)
                    return torch.tensor(loss, dtype=torch.float64)

                @staticmethod
                def backward(ctx, grad_out):
                    theta_phi, theta_f, theta_F = ctx.saved_tensors
                    theta = torch.cat([theta_phi, theta_f, theta_F]).detach().cpu().double().numpy()
                    _, g = ctx.fm.evaluate(theta, grad=True)
                    g = torch.from_numpy(g) * grad_out.detach().cpu().double()
                    n1, n2 = theta_phi.numel(), theta_f.numel()
                    return (g[:n1].to(theta_phi), g[n1:n1 + n2].to(theta_f), g[n1 + n2:].to(theta_F), None)

            cls._fn = _Fn
        return cls._fn

    @classmethod
    def apply(cls, theta_phi, theta_f, theta_F, fm: ForceMatch):
        return cls.function().apply(theta_phi, theta_f, theta_F, fm)
