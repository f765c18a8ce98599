"""The linear time model of the paper's Eq. 6 fitted to GB300 timings.

The paper writes the time of one timestep on a wafer core as a cost per
candidate examined, a cost per interaction evaluated and a fixed cost
(Eq. 6, Table "regression").  The GPU counterpart fits per-atom times of the
pair passes against list entries and interactions per atom, and of the list
build against candidates and list entries per atom, by least squares over a
grid of (r_cut, skin) settings that vary those counts independently
(`bench.py --workload model` measures the points).

This module holds only the host-side arithmetic of the fit, so that it can
be checked on synthetic points with known coefficients.
"""
from __future__ import annotations

import numpy as np


def fit_linear(x_rows, y):
    """Least-squares fit y ~ sum_k c_k x_k + c_0 over the rows of x_rows
    (each row the regressors of one point, without the constant).  Returns
    (coefficients [c_1, ..., c_m, c_0], r^2)."""
    X = np.asarray(x_rows, dtype=np.float64)
    if X.ndim != 2:
        raise ValueError("x_rows must be a 2-D array of regressors")
    y = np.asarray(y, dtype=np.float64)
    if X.shape[0] != y.shape[0] or X.shape[0] < X.shape[1] + 1:
        raise ValueError("need at least one more point than regressors")
    A = np.hstack([X, np.ones((X.shape[0], 1))])
    c, *_ = np.linalg.lstsq(A, y, rcond=None)
    pred = A @ c
    ss_res = float(((y - pred) ** 2).sum())
    ss_tot = float(((y - y.mean()) ** 2).sum())
    r2 = 1.0 - ss_res / ss_tot if ss_tot > 0 else 1.0
    return [float(v) for v in c], r2


def fit_points(points):
    """The four fits of the model from measured points (dicts with n_list,
    n_inter, n_cand and the per-atom times in ns): pair passes, density and
    force against (list entries, interactions); list build against
    (candidates, list entries)."""
    pair_x = [[p["n_list"], p["n_inter"]] for p in points]
    build_x = [[p["n_cand"], p["n_list"]] for p in points]
    out = {}
    for name, key in (("pair_passes", "pair_ns_per_atom"), ("density", "density_ns_per_atom"),
                      ("force", "force_ns_per_atom")):
        (a, b, c), r2 = fit_linear(pair_x, [p[key] for p in points])
        out[name] = {"per_list_entry": a, "per_interaction": b, "fixed": c, "r2": r2}
    (a, b, c), r2 = fit_linear(build_x, [p["build_ns_per_atom"] for p in points])
    out["list_build"] = {"per_candidate": a, "per_list_entry": b, "fixed": c, "r2": r2}
    return out
