"""Force and energy bars shared by the GPU parity tests.

Each force comparison against the oracle's F_ref is held to two measures:

* ``norm``: ||F - F_ref||_2 / ||F_ref||_2 over all 3N components (the error
  metric of the force parity statement: relative in the 2-norm);
* ``atom``: max_i |F_i - F_ref,i| / RMS_i |F_ref,i|, the worst single atom
  in units of the RMS atomic force, so that one wrong atom (or a handful of
  wrong boundary-cell atoms) cannot hide inside a global norm.

Bars, with where the per-atom figure comes from:

* FP64 path: norm 1e-10, atom 1e-9.
* mixed path (FP32 pair arithmetic, FP64 state and sums): norm 2e-5, atom
  1e-4.  The per-atom FP32 error of a force is a sum of ~14 independent pair
  rounding errors, close to an isotropic Gaussian vector.  The largest of N
  such 3-vector magnitudes exceeds their RMS by a factor m with
  P(chi2_3 > 3 m^2) ~ 1/N; at N = 8e5 atoms that gives m ~ 3.2.  A force
  field that just meets the norm bar therefore has its worst atom near
  3.2 x 2e-5 = 6.4e-5 of the RMS force; 1e-4 (5x the norm bar) leaves room
  for non-Gaussian tails and no room for a systematically wrong atom, whose
  error would be of the order of its whole force (~1).
"""
import numpy as np

BARS = {"fp64": (1e-10, 1e-9), "mixed": (2e-5, 1e-4)}


def rel_norm(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_atom(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).reshape(-1, 3)
    b = np.asarray(b, dtype=np.float64).reshape(-1, 3)
    rms = np.sqrt(np.mean(np.sum(b * b, axis=1)))
    return float(np.max(np.linalg.norm(a - b, axis=1)) / rms)


def assert_forces(f, f_ref, precision: str, what: str = "") -> None:
    """Both bars of ``precision`` ("fp64" or "mixed") on an (N, 3) force
    array against the oracle's."""
    norm_bar, atom_bar = BARS[precision]
    e_norm = rel_norm(f, f_ref)
    e_atom = max_atom(f, f_ref)
    assert e_norm < norm_bar, f"{what} force error {e_norm:.3e} (2-norm) >= {norm_bar:g} [{precision}]"
    assert e_atom < atom_bar, f"{what} worst-atom force error {e_atom:.3e} of RMS >= {atom_bar:g} [{precision}]"
