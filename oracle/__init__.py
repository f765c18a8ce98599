"""Python view of the serial FP64 CPU oracle (`oracle/eam_oracle.c`).

TEST INFRASTRUCTURE: only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this package.  It never imports the
CUDA package, and the CUDA package never imports it; both take their inputs
from `paper_2405_07898_gb300.inputs`.

Each wrapper names the part of the paper its C function follows:
Eq. 2 (density), Eq. 3 (energy), Eq. 4 (force), Eq. 5 (integration, as
kick-drift-kick), Section "Neighbor list" (r^2 < r_list^2 filter) and
Section "Periodic Boundary Conditions" (wrap and minimum image).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eam_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)


def _compile(out: str, extra, force: bool) -> str:
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", *extra, "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction: every operation is
    rounded as written; one thread).  This is the build every parity test
    uses."""
    return _compile(_LIB, [], force)


def build_omp(force: bool = False) -> str:
    """The same source built with OpenMP, used only to time the oracle on all
    host cores (its per-atom loops run in parallel; sums over atoms are taken
    in another order, so its energies may differ from build() in rounding)."""
    return _compile(_LIB_OMP, ["-fopenmp"], force)


class _Knots(C.Structure):
    _fields_ = [("n", C.c_int32), ("x0", C.c_double), ("dx", C.c_double), ("y", _dp),
                ("bc_lo", C.c_int32), ("bc_hi", C.c_int32), ("d_lo", C.c_double),
                ("d_hi", C.c_double)]


_lib = None
_lib_omp = None


def lib():
    """The parity build (one thread)."""
    global _lib
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def lib_omp():
    """The all-cores timing build (see build_omp)."""
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = _declare(C.CDLL(build_omp()))
    return _lib_omp


def _declare(L):
    """Argument and result types of the oracle's C functions on library L."""
    L.orc_spline_coeffs.argtypes = [C.c_int32, C.c_double, _dp, C.c_int32, C.c_double,
                                    C.c_int32, C.c_double, _dp]
    L.orc_spline_coeffs.restype = C.c_int
    L.orc_spline_eval.argtypes = [C.c_int32, C.c_double, C.c_double, _dp, C.c_double, _dp, _dp]
    L.orc_spline_eval.restype = C.c_double
    L.orc_pot_create.argtypes = [C.c_int32, _dp, C.POINTER(_Knots), C.POINTER(_Knots),
                                 C.POINTER(_Knots), C.c_double, C.c_double]
    L.orc_pot_create.restype = C.c_void_p
    L.orc_pot_destroy.argtypes = [C.c_void_p]
    L.orc_wrap.argtypes = [C.c_int64, _dp, C.c_int, _dp]
    L.orc_cell_dims.argtypes = [_dp, C.c_int, C.c_double, _ip]
    L.orc_cell_dims.restype = C.c_int
    L.orc_cells.argtypes = [C.c_int64, _dp, C.c_int, C.c_double, _dp, _ip, _ip]
    L.orc_cells.restype = C.c_int
    for name in ("orc_list_cells", "orc_list_brute"):
        fn = getattr(L, name)
        fn.argtypes = [C.c_int64, _dp, C.c_int, C.c_double, _dp, _lp, _ip, C.c_int64]
        fn.restype = C.c_int64
    L.orc_eam_eval.argtypes = [C.c_void_p, C.c_int64, _dp, C.c_int, _dp, _ip, _lp, _ip, _dp, _dp, _dp,
                               _dp, _dp]
    L.orc_eam_eval.restype = C.c_int
    L.orc_density.argtypes = [C.c_void_p, C.c_int64, _dp, C.c_int, _dp, _ip, _lp, _ip, _dp, _dp]
    L.orc_density.restype = C.c_double
    L.orc_force_given_fp.argtypes = [C.c_void_p, C.c_int64, _dp, C.c_int, _dp, _ip, _lp, _ip, _dp, _dp, _dp]
    L.orc_force_given_fp.restype = C.c_double
    L.orc_sys_create.argtypes = [C.c_void_p, C.c_int64, _dp, C.c_int, _dp, _dp, _ip]
    L.orc_sys_create.restype = C.c_void_p
    L.orc_sys_destroy.argtypes = [C.c_void_p]
    L.orc_sys_step.argtypes = [C.c_void_p, C.c_int64, C.c_double, C.c_int32]
    L.orc_sys_step.restype = C.c_int
    L.orc_sys_energy.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_sys_virial.argtypes = [C.c_void_p, _dp]
    L.orc_sys_get.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, _dp, _lp]
    L.orc_spline_basis.argtypes = [C.c_int32, C.c_double, C.c_int32, C.c_int32, _dp]
    L.orc_spline_basis.restype = C.c_int
    L.orc_force_match.argtypes = [C.c_void_p, C.c_int64, _dp, C.c_int, _dp, C.c_double, _dp, C.c_double,
                                  _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_force_match.restype = C.c_int
    return L


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def _l(a):
    return a.ctypes.data_as(_lp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# splines


def spline_coeffs(knots) -> np.ndarray:
    """Per-interval cubic coefficients (a, b, c, d) of the C2 spline through
    `knots` (an `inputs.Knots`), shape (n-1, 4)."""
    y = _f64(knots.y)
    out = np.zeros((knots.n - 1, 4))
    rc = lib().orc_spline_coeffs(knots.n, knots.dx, _d(y), knots.bc_lo, knots.d_lo, knots.bc_hi,
                                 knots.d_hi, _d(out))
    if rc:
        raise ValueError("bad spline knots")
    return out


def spline_eval(knots, coef, x):
    """Value, first and second derivative of the spline at each x."""
    coef = _f64(coef)
    x = np.atleast_1d(_f64(x))
    val = np.empty_like(x)
    der = np.empty_like(x)
    der2 = np.empty_like(x)
    dy = C.c_double()
    d2y = C.c_double()
    for k, xv in enumerate(x):
        val[k] = lib().orc_spline_eval(knots.n, knots.x0, knots.dx, _d(coef), float(xv),
                                       C.byref(dy), C.byref(d2y))
        der[k] = dy.value
        der2[k] = d2y.value
    return val, der, der2


# --------------------------------------------------------------------------
# potential, geometry, evaluation


class Potential:
    """Owns the oracle's own coefficient tables for an `inputs.Potential`.
    `L`: the oracle library to build them in (default the parity build)."""

    def __init__(self, pot, L=None):
        self.src = pot
        self._keep = []
        self.L = L if L is not None else lib()

        def arr(ks):
            out = (_Knots * len(ks))()
            for q, k in enumerate(ks):
                y = _f64(k.y)
                self._keep.append(y)
                out[q] = _Knots(k.n, k.x0, k.dx, _d(y), k.bc_lo, k.bc_hi, k.d_lo, k.d_hi)
            return out

        self._mass = _f64(pot.mass)
        F, f, phi = arr(pot.F), arr(pot.f), arr(pot.phi)
        self.handle = self.L.orc_pot_create(pot.ntypes, _d(self._mass), F, f, phi, pot.r_cut, pot.skin)
        if not self.handle:
            raise ValueError("oracle could not build the potential")
        self.r_cut = pot.r_cut
        self.skin = pot.skin
        self.r_list = pot.r_cut + pot.skin

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and getattr(self, "L", None) is not None:
            self.L.orc_pot_destroy(h)
            self.handle = None


# `open_axes`: one bit per open (non-periodic) axis, 1: x, 2: y, 4: z.


def wrap(pos, box, open_axes: int = 0):
    out = _f64(pos).copy()
    lib().orc_wrap(out.shape[0], _d(_f64(box)), int(open_axes), _d(out))
    return out


def cell_dims(box, r_list, open_axes: int = 0):
    nc = np.zeros(3, dtype=np.int32)
    if lib().orc_cell_dims(_d(_f64(box)), int(open_axes), r_list, _i(nc)):
        raise ValueError("box shorter than 3 r_list along a periodic axis (r_list along an open one)")
    return nc


def cells(pos, box, r_list, open_axes: int = 0):
    """(ncell, cell_start, cell_atoms) for wrapped positions."""
    nc = cell_dims(box, r_list, open_axes)
    ncells = int(np.prod(nc.astype(np.int64)))
    start = np.zeros(ncells + 1, dtype=np.int32)
    atoms = np.zeros(max(pos.shape[0], 1), dtype=np.int32)
    pos = _f64(pos)
    if lib().orc_cells(pos.shape[0], _d(_f64(box)), int(open_axes), r_list, _d(pos), _i(start), _i(atoms)):
        raise ValueError("cells failed")
    return nc, start, atoms[: pos.shape[0]]


def _list(fn, pos, box, r_list, open_axes):
    pos = _f64(pos)
    n = pos.shape[0]
    off = np.zeros(n + 1, dtype=np.int64)
    cap = max(64 * n, 1)
    while True:
        js = np.zeros(cap, dtype=np.int32)
        m = fn(n, _d(_f64(box)), int(open_axes), r_list, _d(pos), _l(off), _i(js), cap)
        if m < 0:
            raise ValueError("neighbour list failed")
        if m <= cap:
            return off, js[:m]
        cap = int(m)


def neighbors_cells(pos, box, r_list, open_axes: int = 0):
    """CSR neighbour list from the 27-cell stencil (positions wrapped)."""
    return _list(lib().orc_list_cells, pos, box, r_list, open_axes)


def neighbors_brute(pos, box, r_list, open_axes: int = 0):
    """CSR neighbour list by testing all pairs."""
    return _list(lib().orc_list_brute, pos, box, r_list, open_axes)


def eam_eval(pot: Potential, pos, box, types, off=None, js=None, open_axes: int = 0):
    """rho, F', forces, (E_embed, E_pair), virial (xx,yy,zz,xy,xz,yz) at pos."""
    pos = _f64(pos)
    n = pos.shape[0]
    types = np.ascontiguousarray(types, dtype=np.int32)
    if off is None:
        off, js = neighbors_cells(wrap(pos, box, open_axes), box, pot.r_list, open_axes)
    rho = np.zeros(n)
    Fp = np.zeros(n)
    force = np.zeros((n, 3))
    energy = np.zeros(2)
    virial = np.zeros(6)
    js = np.ascontiguousarray(js, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    lib().orc_eam_eval(pot.handle, n, _d(_f64(box)), int(open_axes), _d(pos), _i(types), _l(off), _i(js),
                       _d(rho), _d(Fp), _d(force), _d(energy), _d(virial))
    return rho, Fp, force, energy, virial


def density_pass(pot: Potential, pos, box, types, open_axes: int = 0):
    """rho and F' of every atom (Eq. 2) over the 27-cell list of `pos`."""
    pos = _f64(pos)
    n = pos.shape[0]
    off, js = neighbors_cells(pos, box, pot.r_list, open_axes)
    rho = np.zeros(n)
    Fp = np.zeros(n)
    types = np.ascontiguousarray(types, dtype=np.int32)
    pot.L.orc_density(pot.handle, n, _d(_f64(box)), int(open_axes), _d(pos), _i(types), _l(off),
                      _i(np.ascontiguousarray(js, dtype=np.int32)), _d(rho), _d(Fp))
    return rho, Fp


def force_pass(pot: Potential, pos, box, types, Fp, open_axes: int = 0):
    """Forces of Eq. 4 with F' given for every atom."""
    pos = _f64(pos)
    n = pos.shape[0]
    off, js = neighbors_cells(pos, box, pot.r_list, open_axes)
    force = np.zeros((n, 3))
    vir = np.zeros(6)
    types = np.ascontiguousarray(types, dtype=np.int32)
    pot.L.orc_force_given_fp(pot.handle, n, _d(_f64(box)), int(open_axes), _d(pos), _i(types), _l(off),
                             _i(np.ascontiguousarray(js, dtype=np.int32)), _d(_f64(Fp)), _d(force), _d(vir))
    return force


class System:
    """Serial FP64 molecular dynamics of one system (periodic, or open along
    the axes of `open_axes`)."""

    def __init__(self, pot: Potential, box, pos, vel, types, open_axes: int = 0):
        self.pot = pot
        self.L = pot.L
        self.n = int(pos.shape[0])
        self._box = _f64(box)
        pos = _f64(pos)
        vel = _f64(vel) if vel is not None else np.zeros_like(pos)
        types = np.ascontiguousarray(types, dtype=np.int32)
        self.handle = self.L.orc_sys_create(pot.handle, self.n, _d(self._box), int(open_axes), _d(pos),
                                            _d(vel), _i(types))
        if not self.handle:
            raise ValueError("oracle system create failed (box < 3 r_list?)")

    def step(self, nsteps: int, dt: float, rebuild_every: int = 10):
        rc = self.L.orc_sys_step(self.handle, nsteps, dt, rebuild_every)
        if rc:
            raise RuntimeError(f"oracle step failed ({rc})")

    def energy(self):
        pe, ke = C.c_double(), C.c_double()
        self.L.orc_sys_energy(self.handle, C.byref(pe), C.byref(ke))
        return pe.value, ke.value

    def virial(self):
        w = np.zeros(6)
        self.L.orc_sys_virial(self.handle, _d(w))
        return w

    def state(self):
        pos = np.zeros((self.n, 3))
        vel = np.zeros((self.n, 3))
        force = np.zeros((self.n, 3))
        rho = np.zeros(self.n)
        Fp = np.zeros(self.n)
        cnt = np.zeros(2, dtype=np.int64)
        self.L.orc_sys_get(self.handle, _d(pos), _d(vel), _d(force), _d(rho), _d(Fp), _l(cnt))
        return dict(pos=pos, vel=vel, force=force, rho=rho, Fp=Fp, step=int(cnt[0]),
                    rebuilds=int(cnt[1]))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and getattr(self, "L", None) is not None:
            self.L.orc_sys_destroy(h)
            self.handle = None


# --------------------------------------------------------------------------
# differentiation (force matching)


def spline_basis(knots) -> np.ndarray:
    """M with coefficients = M @ y (+ the end-slope part): shape (4(n-1), n)."""
    M = np.zeros((4 * (knots.n - 1), knots.n))
    rc = lib().orc_spline_basis(knots.n, knots.dx, knots.bc_lo, knots.bc_hi, _d(M))
    if rc:
        raise ValueError("spline basis failed")
    return M


def force_match(pot: Potential, pos, box, e_ref: float, f_ref, w: float, open_axes: int = 0):
    """Loss (E - E_ref)^2/N + w sum |F - F_ref|^2 of one single-type
    configuration and dL/d(coefficients) of phi, f, F (each (n-1, 4)); also
    returns E and F."""
    pos = _f64(pos)
    n = pos.shape[0]
    src = pot.src
    g_phi = np.zeros((src.phi[0].n - 1, 4))
    g_f = np.zeros((src.f[0].n - 1, 4))
    g_F = np.zeros((src.F[0].n - 1, 4))
    loss = C.c_double()
    e = C.c_double()
    force = np.zeros((n, 3))
    rc = lib().orc_force_match(pot.handle, n, _d(_f64(box)), int(open_axes), _d(pos), float(e_ref),
                               _d(_f64(f_ref)),
                               float(w), C.byref(loss), _d(g_phi), _d(g_f), _d(g_F), C.byref(e),
                               _d(force))
    if rc:
        raise RuntimeError(f"force_match failed ({rc})")
    return loss.value, (g_phi, g_f, g_F), e.value, force


def force_match_knot_grad(pot: Potential, configs, w: float):
    """Total loss over configs [(pos, box, e_ref, f_ref)] and its gradient
    with respect to the knot values of phi, f and F (concatenated in that
    order): the coefficient gradient mapped through M^T."""
    src = pot.src
    Ms = [spline_basis(src.phi[0]), spline_basis(src.f[0]), spline_basis(src.F[0])]
    total = 0.0
    gk = [np.zeros(src.phi[0].n), np.zeros(src.f[0].n), np.zeros(src.F[0].n)]
    for pos, box, e_ref, f_ref in configs:
        loss, gc, _, _ = force_match(pot, pos, box, e_ref, f_ref, w)
        total += loss
        for q in range(3):
            gk[q] += Ms[q].T @ gc[q].ravel()
    return total, np.concatenate(gk)
