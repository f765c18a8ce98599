"""ctypes binding of the C ABI in include/eammd.h (argument marshalling only;
every step of the method runs in the CUDA library).

PyTorch supplies device memory (its caching allocator, through the
md_options alloc/free callbacks) and the CUDA stream (its current stream).
The library must be built (`paper_2405_07898_gb300.build.build()`); loading
fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)

MD_OK = 0
STATUS = {0: "MD_OK", -1: "MD_ERR_ARG", -2: "MD_ERR_BOX", -3: "MD_ERR_CUDA", -4: "MD_ERR_OOM",
          -5: "MD_ERR_NONFINITE", -6: "MD_ERR_TIMEOUT", -7: "MD_ERR_LIST_OVERFLOW",
          -8: "MD_ERR_CAPACITY"}
PRECISION = {"fp64": 0, "mixed": 1}
PERSIST = {"auto": 0, "off": 1, "on": 2}

# every entry point declared in include/eammd.h
EXPORTS = ("md_options_default", "md_create", "md_step", "md_sync", "md_energy", "md_forces",
           "md_virial", "md_get_state", "md_set_state", "md_neighbors", "md_cells", "md_stats",
           "md_profile", "md_last_error", "md_destroy", "md_bin_cells_noalloc", "md_set_potential",
           "md_force_match", "md_batch_create", "md_batch_step", "md_batch_energy", "md_batch_get_state",
           "md_batch_info", "md_batch_last_error", "md_batch_destroy")

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Spline(C.Structure):
    _fields_ = [("n", C.c_int32), ("x0", C.c_double), ("dx", C.c_double), ("y", _dp),
                ("bc_lo", C.c_int32), ("bc_hi", C.c_int32), ("d_lo", C.c_double),
                ("d_hi", C.c_double)]


class PotentialC(C.Structure):
    _fields_ = [("ntypes", C.c_int32), ("mass", _dp), ("F", C.POINTER(Spline)),
                ("f", C.POINTER(Spline)), ("phi", C.POINTER(Spline)), ("r_cut", C.c_double),
                ("skin", C.c_double)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("rebuild_every", C.c_int32),
                ("list_capacity", C.c_int32), ("use_graphs", C.c_int32),
                ("block_size", C.c_int32), ("lanes_per_atom", C.c_int32),
                ("cuda_stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p),
                ("persistent", C.c_int32),
                ("wait_limit_us", C.c_int32),
                ("open_axes", C.c_int32),
                ("batch_schedule", C.c_int32),
                ("half_list", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("rebuilds", C.c_int64), ("max_neighbors", C.c_int32),
                ("list_capacity", C.c_int32), ("table_out_of_range", C.c_int64),
                ("kernel_launches", C.c_int64), ("lanes_density", C.c_int32),
                ("lanes_force", C.c_int32), ("threads_density", C.c_int32),
                ("threads_force", C.c_int32), ("persistent_blocks", C.c_int32),
                ("persistent_lanes", C.c_int32), ("half_list", C.c_int32), ("record_textures", C.c_int32)]


class Profile(C.Structure):
    _fields_ = [("density_ms", C.c_double), ("force_ms", C.c_double), ("rebuild_ms", C.c_double),
                ("step_ms", C.c_double), ("density_launches", C.c_int64),
                ("force_launches", C.c_int64), ("rebuilds", C.c_int64)]


class Replica(C.Structure):
    _fields_ = [("n", C.c_int64), ("box", C.c_double * 3), ("pos", _dp), ("vel", _dp),
                ("potential", C.c_int32), ("reserved", C.c_int32)]


class BatchInfo(C.Structure):
    _fields_ = [("replicas", C.c_int32), ("blocks", C.c_int32), ("threads_per_block", C.c_int32),
                ("list_capacity", C.c_int32), ("atoms", C.c_int64), ("steps", C.c_int64),
                ("rebuilds", C.c_int64), ("kernel_launches", C.c_int64), ("max_neighbors", C.c_int32),
                ("reserved", C.c_int32)]


class MDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libeammd.so (building it first if asked and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing")
    L = C.CDLL(path)
    L.md_options_default.argtypes = [C.POINTER(Options)]
    L.md_options_default.restype = None
    L.md_create.argtypes = [_dp, C.c_int64, _dp, _dp, _ip, C.POINTER(PotentialC), C.POINTER(Options),
                            C.POINTER(C.c_void_p)]
    L.md_create.restype = C.c_int
    L.md_step.argtypes = [C.c_void_p, C.c_int64, C.c_double]
    L.md_step.restype = C.c_int
    L.md_sync.argtypes = [C.c_void_p]
    L.md_sync.restype = C.c_int
    L.md_energy.argtypes = [C.c_void_p, _dp, _dp]
    L.md_energy.restype = C.c_int
    L.md_forces.argtypes = [C.c_void_p, _dp]
    L.md_forces.restype = C.c_int
    L.md_virial.argtypes = [C.c_void_p, _dp]
    L.md_virial.restype = C.c_int
    L.md_get_state.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, _lp]
    L.md_get_state.restype = C.c_int
    L.md_set_state.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
    L.md_set_state.restype = C.c_int
    L.md_neighbors.argtypes = [C.c_void_p, _lp, _ip, C.c_int64]
    L.md_neighbors.restype = C.c_int
    L.md_cells.argtypes = [C.c_void_p, _ip, _ip, _ip]
    L.md_cells.restype = C.c_int
    L.md_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
    L.md_stats.restype = C.c_int
    L.md_profile.argtypes = [C.c_void_p, C.c_int64, C.c_double, C.POINTER(Profile)]
    L.md_profile.restype = C.c_int
    L.md_last_error.argtypes = [C.c_void_p]
    L.md_last_error.restype = C.c_char_p
    L.md_destroy.argtypes = [C.c_void_p]
    L.md_destroy.restype = None
    L.md_bin_cells_noalloc.argtypes = [_dp, C.c_double, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p]
    L.md_bin_cells_noalloc.restype = C.c_int
    L.md_set_potential.argtypes = [C.c_void_p, C.POINTER(PotentialC)]
    L.md_set_potential.restype = C.c_int
    L.md_force_match.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, _dp, _dp]
    L.md_force_match.restype = C.c_int
    L.md_batch_create.argtypes = [C.c_int32, C.POINTER(Replica), C.c_int32, C.POINTER(PotentialC),
                                  C.POINTER(Options), C.POINTER(C.c_void_p)]
    L.md_batch_create.restype = C.c_int
    L.md_batch_step.argtypes = [C.c_void_p, C.c_int64, C.c_double]
    L.md_batch_step.restype = C.c_int
    L.md_batch_energy.argtypes = [C.c_void_p, _dp, _dp]
    L.md_batch_energy.restype = C.c_int
    L.md_batch_get_state.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    L.md_batch_get_state.restype = C.c_int
    L.md_batch_info.argtypes = [C.c_void_p, C.POINTER(BatchInfo)]
    L.md_batch_info.restype = C.c_int
    L.md_batch_last_error.argtypes = [C.c_void_p]
    L.md_batch_last_error.restype = C.c_char_p
    L.md_batch_destroy.argtypes = [C.c_void_p]
    L.md_batch_destroy.restype = None
    _lib = L
    return L


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    """Host pointer of a numpy array or a (pinned) CPU torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _torch_allocator(stream):
    import torch

    def alloc(nbytes, _ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream)
        except Exception:  # out of memory -> NULL, the library reports MD_ERR_OOM
            return None

    def free(ptr, _ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    return ALLOC_FN(alloc), FREE_FN(free)


def bin_cells_noalloc(box, r_list: float, n: int, d_pos: int, d_cell_start: int, d_cell_atoms: int,
                      stream: int = 0) -> int:
    """md_bin_cells_noalloc: cell bins of n device positions into caller-owned
    device arrays, without any device allocation.  Pointers are integers
    (e.g. torch `data_ptr()`); returns the md_status code."""
    L = load()
    box = _f64(box)
    return L.md_bin_cells_noalloc(_d(box), float(r_list), int(n), C.c_void_p(d_pos),
                                  C.c_void_p(d_cell_start), C.c_void_p(d_cell_atoms), C.c_void_p(stream))


class MD:
    """One periodic EAM system on the GPU (the md_ctx of include/eammd.h).

    `system` is an `inputs.System`.  precision: "mixed" or "fp64".
    With use_torch=True (default when CUDA is available to torch) device
    memory comes from torch's caching allocator, or from `allocator` =
    (alloc(nbytes) -> device pointer or None, free(pointer)) when given, and
    work is queued on a torch stream owned by this object (`self.stream`)."""

    def __init__(self, system, precision: str = "mixed", rebuild_every: int = 10,
                 list_capacity: int = 0, use_graphs: bool = True, block_size: int = 256,
                 lanes_per_atom: int = 0, use_torch: bool | None = None, persistent: str = "auto",
                 wait_limit_us: int = 0, half_list: bool = False, allocator=None):
        L = load()
        self._L = L
        self.n = int(system.n)
        self.system = system
        opt = Options()
        L.md_options_default(C.byref(opt))
        opt.precision = PRECISION[precision]
        opt.rebuild_every = rebuild_every
        opt.list_capacity = list_capacity
        opt.use_graphs = 1 if use_graphs else 0
        opt.block_size = block_size
        opt.lanes_per_atom = lanes_per_atom
        opt.persistent = PERSIST[persistent]
        opt.wait_limit_us = wait_limit_us
        opt.half_list = 1 if half_list else 0
        opt.open_axes = int(getattr(system, "open_axes", 0))
        self._keep = []
        if use_torch is None:
            try:
                import torch
                use_torch = torch.cuda.is_available()
            except Exception:
                use_torch = False
        if use_torch:
            import torch
            torch.cuda.init()
            self.stream = torch.cuda.Stream()
            if allocator is None:
                a, f = _torch_allocator(self.stream)
            else:
                # caller's device allocator: (alloc(nbytes) -> pointer or None,
                # free(pointer)); pointers must be 256-byte aligned
                ua, uf = allocator
                a = ALLOC_FN(lambda nbytes, _ctx: ua(int(nbytes)))
                f = FREE_FN(lambda ptr, _ctx: uf(int(ptr)))
            self._keep += [a, f]
            opt.alloc, opt.free = a, f
            opt.cuda_stream = C.c_void_p(self.stream.cuda_stream)
        pot = system.pot
        pc = self._potential_c(pot)
        box = _f64(system.box)
        pos = _f64(system.pos)
        vel = _f64(system.vel) if system.vel is not None else None
        types = np.ascontiguousarray(system.types, dtype=np.int32)
        h = C.c_void_p()
        rc = L.md_create(_d(box), self.n, _d(pos), _d(vel) if vel is not None else None,
                         types.ctypes.data_as(_ip), C.byref(pc), C.byref(opt), C.byref(h))
        if rc != MD_OK:
            raise MDError(rc, L.md_last_error(None).decode())
        self.h = h
        self.box = box
        self._pot = None

    def _potential_c(self, pot):
        keep = []

        def splines(ks):
            arr = (Spline * len(ks))()
            for q, k in enumerate(ks):
                y = _f64(k.y)
                keep.append(y)
                arr[q] = Spline(k.n, k.x0, k.dx, _d(y), k.bc_lo, k.bc_hi, k.d_lo, k.d_hi)
            keep.append(arr)
            return arr

        mass = _f64(pot.mass)
        keep.append(mass)
        pc = PotentialC(pot.ntypes, _d(mass), splines(pot.F), splines(pot.f), splines(pot.phi),
                        pot.r_cut, pot.skin)
        self._keep.append(keep)
        return pc

    def set_potential(self, pot):
        """md_set_potential: new spline values on the same grids."""
        pc = self._potential_c(pot)
        self._check(self._L.md_set_potential(self.h, C.byref(pc)))
        self._keep.pop()
        self._pot = pot

    def force_match(self, f_ref, e_ref: float, w: float, grad: bool = True):
        """md_force_match: (loss, knot gradient phi|f|F or None)."""
        f_ref = _f64(f_ref)
        loss = C.c_double()
        g = None
        if grad:
            pot = self.system.pot if self._pot is None else self._pot
            g = np.zeros(pot.phi[0].n + pot.f[0].n + pot.F[0].n)
        self._check(self._L.md_force_match(self.h, _d(f_ref), float(e_ref), float(w), C.byref(loss),
                                           _d(g) if g is not None else None))
        return loss.value, g

    def _check(self, rc):
        if rc != MD_OK:
            raise MDError(rc, self._L.md_last_error(self.h).decode())

    def step(self, nsteps: int, dt: float):
        self._check(self._L.md_step(self.h, int(nsteps), float(dt)))

    def sync(self):
        self._check(self._L.md_sync(self.h))

    def energy(self):
        pe, ke = C.c_double(), C.c_double()
        self._check(self._L.md_energy(self.h, C.byref(pe), C.byref(ke)))
        return pe.value, ke.value

    def virial(self):
        w = np.zeros(6)
        self._check(self._L.md_virial(self.h, _d(w)))
        return w

    def forces(self, out=None):
        out = np.zeros((self.n, 3)) if out is None else out
        self._check(self._L.md_forces(self.h, _d(out) if isinstance(out, np.ndarray) else _ptr(out)))
        return out

    def get_state(self, pos=None, vel=None):
        pos = np.zeros((self.n, 3)) if pos is None else pos
        vel = np.zeros((self.n, 3)) if vel is None else vel
        st = C.c_int64()
        self._check(self._L.md_get_state(self.h, _ptr(pos), _ptr(vel), C.byref(st)))
        return pos, vel, st.value

    def set_state(self, pos, vel=None, step: int = 0):
        if isinstance(pos, np.ndarray):
            pos = _f64(pos)
        if isinstance(vel, np.ndarray):
            vel = _f64(vel)
        self._check(self._L.md_set_state(self.h, _ptr(pos), _ptr(vel), int(step)))

    def neighbors(self):
        off = np.zeros(self.n + 1, dtype=np.int64)
        self._check(self._L.md_neighbors(self.h, off.ctypes.data_as(_lp), None, 0))
        js = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
        self._check(self._L.md_neighbors(self.h, off.ctypes.data_as(_lp), js.ctypes.data_as(_ip),
                                         js.shape[0]))
        return off, js[: int(off[-1])]

    def cells(self):
        nc = np.zeros(3, dtype=np.int32)
        self._check(self._L.md_cells(self.h, nc.ctypes.data_as(_ip), None, None))
        ncells = int(np.prod(nc.astype(np.int64)))
        start = np.zeros(ncells + 1, dtype=np.int32)
        atoms = np.zeros(max(self.n, 1), dtype=np.int32)
        self._check(self._L.md_cells(self.h, nc.ctypes.data_as(_ip), start.ctypes.data_as(_ip),
                                     atoms.ctypes.data_as(_ip)))
        return nc, start, atoms[: self.n]

    def stats(self):
        s = Stats()
        self._check(self._L.md_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def profile(self, nsteps: int, dt: float):
        """Average kernel durations (ms) over nsteps eagerly launched steps."""
        p = Profile()
        self._check(self._L.md_profile(self.h, int(nsteps), float(dt), C.byref(p)))
        return {k: getattr(p, k) for k, _ in Profile._fields_}

    def close(self):
        if getattr(self, "h", None):
            self._L.md_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class MDBatch:
    """Independent systems advanced together in one persistent launch
    (md_batch_* of include/eammd.h).  `systems`: inputs.System objects with
    one-type potentials; identical potentials are shared."""

    def __init__(self, systems, rebuild_every: int = 10, list_capacity: int = 0, use_graphs: bool = True,
                 use_torch: bool | None = None, schedule: int = 0):
        L = load()
        self._L = L
        self._keep = []
        self.systems = list(systems)
        pots, pot_index = [], []
        for s in self.systems:
            for q, p in enumerate(pots):
                if p is s.pot:
                    pot_index.append(q)
                    break
            else:
                pots.append(s.pot)
                pot_index.append(len(pots) - 1)
        helper = MD.__new__(MD)
        helper._keep = self._keep
        pc = (PotentialC * len(pots))()
        for q, p in enumerate(pots):
            pc[q] = MD._potential_c(helper, p)
        reps = (Replica * len(self.systems))()
        for r, s in enumerate(self.systems):
            pos = _f64(s.pos)
            vel = _f64(s.vel) if s.vel is not None else None
            self._keep += [pos, vel]
            reps[r].n = s.n
            for a in range(3):
                reps[r].box[a] = float(s.box[a])
            reps[r].pos = _d(pos)
            reps[r].vel = _d(vel) if vel is not None else None
            reps[r].potential = pot_index[r]
        opt = Options()
        L.md_options_default(C.byref(opt))
        opt.precision = 1
        opt.rebuild_every = rebuild_every
        opt.list_capacity = list_capacity
        opt.use_graphs = 1 if use_graphs else 0
        opt.batch_schedule = schedule
        if use_torch is None:
            try:
                import torch
                use_torch = torch.cuda.is_available()
            except Exception:
                use_torch = False
        if use_torch:
            import torch
            torch.cuda.init()
            self.stream = torch.cuda.Stream()
            a, f = _torch_allocator(self.stream)
            self._keep += [a, f]
            opt.alloc, opt.free = a, f
            opt.cuda_stream = C.c_void_p(self.stream.cuda_stream)
        h = C.c_void_p()
        rc = L.md_batch_create(len(self.systems), reps, len(pots), pc, C.byref(opt), C.byref(h))
        if rc != MD_OK:
            raise MDError(rc, L.md_batch_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != MD_OK:
            raise MDError(rc, self._L.md_batch_last_error(self.h).decode())

    def step(self, nsteps: int, dt: float):
        self._check(self._L.md_batch_step(self.h, int(nsteps), float(dt)))

    def energy(self):
        n = len(self.systems)
        pe, ke = np.zeros(n), np.zeros(n)
        self._check(self._L.md_batch_energy(self.h, _d(pe), _d(ke)))
        return pe, ke

    def get_state(self, r: int):
        n = self.systems[r].n
        pos, vel, force = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
        self._check(self._L.md_batch_get_state(self.h, int(r), _ptr(pos), _ptr(vel), _ptr(force)))
        return pos, vel, force

    def info(self):
        i = BatchInfo()
        self._check(self._L.md_batch_info(self.h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in BatchInfo._fields_}

    def close(self):
        if getattr(self, "h", None):
            self._L.md_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
