"""Seeded synthetic inputs for the EAM timestep: lattices, thermal states and
potential knot tables.

This module is shared by the CUDA path, the CPU oracle, the tests and the
benchmark.  It holds none of the method's arithmetic: it only produces the
*inputs* the method consumes (positions, velocities, types, masses and the
knot values of the three EAM functions).  Spline construction, neighbour
search, density, forces, energies and integration are each implemented
separately on the two sides.

Units are metal units throughout: Angstrom, eV, amu, fs, K.

The paper (Section "Computational Molecular Dynamics", Eqs. 2-4) lets rho_i,
F_i and phi_ij be arbitrary splines per atom type; its own benchmarks use
published Cu/W/Ta potentials that are not available here.  The stand-in is
the analytic Johnson form

    f(r)   = fe * exp(-beta  * (r/re - 1))
    phi(r) = A  * exp(-alpha * (r/re - 1)) - B * exp(-kappa * (r/re - 1))
    F(rho) = -E0 * sqrt(rho / rho_e)

with f and phi multiplied by a quintic smoothstep that takes them to zero,
with two continuous derivatives, between r_s = r_cut - 0.5 and r_cut
(the paper only states that the functions vanish beyond the cutoff).
The BCC parameter set (a = 3.30, m = 180.95, r_cut = 4.5) stands in for the
Ta system of Table "Results for 800,000 atom models" (14 interactions per
atom, as there); the FCC set (a = 3.615, m = 63.55, r_cut = 5.0) stands in
for Cu (42 interactions per atom).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# 1 eV/(Angstrom*amu) expressed in Angstrom/fs^2 (CODATA 2018 e and u).
ACCEL_EV_A_AMU = 9.648533215665e-3
# Boltzmann constant in eV/K.
KB_EV = 8.617333262e-5

SEED_BASE = 7898

BC_NATURAL = 0
BC_CLAMPED = 1


@dataclasses.dataclass(frozen=True)
class JohnsonParams:
    """Parameters of one analytic Johnson-form EAM species."""
    name: str
    lattice: str          # "bcc" or "fcc"
    a: float              # lattice constant, Angstrom
    mass: float           # amu
    re: float = 2.86
    alpha: float = 8.5
    beta: float = 4.5
    kappa: float = 4.5
    A: float = 0.6
    B: float = 0.8
    fe: float = 1.0
    E0: float = 3.0
    rho_e: float = 14.0
    r_cut: float = 4.5
    smooth_width: float = 0.5
    skin: float = 0.3

    @property
    def r_s(self) -> float:
        return self.r_cut - self.smooth_width

    @property
    def rho_max(self) -> float:
        return 3.0 * self.rho_e


BCC_TA_LIKE = JohnsonParams(name="bcc_johnson", lattice="bcc", a=3.30, mass=180.95)
FCC_CU_LIKE = JohnsonParams(name="fcc_johnson", lattice="fcc", a=3.615, mass=63.55,
                            re=2.55, E0=3.5, r_cut=5.0)


def smoothstep(r, r_s, r_c):
    """Quintic switch: 1 below r_s, 0 at and above r_c, C2 at both ends."""
    u = np.clip((np.asarray(r, dtype=np.float64) - r_s) / (r_c - r_s), 0.0, 1.0)
    return 1.0 - 10.0 * u**3 + 15.0 * u**4 - 6.0 * u**5


def johnson_f(p: JohnsonParams, r):
    r = np.asarray(r, dtype=np.float64)
    return p.fe * np.exp(-p.beta * (r / p.re - 1.0)) * smoothstep(r, p.r_s, p.r_cut)


def johnson_phi(p: JohnsonParams, r):
    r = np.asarray(r, dtype=np.float64)
    raw = p.A * np.exp(-p.alpha * (r / p.re - 1.0)) - p.B * np.exp(-p.kappa * (r / p.re - 1.0))
    return raw * smoothstep(r, p.r_s, p.r_cut)


def johnson_F(p: JohnsonParams, rho):
    rho = np.asarray(rho, dtype=np.float64)
    return -p.E0 * np.sqrt(np.maximum(rho, 0.0) / p.rho_e)


def johnson_f_slope0(p: JohnsonParams) -> float:
    """df/dr at r = 0 (the switch is identically 1 there)."""
    return -p.beta / p.re * p.fe * math.exp(p.beta)


def johnson_phi_slope0(p: JohnsonParams) -> float:
    return (-p.alpha / p.re * p.A * math.exp(p.alpha)
            + p.kappa / p.re * p.B * math.exp(p.kappa))


@dataclasses.dataclass
class Knots:
    """Values of one function on a uniform grid x0 + k*dx, k = 0..n-1, with
    the end conditions a cubic spline through them should take:
    BC_NATURAL (zero second derivative) or BC_CLAMPED (given slope)."""
    x0: float
    dx: float
    y: np.ndarray
    bc_lo: int = BC_NATURAL
    bc_hi: int = BC_NATURAL
    d_lo: float = 0.0
    d_hi: float = 0.0

    @property
    def n(self) -> int:
        return int(self.y.shape[0])

    @property
    def x(self) -> np.ndarray:
        return self.x0 + self.dx * np.arange(self.n, dtype=np.float64)


@dataclasses.dataclass
class Potential:
    """A multi-type EAM potential given as knot tables.

    F[t], f[t] belong to type t (f is the density an atom of type t
    contributes to its neighbours); phi is packed over type pairs a <= b in
    row-major upper-triangular order."""
    mass: np.ndarray
    F: list
    f: list
    phi: list
    r_cut: float
    skin: float

    @property
    def ntypes(self) -> int:
        return len(self.F)

    @property
    def r_list(self) -> float:
        return self.r_cut + self.skin


def johnson_knots(p: JohnsonParams, n_knots: int = 2000):
    """Tabulate the three Johnson functions on uniform knots.

    f, phi: r in [0, r_cut], clamped at r = 0 with the analytic slope,
    natural at r_cut (where the smoothed functions have zero curvature).
    F: rho in [0, 3 rho_e], natural at both ends."""
    dr = p.r_cut / (n_knots - 1)
    r = dr * np.arange(n_knots, dtype=np.float64)
    f = Knots(0.0, dr, johnson_f(p, r), BC_CLAMPED, BC_NATURAL, johnson_f_slope0(p), 0.0)
    phi = Knots(0.0, dr, johnson_phi(p, r), BC_CLAMPED, BC_NATURAL, johnson_phi_slope0(p), 0.0)
    # exact zeros at the cutoff knot (the switch is 0 there)
    f.y[-1] = 0.0
    phi.y[-1] = 0.0
    drho = p.rho_max / (n_knots - 1)
    rho = drho * np.arange(n_knots, dtype=np.float64)
    F = Knots(0.0, drho, johnson_F(p, rho), BC_NATURAL, BC_NATURAL)
    return F, f, phi


def johnson_potential(p: JohnsonParams, n_knots: int = 2000) -> Potential:
    F, f, phi = johnson_knots(p, n_knots)
    return Potential(mass=np.array([p.mass]), F=[F], f=[f], phi=[phi],
                     r_cut=p.r_cut, skin=p.skin)


# --------------------------------------------------------------------------
# lattices and thermal states


def bcc_lattice(nx: int, ny: int, nz: int, a: float):
    base = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    return _lattice(base, nx, ny, nz, a)


def fcc_lattice(nx: int, ny: int, nz: int, a: float):
    base = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    return _lattice(base, nx, ny, nz, a)


def _lattice(base, nx, ny, nz, a):
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (cells[:, None, :] + base[None, :, :]).reshape(-1, 3) * a
    box = np.array([nx * a, ny * a, nz * a], dtype=np.float64)
    return np.ascontiguousarray(pos), box


def lattice(p: JohnsonParams, nx: int, ny: int, nz: int):
    return bcc_lattice(nx, ny, nz, p.a) if p.lattice == "bcc" else fcc_lattice(nx, ny, nz, p.a)


def displace(pos, box, sigma: float, rng: np.random.Generator):
    """Gaussian displacement of every coordinate, re-wrapped into the box."""
    out = pos + rng.normal(0.0, sigma, size=pos.shape)
    return np.ascontiguousarray(np.mod(out, box))


def maxwell(n: int, mass, temperature: float, rng: np.random.Generator):
    """Maxwell-Boltzmann velocities (Angstrom/fs) with zero total momentum,
    rescaled so that the kinetic temperature over 3N-3 degrees of freedom is
    exactly `temperature`."""
    m = np.broadcast_to(np.asarray(mass, dtype=np.float64), (n,)).astype(np.float64)
    if n < 2 or temperature <= 0.0:
        return np.zeros((n, 3))
    sd = np.sqrt(KB_EV * temperature * ACCEL_EV_A_AMU / m)
    v = rng.normal(size=(n, 3)) * sd[:, None]
    v -= (m[:, None] * v).sum(axis=0) / m.sum()
    ke = 0.5 * (m[:, None] * v * v).sum() / ACCEL_EV_A_AMU
    t_now = 2.0 * ke / ((3 * n - 3) * KB_EV)
    v *= math.sqrt(temperature / t_now)
    return np.ascontiguousarray(v)


@dataclasses.dataclass
class System:
    """One system: the inputs md_create takes.  open_axes has one bit per
    open (non-periodic) axis, 1: x, 2: y, 4: z (0: fully periodic)."""
    box: np.ndarray
    pos: np.ndarray
    vel: np.ndarray
    types: np.ndarray
    pot: Potential
    label: str = ""
    open_axes: int = 0

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def thermal_system(p: JohnsonParams, cells, sigma: float, temperature: float, seed: int,
                   n_knots: int = 2000, label: str = "") -> System:
    pos, box = lattice(p, *cells)
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = displace(pos, box, sigma, rng)
    vel = maxwell(pos.shape[0], p.mass, temperature, rng)
    types = np.zeros(pos.shape[0], dtype=np.int32)
    return System(box=box, pos=pos, vel=vel, types=types, pot=johnson_potential(p, n_knots),
                  label=label or f"{p.lattice}{cells[0]}x{cells[1]}x{cells[2]}")


def slab_system(p: JohnsonParams, cells, open_axes: int, vacuum: float, sigma: float, temperature: float,
                seed: int, n_knots: int = 2000, label: str = "") -> System:
    """A crystal with free surfaces on the open axes: the lattice of `cells`
    unit cells, shifted by `vacuum` (Angstrom) along each open axis inside a
    box that is the lattice extent plus 2 x vacuum there (the lattice period
    along periodic axes); Gaussian displacements (not re-wrapped along open
    axes) and Maxwell velocities."""
    pos, box = lattice(p, *cells)
    box = box.copy()
    rng = np.random.Generator(np.random.PCG64(seed))
    disp = rng.normal(0.0, sigma, size=pos.shape)
    pos = pos + disp
    for a in range(3):
        if (open_axes >> a) & 1:
            pos[:, a] += vacuum
            box[a] += 2.0 * vacuum
        else:
            pos[:, a] = np.mod(pos[:, a], box[a])
    vel = maxwell(pos.shape[0], p.mass, temperature, rng)
    types = np.zeros(pos.shape[0], dtype=np.int32)
    return System(box=box, pos=np.ascontiguousarray(pos), vel=vel, types=types, pot=johnson_potential(p, n_knots),
                  label=label or f"{p.lattice}_slab{cells[0]}x{cells[1]}x{cells[2]}_open{open_axes}",
                  open_axes=open_axes)


# --------------------------------------------------------------------------
# the named workloads


def bcc_2000_fp64() -> System:
    """2,000-atom BCC cube (10x10x10 cells, a = 3.30, L = 33 A), sigma 0.02 A,
    300 K, 2,000-knot tables; integrated 100 steps at dt = 2 fs in FP64."""
    return thermal_system(BCC_TA_LIKE, (10, 10, 10), 0.02, 300.0, SEED_BASE + 0,
                          label="bcc_2000")


def bcc_799496() -> System:
    """799,496-atom BCC system (74x74x73 cells; box 244.2 x 244.2 x 240.9 A),
    sigma 0.02 A, 300 K: the 800k-atom mixed-precision workload."""
    return thermal_system(BCC_TA_LIKE, (74, 74, 73), 0.02, 300.0, SEED_BASE + 1,
                          label="bcc_799496")


def bcc_cube(n: int, temperature: float = 300.0, sigma: float = 0.02, seed: int | None = None) -> System:
    return thermal_system(BCC_TA_LIKE, (n, n, n), sigma, temperature,
                          SEED_BASE + 100 + n if seed is None else seed, label=f"bcc_cube{n}")


def ta_slab_801792() -> System:
    """The size and shape of the paper's tantalum benchmark slab (Table
    "Results for 800,000 atom models": 256 x 261 x 6 BCC unit cells, 801,792
    atoms, open boundaries), with the BCC stand-in potential: all three axes
    open, 6 A of vacuum on each side, sigma 0.02 A, 290 K."""
    return slab_system(BCC_TA_LIKE, (256, 261, 6), 7, 6.0, 0.02, 290.0, SEED_BASE + 600, label="ta_slab_801792")


def cu_slab_801792() -> System:
    """The size and shape of the paper's copper benchmark slab (Table "Results
    for 800,000 atom models": 174 x 192 x 6 FCC unit cells, 801,792 atoms,
    open boundaries), with the FCC stand-in potential (42 interactions per
    atom): all three axes open, 6 A of vacuum on each side, sigma 0.02 A,
    290 K."""
    return slab_system(FCC_CU_LIKE, (174, 192, 6), 7, 6.0, 0.02, 290.0, SEED_BASE + 602, label="cu_slab_801792")


def bcc_slab_small(open_axes: int = 4, seed: int = SEED_BASE + 601) -> System:
    """2,160-atom BCC slab (12 x 10 x 9 cells) for parity tests: open along
    the axes of open_axes with 5 A of vacuum, periodic along the others."""
    return slab_system(BCC_TA_LIKE, (12, 10, 9), open_axes, 5.0, 0.03, 400.0, seed,
                       label=f"bcc_slab_small_open{open_axes}")


def multi_type_system(cells=(6, 6, 6), seed: int = SEED_BASE + 50, n_knots: int = 400) -> System:
    """Two-species BCC alloy for the type-dependent code path: both species
    use Johnson forms with different parameters; the cross pair function is
    the average of the two pure ones (a synthetic choice)."""
    pa = BCC_TA_LIKE
    pb = dataclasses.replace(BCC_TA_LIKE, name="bcc_b", mass=95.95, re=2.75, E0=3.6,
                             fe=1.2, A=0.7)
    pos, box = bcc_lattice(*cells, pa.a)
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = displace(pos, box, 0.03, rng)
    types = (rng.random(pos.shape[0]) < 0.35).astype(np.int32)
    masses = np.array([pa.mass, pb.mass])
    vel = maxwell(pos.shape[0], masses[types], 400.0, rng)
    Fa, fa, phia = johnson_knots(pa, n_knots)
    Fb, fb, phib = johnson_knots(pb, n_knots)
    phiab = Knots(phia.x0, phia.dx, 0.5 * (phia.y + phib.y), BC_CLAMPED, BC_NATURAL,
                  0.5 * (phia.d_lo + phib.d_lo), 0.0)
    pot = Potential(mass=masses, F=[Fa, Fb], f=[fa, fb], phi=[phia, phiab, phib],
                    r_cut=pa.r_cut, skin=pa.skin)
    return System(box=box, pos=pos, vel=vel, types=types, pot=pot, label="bcc_alloy")


# --------------------------------------------------------------------------
# the force-matching workload (differentiation)


def knot_potential(p: JohnsonParams, theta_phi, theta_f, theta_F, n_knots: int) -> Potential:
    """A single-type potential whose phi, f and F are the cubic splines
    through the given knot values on the same grids and end conditions as
    `johnson_knots(p, n_knots)` (the clamped end slopes stay those of the
    Johnson functions; they are not parameters)."""
    F, f, phi = johnson_knots(p, n_knots)
    phi = dataclasses.replace(phi, y=np.ascontiguousarray(theta_phi, dtype=np.float64))
    f = dataclasses.replace(f, y=np.ascontiguousarray(theta_f, dtype=np.float64))
    F = dataclasses.replace(F, y=np.ascontiguousarray(theta_F, dtype=np.float64))
    return Potential(mass=np.array([p.mass]), F=[F], f=[f], phi=[phi], r_cut=p.r_cut, skin=p.skin)


@dataclasses.dataclass
class FitProblem:
    """Force-matching problem: configurations (positions, box), the
    parameter vector theta = (phi knots, f knots, F knots), and the weight w
    of the force term.  References are computed by the caller with the
    2,000-knot Johnson tables."""
    params: JohnsonParams
    n_knots: int
    theta0: np.ndarray
    configs: list
    w: float

    def potential(self, theta) -> Potential:
        n = self.n_knots
        return knot_potential(self.params, theta[:n], theta[n:2 * n], theta[2 * n:], n)


def fit_problem(n_configs: int = 64, cells=(10, 10, 10), n_knots: int = 64, w: float = 0.1,
                seed: int = SEED_BASE + 400) -> FitProblem:
    """64 BCC configurations of 2,000 atoms with thermal displacements
    sigma_c = 0.05 + 0.15 c/63 A, three of them (a seeded choice, ~5%) with
    one vacancy; theta0 = the Johnson knots times (1 + 0.02 xi)."""
    p = BCC_TA_LIKE
    rng = np.random.Generator(np.random.PCG64(seed))
    vac = set(rng.choice(n_configs, size=max(1, round(0.05 * n_configs)), replace=False).tolist())
    configs = []
    for c in range(n_configs):
        pos, box = lattice(p, *cells)
        sigma = 0.05 + 0.15 * c / max(n_configs - 1, 1)
        pos = displace(pos, box, sigma, rng)
        if c in vac:
            pos = np.delete(pos, int(rng.integers(pos.shape[0])), axis=0)
        configs.append((np.ascontiguousarray(pos), box))
    F, f, phi = johnson_knots(p, n_knots)
    theta = np.concatenate([phi.y, f.y, F.y])
    noise = 1.0 + 0.02 * rng.normal(size=theta.shape)
    return FitProblem(params=p, n_knots=n_knots, theta0=theta * noise, configs=configs, w=w)


# --------------------------------------------------------------------------
# the batched workload


def _near_box(cells_wanted: int, min_cells: int):
    nx = max(min_cells, int(round(cells_wanted ** (1.0 / 3.0))))
    ny = max(min_cells, int(round((cells_wanted / nx) ** 0.5)))
    nz = max(min_cells, int(round(cells_wanted / (nx * ny))))
    return nx, ny, nz


def replica_batch(nrep: int = 512, n_min: int = 1024, n_max: int = 16384, seed: int = SEED_BASE):
    """Independent periodic systems of uneven size: target atom counts
    log-uniform in [n_min, n_max], realised as the nearest orthorhombic
    lattice with at least 3 list radii per edge; the first half BCC (a = 3.30),
    the second half FCC (a = 3.615, Cu-like); temperatures uniform in
    [200, 1200] K; replica r uses seed + r."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=nrep))
    temps = rng.uniform(200.0, 1200.0, size=nrep)
    out = []
    for r in range(nrep):
        p = BCC_TA_LIKE if r < nrep // 2 else FCC_CU_LIKE
        per_cell = 2 if p.lattice == "bcc" else 4
        min_cells = int(math.ceil(3.0 * (p.r_cut + p.skin) / p.a))
        cells = _near_box(max(1, int(round(sizes[r] / per_cell))), min_cells)
        out.append(thermal_system(p, cells, 0.02, float(temps[r]), seed + r, label=f"rep{r}"))
    return out


# --------------------------------------------------------------------------
# strong-scaling sweep and the Sigma-5 tilt-boundary bicrystal

SWEEP_CUBES = (8, 11, 15, 21, 28, 39, 54)  # 2 n^3 atoms: 1,024 ... 314,928


def sweep_systems(temperature: float = 1000.0):
    """BCC cubes of 1,024 to 314,928 atoms (geometric), then the 799,496-atom
    box, at the given temperature."""
    out = [bcc_cube(n, temperature=temperature, seed=SEED_BASE + 200 + n) for n in SWEEP_CUBES]
    out.append(thermal_system(BCC_TA_LIKE, (74, 74, 73), 0.02, temperature, SEED_BASE + 274,
                              label="bcc_799496"))
    return out


def sigma5_bicrystal(periods=(25, 10, 25), temperature: float = 1000.0, seed: int = SEED_BASE + 500,
                     min_sep: float = 0.3, sigma: float = 0.02) -> System:
    """Sigma-5 (310)[001] symmetric tilt bicrystal of the BCC stand-in: two
    grains rotated by -+atan(1/3) (18.43 degrees) about z, so that [310] of
    the lower grain and [3-10] of the upper grain both lie along x.  One
    periodic cell of a grain is a sqrt(10) x a sqrt(10) x a with 20 atoms; the
    box holds periods[0] x (2 periods[1]) x periods[2] of them, the grains
    stacked along y (boundaries at y = 0 and y = L_y / 2).  Upper-grain atoms
    closer than min_sep * a to a lower-grain atom are removed.  Gaussian
    displacements of `sigma` Angstrom and Maxwell velocities at
    `temperature`."""
    p = BCC_TA_LIKE
    a = p.a
    s10 = math.sqrt(10.0)
    Lx, Ly, Lz = periods[0] * a * s10, 2 * periods[1] * a * s10, periods[2] * a
    box = np.array([Lx, Ly, Lz])
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    grains = []
    for g, sign in enumerate((1.0, -1.0)):
        # columns: where lattice vectors x, y go; (3, sign, 0) a maps to +x
        c, s = 3.0 / s10, sign * 1.0 / s10
        R = np.array([[c, s], [-s, c]])
        y0, y1 = (0.0, Ly / 2) if g == 0 else (Ly / 2, Ly)
        span = int(math.ceil(max(Lx, Ly) / a)) + 4
        ii, jj = np.meshgrid(np.arange(-span, 2 * span), np.arange(-span, 2 * span), indexing="ij")
        pts = []
        for bvec in basis:
            xy = (np.stack([ii.ravel() + bvec[0], jj.ravel() + bvec[1]], 1) * a) @ R.T
            eps = 1e-7
            keep = (xy[:, 0] >= -eps) & (xy[:, 0] < Lx - eps) & (xy[:, 1] >= y0 - eps) & (xy[:, 1] < y1 - eps)
            xy = xy[keep]
            for k in range(periods[2]):
                z = np.full((xy.shape[0], 1), (k + bvec[2]) * a)
                pts.append(np.hstack([xy, z]))
        grains.append(np.vstack(pts))
    lower, upper = grains

    def inbox(x):
        w = np.mod(x, box)
        return np.where(w >= box, w - box, w)

    from scipy.spatial import cKDTree  # input construction only
    tree = cKDTree(inbox(lower), boxsize=box)
    dist, _ = tree.query(inbox(upper), k=1)
    upper = upper[dist >= min_sep * a]
    pos = inbox(np.vstack([lower, upper]))
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = displace(pos, box, sigma, rng)
    vel = maxwell(pos.shape[0], p.mass, temperature, rng)
    return System(box=box, pos=pos, vel=vel, types=np.zeros(pos.shape[0], np.int32),
                  pot=johnson_potential(p), label="sigma5_bicrystal")
