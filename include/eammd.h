/*
 * eammd.h -- C ABI of the GB300 (sm_103a) Embedded-Atom-Method molecular
 * dynamics library.
 *
 * The library advances periodic systems of atoms under an EAM potential
 * (arXiv 2405.07898, Section "Computational Molecular Dynamics"):
 *   density   rho_i = sum_{j != i, r_ij < r_cut} f_{t_j}(r_ij)               (Eq. 2)
 *   energy    U = 1/2 sum_{i != j} phi_{t_i t_j}(r_ij) + sum_i F_{t_i}(rho_i) (Eq. 3)
 *   force     F_i = sum_j [phi'(r) + F'_i f'_{t_j}(r) + F'_j f'_{t_i}(r)] (x_j - x_i)/r  (Eq. 4)
 *   motion    velocity Verlet, whose half-step velocities are the leap-frog
 *             velocities of Eq. 5,
 * with a cell-binned Verlet neighbour list of radius r_cut + skin (Section
 * "Neighbor list": the squared distance is compared with the squared
 * radius) under periodic boundaries (Section "Periodic Boundary Conditions").
 *
 * Conventions shared by every entry point:
 *   - Units are metal units: Angstrom, eV, amu, fs.
 *   - Host arrays are caller-owned; the library copies what it needs and
 *     never keeps a host pointer past the call.  Per-atom arrays are in the
 *     caller's original atom order, xyz interleaved (n*3 doubles).
 *   - Every call returns an md_status; nothing throws across the ABI.
 *     md_last_error() gives a human-readable message for the last failure.
 *   - Device work is queued on the context's CUDA stream.  md_step returns
 *     once its work is queued; errors raised on the device (neighbour-list
 *     overflow, non-finite forces) are sticky and reported by the next call
 *     that synchronises (md_sync, md_energy, md_forces, md_virial,
 *     md_get_state, md_neighbors, md_cells, md_stats).
 *   - A context is used from one host thread at a time.
 */
#ifndef EAMMD_H
#define EAMMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct md_ctx md_ctx;

typedef enum {
    MD_OK = 0,
    MD_ERR_ARG = -1,          /* invalid argument (null pointer, n < 0, bad table, ...) */
    MD_ERR_BOX = -2,          /* some box edge is shorter than 3 (r_cut + skin) */
    MD_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    MD_ERR_OOM = -4,          /* device allocation failed */
    MD_ERR_NONFINITE = -5,    /* a force or an input coordinate was not finite */
    MD_ERR_TIMEOUT = -6,      /* a bounded device wait gave up */
    MD_ERR_LIST_OVERFLOW = -7,/* an atom had more neighbours than the list capacity */
    MD_ERR_CAPACITY = -8      /* a size is beyond a compiled-in or configured maximum */
} md_status;

/* Uniform-knot cubic spline: knots x0 + k*dx, k = 0..n-1, values y[k].
 * The library builds the C2 interpolating cubic.  bc_lo / bc_hi select
 * the end condition: 0 = natural (zero second derivative), 1 = clamped
 * (first derivative d_lo / d_hi).  Outside [x0, x0+(n-1)dx] the spline
 * continues along its end tangent.  n >= 2, dx > 0. */
typedef struct {
    int32_t n;
    double x0, dx;
    const double *y;
    int32_t bc_lo, bc_hi;
    double d_lo, d_hi;
} md_spline;

/* EAM potential over ntypes atom types (1 <= ntypes <= 8), the
 * type-dependent splines of Section "Computational Molecular Dynamics":
 *   mass[t]  amu;
 *   F[t]     embedding energy of an atom of type t, a function of density;
 *   f[t]     density contributed by an atom of type t at distance r;
 *   phi[q]   pair energy of types (a <= b), q = a*ntypes - a*(a-1)/2 + (b-a).
 * The f and phi tables must start at r <= 0 and extend to at least r_cut.
 * The potential vanishes for r >= r_cut; the list radius is r_cut + skin. */
typedef struct {
    int32_t ntypes;
    const double *mass;
    const md_spline *F;
    const md_spline *f;
    const md_spline *phi;
    double r_cut, skin;
} md_potential;

enum { MD_PRECISION_FP64 = 0, MD_PRECISION_MIXED = 1 };
enum { MD_PERSIST_AUTO = 0, MD_PERSIST_OFF = 1, MD_PERSIST_ON = 2 };

/* Options.  Fill with md_options_default() and change what you need.
 *   precision        MD_PRECISION_FP64: all arithmetic in FP64.
 *                    MD_PRECISION_MIXED: pair distance, spline, density and
 *                    force arithmetic in FP32 on cell-relative coordinates;
 *                    positions, velocities, integration and the energy /
 *                    virial sums over atoms in FP64.
 *   rebuild_every    rebuild the neighbour list after this many steps (10),
 *                    or sooner when an atom has moved more than skin/2.
 *   list_capacity    neighbours per atom the list can hold; 0 = sized from
 *                    the initial configuration.
 *   cuda_stream      cudaStream_t to queue work on; NULL = the library
 *                    creates its own stream.
 *   alloc / free     device allocator callbacks (e.g. a framework caching
 *                    allocator); NULL = cudaMalloc / cudaFree.  alloc must
 *                    return 256-byte aligned device memory or NULL.
 *   use_graphs       1 = replay the step sequence as CUDA graphs with a
 *                    device-side conditional node for the list rebuild;
 *                    0 = launch kernels one by one (same kernels, same results).
 *   block_size       threads per block of the per-atom kernels (0 = 256).
 *   lanes_per_atom   threads that share one atom's neighbour list in the
 *                    density and force passes: 1, 2, 4 or 8; 0 = chosen at
 *                    md_create by timing each together with the threads per
 *                    block (the choice is kept for the process, per
 *                    precision and size class, so contexts of the same shape
 *                    follow the same schedule).  Each lane gathers its
 *                    neighbours' records and spline rows from device memory.
 *                    Results depend on it only through FP summation order.
 *   persistent       MD_PERSIST_AUTO (0): md_step runs as one launch (all
 *                    phases of all steps) for systems of at most 65,536
 *                    atoms, else as CUDA graphs.  The launch is a
 *                    cooperative grid of all resident blocks meeting at grid
 *                    barriers in device memory.  MD_PERSIST_OFF: always the
 *                    graph (or eager) path.  MD_PERSIST_ON: always the
 *                    single launch.  Lanes per atom: lanes_per_atom, or
 *                    timed at md_create over 1, 2, 4, 8 on steps at dt = 0
 *                    (the state is restored).  Positions, velocities and
 *                    forces are bitwise those of the graph path with the
 *                    same lanes per atom; energy sums differ in rounding
 *                    only.  A barrier wait longer than the wait limit ends
 *                    the launch and raises MD_ERR_TIMEOUT.
 *   open_axes        one bit per open (non-periodic) axis: 1 = x, 2 = y,
 *                    4 = z; 0 = fully periodic.  The free-surface slabs of
 *                    the paper's benchmarks (Section "How Performance Was
 *                    Measured": open boundaries).  On an open axis the box is
 *                    the extent of the cell grid (edge >= r_cut + skin,
 *                    against 3 (r_cut + skin) on a periodic axis),
 *                    positions are not wrapped, pair vectors are plain
 *                    differences, and an atom outside the box is binned into
 *                    the edge cell (its list stays complete; keep atoms
 *                    inside the box for the FP32 accuracy bound of the mixed
 *                    path).  Batches are periodic only.
 *   wait_limit_us    longest device-side wait (a grid barrier of the single
 *                    launch) before the kernel gives up and raises
 *                    MD_ERR_TIMEOUT; 0 = 1 s.
 *   batch_schedule   batches only: 0 = threads per block and resident
 *                    blocks per SM timed at md_batch_create (unless
 *                    lanes_per_atom > 0, which takes 512 x 1); 1..5 =
 *                    512 x 1, 256 x 2, 256 x 3, 1024 x 1, 512 x 2.
 *   half_list        0: every atom lists all its neighbours and each pair is
 *                    evaluated from both ends (the default).  1: the
 *                    force-symmetry form (Section "Additional Acceleration"): each pair
 *                    is listed once -- by the atom that sees the other in
 *                    the upper half space (pair vector with d_z > 0, ties
 *                    broken by d_y, then d_x, decided exactly) -- and
 *                    evaluated once; the term for the other atom is added
 *                    to it through per-atom 64-bit fixed-point accumulators
 *                    (2^-32 units of density or eV/Angstrom) by integer
 *                    atomics, whose totals do not depend on arrival order,
 *                    so runs are bitwise reproducible.  Mixed precision with
 *                    one atom type whose f and phi share a knot grid only
 *                    (MD_ERR_ARG otherwise); md_step runs as CUDA graphs
 *                    (or eagerly), never as the single launch; lanes per
 *                    atom are 1.  A pair term beyond 2^24 in magnitude (out
 *                    of the accumulators' range) raises MD_ERR_NONFINITE.
 *                    md_neighbors still reports every atom's full list. */
typedef struct {
    int32_t precision;
    int32_t rebuild_every;
    int32_t list_capacity;
    int32_t use_graphs;
    int32_t block_size;
    int32_t lanes_per_atom;
    void *cuda_stream;
    void *(*alloc)(size_t bytes, void *alloc_ctx);
    void (*free)(void *ptr, void *alloc_ctx);
    void *alloc_ctx;
    int32_t persistent;
    int32_t wait_limit_us;
    int32_t open_axes;
    int32_t batch_schedule;
    int32_t half_list;
} md_options;

void md_options_default(md_options *opt);

/* Create a system of n atoms in the box [0,box[0]) x [0,box[1]) x
 * [0,box[2]), periodic but along the axes of opt->open_axes.  pos: n*3
 * Angstrom (any image along periodic axes: wrapped on entry);
 * vel: n*3 Angstrom/fs or NULL for zero; types: n values in [0, ntypes).
 * Builds the tables, bins the atoms, builds the list and evaluates the
 * forces, energies and virial of the initial state.  Synchronises.
 * Errors: MD_ERR_ARG, MD_ERR_BOX, MD_ERR_NONFINITE, MD_ERR_OOM, MD_ERR_CUDA,
 * MD_ERR_CAPACITY (n >= 2^26). */
md_status md_create(const double box[3], int64_t n, const double *pos, const double *vel,
                    const int32_t *types, const md_potential *pot, const md_options *opt,
                    md_ctx **out);

/* Advance nsteps velocity-Verlet steps of dt fs: per step kick (dt/2),
 * drift (dt), rebuild the list if due, density and force, kick (dt/2).
 * Energies and the virial are evaluated at the last step.  Asynchronous:
 * returns once the work is queued on the context's stream. */
md_status md_step(md_ctx *ctx, int64_t nsteps, double dt);

/* Wait for queued work and report sticky device errors. */
md_status md_sync(md_ctx *ctx);

/* Potential (Eq. 3) and kinetic energy of the current state, eV. */
md_status md_energy(md_ctx *ctx, double *pe, double *ke);

/* Forces of the current state into f (n*3, eV/Angstrom, original order). */
md_status md_forces(md_ctx *ctx, double *f);

/* Virial W_ab = -1/2 sum_i sum_{j != i} s_ij d_a d_b / r_ij (d = x_j - x_i,
 * s_ij the scalar of Eq. 4), ordered xx, yy, zz, xy, xz, yz, eV.  The
 * pressure is (2 KE + W_xx + W_yy + W_zz) / (3 V). */
md_status md_virial(md_ctx *ctx, double w[6]);

/* Current positions (wrapped at the last list build, then advanced),
 * velocities (at the integer step) and the step counter; any pointer may
 * be NULL. */
md_status md_get_state(md_ctx *ctx, double *pos, double *vel, int64_t *step);

/* Replace positions and velocities (original order), rebuild the list and
 * re-evaluate forces and energies.  vel may be NULL for zero.  pos and vel
 * are host arrays (pinned memory makes the copy asynchronous DMA).
 * Synchronises.  Errors: MD_ERR_ARG (pos NULL); MD_ERR_NONFINITE when a
 * value is not finite (checked on the device while loading; the context's
 * state is then undefined until the next successful md_set_state). */
md_status md_set_state(md_ctx *ctx, const double *pos, const double *vel, int64_t step);

/* Neighbour list of the last build in original atom ids, CSR:
 * offsets[n+1] and js[offsets[n]].  js is written only if offsets[n] <= cap;
 * the needed size is always returned in offsets[n]. */
md_status md_neighbors(md_ctx *ctx, int64_t *offsets, int32_t *js, int64_t cap);

/* Cell bins of the last build: ncell[3] cells per axis, cell_start[ncells+1],
 * cell_atoms[n] (original ids, ascending within each cell).  Any array may
 * be NULL to query ncell only. */
md_status md_cells(md_ctx *ctx, int32_t ncell[3], int32_t *cell_start, int32_t *cell_atoms);

/* Counters of the run so far. */
typedef struct {
    int64_t steps;           /* velocity-Verlet steps taken */
    int64_t rebuilds;        /* neighbour-list builds after md_create */
    int32_t max_neighbors;   /* largest list length at the last build */
    int32_t list_capacity;   /* list slots per atom */
    int64_t table_out_of_range; /* embedding lookups beyond the F table */
    int64_t kernel_launches; /* kernels queued by this context so far */
    int32_t lanes_density;   /* lanes per atom of the density pass */
    int32_t lanes_force;     /* lanes per atom of the force pass */
    int32_t threads_density; /* threads per block of the density pass */
    int32_t threads_force;   /* threads per block of the force pass */
    int32_t persistent_blocks; /* blocks of the single-launch md_step (0: graphs) */
    int32_t persistent_lanes;  /* lanes per atom of its pair passes */
    int32_t half_list;         /* 1: pairs listed and evaluated once (md_options.half_list) */
    int32_t record_textures;   /* 1: the density pass gathers neighbour records through texture
                                  objects (mixed precision, record buffers aligned for textures);
                                  0: through ordinary loads.  Results are the same either way. */
} md_stats_t;

md_status md_stats(md_ctx *ctx, md_stats_t *out);

/* Kernel timing: runs nsteps ordinary steps of dt fs (the state advances as
 * with md_step) with kernels launched one by one, each density launch, force
 * launch and list rebuild bracketed by CUDA events on the context's stream,
 * and returns their average durations in milliseconds.  Synchronises. */
typedef struct {
    double density_ms;       /* average density (Eq. 2) kernel */
    double force_ms;         /* average force + integration (Eqs. 4, 5) kernel */
    double rebuild_ms;       /* average full list rebuild (8 kernels) */
    double step_ms;          /* average wall time of one step on the stream */
    int64_t density_launches, force_launches, rebuilds;
} md_profile_t;

md_status md_profile(md_ctx *ctx, int64_t nsteps, double dt, md_profile_t *out);

/* Replace the spline values of the potential (the differentiation form: fit
 * the splines of Section "Computational Molecular Dynamics" to reference
 * data).  Every spline must keep its knot count, x0, dx and end conditions,
 * and ntypes, masses, r_cut and skin must be unchanged.  Forces, energies and
 * the virial of the current positions are re-evaluated.  Synchronises. */
md_status md_set_potential(md_ctx *ctx, const md_potential *pot);

/* Force-matching loss of the current configuration and its gradient with
 * respect to the spline knot values (FP64 context, one atom type):
 *   L = (E - e_ref)^2 / n + w sum_i |F_i - f_ref_i|^2,
 * E the potential energy (Eq. 3) and F the forces (Eq. 4) of the current
 * positions under the current splines.  f_ref: n*3 host array, original atom
 * order.  grad (may be NULL): the derivative of L with respect to the knot
 * values y[k] of phi[0], then f[0], then F[0], in that order (n_phi + n_f +
 * n_F doubles, host memory); the clamped end slopes are not parameters.  The
 * gradient includes the second-order terms through the forces: along
 * g = F - f_ref it differentiates dE/dtheta (the density is recomputed, no
 * per-pair term is stored).  Synchronises.  Errors: MD_ERR_ARG (wrong
 * precision or several types), MD_ERR_CAPACITY (more than 200 KB of
 * per-interval gradient bins, about 6,400 intervals in all). */
md_status md_force_match(md_ctx *ctx, const double *f_ref, double e_ref, double w, double *loss, double *grad);

/* Cell binning that allocates no device memory.  The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc --
 * programs whose device memory is handed out by a fixed pool or budget that
 * may not grow (a framework's caching allocator, an embedded or real-time
 * loop that forbids allocation after start-up because cudaMalloc can
 * synchronise the device).
 * It computes what md_cells reports after md_create for the same positions:
 * wraps d_pos (n*3 doubles, xyz interleaved, device memory) into the box,
 * uses ncell_d = floor(box_d / r_list) cells per axis (each >= 3), and writes
 * d_cell_start[ncells+1] and d_cell_atoms[n] (atom indices, ascending inside
 * each cell; both device memory, caller-owned), queued on cuda_stream (NULL =
 * the legacy default stream); it does not synchronise.  The order inside a
 * cell comes from sorting the distinct keys (cell, index), so its cost is
 * O(n log^2 n) however the atoms crowd into cells.  A non-finite coordinate
 * cannot be detected here (the call does not synchronise): such an atom is
 * binned into cell 0 along that axis, whereas md_create and md_set_state
 * reject non-finite positions with MD_ERR_NONFINITE, so for such input there
 * is no md_cells result to equal.
 * Scratch lives in one static device array of about 2.3 MB that every GPU
 * loading this library holds until the process exits.  Limits: n <= 262,144
 * atoms and ncells <= 65,536; larger inputs return MD_ERR_CAPACITY, and no
 * work is queued.  Other errors: MD_ERR_ARG, MD_ERR_BOX (an axis with fewer
 * than 3 cells), MD_ERR_CUDA (a launch of this call failed; each launch's
 * own status is checked and no earlier error is consumed); this entry point
 * has no context, so md_last_error() does not describe its failures.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call shares the one array: calls that
 * overlap on the GPU (different streams, or different host threads on the
 * same device) race and must be ordered by the caller. */
md_status md_bin_cells_noalloc(const double box[3], double r_list, int64_t n, const double *d_pos,
                               int32_t *d_cell_start, int32_t *d_cell_atoms, void *cuda_stream);

/* ---- batches: many independent systems in one persistent launch ----
 * The batching form of the method: hundreds of periodic systems ("replicas")
 * of uneven size, each with its own box and one-type potential, advanced
 * together.  One thread block runs all phases of all steps of a replica
 * (list rebuild, density, force and integration) with block-level barriers
 * only; blocks take replicas largest first.  Mixed precision only (FP32
 * pair arithmetic, FP64 positions, velocities and sums), the same
 * arithmetic and list rules as a single context. */
typedef struct md_batch md_batch;

typedef struct {
    int64_t n;             /* atoms, >= 1 */
    double box[3];         /* each edge >= 3 (r_cut + skin) of its potential */
    const double *pos;     /* n*3 Angstrom, caller order */
    const double *vel;     /* n*3 Angstrom/fs or NULL */
    int32_t potential;     /* index into the potentials of md_batch_create */
    int32_t reserved;
} md_replica;

typedef struct {
    int32_t replicas, blocks, threads_per_block, list_capacity;
    int64_t atoms, steps, rebuilds, kernel_launches;
    int32_t max_neighbors, reserved;
} md_batch_info_t;

/* pots: npot single-type potentials whose f and phi share a knot grid
 * covering [0, r_cut].  opt: precision must be MD_PRECISION_MIXED;
 * rebuild_every, list_capacity, use_graphs, cuda_stream and alloc/free
 * apply.  Builds every replica's list and evaluates its initial forces and
 * energies.  Synchronises. */
md_status md_batch_create(int32_t nrep, const md_replica *reps, int32_t npot, const md_potential *pots,
                          const md_options *opt, md_batch **out);

/* nsteps velocity-Verlet steps of dt fs for every replica: one kernel launch
 * (replayed from a captured graph when use_graphs).  Energies are evaluated
 * at the last step.  Asynchronous. */
md_status md_batch_step(md_batch *b, int64_t nsteps, double dt);

/* pe[nrep], ke[nrep] (eV) of every replica; either may be NULL. */
md_status md_batch_energy(md_batch *b, double *pe, double *ke);

/* Positions, velocities and forces of replica r (n*3 each, caller order);
 * any pointer may be NULL. */
md_status md_batch_get_state(md_batch *b, int32_t r, double *pos, double *vel, double *force);

md_status md_batch_info(md_batch *b, md_batch_info_t *out);
const char *md_batch_last_error(const md_batch *b);
void md_batch_destroy(md_batch *b);

/* Message for the last failed call on ctx (or of md_create when ctx is NULL). */
const char *md_last_error(const md_ctx *ctx);

/* Free everything the context owns.  Safe on NULL. */
void md_destroy(md_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* EAMMD_H */
