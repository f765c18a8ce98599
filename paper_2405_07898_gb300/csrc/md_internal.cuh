// md_internal.cuh -- device data layout shared by the kernels and the host
// runtime of the EAM library (not part of the public ABI).
//
// Layout in HBM (all per-atom arrays in the current spatially sorted order,
// i.e. grouped by cell, ascending original id inside a cell):
//   xr[set][3]   FP64 SoA, wrapped absolute positions at the last list build
//   d[3]         FP64 SoA, displacement since the last build (x = xr + d)
//   v[set][3]    FP64 SoA, velocities
//   id[set], type[set]   int32: original index and atom type
//   uref[3]      R SoA, xr minus the centre of the atom's cell (|uref| <= h/2)
//   shadow[2]    R4 (u_x, u_y, u_z, F'), u = uref + d: the coordinates the pair
//                kernels read, and the embedding derivative F'(rho_i) that the
//                density pass stores for the force pass; double-buffered
//                across steps
//   fcache[3]    R SoA, forces of the last closed step
//   list         uint32 [capacity][ld] (column k of atom i at k*ld + i):
//                neighbour index in bits 0..25; the stencil offset (dx, dy,
//                dz) of the neighbour's cell as t = d + 1 in {0, 1, 2} in
//                bits 26..27 (x), 28..29 (y), 30..31 (z)
//   nnb          int32 neighbours per atom
//   acc_rho, acc_f  int64 per atom (density) and per atom and axis (force,
//                interleaved xyz): fixed-point sums (2^-32 units) of the pair
//                terms added to an atom from the other end of a half-list
//                pair; zeroed by the pass that reads them (half lists only)
//   own          float4 per atom: the sum of an atom's own half-list terms
//                (density in x; force in x, y, z) (half lists only)
// "set" flips at every list build (the permutation writes the other set),
// "sp" flips at every drift.  Both live in DevState, on the device, so that a
// captured CUDA graph replays correctly whatever the rebuild history.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace eammd {

constexpr int kMaxTypes = 8;
constexpr int kMaxPairs = kMaxTypes * (kMaxTypes + 1) / 2;
constexpr int kCodeShift = 26;
constexpr uint32_t kIndexMask = (1u << kCodeShift) - 1u;

// List entry of neighbour q in the stencil cell at offset (dx, dy, dz).
__host__ __device__ constexpr uint32_t list_entry(uint32_t q, int dx, int dy, int dz)
{
    return q | ((uint32_t)((dx + 1) | ((dy + 1) << 2) | ((dz + 1) << 4)) << kCodeShift);
}
constexpr int kScanBlock = 1024;
constexpr int kEnergySlots = 10;  // embed, pair, ke, virial xx yy zz xy xz yz, spare
constexpr double kAccel = 9.648533215665e-3;  // (eV/Angstrom/amu) -> Angstrom/fs^2

enum : uint32_t { ERR_LIST_OVERFLOW = 1u, ERR_NONFINITE = 2u, ERR_TIMEOUT = 4u };

struct DevState {
    long long step;
    long long rebuilds;
    unsigned long long table_oor;
    int since_build;
    int sp;
    int set;
    int need_rebuild;
    unsigned int maxdisp2;  // bit pattern of a non-negative float (orders as unsigned)
    unsigned int error;
    int max_nnb;
    int pad0;
    long long graph_rebuilds;  // builds run inside a graph's conditional node
    double e_embed, e_pair, ke;
    double virial[6];
};

template <class R> struct V4;
template <> struct V4<float> { using T = float4; };
template <> struct V4<double> { using T = double4_32a; };

// One cubic spline on uniform knots: coefficients (a, b, c, d) of interval k
// at coef[offset + k], S(t) = a + b t + c t^2 + d t^3 with t = x - x_k.
template <class R>
struct SplineDesc {
    int offset, nint;
    R x0, inv_h;
    R h_hi, h_lo;        // h = h_hi + h_lo (the knot spacing to FP64 accuracy in R pairs)
    R x_end;             // last knot
    R y_lo, s_lo;        // value and slope at x0 (continued linearly below)
    R y_end, s_end;      // value and slope at x_end (continued linearly above)
};

template <class R>
struct Tables {
    int ntypes;
    int fused;             // 1: one type whose f and phi share a knot grid (fphi)
    SplineDesc<R> fphi;    // grid of the fused rows: coef2[2k] = f, coef2[2k+1] = phi
    SplineDesc<R> F[kMaxTypes], f[kMaxTypes], phi[kMaxPairs];
};

struct Geom {
    double box[3];
    double half_box[3];
    double inv_cell[3];  // n_d / L_d
    double h[3];         // L_d / n_d
    int ncell[3];
    int ncells;
    double rl2;          // r_list^2
    double screen_lo;    // candidates with r2 below this are in the list for sure
    double screen_hi;    // ... above this are out for sure; in between: exact FP64 test
    double rc2;          // r_cut^2
    int open_mask;       // one bit per open (non-periodic) axis: 1 x, 2 y, 4 z
    // the same in FP32, so that FP32 kernels convert nothing on the FP64 pipe
    float h_f[3];
    float inv_cell_f[3];  // inv_cell rounded to FP32 (the binning estimate)
    float rc2_f;
    float screen_lo_f, screen_hi_f;
};

template <class R>
struct Bufs {
    using R4 = typename V4<R>::T;
    double *xr[2][3];
    double *d[3];
    double *v[2][3];
    int *id[2];
    int *type[2];
    R *uref[3];
    R4 *shadow[2];
    // texture objects over shadow[0] and shadow[1] (FP32 records only; 0 =
    // none): the density pass gathers its neighbours' records through the
    // texture path, which issues them at fewer L1 data-pipe cycles than the
    // load path.  The density pass writes only the F' word of the records,
    // which its gathers do not use, so the non-coherent texture reads of the
    // coordinates are exact.
    unsigned long long tex_shadow[2];
    R *fcache[3];
    int *cell;
    double *center[3];   // cell centres per axis, (c + 1/2) h_d
    // rebuild scratch
    double *xw[3];
    int *cell_old;
    int *slot;
    int *count;
    int *cell_start;
    int *cell_atoms;
    int *block_sums;
    // list
    uint32_t *list;
    int *nnb;
    // half lists: fixed-point accumulators and own partial sums
    unsigned long long *acc_rho;
    unsigned long long *acc_f;
    float4 *own;
    // energy partials [kEnergySlots][nblocks]
    double *partials;
    // state and tables
    DevState *st;
    const R4 *coef;
    const R4 *coef2;     // fused f | phi rows (single-type fast path)
    const R4 *coef_f;    // the f rows alone (coef2 + 2 nint), read by the density pass
    const Tables<R> *tables;
};

struct Launch {
    int n;          // atoms
    int ld;         // list leading dimension (multiple of 32)
    int cap;        // list slots per atom
    int block;      // threads per block of per-atom kernels
    int list_block; // threads per block of the list build (smaller for small systems, to fill the SMs)
    int block_d;    // threads per block of the density pass
    int block_f;    // threads per block of the force pass
    int nblocks;    // ceil(n / block)
    int tpa_d;      // lanes per atom of the density pass (1, 2, 4, 8)
    int tpa_f;      // lanes per atom of the force pass
    int nb_d;       // blocks of the density pass
    int nb_f;       // blocks of the force pass
    int pstride;    // stride between energy slots in partials (>= nb_d, nb_f)
    int nint_fused; // intervals of the fused f|phi table (0: not fused)
    int multi;      // general type-dependent path (several types or unfused tables)
    int half;       // 1: half lists (each pair once, j < i ends added through acc_*)
    int ntypes;
    int rebuild_every;
    double disp2_thr;                 // (skin/2)^2
    double dt;
    double half_kick[kMaxTypes];      // 0.5 dt kAccel / m_t
    double ke_factor[kMaxTypes];      // 0.5 m_t / kAccel
    cudaStream_t stream;
    cudaGraphConditionalHandle cond;  // 0 outside graph capture
    int use_cond;
    unsigned long long wait_ns;       // limit of a device-side wait (grid barrier, bulk-copy barrier)
};

enum StepMode { MODE_MEASURE = 0, MODE_CLOSE = 1, MODE_CLOSE_OPEN = 2 };

// Device words of the persistent step kernel: the grid-barrier arrival
// counter and the two alternating largest-displacement words.
struct PersistScratch {
    unsigned long long arrive;
    unsigned maxdisp[2];
};
constexpr int kPersistentBlock = 256;

// Host-side launchers (rebuild.cu, pair_f32.cu, pair_f64.cu, persistent.cu).  All are asynchronous on L.stream and
// return the number of kernels queued.
template <class R> int launch_rebuild(const Bufs<R> &B, const Geom &G, const Launch &L);
template <class R> int launch_decide(const Bufs<R> &B, const Launch &L);
template <class R> int launch_open(const Bufs<R> &B, const Geom &G, const Launch &L);
template <class R> int launch_density(const Bufs<R> &B, const Geom &G, const Launch &L, bool energy);
template <class R> int launch_force(const Bufs<R> &B, const Geom &G, const Launch &L, int mode, bool energy);
// md_step as one cooperative launch of `grid` blocks with `tpa` lanes per atom
// in the pair passes (persistent.cu); persistent_grid: the blocks that can be
// resident at once for that kernel (0 if it cannot be launched).
template <class R> int persistent_grid(const Launch &L, int tpa);
template <class R>
cudaError_t launch_steps(const Bufs<R> &B, const Geom &G, const Launch &L, long long nsteps, int tpa, int grid,
                         PersistScratch *ps);

template <class R> int launch_reduce(const Bufs<R> &B, const Launch &L);
template <class R>
int launch_load_state(const Bufs<R> &B, const Launch &L, const double *pos, const double *vel, const int *types);
template <class R>
int launch_store_state(const Bufs<R> &B, const Launch &L, double *pos, double *vel, double *force);

// Adjoint of the force-matching loss for one configuration (adjoint.cu).
// All buffers are device memory owned by the context.
struct AdjointArgs {
    double x0[3], h[3];
    int nint[3];
    int off_f, off_F;       // coefficient offsets of f and F in B.coef
    double A, w;
    const double *f_ref;    // n*3, caller order (device)
    double *g, *rho, *drho; // 3n, n, n
    double *block_bins;     // nblocks_warp * 4 * nrows
    double *partials_g;     // >= blocks of k_adj_g
    double *coef_grad;      // 4 * nrows
    double *sq;             // 1
    const double *Mt;       // transposed basis matrices
    int nknots_total;
    const int *knot_func, *func_coef0, *func_ncoef;
    const long long *knot_mt0;
    double *knot_grad;      // nknots_total (nullptr: skip the knot map)
};

int launch_adjoint(const Bufs<double> &B, const Geom &G, const Launch &L, const AdjointArgs &a);
size_t adjoint_smem_bytes(int nrows);
// Permits `bytes` of dynamic shared memory to the adjoint accumulation.
cudaError_t allow_adjoint_smem(size_t bytes);
// Warps that share the 32 atoms of one block of the adjoint accumulation.
constexpr int kAdjWarps = 4;

}  // namespace eammd
