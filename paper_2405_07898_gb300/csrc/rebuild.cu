// rebuild.cu -- sm_103a kernels of the EAM timestep other than the pair
// passes (those are in pair_kernels.cuh):
//   candidate exchange + neighbour list  -> k_bin .. k_build_list (every
//                                           rebuild, Section "Neighbor list")
//   atom swap                            -> the spatial re-sort inside the
//                                           rebuild (k_bin .. k_permute)
//   per-step control                     -> k_decide (rebuild condition),
//                                           k_open (first kick and drift of
//                                           an md_step call), k_reduce
//   state in and out                     -> k_load_state, k_store_state
// R is the pair-arithmetic type: float in the mixed-precision path, double in
// the FP64 path.  Positions, velocities, the drift and all sums over atoms are
// FP64 in both paths.
#include "device_common.cuh"

#include <cuda_runtime.h>

namespace eammd {
namespace {

// --------------------------------------------------------------------------
// list build (every rebuild): wrap, bin, scan, scatter, sort, permute, list

// Wrap x = xr + d into [0, L) exactly as x - L floor(x / L) (for |x| < 2L the
// branch form below gives the same bits), then bin: c_d = floor(x_d n_d/L_d).
template <class R>
__global__ void k_bin(Bufs<R> B, Geom G, int n)
{
    const DevState *st = B.st;
    if (!st->need_rebuild) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = st->set;
    int c[3];
    bool finite = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double L = G.box[a];
        double x = __dadd_rn(B.xr[s][a][i], B.d[a][i]);
        if (x >= 0.0 && x < L) {
        } else if (x < 0.0 && x >= -L) {
            x = __dadd_rn(x, L);
        } else if (x >= L && x < 2.0 * L) {
            x = __dsub_rn(x, L);
        } else {
            double q = floor(__ddiv_rn(x, L));
            x = __dsub_rn(x, __dmul_rn(L, q));
        }
        finite = finite && isfinite(x);
        B.xw[a][i] = x;
        double q = floor(__dmul_rn(x, G.inv_cell[a]));
        int ca = finite ? (int)fmax(fmin(q, (double)(G.ncell[a] - 1)), 0.0) : 0;
        c[a] = ca;
    }
    if (!finite) atomicOr(&B.st->error, ERR_NONFINITE);
    int cell = (c[2] * G.ncell[1] + c[1]) * G.ncell[0] + c[0];
    B.cell_old[i] = cell;
    B.slot[i] = atomicAdd(&B.count[cell], 1);
}

// Per block of kScanBlock cells: total count.
template <class R>
__global__ void k_scan_blocks(Bufs<R> B, int ncells)
{
    if (!B.st->need_rebuild) return;
    __shared__ int sm[32];
    int base = blockIdx.x * kScanBlock;
    int v = 0;
    for (int c = base + threadIdx.x; c < min(base + kScanBlock, ncells); c += blockDim.x) v += B.count[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < (blockDim.x + 31) / 32; ++w) s += sm[w];
        B.block_sums[blockIdx.x] = s;
    }
}

// Exclusive scan of the cell counts: cell_start[c] = sum_{c' < c} count[c'].
// Block b adds the totals of blocks < b, then scans its own kScanBlock cells
// (blockDim.x == kScanBlock).  Counts are zeroed for the next build.
template <class R>
__global__ void k_scan_apply(Bufs<R> B, int ncells)
{
    if (!B.st->need_rebuild) return;
    __shared__ int warp_tot[32];
    __shared__ int prefix;
    const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t < 32) {
        int s = 0;
        for (int k = t; k < b; k += 32) s += B.block_sums[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (t == 0) prefix = s;
    }
    int c = b * kScanBlock + t;
    int v = (c < ncells) ? B.count[c] : 0;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
    }
    __syncthreads();
    int excl = prefix + warp_tot[warp] + incl - v;
    if (c < ncells) {
        B.cell_start[c] = excl;
        B.count[c] = 0;
        if (c == ncells - 1) B.cell_start[ncells] = excl + v;
    }
}

template <class R>
__global__ void k_scatter(Bufs<R> B, int n)
{
    if (!B.st->need_rebuild) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    B.cell_atoms[B.cell_start[B.cell_old[i]] + B.slot[i]] = i;
}

// Within each cell, order atoms by original id (the atomics above leave
// them in arrival order); insertion sort, cells hold a handful of atoms.
template <class R>
__global__ void k_cell_sort(Bufs<R> B, int ncells)
{
    if (!B.st->need_rebuild) return;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const int *id = B.id[B.st->set];
    int s = B.cell_start[c], e = B.cell_start[c + 1];
    for (int q = s + 1; q < e; ++q) {
        int a = B.cell_atoms[q];
        int ka = id[a];
        int r = q - 1;
        while (r >= s && id[B.cell_atoms[r]] > ka) {
            B.cell_atoms[r + 1] = B.cell_atoms[r];
            --r;
        }
        B.cell_atoms[r + 1] = a;
    }
}

// Gather the state into cell order (the other buffer set): positions become
// the wrapped positions, displacements restart at zero, and the cell-centred
// coordinates uref (and this step's shadow) are formed in FP64 and rounded.
template <class R>
__global__ void k_permute(Bufs<R> B, Geom G, int n)
{
    const DevState *st = B.st;
    if (!st->need_rebuild) return;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int s = st->set, t = 1 - s, sp = st->sp;
    int i = B.cell_atoms[p];
    int cell = B.cell_old[i];
    int cc[3] = {cell % G.ncell[0], (cell / G.ncell[0]) % G.ncell[1], cell / (G.ncell[0] * G.ncell[1])};
    R u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double X = B.xw[a][i];
        B.xr[t][a][p] = X;
        u[a] = (R)__dsub_rn(X, B.center[a][cc[a]]);
        B.uref[a][p] = u[a];
        B.v[t][a][p] = B.v[s][a][i];
        B.d[a][p] = 0.0;
    }
    B.shadow[sp][p] = mk4<R>(u[0], u[1], u[2], (R)0);
    B.id[t][p] = B.id[s][i];
    B.type[t][p] = B.type[s][i];
    B.cell[p] = cell;
}

template <class R>
__global__ void k_rebuild_finish(Bufs<R> B, int in_graph)
{
    DevState *st = B.st;
    if (!st->need_rebuild) return;
    st->set = 1 - st->set;
    st->since_build = 0;
    st->rebuilds += 1;
    st->graph_rebuilds += in_graph;
    st->max_nnb = 0;
}

// Exact list test for a candidate near the list radius: the minimum-image
// squared distance with the operations and rounding order of the definition
// (d = x_j - x_i, +-L once, (dx^2 + dy^2) + dz^2, no fused operations).
__device__ __forceinline__ bool exact_in_list(const double *const xr[3], int p, int q, const Geom &G)
{
    double d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = __dsub_rn(xr[a][q], xr[a][p]);
        if (x > G.half_box[a]) x = __dsub_rn(x, G.box[a]);
        else if (x < -G.half_box[a]) x = __dadd_rn(x, G.box[a]);
        d[a] = x;
    }
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
    return r2 < G.rl2;
}

// Verlet list: for each atom the atoms of the 27 surrounding cells (in
// stencil order, ascending id inside a cell) closer than r_list.  The test
// runs in R on the cell-centred coordinates; candidates within the rounding
// margin of r_list are decided by exact_in_list, so the list is bit-identical
// to the FP64 definition.  The stencil loop is unrolled: cell codes and
// shifts are constants of each unrolled iteration.
template <class R>
__global__ void __launch_bounds__(256) k_build_list(Bufs<R> B, Geom G, int n, int ld, int cap)
{
    using R4 = typename V4<R>::T;
    DevState *st = B.st;
    if (!st->need_rebuild) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    int cnt = 0;
    if (p < n) {
        const int sp = st->sp, s = st->set;
        const double *const xr[3] = {B.xr[s][0], B.xr[s][1], B.xr[s][2]};
        const R4 *sw = B.shadow[sp];
        const R lo = g_screen_lo<R>(G), hi = g_screen_hi<R>(G);
        const R hx = g_h<R>(G, 0), hy = g_h<R>(G, 1), hz = g_h<R>(G, 2);
        const int nx = G.ncell[0], ny = G.ncell[1], nz = G.ncell[2];
        const int cell = B.cell[p];
        const int cx = cell % nx, cy = (cell / nx) % ny, cz = cell / (nx * ny);
        const R4 up = sw[p];
        uint32_t *lp = B.list + p;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            int ez = cz + dz;
            ez += (ez < 0) ? nz : ((ez >= nz) ? -nz : 0);
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                int ey = cy + dy;
                ey += (ey < 0) ? ny : ((ey >= ny) ? -ny : 0);
                const int row = (ez * ny + ey) * nx;
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    int ex = cx + dx;
                    ex += (ex < 0) ? nx : ((ex >= nx) ? -nx : 0);
                    const int e = row + ex;
                    const uint32_t code = list_entry(0u, dx, dy, dz);
                    const R ox = (R)dx * hx - up.x, oy = (R)dy * hy - up.y, oz = (R)dz * hz - up.z;
                    const int q1 = B.cell_start[e + 1];
                    for (int q = B.cell_start[e]; q < q1; ++q) {
                        const R4 uq = sw[q];
                        const R ddx = uq.x + ox, ddy = uq.y + oy, ddz = uq.z + oz;
                        const R r2 = fma(ddz, ddz, fma(ddy, ddy, ddx * ddx));
                        if (r2 > hi || q == p) continue;
                        if (r2 < lo || exact_in_list(xr, p, q, G)) {
                            if (cnt < cap) lp[(size_t)cnt * ld] = (uint32_t)q | code;
                            ++cnt;
                        }
                    }
                }
            }
        }
        B.nnb[p] = min(cnt, cap);
        if (cnt > cap) atomicOr(&st->error, ERR_LIST_OVERFLOW);
    }
    // block maximum of the neighbour counts, one atomic per block
    __shared__ int smax[32];
    int m = cnt;
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)((blockDim.x + 31) >> 5); ++w) m = max(m, smax[w]);
        if (m > *(volatile int *)&st->max_nnb) atomicMax(&st->max_nnb, m);
    }
}

// --------------------------------------------------------------------------
// per-step kernels

// Start of a step: account for the drift just taken, flip the shadow buffer
// and decide whether the list must be rebuilt before the force evaluation
// (10 steps since the last build, or an atom moved more than skin/2).
__global__ void k_decide(DevState *st, int rebuild_every, double disp2_thr, cudaGraphConditionalHandle h_if,
                         int use_cond)
{
    st->sp ^= 1;
    st->step += 1;
    st->since_build += 1;
    float md = __uint_as_float(st->maxdisp2);
    st->maxdisp2 = 0u;
    int need = (st->since_build >= rebuild_every) || ((double)md > disp2_thr);
    st->need_rebuild = need;
    if (use_cond) cudaGraphSetConditional(h_if, need ? 1u : 0u);
}

// Opening kick and drift of a step from the forces cached at the last
// closed step: v += F dt/(2m), x += v dt.
template <class R>
__global__ void k_open(Bufs<R> B, Launch L)
{
    using R4 = typename V4<R>::T;
    const DevState *st = B.st;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = st->set, sp = st->sp;
    float d2 = 0.f;
    if (i < L.n) {
        int ti = L.ntypes > 1 ? B.type[s][i] : 0;
        double kq = L.half_kick[ti];
        double dn[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double v = B.v[s][a][i];
            v = fma((double)B.fcache[a][i], kq, v);
            B.v[s][a][i] = v;
            dn[a] = fma(v, L.dt, B.d[a][i]);
            B.d[a][i] = dn[a];
        }
        R u0 = B.uref[0][i] + (R)dn[0], u1 = B.uref[1][i] + (R)dn[1], u2 = B.uref[2][i] + (R)dn[2];
        B.shadow[sp ^ 1][i] = mk4<R>(u0, u1, u2, (R)0);
        float fx = (float)dn[0], fy = (float)dn[1], fz = (float)dn[2];
        d2 = fx * fx + fy * fy + fz * fz;
    }
    block_max_disp(d2, &B.st->maxdisp2);
}

// Fixed-order sum of the per-block partials: block `slot` sums slot 0
// (embedding energy) over the density pass's blocks, or slots 1..8 (pair
// energy, kinetic energy, virial) over the force pass's blocks.
template <class R>
__global__ void __launch_bounds__(1024) k_reduce(Bufs<R> B, int nb_d, int nb_f, int stride)
{
    __shared__ double sm[32];
    const int slot = blockIdx.x;
    const int nb = slot == 0 ? nb_d : nb_f;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += B.partials[(size_t)slot * stride + b];
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
        DevState *st = B.st;
        if (slot == 0) st->e_embed = t;
        else if (slot == 1) st->e_pair = t;
        else if (slot == 2) st->ke = t;
        else st->virial[slot - 3] = t;
    }
}

// Host arrays in, device SoA out: state of md_create / md_set_state in the
// caller's atom order (the next list build sorts it).
template <class R>
__global__ void k_load_state(Bufs<R> B, const double *pos, const double *vel, const int *types, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = B.st->set;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        B.xr[s][a][i] = pos[3 * (size_t)i + a];
        B.d[a][i] = 0.0;
        B.v[s][a][i] = vel ? vel[3 * (size_t)i + a] : 0.0;
    }
    B.id[s][i] = i;
    B.type[s][i] = types[i];
}

// Device SoA (sorted) out to interleaved arrays in the caller's order.
template <class R>
__global__ void k_store_state(Bufs<R> B, double *pos, double *vel, double *force, int n)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int s = B.st->set;
    size_t o = 3 * (size_t)B.id[s][p];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (pos) pos[o + a] = __dadd_rn(B.xr[s][a][p], B.d[a][p]);
        if (vel) vel[o + a] = B.v[s][a][p];
        if (force) force[o + a] = (double)B.fcache[a][p];
    }
}

}  // namespace

// --------------------------------------------------------------------------
// launchers

template <class R>
int launch_rebuild(const Bufs<R> &B, const Geom &G, const Launch &L)
{
    const int b = L.block, nb = blocks_for(L.n, b);
    const int nsb = blocks_for(G.ncells, kScanBlock);
    k_bin<R><<<nb, b, 0, L.stream>>>(B, G, L.n);
    k_scan_blocks<R><<<nsb, 256, 0, L.stream>>>(B, G.ncells);
    k_scan_apply<R><<<nsb, kScanBlock, 0, L.stream>>>(B, G.ncells);
    k_scatter<R><<<nb, b, 0, L.stream>>>(B, L.n);
    k_cell_sort<R><<<blocks_for(G.ncells, 256), 256, 0, L.stream>>>(B, G.ncells);
    k_permute<R><<<nb, b, 0, L.stream>>>(B, G, L.n);
    k_rebuild_finish<R><<<1, 1, 0, L.stream>>>(B, L.use_cond);
    k_build_list<R><<<nb, b, 0, L.stream>>>(B, G, L.n, L.ld, L.cap);
    return 8;
}

template <class R>
int launch_decide(const Bufs<R> &B, const Launch &L)
{
    k_decide<<<1, 1, 0, L.stream>>>(B.st, L.rebuild_every, L.disp2_thr, L.cond, L.use_cond);
    return 1;
}

template <class R>
int launch_open(const Bufs<R> &B, const Geom &G, const Launch &L)
{
    (void)G;
    k_open<R><<<L.nblocks, L.block, 0, L.stream>>>(B, L);
    return 1;
}

template <class R>
int launch_reduce(const Bufs<R> &B, const Launch &L)
{
    k_reduce<R><<<9, 1024, 0, L.stream>>>(B, L.nb_d, L.nb_f, L.pstride);
    return 1;
}

template <class R>
int launch_load_state(const Bufs<R> &B, const Launch &L, const double *pos, const double *vel, const int *types)
{
    k_load_state<R><<<L.nblocks, L.block, 0, L.stream>>>(B, pos, vel, types, L.n);
    return 1;
}

template <class R>
int launch_store_state(const Bufs<R> &B, const Launch &L, double *pos, double *vel, double *force)
{
    k_store_state<R><<<L.nblocks, L.block, 0, L.stream>>>(B, pos, vel, force, L.n);
    return 1;
}

#define EAMMD_INSTANTIATE(R)                                                                   \
    template int launch_rebuild<R>(const Bufs<R> &, const Geom &, const Launch &);              \
    template int launch_decide<R>(const Bufs<R> &, const Launch &);                             \
    template int launch_open<R>(const Bufs<R> &, const Geom &, const Launch &);                 \
    template int launch_reduce<R>(const Bufs<R> &, const Launch &);                             \
    template int launch_load_state<R>(const Bufs<R> &, const Launch &, const double *, const double *, \
                                      const int *);                                             \
    template int launch_store_state<R>(const Bufs<R> &, const Launch &, double *, double *, double *);

EAMMD_INSTANTIATE(float)
EAMMD_INSTANTIATE(double)

}  // namespace eammd
