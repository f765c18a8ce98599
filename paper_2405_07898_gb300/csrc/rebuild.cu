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
#include "rebuild_device.cuh"

#include <cuda_runtime.h>

namespace eammd {
namespace {

// Largest system whose list the graph path builds with a warp per atom.
// Measured with graphs (BCC, 1,000 K): +26 % timesteps/s at 1,024 atoms,
// +14 % at 18,522, +2 % at 43,904, and a loss from 118,638 atoms up.
constexpr int64_t kListWarpMaxAtoms = 32768;

// --------------------------------------------------------------------------
// list build (every rebuild): wrap, bin, scan, scatter, sort, permute, list

template <class R>
__global__ void k_bin(Bufs<R> B, Geom G, int n)
{
    const DevState *st = B.st;
    if (!st->need_rebuild) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) bin_atom<R>(B, G, st->set, i);
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
    if (i < n) scatter_atom<R>(B, i);
}

template <class R>
__global__ void k_cell_sort(Bufs<R> B, int ncells)
{
    if (!B.st->need_rebuild) return;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncells) sort_cell<R>(B, B.st->set, c);
}

template <class R>
__global__ void k_permute(Bufs<R> B, Geom G, int n)
{
    const DevState *st = B.st;
    if (!st->need_rebuild) return;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) permute_atom<R>(B, G, st->set, st->sp, p);
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

// A warp per atom (list_atom_warp), for systems of up to kListWarpMaxAtoms:
// there the thread-per-atom walk waits on load latency.  Above that it is
// bound by instruction issue, which the warp form multiplies (a 799,496-atom
// build took about 780 us with it against 334 us).
template <class R>
__global__ void __launch_bounds__(256) k_build_list_warp(Bufs<R> B, Geom G, int n, int ld, int cap)
{
    DevState *st = B.st;
    if (!st->need_rebuild) return;
    const int p = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);  // the same for a warp's lanes
    const int cnt = (p < n) ? list_atom_warp<R>(B, G, st->set, st->sp, p, ld, cap) : 0;
    block_max_nnb(cnt, &st->max_nnb);
}

template <class R>
__global__ void __launch_bounds__(256) k_build_list(Bufs<R> B, Geom G, int n, int ld, int cap, int half)
{
    DevState *st = B.st;
    if (!st->need_rebuild) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int cnt = (p < n) ? list_atom<R>(B, G, st->set, st->sp, p, ld, cap, half != 0) : 0;
    block_max_nnb(cnt, &st->max_nnb);
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
    const DevState *st = B.st;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float d2 = (i < L.n) ? open_atom<R>(B, L, st->set, st->sp, i) : 0.f;
    block_max_disp(d2, &B.st->maxdisp2);
}

// Fixed-order sum of the per-block partials: block `slot` sums slot 0
// (embedding energy) over the density pass's blocks, or slots 1..8 (pair
// energy, kinetic energy, virial) over the force pass's blocks.
template <class R>
__global__ void __launch_bounds__(1024) k_reduce(Bufs<R> B, int nb_d, int nb_f, int stride)
{
    const int slot = blockIdx.x;
    reduce_slot(B.partials, B.st, slot, slot == 0 ? nb_d : nb_f, stride);
}

// Host arrays in, device SoA out: state of md_create / md_set_state in the
// caller's atom order (the next list build sorts it).
template <class R>
__global__ void k_load_state(Bufs<R> B, const double *pos, const double *vel, const int *types, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = B.st->set;
    bool finite = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double x = pos[3 * (size_t)i + a];
        const double v = vel ? vel[3 * (size_t)i + a] : 0.0;
        finite = finite && isfinite(x) && isfinite(v);
        B.xr[s][a][i] = x;
        B.d[a][i] = 0.0;
        B.v[s][a][i] = v;
    }
    if (!finite) atomicOr(&B.st->error, ERR_NONFINITE);
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
    if (!L.half && (int64_t)L.n <= kListWarpMaxAtoms)
        k_build_list_warp<R><<<blocks_for((int64_t)L.n * 32, 256), 256, 0, L.stream>>>(B, G, L.n, L.ld, L.cap);
    else
        k_build_list<R><<<blocks_for(L.n, L.list_block), L.list_block, 0, L.stream>>>(B, G, L.n, L.ld, L.cap, L.half);
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
