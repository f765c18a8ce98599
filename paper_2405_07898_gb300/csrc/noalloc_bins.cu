// noalloc_bins.cu -- a cell binner that allocates no device memory.
//
// md_bin_cells_noalloc() sorts atoms into cells like the binning stage of the
// list rebuild (cells in x-fastest order, ascending atom index inside a
// cell), but reads the caller's device positions, writes the caller's device
// outputs, and keeps its scratch (one 64-bit sort key per atom, per-cell
// counts, per-block sums) in the file-scope device array below instead of
// memory from cudaMalloc.  Every GPU that loads the library holds that array
// until the process exits.
//
// Order inside a cell: each atom's key is (cell << 32) | index, and the keys
// are put in order by a bitonic sorting network.  The keys are distinct, so
// the result is the one stable order whatever the input; the work is
// O(N log^2 N) for N = the next power of two >= n (at least 2,048), however
// the atoms are spread over the cells.  The per-cell counts come from integer
// atomics, whose totals do not depend on arrival order.
#include "eammd.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

namespace {

constexpr int kNoAllocMaxAtoms = 1 << 18;  // 262,144 atoms
constexpr int kNoAllocMaxCells = 1 << 16;  // 65,536 cells
constexpr int kNbScanBlock = 1024;
constexpr int kNbMaxScanBlocks = kNoAllocMaxCells / kNbScanBlock;
constexpr int kSortChunk = 2048;  // keys one block orders in shared memory
// layout (8-byte words): sort keys [0, A); then (ints) count [0, C) and
// block sums [C, C + B)
constexpr size_t kScratchWords =
    (size_t)kNoAllocMaxAtoms + ((size_t)kNoAllocMaxCells + kNbMaxScanBlocks + 1) / 2;

static __device__ __align__(256) unsigned long long g_bin_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long *g_scratch_addr[kMaxDevices] = {nullptr};

struct BinGeom {
    double box[3];
    double inv_cell[3];
    int ncell[3];
    int ncells;
};

__global__ void k_nb_clear(int *count, int ncells)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncells) count[c] = 0;
}

// periodic image (x kept in [0, L), else x - L floor(x/L)), then
// c_d = min(floor(x_d n_d / L_d), n_d - 1); a non-finite coordinate gives
// cell 0 on its axis.  Keys at and beyond n (up to nsort) are padding that
// orders after every real key.
__global__ void k_nb_bin(const double *pos, int n, int nsort, BinGeom G, unsigned long long *keys, int *count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsort) return;
    if (i >= n) {
        keys[i] = ~0ull;
        return;
    }
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double L = G.box[a];
        double x = pos[3 * (size_t)i + a];
        if (!(x >= 0.0 && x < L)) {
            double q = floor(__ddiv_rn(x, L));
            x = __dsub_rn(x, __dmul_rn(L, q));
        }
        double y = floor(__dmul_rn(x, G.inv_cell[a]));
        c[a] = isfinite(y) ? (int)fmax(fmin(y, (double)(G.ncell[a] - 1)), 0.0) : 0;
    }
    int cell = (c[2] * G.ncell[1] + c[1]) * G.ncell[0] + c[0];
    keys[i] = ((unsigned long long)(unsigned)cell << 32) | (unsigned)i;
    atomicAdd(&count[cell], 1);
}

__global__ void k_nb_block_sums(const int *count, int ncells, int *block_sums)
{
    __shared__ int sm[32];
    int base = blockIdx.x * kNbScanBlock, v = 0;
    for (int c = base + threadIdx.x; c < min(base + kNbScanBlock, ncells); c += blockDim.x) v += count[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += sm[w];
        block_sums[blockIdx.x] = s;
    }
}

// exclusive scan of the counts into cell_start (blockDim.x == kNbScanBlock)
__global__ void k_nb_scan(const int *count, const int *block_sums, int ncells, int *cell_start)
{
    __shared__ int warp_tot[32];
    __shared__ int prefix;
    const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t < 32) {
        int s = 0;
        for (int k = t; k < b; k += 32) s += block_sums[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (t == 0) prefix = s;
    }
    int c = b * kNbScanBlock + t;
    int v = (c < ncells) ? count[c] : 0;
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
        warp_tot[lane] = wi - w;
    }
    __syncthreads();
    int excl = prefix + warp_tot[warp] + incl - v;
    if (c < ncells) {
        cell_start[c] = excl;
        if (c == ncells - 1) cell_start[ncells] = excl + v;
    }
}

// One compare-exchange of the bitonic network: stage k (the length of the
// sequences being merged), distance j.  Element i pairs with i ^ j; the pair
// is put in ascending order when bit k of i is clear, else descending.
__device__ __forceinline__ void bitonic_cx(unsigned long long *a, unsigned i, unsigned j, unsigned k)
{
    const unsigned l = i ^ j;
    if (l <= i) return;
    const unsigned long long x = a[i], y = a[l];
    if ((x > y) == ((i & k) == 0)) {
        a[i] = y;
        a[l] = x;
    }
}

// All steps of distance j < kSortChunk for the stages k in [k_lo, k_hi] on
// one 2,048-key chunk in shared memory (blockDim.x == kSortChunk / 2).  For
// k_lo = 2 this orders each chunk from scratch; for one k > kSortChunk it
// finishes that stage after the global steps of larger distances.
__global__ void k_nb_sort_chunk(unsigned long long *keys, unsigned k_lo, unsigned k_hi)
{
    __shared__ unsigned long long sm[kSortChunk];
    const unsigned base = blockIdx.x * kSortChunk;
    for (unsigned t = threadIdx.x; t < (unsigned)kSortChunk; t += blockDim.x) sm[t] = keys[base + t];
    __syncthreads();
    for (unsigned k = k_lo; k <= k_hi; k <<= 1) {
        for (unsigned j = min(k >> 1, (unsigned)kSortChunk >> 1); j > 0; j >>= 1) {
            // thread t handles the pair whose lower index is the t-th index
            // with bit j clear
            const unsigned t = threadIdx.x;
            const unsigned i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
            const unsigned l = i | j;
            const unsigned long long x = sm[i], y = sm[l];
            const bool up = ((base + i) & k) == 0;
            if ((x > y) == up) {
                sm[i] = y;
                sm[l] = x;
            }
            __syncthreads();
        }
    }
    for (unsigned t = threadIdx.x; t < (unsigned)kSortChunk; t += blockDim.x) keys[base + t] = sm[t];
}

// One step of distance j >= kSortChunk of stage k over all nsort keys.
__global__ void k_nb_sort_step(unsigned long long *keys, unsigned nsort, unsigned j, unsigned k)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nsort) bitonic_cx(keys, i, j, k);
}

__global__ void k_nb_extract(const unsigned long long *keys, int n, int *cell_atoms)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) cell_atoms[q] = (int)(unsigned)(keys[q] & 0xffffffffull);
}

// Each launch reports its own status, and no earlier error of the caller's
// is consumed.
template <class... KArgs, class... Args>
cudaError_t launch(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Device address of the scratch array for the current device, looked up once
// per device (the first call on a device does it, with that device current).
md_status scratch_for_current_device(unsigned long long **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return MD_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return MD_ERR_CAPACITY;  // device ordinal beyond 63
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bin_scratch);
        if (e != cudaSuccess || !p) return MD_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_scratch_addr[dev];
    return MD_OK;
}

}  // namespace

extern "C" md_status md_bin_cells_noalloc(const double box[3], double r_list, int64_t n, const double *d_pos,
                                          int32_t *d_cell_start, int32_t *d_cell_atoms, void *cuda_stream)
{
    if (!box || n < 0 || !(r_list > 0.0) || !std::isfinite(r_list)) return MD_ERR_ARG;
    BinGeom G;
    long long ncells = 1;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0.0) || !std::isfinite(box[a])) return MD_ERR_ARG;
        double q = std::floor(box[a] / r_list);
        if (q < 3.0) return MD_ERR_BOX;                              // fewer than 3 cells on an axis
        if (q > (double)kNoAllocMaxCells) return MD_ERR_CAPACITY;    // beyond the cell maximum
        G.box[a] = box[a];
        G.ncell[a] = (int)q;
        G.inv_cell[a] = (double)G.ncell[a] / box[a];
        ncells *= G.ncell[a];
    }
    if (n > kNoAllocMaxAtoms) return MD_ERR_CAPACITY;        // more than 262,144 atoms
    if (ncells > kNoAllocMaxCells) return MD_ERR_CAPACITY;   // more than 65,536 cells
    if ((n > 0 && (!d_pos || !d_cell_atoms)) || !d_cell_start) return MD_ERR_ARG;
    G.ncells = (int)ncells;
    unsigned long long *scratch = nullptr;
    md_status rc = scratch_for_current_device(&scratch);
    if (rc != MD_OK) return rc;
    unsigned long long *keys = scratch;
    int *count = reinterpret_cast<int *>(scratch + kNoAllocMaxAtoms);
    int *block_sums = count + kNoAllocMaxCells;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int ncb = (G.ncells + 255) / 256;
    const int nsb = (G.ncells + kNbScanBlock - 1) / kNbScanBlock;
    unsigned nsort = kSortChunk;
    while (nsort < (unsigned)n) nsort <<= 1;  // <= kNoAllocMaxAtoms
    cudaError_t e = launch(k_nb_clear, ncb, 256, s, count, G.ncells);
    if (e == cudaSuccess && n > 0)
        e = launch(k_nb_bin, (nsort + 255) / 256, 256, s, d_pos, (int)n, (int)nsort, G, keys, count);
    if (e == cudaSuccess) e = launch(k_nb_block_sums, nsb, 256, s, (const int *)count, G.ncells, block_sums);
    if (e == cudaSuccess)
        e = launch(k_nb_scan, nsb, kNbScanBlock, s, (const int *)count, (const int *)block_sums, G.ncells,
                   (int *)d_cell_start);
    if (n > 0) {
        const unsigned chunks = nsort / kSortChunk;
        if (e == cudaSuccess) e = launch(k_nb_sort_chunk, chunks, kSortChunk / 2, s, keys, 2u, (unsigned)kSortChunk);
        for (unsigned k = 2 * kSortChunk; k <= nsort && e == cudaSuccess; k <<= 1) {
            for (unsigned j = k >> 1; j >= (unsigned)kSortChunk && e == cudaSuccess; j >>= 1)
                e = launch(k_nb_sort_step, nsort / 256, 256, s, keys, nsort, j, k);
            if (e == cudaSuccess) e = launch(k_nb_sort_chunk, chunks, kSortChunk / 2, s, keys, k, k);
        }
        if (e == cudaSuccess)
            e = launch(k_nb_extract, (unsigned)((n + 255) / 256), 256, s, (const unsigned long long *)keys, (int)n,
                       (int *)d_cell_atoms);
    }
    return e == cudaSuccess ? MD_OK : MD_ERR_CUDA;
}
