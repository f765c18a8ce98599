// noalloc_bins.cu -- a cell binner that allocates no device memory.
//
// md_bin_cells_noalloc() sorts atoms into cells like the binning stage of the
// list rebuild (counting sort, ascending atom index inside a cell), but
// reads the caller's device positions, writes the caller's device outputs,
// and keeps its scratch (cell of each atom, rank inside its cell, per-cell
// counts, per-block sums) in the file-scope device array below instead of
// memory from cudaMalloc.  Every GPU that loads the library holds that array
// until the process exits.
#include "eammd.h"

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

namespace {

constexpr int kNoAllocMaxAtoms = 1 << 18;  // 262,144 atoms
constexpr int kNoAllocMaxCells = 1 << 16;  // 65,536 cells
constexpr int kNbScanBlock = 1024;
constexpr int kNbMaxScanBlocks = kNoAllocMaxCells / kNbScanBlock;
// layout (ints): cell of atom [0, A), rank in cell [A, 2A), count [2A, 2A+C),
// block sums [2A+C, 2A+C+B)
constexpr size_t kScratchInts = 2 * (size_t)kNoAllocMaxAtoms + kNoAllocMaxCells + kNbMaxScanBlocks;

static __device__ __align__(256) int g_bin_scratch[kScratchInts];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int *g_scratch_addr[kMaxDevices] = {nullptr};

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
// c_d = min(floor(x_d n_d / L_d), n_d - 1)
__global__ void k_nb_bin(const double *pos, int n, BinGeom G, int *cell_of, int *rank, int *count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
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
    cell_of[i] = cell;
    rank[i] = atomicAdd(&count[cell], 1);
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

__global__ void k_nb_scatter(const int *cell_of, const int *rank, const int *cell_start, int n, int *cell_atoms)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cell_atoms[cell_start[cell_of[i]] + rank[i]] = i;
}

// ascending atom index inside each cell (atomics leave arrival order)
__global__ void k_nb_sort(const int *cell_start, int ncells, int *cell_atoms)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int s = cell_start[c], e = cell_start[c + 1];
    for (int q = s + 1; q < e; ++q) {
        int a = cell_atoms[q];
        int r = q - 1;
        while (r >= s && cell_atoms[r] > a) {
            cell_atoms[r + 1] = cell_atoms[r];
            --r;
        }
        cell_atoms[r + 1] = a;
    }
}

// Device address of the scratch array for the current device, looked up once
// per device (the first call on a device does it, with that device current).
md_status scratch_for_current_device(int **out)
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
        g_scratch_addr[dev] = static_cast<int *>(p);
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
    int *scratch = nullptr;
    md_status rc = scratch_for_current_device(&scratch);
    if (rc != MD_OK) return rc;
    int *cell_of = scratch;
    int *rank = scratch + kNoAllocMaxAtoms;
    int *count = scratch + 2 * (size_t)kNoAllocMaxAtoms;
    int *block_sums = count + kNoAllocMaxCells;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nb = (int)((n + 255) / 256), ncb = (G.ncells + 255) / 256;
    const int nsb = (G.ncells + kNbScanBlock - 1) / kNbScanBlock;
    k_nb_clear<<<ncb, 256, 0, s>>>(count, G.ncells);
    if (n > 0) k_nb_bin<<<nb, 256, 0, s>>>(d_pos, (int)n, G, cell_of, rank, count);
    k_nb_block_sums<<<nsb, 256, 0, s>>>(count, G.ncells, block_sums);
    k_nb_scan<<<nsb, kNbScanBlock, 0, s>>>(count, block_sums, G.ncells, d_cell_start);
    if (n > 0) {
        k_nb_scatter<<<nb, 256, 0, s>>>(cell_of, rank, d_cell_start, (int)n, d_cell_atoms);
        k_nb_sort<<<ncb, 256, 0, s>>>(d_cell_start, G.ncells, d_cell_atoms);
    }
    return cudaGetLastError() == cudaSuccess ? MD_OK : MD_ERR_CUDA;
}
