// rebuild_device.cuh -- per-element device functions of the list rebuild,
// the opening kick and the energy reduction.  The kernels of rebuild.cu launch
// them one element per thread; the persistent step kernel (persistent.cu)
// runs them in grid-stride loops between grid barriers.  Every function takes
// the buffer set `s` and the record buffer `sp` explicitly.
#pragma once

#include "device_common.cuh"

namespace eammd {
namespace {

// x as a float truncated toward zero, from its bits by integer operations
// (the FP64 pipe of this GPU is narrow): 0 below 2^-126, +-inf above the
// float range.
__device__ __forceinline__ float trunc_to_float(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned e = (hi >> 20) & 0x7ffu;
    if (e < 897u) return 0.f;
    if (e > 1150u) return __uint_as_float((hi & 0x80000000u) | 0x7f800000u);
    return __uint_as_float((hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// Cell index floor(RN(x inv)) clamped to [0, n - 1], for finite x.  The FP32
// product of the truncated x and the rounded inv is within 2^-21.8 |q| of the
// FP64 product (truncation 2^-23, two roundings 2^-24 each); where it lies
// farther than 2^-20 max(|q|, 1) from every integer both have the same floor,
// elsewhere the FP64 product decides.
__device__ __forceinline__ int cell_index(double x, double inv, float inv_f, int n)
{
    const float q32 = trunc_to_float(x) * inv_f;
    const float f = floorf(q32), frac = q32 - f;
    const float tol = 0x1p-20f * fmaxf(fabsf(q32), 1.0f);
    if (frac > tol && frac < 1.0f - tol) return min(max((int)f, 0), n - 1);
    const double q = floor(__dmul_rn(x, inv));
    return (int)fmax(fmin(q, (double)(n - 1)), 0.0);
}

// Periodic image of x = xr + d on periodic axes: kept when already in
// [0, L), else x - L floor(x / L); then bin: c_d = floor(x_d n_d/L_d) clamped
// to [0, n_d - 1].  The box test compares bit patterns (non-negative doubles
// order as their bits; -0 is inside).  The slot inside the cell is the
// arrival order (fixed by sort_cell).
template <class R>
__device__ __forceinline__ void bin_atom(const Bufs<R> &B, const Geom &G, int s, int i)
{
    int c[3];
    bool finite = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double L = G.box[a];
        double x = __dadd_rn(B.xr[s][a][i], B.d[a][i]);
        const long long xb = __double_as_longlong(x);
        const bool inside = (xb >= 0 && xb < __double_as_longlong(L)) || xb == (long long)0x8000000000000000ull;
        if (!((G.open_mask >> a) & 1) && !inside) {
            // (open axis: not wrapped; outside the box, the edge cell takes it)
            const double q = floor(__ddiv_rn(x, L));
            x = __dsub_rn(x, __dmul_rn(L, q));
        }
        finite = finite && ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff;
        B.xw[a][i] = x;
        c[a] = finite ? cell_index(x, G.inv_cell[a], G.inv_cell_f[a], G.ncell[a]) : 0;
    }
    if (!finite) atomicOr(&B.st->error, ERR_NONFINITE);
    int cell = (c[2] * G.ncell[1] + c[1]) * G.ncell[0] + c[0];
    B.cell_old[i] = cell;
    // one atomic per distinct cell among the warp's active lanes (atoms in
    // cell order mostly share cells); the lanes of a cell take consecutive
    // slots from it in lane order
    const unsigned peers = __match_any_sync(__activemask(), cell);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&B.count[cell], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    B.slot[i] = base + __popc(peers & ((1u << lane) - 1u));
}

// Exclusive scan of all cell counts by one block (any size): cell_start[c] =
// sum_{c' < c} count[c'], counts zeroed for the next build.  Each thread
// scans a contiguous chunk; the chunk totals are scanned across the block.
template <class R>
__device__ __forceinline__ void scan_cells_block(const Bufs<R> &B, int ncells)
{
    __shared__ int tot[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int per = (ncells + nt - 1) / nt;
    const int c0 = min(t * per, ncells), c1 = min(c0 + per, ncells);
    int sum = 0;
    for (int c = c0; c < c1; ++c) sum += B.count[c];
    tot[t] = sum;
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int k = 0; k < nt; ++k) {
            const int v = tot[k];
            tot[k] = run;
            run += v;
        }
        B.cell_start[ncells] = run;
    }
    __syncthreads();
    int run = tot[t];
    for (int c = c0; c < c1; ++c) {
        const int v = B.count[c];
        B.cell_start[c] = run;
        B.count[c] = 0;
        run += v;
    }
    __syncthreads();
}

template <class R>
__device__ __forceinline__ void scatter_atom(const Bufs<R> &B, int i)
{
    B.cell_atoms[B.cell_start[B.cell_old[i]] + B.slot[i]] = i;
}

// Within cell c, order atoms by original id (the atomics of bin_atom leave
// them in arrival order); insertion sort, cells hold a handful of atoms.
template <class R>
__device__ __forceinline__ void sort_cell(const Bufs<R> &B, int s, int c)
{
    const int *id = B.id[s];
    int lo = B.cell_start[c], hi = B.cell_start[c + 1];
    for (int q = lo + 1; q < hi; ++q) {
        int a = B.cell_atoms[q];
        int ka = id[a];
        int r = q - 1;
        while (r >= lo && id[B.cell_atoms[r]] > ka) {
            B.cell_atoms[r + 1] = B.cell_atoms[r];
            --r;
        }
        B.cell_atoms[r + 1] = a;
    }
}

// Gather the state of atom p (cell order) into the other buffer set:
// positions become the wrapped positions, displacements restart at zero, and
// the cell-centred coordinates uref (and record buffer sp) are formed in FP64
// and rounded.
template <class R>
__device__ __forceinline__ void permute_atom(const Bufs<R> &B, const Geom &G, int s, int sp, int p)
{
    const int t = 1 - s;
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

// Exact list test for a candidate near the list radius: the minimum-image
// squared distance with the operations and rounding order of the definition
// (d = x_j - x_i, +-L once on periodic axes, (dx^2 + dy^2) + dz^2, no fused
// operations).
__device__ __forceinline__ bool exact_in_list(const double *const xr[3], int p, int q, const Geom &G)
{
    double d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = __dsub_rn(xr[a][q], xr[a][p]);
        if (!((G.open_mask >> a) & 1)) {
            if (x > G.half_box[a]) x = __dsub_rn(x, G.box[a]);
            else if (x < -G.half_box[a]) x = __dadd_rn(x, G.box[a]);
        }
        d[a] = x;
    }
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
    return r2 < G.rl2;
}

// Whether the pair vector d = x_q - x_p (minimum image) lies in the upper
// half space: d_z > 0, or d_z = 0 and d_y > 0, or d_z = d_y = 0 and d_x > 0.
// (dx, dy, dz) is the R-precision vector of the screen; where d_z is clearly
// away from zero (far beyond its rounding error) it decides, elsewhere the
// FP64 components of the definition do.  FP64 subtraction and the image
// shift are exactly antisymmetric, so the answers for (p, q) and (q, p) are
// complements: a pair is kept by exactly one of its atoms.
template <class R>
__device__ __forceinline__ bool upper_half(R dx, R dy, R dz, const double *const xr[3], int p, int q,
                                           const Geom &G)
{
    (void)dx;
    (void)dy;
    const R tol = (R)1e-4;
    if (dz > tol) return true;
    if (dz < -tol) return false;
    double d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = __dsub_rn(xr[a][q], xr[a][p]);
        if (!((G.open_mask >> a) & 1)) {
            if (x > G.half_box[a]) x = __dsub_rn(x, G.box[a]);
            else if (x < -G.half_box[a]) x = __dadd_rn(x, G.box[a]);
        }
        d[a] = x;
    }
    if (d[2] != 0.0) return d[2] > 0.0;
    if (d[1] != 0.0) return d[1] > 0.0;
    return d[0] > 0.0;
}

// Verlet list of atom p: the atoms of the 27 surrounding cells (in stencil
// order, ascending id inside a cell; cells beyond an open edge do not exist)
// closer than r_list.  The test runs in R
// on the cell-centred coordinates; candidates within the rounding margin of
// r_list are decided by exact_in_list, so the list is bit-identical to the
// FP64 definition.  The 9 rows of the stencil are unrolled; the 3 cells of a
// row are a loop (a fully unrolled stencil outgrows the instruction cache).
// Returns the neighbour count (the list keeps at most cap of them; more
// raises ERR_LIST_OVERFLOW).  half: keep each pair once, in the same order:
// only the neighbours q whose pair vector x_q - x_p lies in the upper half
// space (upper_half).  Every atom's neighbourhood is close to centrally
// symmetric, so each lists about half its neighbours.
template <class R>
__device__ __forceinline__ int list_atom(const Bufs<R> &B, const Geom &G, int s, int sp, int p, int ld, int cap,
                                         bool half = false)
{
    using R4 = typename V4<R>::T;
    int cnt = 0;
    const double *const xr[3] = {B.xr[s][0], B.xr[s][1], B.xr[s][2]};
    const R4 *sw = B.shadow[sp];
    const R lo = g_screen_lo<R>(G), hi = g_screen_hi<R>(G);
    const R hx = g_h<R>(G, 0), hy = g_h<R>(G, 1), hz = g_h<R>(G, 2);
    const int nx = G.ncell[0], ny = G.ncell[1], nz = G.ncell[2];
    const int cell = B.cell[p];
    const int cx = cell % nx, cy = (cell / nx) % ny, cz = cell / (nx * ny);
    const R4 up = sw[p];
    uint32_t *lp = B.list + p;
    const bool open_x = G.open_mask & 1, open_y = (G.open_mask >> 1) & 1, open_z = (G.open_mask >> 2) & 1;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        int ez = cz + dz;
        if (ez < 0 || ez >= nz) {
            if (open_z) continue;  // no cell beyond an open edge
            ez += (ez < 0) ? nz : -nz;
        }
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            int ey = cy + dy;
            if (ey < 0 || ey >= ny) {
                if (open_y) continue;
                ey += (ey < 0) ? ny : -ny;
            }
            const int row = (ez * ny + ey) * nx;
#pragma unroll 1
            for (int dx = -1; dx <= 1; ++dx) {
                int ex = cx + dx;
                if (ex < 0 || ex >= nx) {
                    if (open_x) continue;
                    ex += (ex < 0) ? nx : -nx;
                }
                const int e = row + ex;
                const uint32_t code = list_entry(0u, dx, dy, dz);
                const R ox = (R)dx * hx - up.x, oy = (R)dy * hy - up.y, oz = (R)dz * hz - up.z;
                const int q1 = B.cell_start[e + 1];
                for (int q = B.cell_start[e]; q < q1; ++q) {
                    const R4 uq = sw[q];
                    const R ddx = uq.x + ox, ddy = uq.y + oy, ddz = uq.z + oz;
                    const R r2 = fma(ddz, ddz, fma(ddy, ddy, ddx * ddx));
                    if (r2 > hi || q == p) continue;
                    if (half && !upper_half(ddx, ddy, ddz, xr, p, q, G)) continue;
                    if (r2 < lo || exact_in_list(xr, p, q, G)) {
                        if (cnt < cap) lp[(size_t)cnt * ld] = (uint32_t)q | code;
                        ++cnt;
                    }
                }
            }
        }
    }
    B.nnb[p] = min(cnt, cap);
    if (cnt > cap) atomicOr(&B.st->error, ERR_LIST_OVERFLOW);
    return cnt;
}

// list_atom with the 32 lanes of a warp on atom p: lane c < 27 walks
// stencil cell c = 9 (dz + 1) + 3 (dy + 1) + (dx + 1) -- the stencil order --
// issuing its candidates' record loads four at a time, and an exclusive warp
// prefix sum of the cells' hit counts gives each cell its place in the list,
// so the list is the one list_atom writes, entry for entry.  The walk per
// atom is a few rounds of independent loads (the cells in parallel) instead
// of a chain of ~27: for systems of a few thousand atoms, whose records were
// just written by other SMs, the chain's L2 round trips are the cost of the
// build.  A cell's decisions are kept as a bit mask for its first 64
// candidates and recomputed beyond them.  All 32 lanes must call; every lane
// returns the count.
template <class R>
__device__ __forceinline__ int list_atom_warp(const Bufs<R> &B, const Geom &G, int s, int sp, int p, int ld,
                                              int cap)
{
    using R4 = typename V4<R>::T;
    constexpr int UQ = 4;  // candidate loads in flight per lane
    const int lane = (int)(threadIdx.x & 31u);
    const double *const xr[3] = {B.xr[s][0], B.xr[s][1], B.xr[s][2]};
    const R4 *sw = B.shadow[sp];
    const R lo = g_screen_lo<R>(G), hi = g_screen_hi<R>(G);
    const R hx = g_h<R>(G, 0), hy = g_h<R>(G, 1), hz = g_h<R>(G, 2);
    const int nx = G.ncell[0], ny = G.ncell[1], nz = G.ncell[2];
    const int cell = B.cell[p];
    const int cx = cell % nx, cy = (cell / nx) % ny, cz = cell / (nx * ny);
    const R4 up = sw[p];
    const int dz = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dx = lane % 3 - 1;
    int ex = cx + dx, ey = cy + dy, ez = cz + dz;
    bool valid = lane < 27;
    if (ex < 0 || ex >= nx) {
        if (G.open_mask & 1) valid = false;
        else ex += (ex < 0) ? nx : -nx;
    }
    if (ey < 0 || ey >= ny) {
        if ((G.open_mask >> 1) & 1) valid = false;
        else ey += (ey < 0) ? ny : -ny;
    }
    if (ez < 0 || ez >= nz) {
        if ((G.open_mask >> 2) & 1) valid = false;
        else ez += (ez < 0) ? nz : -nz;
    }
    int q0 = 0, q1 = 0;
    if (valid) {
        const int e = (ez * ny + ey) * nx + ex;
        q0 = B.cell_start[e];
        q1 = B.cell_start[e + 1];
    }
    const R ox = (R)dx * hx - up.x, oy = (R)dy * hy - up.y, oz = (R)dz * hz - up.z;
    auto in_list = [&](const R4 &uq, int q) -> bool {
        const R ddx = uq.x + ox, ddy = uq.y + oy, ddz = uq.z + oz;
        const R r2 = fma(ddz, ddz, fma(ddy, ddy, ddx * ddx));
        return !(r2 > hi || q == p) && (r2 < lo || exact_in_list(xr, p, q, G));
    };
    unsigned long long bits = 0ull;
    int hits = 0;
    for (int q = q0; q < q1; q += UQ) {
        R4 u[UQ];
#pragma unroll
        for (int k = 0; k < UQ; ++k) u[k] = sw[min(q + k, q1 - 1)];
#pragma unroll
        for (int k = 0; k < UQ; ++k) {
            if (q + k < q1 && in_list(u[k], q + k)) {
                if (q + k - q0 < 64) bits |= 1ull << (q + k - q0);
                ++hits;
            }
        }
    }
    int incl = hits;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int pos = incl - hits;
    uint32_t *lp = B.list + p;
    const uint32_t code = list_entry(0u, dx, dy, dz);
    while (bits) {
        const int k = __ffsll((long long)bits) - 1;
        bits &= bits - 1ull;
        if (pos < cap) lp[(size_t)pos * ld] = (uint32_t)(q0 + k) | code;
        ++pos;
    }
    for (int q = q0 + 64; q < q1; ++q)
        if (in_list(sw[q], q)) {
            if (pos < cap) lp[(size_t)pos * ld] = (uint32_t)q | code;
            ++pos;
        }
    if (lane == 0) {
        B.nnb[p] = min(total, cap);
        if (total > cap) atomicOr(&B.st->error, ERR_LIST_OVERFLOW);
    }
    return total;
}

// Block maximum of the neighbour counts into st->max_nnb (one atomic per
// block).  All threads must call.
__device__ __forceinline__ void block_max_nnb(int cnt, int *dst)
{
    __shared__ int smax[32];
    int m = cnt;
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)((blockDim.x + 31) >> 5); ++w) m = max(m, smax[w]);
        if (m > *(volatile int *)dst) atomicMax(dst, m);
    }
    __syncthreads();
}

// Opening kick and drift of atom i from the forces cached at the last closed
// step: v += F dt/(2m), x += v dt; record buffer sp ^ 1 gets the new
// coordinates.  Returns the squared displacement since the last build (FP32).
template <class R>
__device__ __forceinline__ float open_atom(const Bufs<R> &B, const Launch &L, int s, int sp, int i)
{
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
    return fx * fx + fy * fy + fz * fz;
}

// Sum of partials[slot * stride + b], b < nb, by one block (any size) in a
// fixed order; the result goes to the DevState field of the slot (0: embedding
// energy, 1: pair energy, 2: kinetic energy, 3..8: virial).
__device__ __forceinline__ void reduce_slot(const double *partials, DevState *st, int slot, int nb, int stride)
{
    __shared__ double sm[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partials[(size_t)slot * stride + b];
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
        if (slot == 0) st->e_embed = t;
        else if (slot == 1) st->e_pair = t;
        else if (slot == 2) st->ke = t;
        else st->virial[slot - 3] = t;
    }
    __syncthreads();
}

}  // namespace
}  // namespace eammd
