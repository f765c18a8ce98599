// kernels.cu -- sm_103a kernels of the EAM timestep.
//
// One step of the method (arXiv 2405.07898, Section "Locality-preserving Atom
// Mapping", the five-stage timestep) maps onto these kernels:
//   candidate exchange + neighbour list  -> k_bin .. k_build_list (every
//                                           rebuild, Section "Neighbor list")
//   embedding calculation and exchange   -> k_density: rho_i (Eq. 2) and
//                                           F'(rho_i), written to HBM; the
//                                           kernel boundary is the exchange
//   force calculation and integration    -> k_force: Eq. 4 and the two
//                                           velocity-Verlet half kicks and the
//                                           drift (Eq. 5), fused
//   atom swap                            -> the spatial re-sort inside the
//                                           rebuild (k_bin .. k_permute)
// R is the pair-arithmetic type: float in the mixed-precision path, double in
// the FP64 path.  Positions, velocities, the drift and all sums over atoms are
// FP64 in both paths.
#include "md_internal.cuh"

#include <cuda_runtime.h>
#include <type_traits>

namespace eammd {
namespace {

template <class R> __device__ __forceinline__ typename V4<R>::T mk4(R x, R y, R z, R w);
template <> __device__ __forceinline__ float4 mk4<float>(float x, float y, float z, float w)
{
    return make_float4(x, y, z, w);
}
template <> __device__ __forceinline__ double4_32a mk4<double>(double x, double y, double z, double w)
{
    return make_double4_32a(x, y, z, w);
}

// 1/r and r from r^2: one MUFU reciprocal square root in FP32, IEEE sqrt and
// division in FP64.
__device__ __forceinline__ void inv_r(float r2, float &rinv, float &r)
{
    rinv = rsqrtf(r2);
    r = r2 * rinv;
}
__device__ __forceinline__ void inv_r(double r2, double &rinv, double &r)
{
    r = sqrt(r2);
    rinv = 1.0 / r;
}

// Cubic spline in r on a table that covers [x0, x_end] with x0 <= 0 and
// x_end >= r_cut (checked on the host), for 0 <= r < r_cut.
template <class R>
__device__ __forceinline__ void spline_r(const SplineDesc<R> &s, const typename V4<R>::T *coef, R x,
                                         R &val, R &der)
{
    R u = (x - s.x0) * s.inv_h;
    int k = min((int)u, s.nint - 1);
    R kf = (R)k;
    R t = fma(-kf, s.h_lo, fma(-kf, s.h_hi, x - s.x0));
    typename V4<R>::T c = coef[s.offset + k];
    val = fma(t, fma(t, fma(t, c.w, c.z), c.y), c.x);
    der = fma(t, fma(t, (R)3 * c.w, (R)2 * c.z), c.y);
}

template <class R>
__device__ __forceinline__ R spline_r_der(const SplineDesc<R> &s, const typename V4<R>::T *coef, R x)
{
    R u = (x - s.x0) * s.inv_h;
    int k = min((int)u, s.nint - 1);
    R kf = (R)k;
    R t = fma(-kf, s.h_lo, fma(-kf, s.h_hi, x - s.x0));
    typename V4<R>::T c = coef[s.offset + k];
    return fma(t, fma(t, (R)3 * c.w, (R)2 * c.z), c.y);
}

// Cubic spline anywhere: outside the knot range it continues along the end
// tangent (used for the embedding function, whose argument is unbounded).
template <class R>
__device__ __forceinline__ bool spline_any(const SplineDesc<R> &s, const typename V4<R>::T *coef, R x,
                                           R &val, R &der)
{
    if (x < s.x0) {
        val = s.y_lo + s.s_lo * (x - s.x0);
        der = s.s_lo;
        return true;
    }
    if (x > s.x_end) {
        val = s.y_end + s.s_end * (x - s.x_end);
        der = s.s_end;
        return true;
    }
    spline_r(s, coef, x, val, der);
    return false;
}

__device__ __forceinline__ int pair_index(int nt, int a, int b)
{
    int lo = min(a, b), hi = max(a, b);
    return lo * nt - lo * (lo - 1) / 2 + (hi - lo);
}

// Shift of the 27 stencil cells, code = (dz+1)*9 + (dy+1)*3 + (dx+1):
// u_j + shift(code) - u_i is the displacement x_j - x_i of a listed pair.
template <class R>
__device__ __forceinline__ void fill_shift(typename V4<R>::T *sh, const Geom &G)
{
    for (int c = threadIdx.x; c < 27; c += blockDim.x) {
        int dx = c % 3 - 1, dy = (c / 3) % 3 - 1, dz = c / 9 - 1;
        sh[c] = mk4<R>((R)dx * (R)G.h[0], (R)dy * (R)G.h[1], (R)dz * (R)G.h[2], (R)0);
    }
    __syncthreads();
}

// Block-wide sums of NV doubles in a fixed order; thread 0 stores them to
// partials[(slot0 + k) * nblocks + blockIdx.x].  All threads must call.
template <int NV>
__device__ __forceinline__ void block_sums(double (&v)[NV], double *partials, int nblocks, int slot0)
{
    __shared__ double sm[32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sm[w][k];
            partials[(size_t)(slot0 + k) * nblocks + blockIdx.x] = s;
        }
    }
}

__device__ __forceinline__ void block_max_disp(float d2, unsigned int *dst)
{
    __shared__ float sm[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if (lane == 0) sm[warp] = d2;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < nw; ++w) m = fmaxf(m, sm[w]);
        if (m > 0.f) atomicMax(dst, __float_as_uint(m));
    }
}

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
// to the FP64 definition.
template <class R>
__global__ void k_build_list(Bufs<R> B, Geom G, int n, int ld, int cap)
{
    using R4 = typename V4<R>::T;
    __shared__ R4 sh[27];
    DevState *st = B.st;
    if (!st->need_rebuild) return;
    fill_shift<R>(sh, G);
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    int cnt = 0;
    if (p < n) {
        const int sp = st->sp, s = st->set;
        const double *const xr[3] = {B.xr[s][0], B.xr[s][1], B.xr[s][2]};
        const R4 *sw = B.shadow[sp];
        const R lo = (R)G.screen_lo, hi = (R)G.screen_hi;
        int cell = B.cell[p];
        int cx = cell % G.ncell[0], cy = (cell / G.ncell[0]) % G.ncell[1], cz = cell / (G.ncell[0] * G.ncell[1]);
        R4 up = sw[p];
        for (int code = 0; code < 27; ++code) {
            int ex = cx + code % 3 - 1, ey = cy + (code / 3) % 3 - 1, ez = cz + code / 9 - 1;
            ex += (ex < 0) ? G.ncell[0] : ((ex >= G.ncell[0]) ? -G.ncell[0] : 0);
            ey += (ey < 0) ? G.ncell[1] : ((ey >= G.ncell[1]) ? -G.ncell[1] : 0);
            ez += (ez < 0) ? G.ncell[2] : ((ez >= G.ncell[2]) ? -G.ncell[2] : 0);
            int e = (ez * G.ncell[1] + ey) * G.ncell[0] + ex;
            R4 shf = sh[code];
            int q1 = B.cell_start[e + 1];
            for (int q = B.cell_start[e]; q < q1; ++q) {
                if (q == p) continue;
                R4 uq = sw[q];
                R dx = (uq.x - up.x) + shf.x;
                R dy = (uq.y - up.y) + shf.y;
                R dz = (uq.z - up.z) + shf.z;
                R r2 = fma(dz, dz, fma(dy, dy, dx * dx));
                bool in = (r2 < lo) ? true : ((r2 > hi) ? false : exact_in_list(xr, p, q, G));
                if (in) {
                    if (cnt < cap) B.list[(size_t)cnt * ld + p] = (uint32_t)q | ((uint32_t)code << kCodeShift);
                    ++cnt;
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
        atomicMax(&st->max_nnb, m);
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

// Density pass, Eq. 2: rho_i = sum over listed j with r < r_cut of
// f_{t_j}(r_ij); then F'(rho_i) (and F(rho_i) when energies are wanted).
template <class R, bool MULTI, bool ENERGY>
__global__ void __launch_bounds__(256) k_density(Bufs<R> B, Geom G, Launch L)
{
    using R4 = typename V4<R>::T;
    __shared__ R4 sh[27];
    fill_shift<R>(sh, G);
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    const R4 *sw = B.shadow[sp];
    const Tables<R> &T = *B.tables;
    const R4 *coef = B.coef;
    const R rc2 = (R)G.rc2;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double e_embed = 0.0;
    if (i < L.n) {
        R4 ui = sw[i];
        int nn = B.nnb[i];
        int ti = MULTI ? B.type[s][i] : 0;
        SplineDesc<R> f0 = T.f[0];
        R rho = (R)0;
        const uint32_t *lp = B.list + i;
        for (int k = 0; k < nn; ++k) {
            uint32_t e = lp[(size_t)k * L.ld];
            int j = (int)(e & kIndexMask);
            R4 uj = sw[j];
            R4 shf = sh[e >> kCodeShift];
            R dx = (uj.x - ui.x) + shf.x;
            R dy = (uj.y - ui.y) + shf.y;
            R dz = (uj.z - ui.z) + shf.z;
            R r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            if (r2 < rc2) {
                R rinv, r;
                inv_r(r2, rinv, r);
                R val, der;
                if (MULTI) spline_r(T.f[B.type[s][j]], coef, r, val, der);
                else spline_r(f0, coef, r, val, der);
                rho += val;
            }
        }
        R Fv, Fd;
        if (spline_any(T.F[ti], coef, rho, Fv, Fd)) atomicAdd(&B.st->table_oor, 1ull);
        B.Fp[i] = Fd;
        e_embed = (double)Fv;
    }
    if (ENERGY) {
        double v[1] = {e_embed};
        block_sums<1>(v, B.partials, L.nblocks, 0);
    }
}

// Force pass, Eq. 4, fused with the integration of Eq. 5:
//   s_ij = phi'_{t_i t_j}(r) + F'_i f'_{t_j}(r) + F'_j f'_{t_i}(r),
//   F_i  = sum_j s_ij (x_j - x_i) / r,
// then (MODE_CLOSE*) the closing half kick v += F dt/(2m), and
// (MODE_CLOSE_OPEN) the next step's opening half kick and drift
// x += v dt, writing the next shadow coordinates and the displacement
// since the last list build.  MODE_MEASURE only stores the forces.
template <class R, bool MULTI, int MODE, bool ENERGY>
__global__ void __launch_bounds__(256) k_force(Bufs<R> B, Geom G, Launch L)
{
    using R4 = typename V4<R>::T;
    __shared__ R4 sh[27];
    fill_shift<R>(sh, G);
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    const R4 *sw = B.shadow[sp];
    const Tables<R> &T = *B.tables;
    const R4 *coef = B.coef;
    const R rc2 = (R)G.rc2;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // pair, ke, virial x6, spare
    float d2 = 0.f;
    if (i < L.n) {
        R4 ui = sw[i];
        R Fpi = B.Fp[i];
        int nn = B.nnb[i];
        int ti = MULTI ? B.type[s][i] : 0;
        SplineDesc<R> f0 = T.f[0], p0 = T.phi[0];
        R fx = 0, fy = 0, fz = 0;
        R ep = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
        const uint32_t *lp = B.list + i;
        for (int k = 0; k < nn; ++k) {
            uint32_t e = lp[(size_t)k * L.ld];
            int j = (int)(e & kIndexMask);
            R4 uj = sw[j];
            R4 shf = sh[e >> kCodeShift];
            R dx = (uj.x - ui.x) + shf.x;
            R dy = (uj.y - ui.y) + shf.y;
            R dz = (uj.z - ui.z) + shf.z;
            R r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            if (r2 < rc2) {
                R rinv, r;
                inv_r(r2, rinv, r);
                R Fpj = B.Fp[j];
                R phv, phd, fdj, fdi;
                if (MULTI) {
                    int tj = B.type[s][j];
                    spline_r(T.phi[pair_index(L.ntypes, ti, tj)], coef, r, phv, phd);
                    fdj = spline_r_der(T.f[tj], coef, r);
                    fdi = (tj == ti) ? fdj : spline_r_der(T.f[ti], coef, r);
                } else {
                    spline_r(p0, coef, r, phv, phd);
                    fdj = spline_r_der(f0, coef, r);
                    fdi = fdj;
                }
                R sij = fma(Fpj, fdi, fma(Fpi, fdj, phd));
                R sr = sij * rinv;
                fx = fma(sr, dx, fx);
                fy = fma(sr, dy, fy);
                fz = fma(sr, dz, fz);
                if (ENERGY) {
                    R hs = (R)(-0.5) * sr;
                    ep += (R)0.5 * phv;
                    w0 = fma(hs * dx, dx, w0);
                    w1 = fma(hs * dy, dy, w1);
                    w2 = fma(hs * dz, dz, w2);
                    w3 = fma(hs * dx, dy, w3);
                    w4 = fma(hs * dx, dz, w4);
                    w5 = fma(hs * dy, dz, w5);
                }
            }
        }
        if (!isfinite(fx + fy + fz)) atomicOr(&B.st->error, ERR_NONFINITE);
        R f[3] = {fx, fy, fz};
        double kq = L.half_kick[ti];
        double v[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = B.v[s][a][i];
        if (MODE == MODE_MEASURE || MODE == MODE_CLOSE) {
#pragma unroll
            for (int a = 0; a < 3; ++a) B.fcache[a][i] = f[a];
        }
        if (MODE != MODE_MEASURE) {
            if (std::is_same<R, float>::value && MODE == MODE_CLOSE_OPEN && !ENERGY) {
                // both half kicks at once: 2 * (F dt/(2m)) is exact in FP32
#pragma unroll
                for (int a = 0; a < 3; ++a) v[a] += (double)((R)2 * (f[a] * (R)kq));
            } else {
#pragma unroll
                for (int a = 0; a < 3; ++a) v[a] = fma((double)f[a], kq, v[a]);
            }
        }
        if (ENERGY) {
            double m2 = L.ke_factor[ti];
            acc[1] = m2 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            acc[0] = (double)ep;
            acc[2] = (double)w0; acc[3] = (double)w1; acc[4] = (double)w2;
            acc[5] = (double)w3; acc[6] = (double)w4; acc[7] = (double)w5;
        }
        if (MODE == MODE_CLOSE_OPEN && (ENERGY || !std::is_same<R, float>::value)) {
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] = fma((double)f[a], kq, v[a]);
        }
        if (MODE != MODE_MEASURE) {
#pragma unroll
            for (int a = 0; a < 3; ++a) B.v[s][a][i] = v[a];
        }
        if (MODE == MODE_CLOSE_OPEN) {
            double dn[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                dn[a] = fma(v[a], L.dt, B.d[a][i]);
                B.d[a][i] = dn[a];
            }
            R u0 = B.uref[0][i] + (R)dn[0], u1 = B.uref[1][i] + (R)dn[1], u2 = B.uref[2][i] + (R)dn[2];
            B.shadow[sp ^ 1][i] = mk4<R>(u0, u1, u2, (R)0);
            float gx = (float)dn[0], gy = (float)dn[1], gz = (float)dn[2];
            d2 = gx * gx + gy * gy + gz * gz;
        }
    }
    if (ENERGY) {
        double v8[8] = {acc[0], acc[1], acc[2], acc[3], acc[4], acc[5], acc[6], acc[7]};
        block_sums<8>(v8, B.partials, L.nblocks, 1);
    }
    if (MODE == MODE_CLOSE_OPEN) block_max_disp(d2, &B.st->maxdisp2);
}

// Fixed-order sum of the per-block partials: energies and virial.
template <class R>
__global__ void k_reduce(Bufs<R> B, int nblocks)
{
    __shared__ double sm[256];
    double out[9];
    for (int slot = 0; slot < 9; ++slot) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += B.partials[(size_t)slot * nblocks + b];
        sm[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
            __syncthreads();
        }
        out[slot] = sm[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        DevState *st = B.st;
        st->e_embed = out[0];
        st->e_pair = out[1];
        st->ke = out[2];
        for (int k = 0; k < 6; ++k) st->virial[k] = out[3 + k];
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

inline int blocks_for(int n, int b) { return (n + b - 1) / b; }

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
int launch_density(const Bufs<R> &B, const Geom &G, const Launch &L, bool energy)
{
    const bool multi = L.ntypes > 1;
    if (multi) {
        if (energy) k_density<R, true, true><<<L.nblocks, L.block, 0, L.stream>>>(B, G, L);
        else k_density<R, true, false><<<L.nblocks, L.block, 0, L.stream>>>(B, G, L);
    } else {
        if (energy) k_density<R, false, true><<<L.nblocks, L.block, 0, L.stream>>>(B, G, L);
        else k_density<R, false, false><<<L.nblocks, L.block, 0, L.stream>>>(B, G, L);
    }
    return 1;
}

template <class R, bool MULTI>
static void force_dispatch(const Bufs<R> &B, const Geom &G, const Launch &L, int mode, bool energy)
{
    dim3 g(L.nblocks), b(L.block);
    if (mode == MODE_MEASURE) {
        k_force<R, MULTI, MODE_MEASURE, true><<<g, b, 0, L.stream>>>(B, G, L);
    } else if (mode == MODE_CLOSE) {
        if (energy) k_force<R, MULTI, MODE_CLOSE, true><<<g, b, 0, L.stream>>>(B, G, L);
        else k_force<R, MULTI, MODE_CLOSE, false><<<g, b, 0, L.stream>>>(B, G, L);
    } else {
        if (energy) k_force<R, MULTI, MODE_CLOSE_OPEN, true><<<g, b, 0, L.stream>>>(B, G, L);
        else k_force<R, MULTI, MODE_CLOSE_OPEN, false><<<g, b, 0, L.stream>>>(B, G, L);
    }
}

template <class R>
int launch_force(const Bufs<R> &B, const Geom &G, const Launch &L, int mode, bool energy)
{
    if (L.ntypes > 1) force_dispatch<R, true>(B, G, L, mode, energy);
    else force_dispatch<R, false>(B, G, L, mode, energy);
    return 1;
}

template <class R>
int launch_reduce(const Bufs<R> &B, const Launch &L)
{
    k_reduce<R><<<1, 256, 0, L.stream>>>(B, L.nblocks);
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
    template int launch_density<R>(const Bufs<R> &, const Geom &, const Launch &, bool);        \
    template int launch_force<R>(const Bufs<R> &, const Geom &, const Launch &, int, bool);     \
    template int launch_reduce<R>(const Bufs<R> &, const Launch &);                             \
    template int launch_load_state<R>(const Bufs<R> &, const Launch &, const double *, const double *, \
                                      const int *);                                             \
    template int launch_store_state<R>(const Bufs<R> &, const Launch &, double *, double *, double *);

EAMMD_INSTANTIATE(float)
EAMMD_INSTANTIATE(double)

}  // namespace eammd
