// pair_kernels.cuh -- the density and force passes of the EAM timestep.
//
// Two schedules share the per-atom work:
//   * atom-parallel (k_density, k_force): TPA lanes cooperate on one atom;
//     lane l walks list columns l, l+TPA, ... a few at a time (every gather
//     of a round issued before any is used: three pairs a round in the
//     density pass, two in the force pass with the next round in flight),
//     the lanes' sums meet by warp shuffles; neighbour records are gathered
//     from global memory;
//   * row-staged (k_density_rows, k_force_rows): one block per row of cells
//     (all cx for a fixed cy, cz) first copies the records of the 3 x 3 rows
//     around it -- every neighbour its atoms can have -- into shared memory
//     with coalesced loads, then gathers from there.  A list entry's stencil
//     code names the row its neighbour lives in, so the shared-memory slot is
//     the neighbour's index minus that row's base.  Blocks whose neighbourhood
//     exceeds the staging capacity gather from global memory instead.
// The neighbour record is the 16-byte shadow (u_x, u_y, u_z, F'_j): one
// gather gives the force pass both the position and the embedding derivative
// the density pass stored.  With one atom type whose f and phi share a knot
// grid, both splines of an interval sit in one 32-byte row (coef2), read with
// one 256-bit load.
#pragma once

#include "device_common.cuh"

#include <type_traits>

namespace eammd {
namespace {

template <class R> struct PairIn {
    R dx, dy, dz, r2;
};

template <class R>
__device__ __forceinline__ PairIn<R> pair_vector(const typename V4<R>::T &ui, const typename V4<R>::T &uj,
                                                 const Shift<R> &shf)
{
    PairIn<R> p;
    p.dx = (uj.x - ui.x) + shf.x;
    p.dy = (uj.y - ui.y) + shf.y;
    p.dz = (uj.z - ui.z) + shf.z;
    p.r2 = fma(p.dz, p.dz, fma(p.dy, p.dy, p.dx * p.dx));
    return p;
}

// Both 16-byte halves of a 32-byte fused row with one 256-bit load.
template <class R>
__device__ __forceinline__ void load_row2(const typename V4<R>::T *row, typename V4<R>::T &a, typename V4<R>::T &b);
template <>
__device__ __forceinline__ void load_row2<float>(const float4 *row, float4 &a, float4 &b)
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(row));
}
template <>
__device__ __forceinline__ void load_row2<double>(const double4_32a *row, double4_32a &a, double4_32a &b)
{
    a = row[0];
    b = row[1];
}

template <int TPA, class T>
__device__ __forceinline__ T lane_sum(T v)
{
#pragma unroll
    for (int o = TPA / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Where a list entry's neighbour record is read from.
template <class R>
struct GlobalFetch {
    const typename V4<R>::T *sw;
    __device__ __forceinline__ typename V4<R>::T operator()(uint32_t e) const { return sw[e & kIndexMask]; }
};

template <class R>
struct StagedFetch {
    const typename V4<R>::T *stage;
    const int *base;  // per neighbour row (entry_row): first atom index minus its stage offset
    __device__ __forceinline__ typename V4<R>::T operator()(uint32_t e) const
    {
        return stage[(int)(e & kIndexMask) - base[entry_row(e)]];
    }
};

// Where the spline rows of the one-type path are read from: coef2 in device
// memory (row 2k: f, row 2k+1: phi, both in one 32-byte load; the density
// pass reads the f rows alone from coef_f, where a 128-byte line holds eight
// intervals instead of four) or a copy in shared memory with the f and phi
// rows in two arrays, so that 16-byte reads at scattered rows spread over
// all banks.
template <class R>
struct TabGlobal {
    const typename V4<R>::T *coef2;
    const typename V4<R>::T *coef_f;  // f rows alone: more intervals per cache line
    __device__ __forceinline__ typename V4<R>::T f(int kk) const { return coef_f[kk]; }
    __device__ __forceinline__ void fphi(int kk, typename V4<R>::T &cf, typename V4<R>::T &cp) const
    {
        load_row2<R>(coef2 + 2 * kk, cf, cp);
    }
};
struct TabShared {
    const float4 *f_rows, *phi_rows;
    __device__ __forceinline__ float4 f(int kk) const { return f_rows[kk]; }
    __device__ __forceinline__ void fphi(int kk, float4 &cf, float4 &cp) const
    {
        cf = f_rows[kk];
        cp = phi_rows[kk];
    }
};

// Where list column k of the lane's atom is read from.
struct ListGlobal {
    const uint32_t *lp;  // list + i
    int ld;
    __device__ __forceinline__ uint32_t operator()(int k) const { return lp[(size_t)k * ld]; }
};
struct ListTile {
    const uint32_t *tp;  // tile + (i - i0)
    int width;           // atoms per tile column
    __device__ __forceinline__ uint32_t operator()(int k) const { return tp[k * width]; }
};

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of an mbarrier for at most limit_ns.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns)
{
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s: for copies still in flight after a timeout

// Columns 0 .. ncol-1 of the list of atoms [i0, i0 + width) into the block's
// tile (column k at tile + k * width) by bulk asynchronous copies, one per
// column, that complete on one mbarrier.  Every column is a contiguous,
// 128-byte aligned run of the list (ld and width are multiples of 32 atoms).
// Returns false (and flags ERR_TIMEOUT) if the copies did not land within
// wait_ns; the caller then reads the list from device memory.
__device__ __forceinline__ bool stage_list(const uint32_t *list, int ld, int i0, int width, int ncol,
                                           uint32_t *tile, unsigned int *err, uint64_t wait_ns)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t bar_a = (uint32_t)__cvta_generic_to_shared(&bar);
    const int w = min(width, ld - i0);
    const uint32_t col_bytes = (uint32_t)w * 4u;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(col_bytes * (uint32_t)ncol)
                     : "memory");
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int k = threadIdx.x; k < ncol; k += 32) {
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(tile + (size_t)k * width);
            const uint32_t *src = list + (size_t)k * ld + i0;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                "l"(src), "r"(col_bytes), "r"(bar_a)
                : "memory");
        }
    }
    if (mbar_wait(bar_a, 0, wait_ns)) return true;
    atomicOr(err, ERR_TIMEOUT);
    mbar_wait(bar_a, 0, kWaitLimitNs);  // the copies still own the tile
    return false;
}

// This lane's part of rho_i = sum over listed j with r < r_cut of f_{t_j}(r_ij)
// (Eq. 2).
// In the force pass the list columns of the first round are read before the
// neighbour count is known (every column below cap lies inside the list);
// while a round is computed, the next round's records and the columns of the
// round after are in flight.  Columns at or beyond nn never address a record.
template <class R, bool MULTI, int TPA, int U, class List, class Fetch, class Tab>
__device__ __forceinline__ R density_lane(const Bufs<R> &B, const R (&h)[3], R rc2, int s, const int *nnb_i,
                                          int cap, int l, const typename V4<R>::T &ui, const List &list,
                                          const Fetch &fetch, const Tab &tab)
{
    using R4 = typename V4<R>::T;
    const Tables<R> &T = *B.tables;
    const SplineDesc<R> g = MULTI ? T.f[0] : T.fphi;
    R rho = (R)0;
    (void)cap;
    const int nn = *nnb_i;
    // U pairs per round (columns k, k + TPA, ...), all gathers issued before
    // any is used; the sum runs in column order
    for (int k = l; k < nn; k += U * TPA) {
        uint32_t e[U];
#pragma unroll
        for (int q = 0; q < U; ++q) e[q] = (k + q * TPA < nn) ? list(k + q * TPA) : 0u;
        R4 u[U];
#pragma unroll
        for (int q = 0; q < U; ++q) u[q] = fetch(q == 0 || k + q * TPA < nn ? e[q] : e[0]);
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const PairIn<R> p = pair_vector<R>(ui, u[q], entry_shift<R>(e[q], h));
            if ((q == 0 || k + q * TPA < nn) && p.r2 < rc2) {
                R rinv, r;
                inv_r(p.r2, rinv, r);
                if (MULTI) {
                    R val, der;
                    const int j = (int)(e[q] & kIndexMask);
                    spline_r(T.f[B.type[s][j]], B.coef, r, val, der);
                    rho += val;
                } else {
                    R t;
                    const int kk = segment(g, r, t);
                    const R4 c = tab.f(kk);
                    rho += fma(t, fma(t, fma(t, c.w, c.z), c.y), c.x);
                }
            }
        }
    }
    return rho;
}

// F'(rho_i) into the atom's record (w word) and F(rho_i) for the energy.
template <class R>
__device__ __forceinline__ R embed(const Bufs<R> &B, typename V4<R>::T *sw, int i, int ti, R rho)
{
    const Tables<R> &T = *B.tables;
    R Fv, Fd;
    if (spline_any(T.F[ti], B.coef, rho, Fv, Fd)) atomicAdd(&B.st->table_oor, 1ull);
    // the force pass reads w with the coordinates; the density pass never does
    reinterpret_cast<R *>(sw + i)[3] = Fd;
    return Fv;
}

// This lane's part of the force of Eq. 4,
//   s_ij = phi'_{t_i t_j}(r) + F'_i f'_{t_j}(r) + F'_j f'_{t_i}(r),
//   F_i  = sum_j s_ij (x_j - x_i) / r,
// and, when ENERGY, of the pair energy and the virial (e7: pair energy, then
// W xx yy zz xy xz yz).
template <class R, bool MULTI, bool ENERGY, int TPA, int U, class List, class Fetch, class Tab>
__device__ __forceinline__ void force_lane(const Bufs<R> &B, const Launch &L, const R (&h)[3], R rc2,
                                           int s, const int *nnb_i, int l, int ti, const typename V4<R>::T &ui,
                                           const List &list, const Fetch &fetch, R (&f)[3], R (&e7)[7],
                                           const Tab &tab)
{
    using R4 = typename V4<R>::T;
    const Tables<R> &T = *B.tables;
    const SplineDesc<R> g = T.fphi;
    const R Fpi = ui.w;
    constexpr int W = U * TPA;  // columns per round
    uint32_t e[U], en[U];
    R4 u[U];
#pragma unroll
    for (int q = 0; q < U; ++q) e[q] = (l + q * TPA < L.cap) ? list(l + q * TPA) : 0u;
    const int nn = *nnb_i;
#pragma unroll
    for (int q = 0; q < U; ++q) en[q] = (l + W + q * TPA < nn) ? list(l + W + q * TPA) : 0u;
#pragma unroll
    for (int q = 0; q < U; ++q) u[q] = (l < nn) ? fetch(q == 0 || l + q * TPA < nn ? e[q] : e[0]) : ui;
    for (int k = l; k < nn; k += W) {
        // in flight while this round is computed: the next round's records
        // and the columns of the round after
        const int k1 = k + W;
        R4 un[U];
        uint32_t e2[U];
#pragma unroll
        for (int q = 0; q < U; ++q) un[q] = (k1 < nn) ? fetch(q == 0 || k1 + q * TPA < nn ? en[q] : en[0]) : ui;
#pragma unroll
        for (int q = 0; q < U; ++q) e2[q] = (k1 + W + q * TPA < nn) ? list(k1 + W + q * TPA) : 0u;
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const PairIn<R> p = pair_vector<R>(ui, u[q], entry_shift<R>(e[q], h));
            if ((q == 0 || k + q * TPA < nn) && p.r2 < rc2) {
                R rinv, r;
                inv_r(p.r2, rinv, r);
                const R Fpj = u[q].w;
                R phv, phd, fdj, fdi;
                if (MULTI) {
                    const int j = (int)(e[q] & kIndexMask);
                    const int tj = B.type[s][j];
                    spline_r(T.phi[pair_index(L.ntypes, ti, tj)], B.coef, r, phv, phd);
                    fdj = spline_r_der(T.f[tj], B.coef, r);
                    fdi = (tj == ti) ? fdj : spline_r_der(T.f[ti], B.coef, r);
                } else {
                    R t;
                    const int kk = segment(g, r, t);
                    R4 cf, cp;
                    tab.fphi(kk, cf, cp);
                    fdj = fma(t, fma(t, (R)3 * cf.w, (R)2 * cf.z), cf.y);
                    fdi = fdj;
                    phd = fma(t, fma(t, (R)3 * cp.w, (R)2 * cp.z), cp.y);
                    phv = ENERGY ? fma(t, fma(t, fma(t, cp.w, cp.z), cp.y), cp.x) : (R)0;
                }
                const R sij = fma(Fpj, fdi, fma(Fpi, fdj, phd));
                const R sr = sij * rinv;
                f[0] = fma(sr, p.dx, f[0]);
                f[1] = fma(sr, p.dy, f[1]);
                f[2] = fma(sr, p.dz, f[2]);
                if (ENERGY) {
                    const R hs = (R)(-0.5) * sr;
                    e7[0] += (R)0.5 * phv;
                    e7[1] = fma(hs * p.dx, p.dx, e7[1]);
                    e7[2] = fma(hs * p.dy, p.dy, e7[2]);
                    e7[3] = fma(hs * p.dz, p.dz, e7[3]);
                    e7[4] = fma(hs * p.dx, p.dy, e7[4]);
                    e7[5] = fma(hs * p.dx, p.dz, e7[5]);
                    e7[6] = fma(hs * p.dy, p.dz, e7[6]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            e[q] = en[q];
            en[q] = e2[q];
            u[q] = un[q];
        }
    }
}

// Integration of Eq. 5 for the components this lane owns (c = l, l + TPA,
// ... < 3) once the lanes' forces are summed: MODE_CLOSE* applies the closing
// half kick v += F dt/(2m); MODE_CLOSE_OPEN also the next step's opening
// half kick and the drift x += v dt, writing the next record and the
// displacement since the last list build; MODE_MEASURE only stores F.
template <class R, int MODE, bool ENERGY, int TPA>
__device__ __forceinline__ void integrate(const Bufs<R> &B, const Launch &L, int s, int sp, int i, int l, int ti,
                                          const R (&f)[3], double &ke, float &d2)
{
    if (l == 0 && !isfinite(f[0] + f[1] + f[2])) atomicOr(&B.st->error, ERR_NONFINITE);
    const double kq = L.half_kick[ti];
    for (int c = l; c < 3; c += TPA) {
        const R fc = (c == 0) ? f[0] : ((c == 1) ? f[1] : f[2]);
        if (MODE == MODE_MEASURE || MODE == MODE_CLOSE) B.fcache[c][i] = fc;
        double v = B.v[s][c][i];
        if (MODE != MODE_MEASURE) {
            if (std::is_same<R, float>::value && MODE == MODE_CLOSE_OPEN && !ENERGY) {
                // both half kicks at once: 2 (F dt/(2m)) is exact in FP32
                v += (double)((R)2 * (fc * (R)kq));
            } else {
                v = fma((double)fc, kq, v);
            }
        }
        if (ENERGY) ke += L.ke_factor[ti] * v * v;
        if (MODE == MODE_CLOSE_OPEN && (ENERGY || !std::is_same<R, float>::value)) v = fma((double)fc, kq, v);
        if (MODE != MODE_MEASURE) B.v[s][c][i] = v;
        if (MODE == MODE_CLOSE_OPEN) {
            const double dn = fma(v, L.dt, B.d[c][i]);
            B.d[c][i] = dn;
            reinterpret_cast<R *>(B.shadow[sp ^ 1] + i)[c] = B.uref[c][i] + (R)dn;
            const float gc = (float)dn;
            d2 += gc * gc;
        }
    }
}

template <class R, bool ENERGY>
__device__ __forceinline__ void force_block_end(const Bufs<R> &B, const Launch &L, const R (&e7)[7], double ke,
                                                float d2max, bool open)
{
    if (ENERGY) {
        // the kinetic energy is formed in FP64 and carried as a pair of R
        const R ke_hi = (R)ke;
        const R ke_lo = (R)(ke - (double)ke_hi);
        const R v8[8] = {e7[0], ke_hi, e7[1], e7[2], e7[3], e7[4], e7[5], e7[6]};
        const R lo8[8] = {0, ke_lo, 0, 0, 0, 0, 0, 0};
        block_sums_t<8, R>(v8, B.partials, L.pstride, 1, lo8);
    }
    if (open) block_max_disp(d2max, &B.st->maxdisp2);
}

// ---- L2 prefetch of a warp's streams ----

constexpr bool kPrefetchWarpStreams = true;

__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p)));
}

// Ask L2 for the lines a warp of the atom-parallel passes streams from
// device memory, atoms [a0, a0 + m): the list columns up to the longest list
// of the last build and, in the force pass, the velocities, displacements
// and reference coordinates its integration reads.  A hint: nothing waits on
// it, and every address lies inside its array.
template <class R, bool FORCE>
__device__ __forceinline__ void prefetch_warp_streams(const Bufs<R> &B, const Launch &L, int s, int a0, int m,
                                                      int ncol)
{
    if (!kPrefetchWarpStreams || a0 >= L.n) return;
    const int lane = threadIdx.x & 31;
    for (int k = lane; k < ncol; k += 32) prefetch_l2(B.list + (size_t)k * L.ld + a0);
    if (FORCE) {
        // 128-byte lines: 16 doubles or 128 / sizeof(R) reference coordinates
        const int last = min(a0 + m, L.n) - 1;
        const int k = lane;
        if (k < 6) {
            const int c = k % 3;
            const int a = (k < 3) ? a0 : min(a0 + 16, last);
            prefetch_l2(B.v[s][c] + a);
            prefetch_l2(B.d[c] + a);
        } else if (k < 9) {
            prefetch_l2(B.uref[k - 6] + a0);
        } else if (k < 12 && sizeof(R) == 8) {
            prefetch_l2(B.uref[k - 9] + min(a0 + 16, last));
        }
    }
}

// ---- atom-parallel schedule ----

// Pairs in flight per lane: the type-dependent path needs more registers a pair.
template <bool MULTI> struct PairsInFlight {
    static constexpr int density = MULTI ? 2 : 3;
    static constexpr int force = 2;
};

extern __shared__ __align__(32) unsigned char dyn[];

// LS: the block's list tile is brought into shared memory by bulk copies
// first (one-type path only), so that the lanes' gathers do not wait on the
// list stream.
template <class R, bool MULTI, bool ENERGY, int TPA, bool LS>
__global__ void __launch_bounds__(256) k_density(Bufs<R> B, Geom G, Launch L)
{
    using R4 = typename V4<R>::T;
    constexpr int U = PairsInFlight<MULTI>::density;
    R h[3];
    load_h<R>(G, h);
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    R4 *sw = B.shadow[sp];
    const int width = blockDim.x / TPA;
    const int i0 = blockIdx.x * width;
    uint32_t *tile = reinterpret_cast<uint32_t *>(dyn);
    if (!LS) prefetch_warp_streams<R, false>(B, L, s, i0 + (threadIdx.x >> 5) * (32 / TPA), 32 / TPA, min(st->max_nnb, L.cap));
    const bool tiled = LS && stage_list(B.list, L.ld, i0, width, min(st->max_nnb, L.cap), tile, &B.st->error, L.wait_ns);
    const int i = i0 + threadIdx.x / TPA, l = threadIdx.x % TPA;
    const bool active = i < L.n;
    const int ti = (MULTI && active) ? B.type[s][i] : 0;
    const R rc2 = g_rc2<R>(G);
    R rho = (R)0;
    if (active) {
        if (tiled)
            rho = density_lane<R, MULTI, TPA, U>(B, h, rc2, s, B.nnb + i, L.cap, l, sw[i], ListTile{tile + (i - i0), width},
                                                 GlobalFetch<R>{sw}, TabGlobal<R>{B.coef2, B.coef_f});
        else
            rho = density_lane<R, MULTI, TPA, U>(B, h, rc2, s, B.nnb + i, L.cap, l, sw[i], ListGlobal{B.list + i, L.ld},
                                                 GlobalFetch<R>{sw}, TabGlobal<R>{B.coef2, B.coef_f});
    }
    rho = lane_sum<TPA>(rho);
    R e_embed = (R)0;
    if (active && l == 0) e_embed = embed<R>(B, sw, i, ti, rho);
    if (ENERGY) {
        const R v[1] = {e_embed};
        block_sums_t<1, R>(v, B.partials, L.pstride, 0);
    }
}

template <class R, bool MULTI, int MODE, bool ENERGY, int TPA, bool LS>
__global__ void __launch_bounds__(256) k_force(Bufs<R> B, Geom G, Launch L)
{
    using R4 = typename V4<R>::T;
    constexpr int U = PairsInFlight<MULTI>::force;
    R h[3];
    load_h<R>(G, h);
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    const R4 *sw = B.shadow[sp];
    const int width = blockDim.x / TPA;
    const int i0 = blockIdx.x * width;
    uint32_t *tile = reinterpret_cast<uint32_t *>(dyn);
    prefetch_warp_streams<R, true>(B, L, s, i0 + (threadIdx.x >> 5) * (32 / TPA), 32 / TPA, LS ? 0 : min(st->max_nnb, L.cap));
    const bool tiled = LS && stage_list(B.list, L.ld, i0, width, min(st->max_nnb, L.cap), tile, &B.st->error, L.wait_ns);
    const int i = i0 + threadIdx.x / TPA, l = threadIdx.x % TPA;
    const bool active = i < L.n;
    const int ti = (MULTI && active) ? B.type[s][i] : 0;
    const R rc2 = g_rc2<R>(G);
    R f[3] = {0, 0, 0};
    R e7[7] = {0, 0, 0, 0, 0, 0, 0};
    if (active) {
        if (tiled)
            force_lane<R, MULTI, ENERGY, TPA, U>(B, L, h, rc2, s, B.nnb + i, l, ti, sw[i], ListTile{tile + (i - i0), width},
                                                 GlobalFetch<R>{sw}, f, e7, TabGlobal<R>{B.coef2, B.coef_f});
        else
            force_lane<R, MULTI, ENERGY, TPA, U>(B, L, h, rc2, s, B.nnb + i, l, ti, sw[i], ListGlobal{B.list + i, L.ld},
                                                 GlobalFetch<R>{sw}, f, e7, TabGlobal<R>{B.coef2, B.coef_f});
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] = lane_sum<TPA>(f[c]);
    double ke = 0.0;
    float d2 = 0.f;
    if (active) integrate<R, MODE, ENERGY, TPA>(B, L, s, sp, i, l, ti, f, ke, d2);
    force_block_end<R, ENERGY>(B, L, e7, ke, lane_sum<TPA>(d2), MODE == MODE_CLOSE_OPEN);
}

// ---- row-staged schedule (one atom type, fused tables) ----

// Ranges of the 3 x 3 rows around row (cy, cz) and the stage layout; the
// records are copied in when they fit.  Returns whether the block stages.
template <class R>
__device__ __forceinline__ bool stage_rows(const Bufs<R> &B, const Geom &G, const Launch &L, const typename V4<R>::T *sw,
                                           typename V4<R>::T *stage, int *base, int *rstart, int *rcount, int row)
{
    __shared__ int off[10];
    __shared__ int ok;
    const int nx = G.ncell[0], ny = G.ncell[1], nz = G.ncell[2];
    const int cy = row % ny, cz = row / ny;
    if (threadIdx.x < 9) {
        const int t = threadIdx.x;
        int ey = cy + t % 3 - 1, ez = cz + t / 3 - 1;
        const bool gone = ((ey < 0 || ey >= ny) && ((G.open_mask >> 1) & 1)) ||
                          ((ez < 0 || ez >= nz) && ((G.open_mask >> 2) & 1));
        ey += (ey < 0) ? ny : ((ey >= ny) ? -ny : 0);
        ez += (ez < 0) ? nz : ((ez >= nz) ? -nz : 0);
        const int r = ez * ny + ey;
        const int s0 = B.cell_start[r * nx], s1 = B.cell_start[(r + 1) * nx];
        rstart[t] = s0;
        rcount[t] = gone ? 0 : s1 - s0;  // no row beyond an open edge
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        off[0] = 0;
        for (int t = 0; t < 9; ++t) off[t + 1] = off[t] + rcount[t];
        ok = off[9] <= L.stage_cap;
        for (int t = 0; t < 9; ++t) base[t] = rstart[t] - off[t];
    }
    __syncthreads();
    if (!ok) return false;
    for (int t = 0; t < 9; ++t) {
        const int n0 = rcount[t], s0 = rstart[t], o = off[t];
        for (int k = threadIdx.x; k < n0; k += blockDim.x) stage[o + k] = sw[s0 + k];
    }
    __syncthreads();
    return true;
}

template <class R, bool ENERGY, int TPA>
__global__ void __launch_bounds__(256) k_density_rows(Bufs<R> B, Geom G, Launch L)
{
    using R4 = typename V4<R>::T;
    R4 *stage = reinterpret_cast<R4 *>(dyn);
    __shared__ int base[9], rstart[9], rcount[9];
    R h[3];
    load_h<R>(G, h);
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    R4 *sw = B.shadow[sp];
    const bool staged = stage_rows<R>(B, G, L, sw, stage, base, rstart, rcount, blockIdx.x);
    const int a0 = rstart[4], a1 = a0 + rcount[4];  // this row: entry_row 4 is (dy, dz) = (0, 0)
    const R rc2 = g_rc2<R>(G);
    const int per = blockDim.x / TPA;
    const int l = threadIdx.x % TPA;
    R e_embed = (R)0;
    for (int c0 = a0; c0 < a1; c0 += per) {
        const int i = c0 + threadIdx.x / TPA;
        const bool active = i < a1;
        R rho = (R)0;
        if (active) {
                const ListGlobal list{B.list + i, L.ld};
            if (staged)
                rho = density_lane<R, false, TPA, 4>(B, h, rc2, s, B.nnb + i, L.cap, l, stage[i - base[4]], list,
                                                     StagedFetch<R>{stage, base}, TabGlobal<R>{B.coef2, B.coef_f});
            else
                rho = density_lane<R, false, TPA, 4>(B, h, rc2, s, B.nnb + i, L.cap, l, sw[i], list, GlobalFetch<R>{sw},
                                                     TabGlobal<R>{B.coef2, B.coef_f});
        }
        rho = lane_sum<TPA>(rho);
        if (active && l == 0) e_embed += embed<R>(B, sw, i, 0, rho);
    }
    if (ENERGY) {
        const R v[1] = {e_embed};
        block_sums_t<1, R>(v, B.partials, L.pstride, 0);
    }
}

template <class R, int MODE, bool ENERGY, int TPA>
__global__ void __launch_bounds__(256) k_force_rows(Bufs<R> B, Geom G, Launch L)
{
    using R4 = typename V4<R>::T;
    R4 *stage = reinterpret_cast<R4 *>(dyn);
    __shared__ int base[9], rstart[9], rcount[9];
    R h[3];
    load_h<R>(G, h);
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    const R4 *sw = B.shadow[sp];
    const bool staged = stage_rows<R>(B, G, L, sw, stage, base, rstart, rcount, blockIdx.x);
    const int a0 = rstart[4], a1 = a0 + rcount[4];
    const R rc2 = g_rc2<R>(G);
    const int per = blockDim.x / TPA;
    const int l = threadIdx.x % TPA;
    R e7[7] = {0, 0, 0, 0, 0, 0, 0};
    double ke = 0.0;
    float d2max = 0.f;
    for (int c0 = a0; c0 < a1; c0 += per) {
        const int i = c0 + threadIdx.x / TPA;
        const bool active = i < a1;
        R f[3] = {0, 0, 0};
        if (active) {
                const ListGlobal list{B.list + i, L.ld};
            if (staged)
                force_lane<R, false, ENERGY, TPA, 4>(B, L, h, rc2, s, B.nnb + i, l, 0, stage[i - base[4]], list,
                                                     StagedFetch<R>{stage, base}, f, e7, TabGlobal<R>{B.coef2, B.coef_f});
            else
                force_lane<R, false, ENERGY, TPA, 4>(B, L, h, rc2, s, B.nnb + i, l, 0, sw[i], list, GlobalFetch<R>{sw}, f,
                                                     e7, TabGlobal<R>{B.coef2, B.coef_f});
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) f[c] = lane_sum<TPA>(f[c]);
        float d2 = 0.f;
        if (active) integrate<R, MODE, ENERGY, TPA>(B, L, s, sp, i, l, 0, f, ke, d2);
        d2max = fmaxf(d2max, lane_sum<TPA>(d2));
    }
    force_block_end<R, ENERGY>(B, L, e7, ke, d2max, MODE == MODE_CLOSE_OPEN);
}

// ---- spline rows in shared memory (FP32, one atom type, fused tables) ----
//
// Persistent blocks: each block copies the f rows (density) or the f and phi
// rows (force) of the fused table into shared memory once, then walks tiles
// of blockDim / TPA atoms, tile = blockIdx.x, blockIdx.x + gridDim.x, ...;
// the grid is what fits on the GPU at once, so there is no partial last wave.

__device__ __forceinline__ void copy_rows(const float4 *coef2, int nint, float4 *f_rows, float4 *phi_rows)
{
    for (int k = threadIdx.x; k < nint; k += blockDim.x) {
        f_rows[k] = coef2[2 * k];
        if (phi_rows) phi_rows[k] = coef2[2 * k + 1];
    }
}

template <bool ENERGY, int TPA>
__global__ void __launch_bounds__(256) k_density_tab(Bufs<float> B, Geom G, Launch L)
{
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    const int width = blockDim.x / TPA, l = threadIdx.x % TPA;
    const int ntiles = (L.n + width - 1) / width;
    // the warp's list columns are asked of L2 one tile ahead; the first
    // tile's request overlaps the table copy
    const int wa = (threadIdx.x >> 5) * (32 / TPA), ncol = min(st->max_nnb, L.cap);
    prefetch_warp_streams<float, false>(B, L, s, blockIdx.x * width + wa, 32 / TPA, ncol);
    float4 *f_rows = reinterpret_cast<float4 *>(dyn);
    const int nint = B.tables->fphi.nint;
    copy_rows(B.coef2, nint, f_rows, nullptr);
    __syncthreads();
    float h[3];
    load_h<float>(G, h);
    float4 *sw = B.shadow[sp];
    const float rc2 = g_rc2<float>(G);
    const TabShared tab{f_rows, nullptr};
    float e_embed = 0.f;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (tile + (int)gridDim.x < ntiles)
            prefetch_warp_streams<float, false>(B, L, s, (tile + gridDim.x) * width + wa, 32 / TPA, ncol);
        const int i = tile * width + threadIdx.x / TPA;
        const bool active = i < L.n;
        float rho = 0.f;
        if (active)
            rho = density_lane<float, false, TPA, PairsInFlight<false>::density>(
                B, h, rc2, s, B.nnb + i, L.cap, l, sw[i], ListGlobal{B.list + i, L.ld}, GlobalFetch<float>{sw}, tab);
        rho = lane_sum<TPA>(rho);
        if (active && l == 0) e_embed += embed<float>(B, sw, i, 0, rho);
    }
    if (ENERGY) {
        const float v[1] = {e_embed};
        block_sums_t<1, float>(v, B.partials, L.pstride, 0);
    }
}

template <int MODE, bool ENERGY, int TPA>
__global__ void __launch_bounds__(256) k_force_tab(Bufs<float> B, Geom G, Launch L)
{
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    const int width = blockDim.x / TPA, l = threadIdx.x % TPA;
    const int ntiles = (L.n + width - 1) / width;
    const int wa = (threadIdx.x >> 5) * (32 / TPA), ncol = min(st->max_nnb, L.cap);
    prefetch_warp_streams<float, true>(B, L, s, blockIdx.x * width + wa, 32 / TPA, ncol);
    const int nint = B.tables->fphi.nint;
    float4 *f_rows = reinterpret_cast<float4 *>(dyn);
    float4 *phi_rows = f_rows + nint;
    copy_rows(B.coef2, nint, f_rows, phi_rows);
    __syncthreads();
    float h[3];
    load_h<float>(G, h);
    const float4 *sw = B.shadow[sp];
    const float rc2 = g_rc2<float>(G);
    const TabShared tab{f_rows, phi_rows};
    float e7[7] = {0, 0, 0, 0, 0, 0, 0};
    double ke = 0.0;
    float d2max = 0.f;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (tile + (int)gridDim.x < ntiles)
            prefetch_warp_streams<float, true>(B, L, s, (tile + gridDim.x) * width + wa, 32 / TPA, ncol);
        const int i = tile * width + threadIdx.x / TPA;
        const bool active = i < L.n;
        float f[3] = {0, 0, 0};
        if (active)
            force_lane<float, false, ENERGY, TPA, PairsInFlight<false>::force>(B, L, h, rc2, s, B.nnb + i, l, 0, sw[i],
                                                     ListGlobal{B.list + i, L.ld}, GlobalFetch<float>{sw}, f, e7, tab);
#pragma unroll
        for (int c = 0; c < 3; ++c) f[c] = lane_sum<TPA>(f[c]);
        float d2 = 0.f;
        if (active) integrate<float, MODE, ENERGY, TPA>(B, L, s, sp, i, l, 0, f, ke, d2);
        d2max = fmaxf(d2max, lane_sum<TPA>(d2));
    }
    force_block_end<float, ENERGY>(B, L, e7, ke, d2max, MODE == MODE_CLOSE_OPEN);
}

// ---- dispatch ----

template <class R, bool MULTI, bool ENERGY>
void density_tpa(const Bufs<R> &B, const Geom &G, const Launch &L)
{
    if (!MULTI && L.staged_d) {
        const size_t sm = (size_t)L.stage_cap * sizeof(typename V4<R>::T);
        dim3 g(L.nrows), b(L.block_d);
        switch (L.tpa_d) {
        case 1: k_density_rows<R, ENERGY, 1><<<g, b, sm, L.stream>>>(B, G, L); break;
        case 2: k_density_rows<R, ENERGY, 2><<<g, b, sm, L.stream>>>(B, G, L); break;
        default: k_density_rows<R, ENERGY, 4><<<g, b, sm, L.stream>>>(B, G, L); break;
        }
        return;
    }
    if constexpr (std::is_same<R, float>::value && !MULTI) {
        if (L.tab_d) {
            const size_t sm = table_smem_bytes(L, false);
            dim3 g(L.nb_d), b(L.block_d);
            switch (L.tpa_d) {
            case 1: k_density_tab<ENERGY, 1><<<g, b, sm, L.stream>>>(B, G, L); break;
            case 2: k_density_tab<ENERGY, 2><<<g, b, sm, L.stream>>>(B, G, L); break;
            default: k_density_tab<ENERGY, 4><<<g, b, sm, L.stream>>>(B, G, L); break;
            }
            return;
        }
    }
    dim3 g(L.nb_d), b(L.block_d);
    if (!MULTI && L.tiled_d && list_tile_bytes(L, L.tpa_d, L.block_d) <= (size_t)kSharedLimitBytes) {
        const size_t sm = list_tile_bytes(L, L.tpa_d, L.block_d);
        switch (L.tpa_d) {
        case 1: k_density<R, MULTI, ENERGY, 1, true><<<g, b, sm, L.stream>>>(B, G, L); break;
        case 2: k_density<R, MULTI, ENERGY, 2, true><<<g, b, sm, L.stream>>>(B, G, L); break;
        default: k_density<R, MULTI, ENERGY, 4, true><<<g, b, sm, L.stream>>>(B, G, L); break;
        }
        return;
    }
    switch (L.tpa_d) {
    case 1: k_density<R, MULTI, ENERGY, 1, false><<<g, b, 0, L.stream>>>(B, G, L); break;
    case 2: k_density<R, MULTI, ENERGY, 2, false><<<g, b, 0, L.stream>>>(B, G, L); break;
    case 4: k_density<R, MULTI, ENERGY, 4, false><<<g, b, 0, L.stream>>>(B, G, L); break;
    default: k_density<R, MULTI, ENERGY, 8, false><<<g, b, 0, L.stream>>>(B, G, L); break;
    }
}

template <class R, bool MULTI, int MODE, bool ENERGY>
void force_tpa(const Bufs<R> &B, const Geom &G, const Launch &L)
{
    if (!MULTI && L.staged_f) {
        const size_t sm = (size_t)L.stage_cap * sizeof(typename V4<R>::T);
        dim3 g(L.nrows), b(L.block_f);
        switch (L.tpa_f) {
        case 1: k_force_rows<R, MODE, ENERGY, 1><<<g, b, sm, L.stream>>>(B, G, L); break;
        case 2: k_force_rows<R, MODE, ENERGY, 2><<<g, b, sm, L.stream>>>(B, G, L); break;
        default: k_force_rows<R, MODE, ENERGY, 4><<<g, b, sm, L.stream>>>(B, G, L); break;
        }
        return;
    }
    if constexpr (std::is_same<R, float>::value && !MULTI) {
        if (L.tab_f) {
            const size_t sm = table_smem_bytes(L, true);
            dim3 g(L.nb_f), b(L.block_f);
            switch (L.tpa_f) {
            case 1: k_force_tab<MODE, ENERGY, 1><<<g, b, sm, L.stream>>>(B, G, L); break;
            case 2: k_force_tab<MODE, ENERGY, 2><<<g, b, sm, L.stream>>>(B, G, L); break;
            default: k_force_tab<MODE, ENERGY, 4><<<g, b, sm, L.stream>>>(B, G, L); break;
            }
            return;
        }
    }
    dim3 g(L.nb_f), b(L.block_f);
    if (!MULTI && L.tiled_f && list_tile_bytes(L, L.tpa_f, L.block_f) <= (size_t)kSharedLimitBytes) {
        const size_t sm = list_tile_bytes(L, L.tpa_f, L.block_f);
        switch (L.tpa_f) {
        case 1: k_force<R, MULTI, MODE, ENERGY, 1, true><<<g, b, sm, L.stream>>>(B, G, L); break;
        case 2: k_force<R, MULTI, MODE, ENERGY, 2, true><<<g, b, sm, L.stream>>>(B, G, L); break;
        default: k_force<R, MULTI, MODE, ENERGY, 4, true><<<g, b, sm, L.stream>>>(B, G, L); break;
        }
        return;
    }
    switch (L.tpa_f) {
    case 1: k_force<R, MULTI, MODE, ENERGY, 1, false><<<g, b, 0, L.stream>>>(B, G, L); break;
    case 2: k_force<R, MULTI, MODE, ENERGY, 2, false><<<g, b, 0, L.stream>>>(B, G, L); break;
    case 4: k_force<R, MULTI, MODE, ENERGY, 4, false><<<g, b, 0, L.stream>>>(B, G, L); break;
    default: k_force<R, MULTI, MODE, ENERGY, 8, false><<<g, b, 0, L.stream>>>(B, G, L); break;
    }
}

template <class R, bool MULTI>
void force_modes(const Bufs<R> &B, const Geom &G, const Launch &L, int mode, bool energy)
{
    if (mode == MODE_MEASURE) {
        if (energy) force_tpa<R, MULTI, MODE_MEASURE, true>(B, G, L);
        else force_tpa<R, MULTI, MODE_MEASURE, false>(B, G, L);
    } else if (mode == MODE_CLOSE) {
        if (energy) force_tpa<R, MULTI, MODE_CLOSE, true>(B, G, L);
        else force_tpa<R, MULTI, MODE_CLOSE, false>(B, G, L);
    } else {
        if (energy) force_tpa<R, MULTI, MODE_CLOSE_OPEN, true>(B, G, L);
        else force_tpa<R, MULTI, MODE_CLOSE_OPEN, false>(B, G, L);
    }
}

// Shared-memory opt-in of the row-staged kernels for `bytes` of stage.
template <class K>
cudaError_t allow_bytes(K kernel, int bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <class R, int MODE, bool ENERGY>
cudaError_t allow_tiled_force(int bytes)
{
    cudaError_t e = allow_bytes(k_force<R, false, MODE, ENERGY, 1, true>, bytes);
    if (e == cudaSuccess) e = allow_bytes(k_force<R, false, MODE, ENERGY, 2, true>, bytes);
    if (e == cudaSuccess) e = allow_bytes(k_force<R, false, MODE, ENERGY, 4, true>, bytes);
    return e;
}

template <class R, bool ENERGY>
cudaError_t allow_tiled_density(int bytes)
{
    cudaError_t e = allow_bytes(k_density<R, false, ENERGY, 1, true>, bytes);
    if (e == cudaSuccess) e = allow_bytes(k_density<R, false, ENERGY, 2, true>, bytes);
    if (e == cudaSuccess) e = allow_bytes(k_density<R, false, ENERGY, 4, true>, bytes);
    return e;
}

template <int MODE>
cudaError_t allow_tab_force(int bytes)
{
    cudaError_t e = cudaSuccess;
    for (int t : {1, 2, 4}) {
        if (e != cudaSuccess) break;
        e = allow_bytes(t == 1 ? k_force_tab<MODE, false, 1> : (t == 2 ? k_force_tab<MODE, false, 2> : k_force_tab<MODE, false, 4>), bytes);
        if (e == cudaSuccess)
            e = allow_bytes(t == 1 ? k_force_tab<MODE, true, 1> : (t == 2 ? k_force_tab<MODE, true, 2> : k_force_tab<MODE, true, 4>), bytes);
    }
    return e;
}

template <class R, int MODE, bool ENERGY>
cudaError_t allow_rows_force(int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(k_force_rows<R, MODE, ENERGY, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_force_rows<R, MODE, ENERGY, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_force_rows<R, MODE, ENERGY, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

template <class R, bool ENERGY>
cudaError_t allow_rows_density(int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(k_density_rows<R, ENERGY, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_density_rows<R, ENERGY, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_density_rows<R, ENERGY, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

}  // namespace

template <class R>
int launch_density(const Bufs<R> &B, const Geom &G, const Launch &L, bool energy)
{
    if (L.multi) {
        if (energy) density_tpa<R, true, true>(B, G, L);
        else density_tpa<R, true, false>(B, G, L);
    } else {
        if (energy) density_tpa<R, false, true>(B, G, L);
        else density_tpa<R, false, false>(B, G, L);
    }
    return 1;
}

template <class R>
int launch_force(const Bufs<R> &B, const Geom &G, const Launch &L, int mode, bool energy)
{
    if (L.multi) force_modes<R, true>(B, G, L, mode, energy);
    else force_modes<R, false>(B, G, L, mode, energy);
    return 1;
}

// Resident blocks per SM of the shared-table passes (the hot force variant).
inline int table_blocks_per_sm(const Launch &L, bool force, int tpa, int block)
{
    int nb = 0;
    const size_t sm = table_smem_bytes(L, force);
    cudaError_t e;
    if (force)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, tpa == 1 ? k_force_tab<MODE_CLOSE_OPEN, false, 1>
                          : (tpa == 2 ? k_force_tab<MODE_CLOSE_OPEN, false, 2> : k_force_tab<MODE_CLOSE_OPEN, false, 4>),
            block, sm);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, tpa == 1 ? k_density_tab<false, 1> : (tpa == 2 ? k_density_tab<false, 2> : k_density_tab<false, 4>),
            block, sm);
    return e == cudaSuccess ? nb : 0;
}

template <class R>
cudaError_t allow_shared_staging(int bytes)
{
    cudaError_t e = allow_rows_density<R, false>(bytes);
    if (e == cudaSuccess) e = allow_rows_density<R, true>(bytes);
    if (e == cudaSuccess) e = allow_rows_force<R, MODE_MEASURE, false>(bytes);
    if (e == cudaSuccess) e = allow_rows_force<R, MODE_MEASURE, true>(bytes);
    if (e == cudaSuccess) e = allow_rows_force<R, MODE_CLOSE, false>(bytes);
    if (e == cudaSuccess) e = allow_rows_force<R, MODE_CLOSE, true>(bytes);
    if (e == cudaSuccess) e = allow_rows_force<R, MODE_CLOSE_OPEN, false>(bytes);
    if (e == cudaSuccess) e = allow_rows_force<R, MODE_CLOSE_OPEN, true>(bytes);
    if (e == cudaSuccess) e = allow_tiled_density<R, false>(bytes);
    if (e == cudaSuccess) e = allow_tiled_density<R, true>(bytes);
    if (e == cudaSuccess) e = allow_tiled_force<R, MODE_MEASURE, false>(bytes);
    if (e == cudaSuccess) e = allow_tiled_force<R, MODE_MEASURE, true>(bytes);
    if (e == cudaSuccess) e = allow_tiled_force<R, MODE_CLOSE, false>(bytes);
    if (e == cudaSuccess) e = allow_tiled_force<R, MODE_CLOSE, true>(bytes);
    if (e == cudaSuccess) e = allow_tiled_force<R, MODE_CLOSE_OPEN, false>(bytes);
    if (e == cudaSuccess) e = allow_tiled_force<R, MODE_CLOSE_OPEN, true>(bytes);
    if constexpr (std::is_same<R, float>::value) {
        for (int t : {1, 2, 4}) {
            if (e != cudaSuccess) break;
            e = allow_bytes(t == 1 ? k_density_tab<false, 1> : (t == 2 ? k_density_tab<false, 2> : k_density_tab<false, 4>), bytes);
            if (e == cudaSuccess)
                e = allow_bytes(t == 1 ? k_density_tab<true, 1> : (t == 2 ? k_density_tab<true, 2> : k_density_tab<true, 4>), bytes);
        }
        if (e == cudaSuccess) e = allow_tab_force<MODE_MEASURE>(bytes);
        if (e == cudaSuccess) e = allow_tab_force<MODE_CLOSE>(bytes);
        if (e == cudaSuccess) e = allow_tab_force<MODE_CLOSE_OPEN>(bytes);
    }
    return e;
}


}  // namespace eammd
