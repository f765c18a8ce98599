// pair_kernels.cuh -- the density and force passes of the EAM timestep.
//
// Atom-parallel schedule (k_density, k_force): TPA lanes cooperate on one
// atom; lane l walks list columns l, l+TPA, ... a few at a time (every
// gather of a round issued before any is used: three pairs a round in the
// density pass, two in the force pass with the next round in flight), and
// the lanes' sums meet by warp shuffles.  Neighbour records and spline rows
// are gathered from global memory through L1.
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

// The same, through the texture path (FP32 records, density pass).
struct TexFetch {
    cudaTextureObject_t t;
    __device__ __forceinline__ float4 operator()(uint32_t e) const
    {
        return tex1Dfetch<float4>(t, (int)(e & kIndexMask));
    }
};

// Where the spline rows of the one-type path are read from: coef2 in device
// memory (row 2k: f, row 2k+1: phi, both in one 32-byte load); the density
// pass reads the f rows alone from coef_f, where a 128-byte line holds eight
// intervals instead of four.
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
// Where list column k of the lane's atom is read from.
struct ListGlobal {
    const uint32_t *lp;  // list + i
    int ld;
    __device__ __forceinline__ uint32_t operator()(int k) const { return lp[(size_t)k * ld]; }
};
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
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

template <class R, bool MULTI, bool ENERGY, int TPA, bool TEX>
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
    prefetch_warp_streams<R, false>(B, L, s, i0 + (threadIdx.x >> 5) * (32 / TPA), 32 / TPA, min(st->max_nnb, L.cap));
    const int i = i0 + threadIdx.x / TPA, l = threadIdx.x % TPA;
    const bool active = i < L.n;
    const int ti = (MULTI && active) ? B.type[s][i] : 0;
    const R rc2 = g_rc2<R>(G);
    R rho = (R)0;
    if (active) {
        if constexpr (TEX)
            rho = density_lane<R, MULTI, TPA, U>(B, h, rc2, s, B.nnb + i, L.cap, l, sw[i],
                                                 ListGlobal{B.list + i, L.ld},
                                                 TexFetch{(cudaTextureObject_t)B.tex_shadow[sp]},
                                                 TabGlobal<R>{B.coef2, B.coef_f});
        else
            rho = density_lane<R, MULTI, TPA, U>(B, h, rc2, s, B.nnb + i, L.cap, l, sw[i],
                                                 ListGlobal{B.list + i, L.ld}, GlobalFetch<R>{sw},
                                                 TabGlobal<R>{B.coef2, B.coef_f});
    }
    rho = lane_sum<TPA>(rho);
    R e_embed = (R)0;
    if (active && l == 0) e_embed = embed<R>(B, sw, i, ti, rho);
    if (ENERGY) {
        const R v[1] = {e_embed};
        block_sums_t<1, R>(v, B.partials, L.pstride, 0);
    }
}

template <class R, bool MULTI, int MODE, bool ENERGY, int TPA>
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
    prefetch_warp_streams<R, true>(B, L, s, i0 + (threadIdx.x >> 5) * (32 / TPA), 32 / TPA, min(st->max_nnb, L.cap));
    const int i = i0 + threadIdx.x / TPA, l = threadIdx.x % TPA;
    const bool active = i < L.n;
    const int ti = (MULTI && active) ? B.type[s][i] : 0;
    const R rc2 = g_rc2<R>(G);
    R f[3] = {0, 0, 0};
    R e7[7] = {0, 0, 0, 0, 0, 0, 0};
    if (active)
        force_lane<R, MULTI, ENERGY, TPA, U>(B, L, h, rc2, s, B.nnb + i, l, ti, sw[i], ListGlobal{B.list + i, L.ld},
                                             GlobalFetch<R>{sw}, f, e7, TabGlobal<R>{B.coef2, B.coef_f});
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] = lane_sum<TPA>(f[c]);
    double ke = 0.0;
    float d2 = 0.f;
    if (active) integrate<R, MODE, ENERGY, TPA>(B, L, s, sp, i, l, ti, f, ke, d2);
    force_block_end<R, ENERGY>(B, L, e7, ke, lane_sum<TPA>(d2), MODE == MODE_CLOSE_OPEN);
}

// ---- half lists (force symmetry): each pair once, the other end's term
// added through fixed-point accumulators ----
//
// A pair (i, j) sits in one list only: that of the atom that sees the other
// in the upper half space (the list build decides it exactly).  Its
// density term f(r) (one type: the same for both ends) and its force term
// s_ij (x_j - x_i)/r are formed once; i keeps its share in registers (a sum
// in a fixed order, stored in own[i]), j's share goes into acc_*[j] as a
// 64-bit integer in units of 2^-32 by an atomic add.  Integer sums do not
// depend on the order of the adds, so the totals, and every result, are
// bitwise reproducible.  A second pass per quantity adds own and acc (FP64),
// zeroes acc for the next use, and carries on as the full-list passes do:
// the embedding derivative F'(rho) into the record, or the integration.

constexpr float kFixScale = 4294967296.0f;       // 2^32 fixed-point units per unit
constexpr double kFixUnit = 1.0 / 4294967296.0;  // one unit
constexpr float kFixLimit = 16777216.0f;         // 2^24: largest pair term the accumulators take

__device__ __forceinline__ unsigned long long to_fixed(float x)
{
    return (unsigned long long)__float2ll_rn(x * kFixScale);
}

__device__ __forceinline__ double from_fixed(unsigned long long a)
{
    return (double)(long long)a * kFixUnit;
}

// rho_i's own terms and the scatter of j's; one lane per atom.
__global__ void __launch_bounds__(256) k_density_half(Bufs<float> B, Geom G, Launch L)
{
    constexpr int U = 3;
    float h[3];
    load_h<float>(G, h);
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    const float4 *sw = B.shadow[sp];
    const int i0 = blockIdx.x * blockDim.x;
    prefetch_warp_streams<float, false>(B, L, s, i0 + (threadIdx.x & ~31), 32, min(st->max_nnb, L.cap));
    const int i = i0 + threadIdx.x;
    if (i >= L.n) return;
    const SplineDesc<float> g = B.tables->fphi;
    const float rc2 = g_rc2<float>(G);
    const float4 ui = sw[i];
    const uint32_t *lp = B.list + i;
    const int nn = B.nnb[i];
    float rho = 0.f;
    bool range_ok = true;
    for (int k = 0; k < nn; k += U) {
        uint32_t e[U];
        float4 u[U];
#pragma unroll
        for (int q = 0; q < U; ++q) e[q] = (k + q < nn) ? lp[(size_t)(k + q) * L.ld] : 0u;
#pragma unroll
        for (int q = 0; q < U; ++q) u[q] = sw[(q == 0 || k + q < nn ? e[q] : e[0]) & kIndexMask];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const PairIn<float> pv = pair_vector<float>(ui, u[q], entry_shift<float>(e[q], h));
            if ((q == 0 || k + q < nn) && pv.r2 < rc2) {
                float rinv, r;
                inv_r(pv.r2, rinv, r);
                float t;
                const int kk = segment(g, r, t);
                const float4 c = B.coef_f[kk];
                const float v = fma(t, fma(t, fma(t, c.w, c.z), c.y), c.x);
                rho += v;
                range_ok = range_ok && fabsf(v) < kFixLimit;
                atomicAdd(B.acc_rho + (e[q] & kIndexMask), to_fixed(v));
            }
        }
    }
    if (!range_ok) atomicOr(&B.st->error, ERR_NONFINITE);
    B.own[i].x = rho;
}

// rho_i = own + accumulated, F'(rho_i) into the record, F(rho_i) for the
// energy; the accumulator is zeroed for the next pass.
template <bool ENERGY>
__global__ void __launch_bounds__(256) k_embed_half(Bufs<float> B, Launch L)
{
    const DevState *st = B.st;
    float4 *sw = B.shadow[st->sp];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float e_embed = 0.f;
    if (i < L.n) {
        const double rho = (double)B.own[i].x + from_fixed(B.acc_rho[i]);
        B.acc_rho[i] = 0ull;
        e_embed = embed<float>(B, sw, i, 0, (float)rho);
    }
    if (ENERGY) {
        const float v[1] = {e_embed};
        block_sums_t<1, float>(v, B.partials, L.pstride, 0);
    }
}

// F_i's own terms of Eq. 4 and the scatter of j's (-s_ij d / r); with ENERGY
// the pair energy phi(r) and the virial of each pair, counted once.
template <bool ENERGY>
__global__ void __launch_bounds__(256) k_force_half(Bufs<float> B, Geom G, Launch L)
{
    constexpr int U = 2;
    float h[3];
    load_h<float>(G, h);
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    const float4 *sw = B.shadow[sp];
    const int i0 = blockIdx.x * blockDim.x;
    prefetch_warp_streams<float, true>(B, L, s, i0 + (threadIdx.x & ~31), 32, min(st->max_nnb, L.cap));
    const int i = i0 + threadIdx.x;
    const SplineDesc<float> g = B.tables->fphi;
    const float rc2 = g_rc2<float>(G);
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    float e7[7] = {0, 0, 0, 0, 0, 0, 0};
    if (i < L.n) {
        const float4 ui = sw[i];
        const float Fpi = ui.w;
        const uint32_t *lp = B.list + i;
        const int nn = B.nnb[i];
        bool range_ok = true;
        for (int k = 0; k < nn; k += U) {
            uint32_t e[U];
            float4 u[U];
#pragma unroll
            for (int q = 0; q < U; ++q) e[q] = (k + q < nn) ? lp[(size_t)(k + q) * L.ld] : 0u;
#pragma unroll
            for (int q = 0; q < U; ++q) u[q] = sw[(q == 0 || k + q < nn ? e[q] : e[0]) & kIndexMask];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const PairIn<float> pv = pair_vector<float>(ui, u[q], entry_shift<float>(e[q], h));
                if ((q == 0 || k + q < nn) && pv.r2 < rc2) {
                    float rinv, r;
                    inv_r(pv.r2, rinv, r);
                    float t;
                    const int kk = segment(g, r, t);
                    float4 cf, cp;
                    load_row2<float>(B.coef2 + 2 * kk, cf, cp);
                    const float fd = fma(t, fma(t, 3.f * cf.w, 2.f * cf.z), cf.y);
                    const float pd = fma(t, fma(t, 3.f * cp.w, 2.f * cp.z), cp.y);
                    const float sr = fma(u[q].w + Fpi, fd, pd) * rinv;
                    const float gx = sr * pv.dx, gy = sr * pv.dy, gz = sr * pv.dz;
                    f0 += gx;
                    f1 += gy;
                    f2 += gz;
                    range_ok = range_ok && fabsf(gx) < kFixLimit && fabsf(gy) < kFixLimit && fabsf(gz) < kFixLimit;
                    unsigned long long *aj = B.acc_f + 3 * (size_t)(e[q] & kIndexMask);
                    atomicAdd(aj + 0, to_fixed(-gx));
                    atomicAdd(aj + 1, to_fixed(-gy));
                    atomicAdd(aj + 2, to_fixed(-gz));
                    if (ENERGY) {
                        e7[0] += fma(t, fma(t, fma(t, cp.w, cp.z), cp.y), cp.x);
                        const float hs = -sr;
                        e7[1] = fma(hs * pv.dx, pv.dx, e7[1]);
                        e7[2] = fma(hs * pv.dy, pv.dy, e7[2]);
                        e7[3] = fma(hs * pv.dz, pv.dz, e7[3]);
                        e7[4] = fma(hs * pv.dx, pv.dy, e7[4]);
                        e7[5] = fma(hs * pv.dx, pv.dz, e7[5]);
                        e7[6] = fma(hs * pv.dy, pv.dz, e7[6]);
                    }
                }
            }
        }
        if (!range_ok) atomicOr(&B.st->error, ERR_NONFINITE);
        B.own[i] = make_float4(f0, f1, f2, 0.f);
    }
    if (ENERGY) {
        const float pe[1] = {e7[0]};
        block_sums_t<1, float>(pe, B.partials, L.pstride, 1);
        const float w6[6] = {e7[1], e7[2], e7[3], e7[4], e7[5], e7[6]};
        block_sums_t<6, float>(w6, B.partials, L.pstride, 3);
    }
}

// F_i = own + accumulated (zeroed for the next pass), then the integration
// of the full-list force pass (kicks, drift, next record, cached forces,
// kinetic energy and largest displacement as MODE asks).
template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(256) k_integrate_half(Bufs<float> B, Launch L)
{
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    float d2 = 0.f;
    if (i < L.n) {
        const float4 o = B.own[i];
        unsigned long long *ai = B.acc_f + 3 * (size_t)i;
        const float f[3] = {(float)((double)o.x + from_fixed(ai[0])), (float)((double)o.y + from_fixed(ai[1])),
                            (float)((double)o.z + from_fixed(ai[2]))};
        ai[0] = 0ull;
        ai[1] = 0ull;
        ai[2] = 0ull;
        integrate<float, MODE, ENERGY, 1>(B, L, s, sp, i, 0, 0, f, ke, d2);
    }
    if (ENERGY) {
        const float ke_hi = (float)ke;
        const float v[1] = {ke_hi};
        const float lo[1] = {(float)(ke - (double)ke_hi)};
        block_sums_t<1, float>(v, B.partials, L.pstride, 2, lo);
    }
    if (MODE == MODE_CLOSE_OPEN) block_max_disp(d2, &B.st->maxdisp2);
}

template <int MODE, bool ENERGY>
void force_half(const Bufs<float> &B, const Geom &G, const Launch &L)
{
    dim3 g(L.nb_f), b(L.block_f);
    k_force_half<ENERGY><<<g, b, 0, L.stream>>>(B, G, L);
    k_integrate_half<MODE, ENERGY><<<g, b, 0, L.stream>>>(B, L);
}

// ---- dispatch ----

template <class R, bool MULTI, bool ENERGY, bool TEX>
void density_tpa_fetch(const Bufs<R> &B, const Geom &G, const Launch &L)
{
    dim3 g(L.nb_d), b(L.block_d);
    switch (L.tpa_d) {
    case 1: k_density<R, MULTI, ENERGY, 1, TEX><<<g, b, 0, L.stream>>>(B, G, L); break;
    case 2: k_density<R, MULTI, ENERGY, 2, TEX><<<g, b, 0, L.stream>>>(B, G, L); break;
    case 4: k_density<R, MULTI, ENERGY, 4, TEX><<<g, b, 0, L.stream>>>(B, G, L); break;
    default: k_density<R, MULTI, ENERGY, 8, TEX><<<g, b, 0, L.stream>>>(B, G, L); break;
    }
}

// Records through the texture path where both record buffers have a texture
// object (FP32), through the load path otherwise (FP64).
template <class R, bool MULTI, bool ENERGY>
void density_tpa(const Bufs<R> &B, const Geom &G, const Launch &L)
{
    if constexpr (std::is_same<R, float>::value) {
        if (B.tex_shadow[0] && B.tex_shadow[1]) {
            density_tpa_fetch<R, MULTI, ENERGY, true>(B, G, L);
            return;
        }
    }
    density_tpa_fetch<R, MULTI, ENERGY, false>(B, G, L);
}

template <class R, bool MULTI, int MODE, bool ENERGY>
void force_tpa(const Bufs<R> &B, const Geom &G, const Launch &L)
{
    dim3 g(L.nb_f), b(L.block_f);
    switch (L.tpa_f) {
    case 1: k_force<R, MULTI, MODE, ENERGY, 1><<<g, b, 0, L.stream>>>(B, G, L); break;
    case 2: k_force<R, MULTI, MODE, ENERGY, 2><<<g, b, 0, L.stream>>>(B, G, L); break;
    case 4: k_force<R, MULTI, MODE, ENERGY, 4><<<g, b, 0, L.stream>>>(B, G, L); break;
    default: k_force<R, MULTI, MODE, ENERGY, 8><<<g, b, 0, L.stream>>>(B, G, L); break;
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

}  // namespace

template <class R>
int launch_density(const Bufs<R> &B, const Geom &G, const Launch &L, bool energy)
{
    if constexpr (std::is_same<R, float>::value) {
        if (L.half) {
            dim3 g(L.nb_d), b(L.block_d);
            k_density_half<<<g, b, 0, L.stream>>>(B, G, L);
            if (energy) k_embed_half<true><<<g, b, 0, L.stream>>>(B, L);
            else k_embed_half<false><<<g, b, 0, L.stream>>>(B, L);
            return 2;
        }
    }
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
    if constexpr (std::is_same<R, float>::value) {
        if (L.half) {
            if (mode == MODE_MEASURE) {
                if (energy) force_half<MODE_MEASURE, true>(B, G, L);
                else force_half<MODE_MEASURE, false>(B, G, L);
            } else if (mode == MODE_CLOSE) {
                if (energy) force_half<MODE_CLOSE, true>(B, G, L);
                else force_half<MODE_CLOSE, false>(B, G, L);
            } else {
                if (energy) force_half<MODE_CLOSE_OPEN, true>(B, G, L);
                else force_half<MODE_CLOSE_OPEN, false>(B, G, L);
            }
            return 2;
        }
    }
    if (L.multi) force_modes<R, true>(B, G, L, mode, energy);
    else force_modes<R, false>(B, G, L, mode, energy);
    return 1;
}


}  // namespace eammd
