// pair_kernels.cuh -- the density and force passes of the EAM timestep.
//
// Two schedules share the per-atom work:
//   * atom-parallel (k_density, k_force): TPA lanes cooperate on one atom;
//     lane l walks list columns l, l+TPA, ... two at a time (both gathers
//     issued before either is used), the lanes' sums meet by warp shuffles;
//     neighbour records are gathered from global memory;
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
                                                 const typename V4<R>::T &shf)
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
    const int *base;  // per neighbour row t = code / 3: first atom index minus its stage offset
    __device__ __forceinline__ typename V4<R>::T operator()(uint32_t e) const
    {
        const int t = (int)(e >> kCodeShift) / 3;
        return stage[(int)(e & kIndexMask) - base[t]];
    }
};

// This lane's part of rho_i = sum over listed j with r < r_cut of f_{t_j}(r_ij)
// (Eq. 2).
template <class R, bool MULTI, int TPA, class Fetch>
__device__ __forceinline__ R density_lane(const Bufs<R> &B, const Launch &L, const typename V4<R>::T *sh, R rc2,
                                          int s, int i, int l, const typename V4<R>::T &ui, const Fetch &fetch)
{
    using R4 = typename V4<R>::T;
    const Tables<R> &T = *B.tables;
    const SplineDesc<R> g = MULTI ? T.f[0] : T.fphi;
    const int nn = B.nnb[i];
    const uint32_t *lp = B.list + i;
    R rho = (R)0;
    for (int k = l; k < nn; k += 2 * TPA) {
        const bool two = k + TPA < nn;
        const uint32_t e0 = lp[(size_t)k * L.ld];
        const uint32_t e1 = two ? lp[(size_t)(k + TPA) * L.ld] : e0;
        const R4 u0 = fetch(e0);
        const R4 u1 = fetch(e1);
        const PairIn<R> p0 = pair_vector<R>(ui, u0, sh[e0 >> kCodeShift]);
        const PairIn<R> p1 = pair_vector<R>(ui, u1, sh[e1 >> kCodeShift]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const PairIn<R> &p = q ? p1 : p0;
            if ((q == 0 || two) && p.r2 < rc2) {
                R rinv, r;
                inv_r(p.r2, rinv, r);
                if (MULTI) {
                    R val, der;
                    const int j = (int)((q ? e1 : e0) & kIndexMask);
                    spline_r(T.f[B.type[s][j]], B.coef, r, val, der);
                    rho += val;
                } else {
                    R t;
                    const int kk = segment(g, r, t);
                    const R4 c = B.coef2[2 * kk];
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
template <class R, bool MULTI, bool ENERGY, int TPA, class Fetch>
__device__ __forceinline__ void force_lane(const Bufs<R> &B, const Launch &L, const typename V4<R>::T *sh, R rc2,
                                           int s, int i, int l, int ti, const typename V4<R>::T &ui,
                                           const Fetch &fetch, R (&f)[3], R (&e7)[7])
{
    using R4 = typename V4<R>::T;
    const Tables<R> &T = *B.tables;
    const SplineDesc<R> g = T.fphi;
    const R Fpi = ui.w;
    const int nn = B.nnb[i];
    const uint32_t *lp = B.list + i;
    for (int k = l; k < nn; k += 2 * TPA) {
        const bool two = k + TPA < nn;
        const uint32_t e0 = lp[(size_t)k * L.ld];
        const uint32_t e1 = two ? lp[(size_t)(k + TPA) * L.ld] : e0;
        const R4 u0 = fetch(e0);
        const R4 u1 = fetch(e1);
        const PairIn<R> p0 = pair_vector<R>(ui, u0, sh[e0 >> kCodeShift]);
        const PairIn<R> p1 = pair_vector<R>(ui, u1, sh[e1 >> kCodeShift]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const PairIn<R> &p = q ? p1 : p0;
            if ((q == 0 || two) && p.r2 < rc2) {
                R rinv, r;
                inv_r(p.r2, rinv, r);
                const R Fpj = q ? u1.w : u0.w;
                R phv, phd, fdj, fdi;
                if (MULTI) {
                    const int j = (int)((q ? e1 : e0) & kIndexMask);
                    const int tj = B.type[s][j];
                    spline_r(T.phi[pair_index(L.ntypes, ti, tj)], B.coef, r, phv, phd);
                    fdj = spline_r_der(T.f[tj], B.coef, r);
                    fdi = (tj == ti) ? fdj : spline_r_der(T.f[ti], B.coef, r);
                } else {
                    R t;
                    const int kk = segment(g, r, t);
                    R4 cf, cp;
                    load_row2<R>(B.coef2 + 2 * kk, cf, cp);
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

// ---- atom-parallel schedule ----

template <class R, bool MULTI, bool ENERGY, int TPA>
__global__ void __launch_bounds__(256) k_density(Bufs<R> B, Geom G, Launch L)
{
    using R4 = typename V4<R>::T;
    __shared__ R4 sh[27];
    fill_shift<R>(sh, G);
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    R4 *sw = B.shadow[sp];
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / TPA, l = gt % TPA;
    const bool active = i < L.n;
    const int ti = (MULTI && active) ? B.type[s][i] : 0;
    R rho = active ? density_lane<R, MULTI, TPA>(B, L, sh, g_rc2<R>(G), s, i, l, sw[i], GlobalFetch<R>{sw}) : (R)0;
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
    __shared__ R4 sh[27];
    fill_shift<R>(sh, G);
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    const R4 *sw = B.shadow[sp];
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / TPA, l = gt % TPA;
    const bool active = i < L.n;
    const int ti = (MULTI && active) ? B.type[s][i] : 0;
    R f[3] = {0, 0, 0};
    R e7[7] = {0, 0, 0, 0, 0, 0, 0};
    if (active)
        force_lane<R, MULTI, ENERGY, TPA>(B, L, sh, g_rc2<R>(G), s, i, l, ti, sw[i], GlobalFetch<R>{sw}, f, e7);
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
        ey += (ey < 0) ? ny : ((ey >= ny) ? -ny : 0);
        ez += (ez < 0) ? nz : ((ez >= nz) ? -nz : 0);
        const int r = ez * ny + ey;
        const int s0 = B.cell_start[r * nx], s1 = B.cell_start[(r + 1) * nx];
        rstart[t] = s0;
        rcount[t] = s1 - s0;
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
    extern __shared__ __align__(32) unsigned char dyn[];
    R4 *stage = reinterpret_cast<R4 *>(dyn);
    __shared__ R4 sh[27];
    __shared__ int base[9], rstart[9], rcount[9];
    fill_shift<R>(sh, G);
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    R4 *sw = B.shadow[sp];
    const bool staged = stage_rows<R>(B, G, L, sw, stage, base, rstart, rcount, blockIdx.x);
    const int a0 = rstart[4], a1 = a0 + rcount[4];  // this row: t = 4 is (dy, dz) = (0, 0)
    const R rc2 = g_rc2<R>(G);
    const int per = blockDim.x / TPA;
    const int l = threadIdx.x % TPA;
    R e_embed = (R)0;
    for (int c0 = a0; c0 < a1; c0 += per) {
        const int i = c0 + threadIdx.x / TPA;
        const bool active = i < a1;
        R rho = (R)0;
        if (active) {
            if (staged) {
                const R4 ui = stage[i - base[4]];
                rho = density_lane<R, false, TPA>(B, L, sh, rc2, s, i, l, ui, StagedFetch<R>{stage, base});
            } else {
                rho = density_lane<R, false, TPA>(B, L, sh, rc2, s, i, l, sw[i], GlobalFetch<R>{sw});
            }
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
    extern __shared__ __align__(32) unsigned char dyn[];
    R4 *stage = reinterpret_cast<R4 *>(dyn);
    __shared__ R4 sh[27];
    __shared__ int base[9], rstart[9], rcount[9];
    fill_shift<R>(sh, G);
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
            if (staged)
                force_lane<R, false, ENERGY, TPA>(B, L, sh, rc2, s, i, l, 0, stage[i - base[4]],
                                                  StagedFetch<R>{stage, base}, f, e7);
            else
                force_lane<R, false, ENERGY, TPA>(B, L, sh, rc2, s, i, l, 0, sw[i], GlobalFetch<R>{sw}, f, e7);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) f[c] = lane_sum<TPA>(f[c]);
        float d2 = 0.f;
        if (active) integrate<R, MODE, ENERGY, TPA>(B, L, s, sp, i, l, 0, f, ke, d2);
        d2max = fmaxf(d2max, lane_sum<TPA>(d2));
    }
    force_block_end<R, ENERGY>(B, L, e7, ke, d2max, MODE == MODE_CLOSE_OPEN);
}

// ---- dispatch ----

template <class R, bool MULTI, bool ENERGY>
void density_tpa(const Bufs<R> &B, const Geom &G, const Launch &L)
{
    if (!MULTI && L.staged_d) {
        const size_t sm = (size_t)L.stage_cap * sizeof(typename V4<R>::T);
        dim3 g(L.nrows), b(L.block);
        switch (L.tpa_d) {
        case 1: k_density_rows<R, ENERGY, 1><<<g, b, sm, L.stream>>>(B, G, L); break;
        case 2: k_density_rows<R, ENERGY, 2><<<g, b, sm, L.stream>>>(B, G, L); break;
        default: k_density_rows<R, ENERGY, 4><<<g, b, sm, L.stream>>>(B, G, L); break;
        }
        return;
    }
    dim3 g(L.nb_d), b(L.block);
    switch (L.tpa_d) {
    case 1: k_density<R, MULTI, ENERGY, 1><<<g, b, 0, L.stream>>>(B, G, L); break;
    case 2: k_density<R, MULTI, ENERGY, 2><<<g, b, 0, L.stream>>>(B, G, L); break;
    case 4: k_density<R, MULTI, ENERGY, 4><<<g, b, 0, L.stream>>>(B, G, L); break;
    default: k_density<R, MULTI, ENERGY, 8><<<g, b, 0, L.stream>>>(B, G, L); break;
    }
}

template <class R, bool MULTI, int MODE, bool ENERGY>
void force_tpa(const Bufs<R> &B, const Geom &G, const Launch &L)
{
    if (!MULTI && L.staged_f) {
        const size_t sm = (size_t)L.stage_cap * sizeof(typename V4<R>::T);
        dim3 g(L.nrows), b(L.block);
        switch (L.tpa_f) {
        case 1: k_force_rows<R, MODE, ENERGY, 1><<<g, b, sm, L.stream>>>(B, G, L); break;
        case 2: k_force_rows<R, MODE, ENERGY, 2><<<g, b, sm, L.stream>>>(B, G, L); break;
        default: k_force_rows<R, MODE, ENERGY, 4><<<g, b, sm, L.stream>>>(B, G, L); break;
        }
        return;
    }
    dim3 g(L.nb_f), b(L.block);
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

// Shared-memory opt-in of the row-staged kernels for `bytes` of stage.
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

template <class R>
cudaError_t allow_row_staging(int bytes)
{
    cudaError_t e = allow_rows_density<R, false>(bytes);
    if (e == cudaSuccess) e = allow_rows_density<R, true>(bytes);
    if (e == cudaSuccess) e = allow_rows_force<R, MODE_MEASURE, false>(bytes);
    if (e == cudaSuccess) e = allow_rows_force<R, MODE_MEASURE, true>(bytes);
    if (e == cudaSuccess) e = allow_rows_force<R, MODE_CLOSE, false>(bytes);
    if (e == cudaSuccess) e = allow_rows_force<R, MODE_CLOSE, true>(bytes);
    if (e == cudaSuccess) e = allow_rows_force<R, MODE_CLOSE_OPEN, false>(bytes);
    if (e == cudaSuccess) e = allow_rows_force<R, MODE_CLOSE_OPEN, true>(bytes);
    return e;
}

}  // namespace eammd
