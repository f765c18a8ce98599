// pair_kernels.cuh -- the density and force passes of the EAM timestep.
//
// TPA lanes cooperate on one atom: lane l walks list columns l, l+TPA, ...
// two at a time (both gathers issued before either is used), and the lanes'
// partial sums are combined with warp shuffles.  Splitting an atom's ~26
// neighbours over lanes shortens each thread's chain of dependent loads (list
// entry -> neighbour record -> spline row), which is what bounds a
// thread-per-atom loop.  The neighbour record is the 16-byte shadow
// (u_x, u_y, u_z, F'_j): one gather gives the force pass both the position and
// the embedding derivative the density pass stored.
//
// With a single atom type whose f and phi share a knot grid, both splines of
// an interval sit in one 32-byte row (coef2): the force pass reads f' and phi'
// of a pair from one sector.
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

// Density pass, Eq. 2: rho_i = sum over listed j with r < r_cut of
// f_{t_j}(r_ij); then F'(rho_i) into the shadow record's w (and F(rho_i)
// into the energy partials when energies are wanted).
template <class R, bool MULTI, bool ENERGY, int TPA>
__global__ void __launch_bounds__(256) k_density(Bufs<R> B, Geom G, Launch L)
{
    using R4 = typename V4<R>::T;
    __shared__ R4 sh[27];
    fill_shift<R>(sh, G);
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    R4 *sw = B.shadow[sp];
    const Tables<R> &T = *B.tables;
    const R rc2 = g_rc2<R>(G);
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / TPA, l = gt % TPA;
    const bool active = i < L.n;
    R rho = (R)0;
    int ti = 0;
    if (active) {
        const R4 ui = sw[i];
        const int nn = B.nnb[i];
        ti = MULTI ? B.type[s][i] : 0;
        const SplineDesc<R> g = MULTI ? T.f[0] : T.fphi;
        const uint32_t *lp = B.list + i;
        for (int k = l; k < nn; k += 2 * TPA) {
            const bool two = k + TPA < nn;
            const uint32_t e0 = lp[(size_t)k * L.ld];
            const uint32_t e1 = two ? lp[(size_t)(k + TPA) * L.ld] : e0;
            const R4 u0 = sw[e0 & kIndexMask];
            const R4 u1 = sw[e1 & kIndexMask];
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
                        int j = (int)((q ? e1 : e0) & kIndexMask);
                        spline_r(T.f[B.type[s][j]], B.coef, r, val, der);
                        rho += val;
                    } else {
                        R t;
                        int kk = segment(g, r, t);
                        R4 c = B.coef2[2 * kk];
                        rho += fma(t, fma(t, fma(t, c.w, c.z), c.y), c.x);
                    }
                }
            }
        }
    }
    rho = lane_sum<TPA>(rho);
    R e_embed = (R)0;
    if (active && l == 0) {
        R Fv, Fd;
        if (spline_any(T.F[ti], B.coef, rho, Fv, Fd)) atomicAdd(&B.st->table_oor, 1ull);
        // the w word of this atom's record: the force pass reads it with the
        // coordinates (the density pass itself never uses w)
        reinterpret_cast<R *>(sw + i)[3] = Fd;
        e_embed = Fv;
    }
    if (ENERGY) {
        const R v[1] = {e_embed};
        block_sums_t<1, R>(v, B.partials, L.pstride, 0);
    }
}

// Force pass, Eq. 4, fused with the integration of Eq. 5:
//   s_ij = phi'_{t_i t_j}(r) + F'_i f'_{t_j}(r) + F'_j f'_{t_i}(r),
//   F_i  = sum_j s_ij (x_j - x_i) / r,
// then (MODE_CLOSE*) the closing half kick v += F dt/(2m), and
// (MODE_CLOSE_OPEN) the next step's opening half kick and drift
// x += v dt, writing the next shadow coordinates and the displacement
// since the last list build.  MODE_MEASURE only stores the forces.
// After the lane reduction, lane c of an atom (c < 3, or every lane for
// c = l, l + TPA, ... when TPA < 3) integrates component c in FP64.
template <class R, bool MULTI, int MODE, bool ENERGY, int TPA>
__global__ void __launch_bounds__(256) k_force(Bufs<R> B, Geom G, Launch L)
{
    using R4 = typename V4<R>::T;
    __shared__ R4 sh[27];
    fill_shift<R>(sh, G);
    const DevState *st = B.st;
    const int sp = st->sp, s = st->set;
    const R4 *sw = B.shadow[sp];
    const Tables<R> &T = *B.tables;
    const R rc2 = g_rc2<R>(G);
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / TPA, l = gt % TPA;
    const bool active = i < L.n;
    R fx = 0, fy = 0, fz = 0;
    R ep = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    int ti = 0;
    if (active) {
        const R4 ui = sw[i];
        const R Fpi = ui.w;
        const int nn = B.nnb[i];
        ti = MULTI ? B.type[s][i] : 0;
        const SplineDesc<R> g = T.fphi;
        const uint32_t *lp = B.list + i;
        for (int k = l; k < nn; k += 2 * TPA) {
            const bool two = k + TPA < nn;
            const uint32_t e0 = lp[(size_t)k * L.ld];
            const uint32_t e1 = two ? lp[(size_t)(k + TPA) * L.ld] : e0;
            const R4 u0 = sw[e0 & kIndexMask];
            const R4 u1 = sw[e1 & kIndexMask];
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
                        int j = (int)((q ? e1 : e0) & kIndexMask);
                        int tj = B.type[s][j];
                        spline_r(T.phi[pair_index(L.ntypes, ti, tj)], B.coef, r, phv, phd);
                        fdj = spline_r_der(T.f[tj], B.coef, r);
                        fdi = (tj == ti) ? fdj : spline_r_der(T.f[ti], B.coef, r);
                    } else {
                        R t;
                        int kk = segment(g, r, t);
                        R4 cf, cp;
                        load_row2<R>(B.coef2 + 2 * kk, cf, cp);
                        fdj = fma(t, fma(t, (R)3 * cf.w, (R)2 * cf.z), cf.y);
                        fdi = fdj;
                        phd = fma(t, fma(t, (R)3 * cp.w, (R)2 * cp.z), cp.y);
                        phv = ENERGY ? fma(t, fma(t, fma(t, cp.w, cp.z), cp.y), cp.x) : (R)0;
                    }
                    const R sij = fma(Fpj, fdi, fma(Fpi, fdj, phd));
                    const R sr = sij * rinv;
                    fx = fma(sr, p.dx, fx);
                    fy = fma(sr, p.dy, fy);
                    fz = fma(sr, p.dz, fz);
                    if (ENERGY) {
                        const R hs = (R)(-0.5) * sr;
                        ep += (R)0.5 * phv;
                        w0 = fma(hs * p.dx, p.dx, w0);
                        w1 = fma(hs * p.dy, p.dy, w1);
                        w2 = fma(hs * p.dz, p.dz, w2);
                        w3 = fma(hs * p.dx, p.dy, w3);
                        w4 = fma(hs * p.dx, p.dz, w4);
                        w5 = fma(hs * p.dy, p.dz, w5);
                    }
                }
            }
        }
    }
    fx = lane_sum<TPA>(fx);
    fy = lane_sum<TPA>(fy);
    fz = lane_sum<TPA>(fz);
    double ke = 0.0;
    float d2 = 0.f;
    if (active) {
        if (l == 0 && !isfinite(fx + fy + fz)) atomicOr(&B.st->error, ERR_NONFINITE);
        const double kq = L.half_kick[ti];
        for (int c = l; c < 3; c += TPA) {
            const R fc = (c == 0) ? fx : ((c == 1) ? fy : fz);
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
    if (ENERGY) {
        // the kinetic energy is formed in FP64 and carried as a pair of R
        const R ke_hi = (R)ke;
        const R ke_lo = (R)(ke - (double)ke_hi);
        const R v8[8] = {ep, ke_hi, w0, w1, w2, w3, w4, w5};
        const R lo8[8] = {0, ke_lo, 0, 0, 0, 0, 0, 0};
        block_sums_t<8, R>(v8, B.partials, L.pstride, 1, lo8);
    }
    if (MODE == MODE_CLOSE_OPEN) block_max_disp(lane_sum<TPA>(d2), &B.st->maxdisp2);
}

template <class R, bool MULTI, bool ENERGY>
void density_tpa(const Bufs<R> &B, const Geom &G, const Launch &L)
{
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

}  // namespace eammd
