// device_common.cuh -- device helpers shared by the kernels of the EAM
// library: vector construction, 1/r, cubic spline lookups, the 27-cell
// stencil shifts and fixed-order block reductions.
#pragma once

#include "md_internal.cuh"

#include <cuda_runtime.h>

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

// Interval k and local coordinate t = x - x_k of x on a uniform table, for
// x0 <= x (capped to the last interval).
template <class R>
__device__ __forceinline__ int segment(const SplineDesc<R> &s, R x, R &t)
{
    R u = (x - s.x0) * s.inv_h;
    int k = min((int)u, s.nint - 1);
    R kf = (R)k;
    t = fma(-kf, s.h_lo, fma(-kf, s.h_hi, x - s.x0));
    return k;
}

__device__ __forceinline__ int pair_index(int nt, int a, int b)
{
    int lo = min(a, b), hi = max(a, b);
    return lo * nt - lo * (lo - 1) / 2 + (hi - lo);
}

// Geometry constants in the pair type (FP32 kernels read the FP32 copies).
template <class R> __device__ __forceinline__ R g_rc2(const Geom &G);
template <> __device__ __forceinline__ float g_rc2<float>(const Geom &G) { return G.rc2_f; }
template <> __device__ __forceinline__ double g_rc2<double>(const Geom &G) { return G.rc2; }
template <class R> __device__ __forceinline__ R g_h(const Geom &G, int a);
template <> __device__ __forceinline__ float g_h<float>(const Geom &G, int a) { return G.h_f[a]; }
template <> __device__ __forceinline__ double g_h<double>(const Geom &G, int a) { return G.h[a]; }
template <class R> __device__ __forceinline__ R g_screen_lo(const Geom &G);
template <> __device__ __forceinline__ float g_screen_lo<float>(const Geom &G) { return G.screen_lo_f; }
template <> __device__ __forceinline__ double g_screen_lo<double>(const Geom &G) { return G.screen_lo; }
template <class R> __device__ __forceinline__ R g_screen_hi(const Geom &G);
template <> __device__ __forceinline__ float g_screen_hi<float>(const Geom &G) { return G.screen_hi_f; }
template <> __device__ __forceinline__ double g_screen_hi<double>(const Geom &G) { return G.screen_hi; }

// Shift of a list entry's stencil cell: u_j + shift - u_i is the
// displacement x_j - x_i of the pair.  Per axis -h, 0 or h from the entry's
// 2-bit field (the same values as (R)d * h for d = -1, 0, 1), so the kernels
// keep no table of shifts.
template <class R> struct Shift {
    R x, y, z;
};
template <class R>
__device__ __forceinline__ R axis_shift(uint32_t e, int axis, R h)
{
    const uint32_t t = (e >> (kCodeShift + 2 * axis)) & 3u;
    return t == 1u ? (R)0 : (t == 0u ? -h : h);
}
template <class R>
__device__ __forceinline__ Shift<R> entry_shift(uint32_t e, const R (&h)[3])
{
    return Shift<R>{axis_shift<R>(e, 0, h[0]), axis_shift<R>(e, 1, h[1]), axis_shift<R>(e, 2, h[2])};
}
// FP32: t in {0, 1, 2} placed in the low mantissa bits of 1.5 * 2^23 gives
// the float 1.5 * 2^23 + t exactly; subtracting 1.5 * 2^23 + 1 leaves t - 1 in
// {-1, 0, 1} exactly, and (t - 1) * h is the same -h, 0 or h as above.
template <>
__device__ __forceinline__ Shift<float> entry_shift<float>(uint32_t e, const float (&h)[3])
{
    const uint32_t c = e >> kCodeShift;
    const float mx = __uint_as_float((c & 3u) | 0x4B400000u) - 12582913.0f;
    const float my = __uint_as_float(((c >> 2) & 3u) | 0x4B400000u) - 12582913.0f;
    const float mz = __uint_as_float((c >> 4) | 0x4B400000u) - 12582913.0f;
    return Shift<float>{mx * h[0], my * h[1], mz * h[2]};
}
template <class R>
__device__ __forceinline__ void load_h(const Geom &G, R (&h)[3])
{
    h[0] = g_h<R>(G, 0);
    h[1] = g_h<R>(G, 1);
    h[2] = g_h<R>(G, 2);
}

// Error-free sum of two floats (Knuth's TwoSum): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Warp sum of FP32 values carried as unevaluated float pairs (hi + lo), so
// the 32-atom partial keeps about twice FP32 precision without touching the
// FP64 pipe; the result is exact to ~2^-44 relative.
__device__ __forceinline__ double warp_sum_ff(float v, float v_lo = 0.f)
{
    float hi = v, lo = v_lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        float olo = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, ohi, s, e);
        hi = s;
        lo = lo + olo + e;
    }
    return (double)hi + (double)lo;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sums of NV per-thread values in a fixed order: warps reduce in
// registers (FP32 values as float pairs, FP64 values in FP64), then thread 0
// adds the warp sums in FP64 and stores them to
// partials[(slot0 + k) * stride + blockIdx.x].  All threads must call.
template <int NV, class T>
__device__ __forceinline__ void block_sums_t(const T (&v)[NV], double *partials, int stride, int slot0,
                                             const T *v_lo = nullptr)
{
    __shared__ double sm[32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s;
        if constexpr (sizeof(T) == sizeof(float)) s = warp_sum_ff(v[k], v_lo ? v_lo[k] : 0.f);
        else s = warp_sum_d(v[k] + (v_lo ? v_lo[k] : 0.0));
        if (lane == 0) sm[warp][k] = s;
    }
    __syncthreads();
    // lane k of warp 0 adds value k over the warps, in warp order
    if (threadIdx.x < NV) {
        const int k = threadIdx.x;
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sm[w][k];
        partials[(size_t)(slot0 + k) * stride + blockIdx.x] = s;
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

inline int blocks_for(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace
}  // namespace eammd
