// batch.cu -- many independent periodic systems ("replicas") advanced in one
// persistent launch.
//
// Each thread block takes a replica from a queue ordered largest first and
// runs every phase of every step of that replica itself -- list rebuild
// (wrap, bin, scan, scatter, sort, permute, list), density (Eq. 2), force
// (Eq. 4) fused with the velocity-Verlet kicks and drift (Eq. 5) -- with
// block-level barriers only, so replicas never wait on each other and small
// systems pay no launch per step.  Arithmetic follows the mixed-precision
// path of the single-system kernels: FP32 pair math on cell-centred
// coordinates, FP64 positions, velocities and cross-atom sums.  The list,
// its stencil codes and the exact FP64 test near r_list are those of the
// single-system path, so every replica's list equals the FP64 definition.
#include "eammd.h"
#include "device_common.cuh"
#include "spline_host.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace eammd {
namespace {

constexpr int kMaxBatchWarps = 32;  // blocks of up to 1024 threads
constexpr int kBatchDensityPairs = 4;  // pairs in flight per lane in the density phase (3: 2.09 G atom-steps/s, 4: 2.14 G)

struct RepParam {
    int n;          // atoms
    int atom_off;   // first atom in the concatenated per-atom arrays
    int ld;         // list leading dimension (multiple of 32)
    int ncells;
    int cell_off;   // first cell in `count`
    int cs_off;     // first entry in `cell_start` (ncells + 1 entries)
    int pot;        // potential index
    int pad;
    long long list_off;
    int ncell[3];
    double box[3], half_box[3], inv_cell[3], h[3];
    double centre0[3];  // centre of cell 0 (h/2); cell c's centre is (c + 1/2) h
    float h_f[3];
    float rc2_f, screen_lo_f, screen_hi_f;
    double rl2;
    double kick_per_dt;  // 0.5 kAccel / m: times dt, the half-kick factor
    double ke_factor;    // 0.5 m / kAccel
    double disp2_thr;    // (skin/2)^2
};

struct RepState {
    long long step, rebuilds;
    int set, sp, since_build, max_nnb;
    unsigned int error;
    float maxdisp2;
    double e_embed, e_pair, ke;
};

struct BatchBufs {
    double *xr[2][3], *v[2][3], *d[3], *xw[3];
    int *id[2];
    float *uref[3];
    float4 *shadow[2];
    float *fcache[3];
    int *cell, *cell_old, *slot, *cell_atoms;  // per atom
    int *count, *cell_start;                   // per replica cells
    uint32_t *list;
    int *nnb;
    const float4 *coef;                  // F rows of every potential
    const float4 *coef2;                 // fused f | phi rows of every potential
    const float4 *coef_f;                // the f rows alone (density pass), same interval index
    const SplineDesc<float> *fphi, *Fd;  // per potential (offsets in rows)
    const RepParam *par;
    RepState *st;
    const int *order;  // replicas, largest first
    int *queue;
    int nrep, cap, rebuild_every;
};

enum { BATCH_INIT = 0, BATCH_RUN = 1 };

struct Smem {
    RepParam P;
    float4 shift[27];
    double red_d[kMaxBatchWarps];
    float red_f[kMaxBatchWarps];
    int red_i[32];
    int chunk;
    int carry;
    int need;
    int rep;
    float4 cell_u[kMaxBatchWarps][32];
};

__device__ __forceinline__ int nwarps() { return (int)(blockDim.x >> 5); }

__device__ __forceinline__ float block_max_f(float v, Smem &S)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) S.red_f[threadIdx.x >> 5] = v;
    __syncthreads();
    float m = 0.f;
    for (int w = 0; w < nwarps(); ++w) m = fmaxf(m, S.red_f[w]);
    __syncthreads();
    return m;
}

__device__ __forceinline__ int block_max_i(int v, Smem &S)
{
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) S.red_i[threadIdx.x >> 5] = v;
    __syncthreads();
    int m = 0;
    for (int w = 0; w < nwarps(); ++w) m = max(m, S.red_i[w]);
    __syncthreads();
    return m;
}

// FP64 block sum of per-thread float pairs: warps in float pairs, then FP64
// over the warps in warp order.
__device__ __forceinline__ double block_sum_ff(float hi, float lo, Smem &S)
{
    const double s = warp_sum_ff(hi, lo);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) S.red_d[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nwarps(); ++w) t += S.red_d[w];
    __syncthreads();
    return t;
}

// ---- list rebuild of one replica (all threads of the block take part) ----

__device__ void rb_bin(const BatchBufs &B, const RepParam &P, int s)
{
    for (int i = threadIdx.x; i < P.n; i += blockDim.x) {
        const int g = P.atom_off + i;
        int c[3];
        bool finite = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double L = P.box[a];
            double x = __dadd_rn(B.xr[s][a][g], B.d[a][g]);
            if (!(x >= 0.0 && x < L)) {  // kept when already in [0, L)
                const double q = floor(__ddiv_rn(x, L));
                x = __dsub_rn(x, __dmul_rn(L, q));
            }
            finite = finite && isfinite(x);
            B.xw[a][g] = x;
            const double q = floor(__dmul_rn(x, P.inv_cell[a]));
            c[a] = finite ? (int)fmax(fmin(q, (double)(P.ncell[a] - 1)), 0.0) : 0;
        }
        const int cell = (c[2] * P.ncell[1] + c[1]) * P.ncell[0] + c[0];
        B.cell_old[g] = cell;
        B.slot[g] = atomicAdd(&B.count[P.cell_off + cell], 1);
    }
}

// Exclusive scan of the counts into cell_start[0..ncells]; counts are zeroed.
__device__ void rb_scan(const BatchBufs &B, const RepParam &P, Smem &S)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int *cnt = B.count + P.cell_off;
    int *start = B.cell_start + P.cs_off;
    if (threadIdx.x == 0) S.carry = 0;
    __syncthreads();
    for (int base = 0; base < P.ncells; base += blockDim.x) {
        const int c = base + threadIdx.x;
        const int v = (c < P.ncells) ? cnt[c] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) S.red_i[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int w = (lane < nwarps()) ? S.red_i[lane] : 0;
            int wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            S.red_i[lane] = wi - w;  // exclusive prefix of the warp totals
            if (lane == 31) S.chunk = wi;
        }
        __syncthreads();
        const int excl = S.carry + S.red_i[warp] + incl - v;
        if (c < P.ncells) {
            start[c] = excl;
            cnt[c] = 0;
        }
        const int chunk_total = S.chunk;
        __syncthreads();
        if (threadIdx.x == 0) S.carry += chunk_total;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[P.ncells] = S.carry;
}

__device__ void rb_scatter(const BatchBufs &B, const RepParam &P)
{
    const int *start = B.cell_start + P.cs_off;
    for (int i = threadIdx.x; i < P.n; i += blockDim.x) {
        const int g = P.atom_off + i;
        B.cell_atoms[P.atom_off + start[B.cell_old[g]] + B.slot[g]] = i;
    }
}

__device__ void rb_sort(const BatchBufs &B, const RepParam &P, int s)
{
    const int *start = B.cell_start + P.cs_off;
    const int *id = B.id[s] + P.atom_off;
    int *ca = B.cell_atoms + P.atom_off;
    for (int c = threadIdx.x; c < P.ncells; c += blockDim.x) {
        const int s0 = start[c], e0 = start[c + 1];
        for (int q = s0 + 1; q < e0; ++q) {
            const int a = ca[q];
            const int ka = id[a];
            int r = q - 1;
            while (r >= s0 && id[ca[r]] > ka) {
                ca[r + 1] = ca[r];
                --r;
            }
            ca[r + 1] = a;
        }
    }
}

__device__ void rb_permute(const BatchBufs &B, const RepParam &P, int s, int sp)
{
    const int t = 1 - s;
    for (int p = threadIdx.x; p < P.n; p += blockDim.x) {
        const int gp = P.atom_off + p;
        const int gi = P.atom_off + B.cell_atoms[gp];
        const int cell = B.cell_old[gi];
        const int cc[3] = {cell % P.ncell[0], (cell / P.ncell[0]) % P.ncell[1], cell / (P.ncell[0] * P.ncell[1])};
        float u[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double X = B.xw[a][gi];
            B.xr[t][a][gp] = X;
            const double ctr = __dmul_rn((double)cc[a] + 0.5, P.h[a]);
            u[a] = (float)__dsub_rn(X, ctr);
            B.uref[a][gp] = u[a];
            B.v[t][a][gp] = B.v[s][a][gi];
            B.d[a][gp] = 0.0;
        }
        B.shadow[sp][gp] = make_float4(u[0], u[1], u[2], 0.f);
        B.id[t][gp] = B.id[s][gi];
        B.cell[gp] = cell;
    }
}

// exact list decision as in the single-system path
__device__ __forceinline__ bool rb_exact(const BatchBufs &B, const RepParam &P, int set, int gp, int gq)
{
    double d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = __dsub_rn(B.xr[set][a][gq], B.xr[set][a][gp]);
        if (x > P.half_box[a]) x = __dsub_rn(x, P.box[a]);
        else if (x < -P.half_box[a]) x = __dadd_rn(x, P.box[a]);
        d[a] = x;
    }
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
    return r2 < P.rl2;
}

// Verlet list, one warp per cell (warps stride over the replica's cells);
// same candidate order and ballot append as the single-system builder.
__device__ void rb_list(const BatchBufs &B, Smem &S, int set, int sp, int cap, RepState *st)
{
    Smem &W = S;
    const RepParam &P = S.P;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float4 *sw = B.shadow[sp] + P.atom_off;
    const unsigned lt = (1u << lane) - 1u;
    int my_max = 0;
    for (int c = warp; c < P.ncells; c += nwarps()) {
        const int cx = c % P.ncell[0], cy = (c / P.ncell[0]) % P.ncell[1], cz = c / (P.ncell[0] * P.ncell[1]);
        int e_start = 0, e_cnt = 0;
        if (lane < 27) {
            int ex = cx + lane % 3 - 1, ey = cy + (lane / 3) % 3 - 1, ez = cz + lane / 9 - 1;
            ex += (ex < 0) ? P.ncell[0] : ((ex >= P.ncell[0]) ? -P.ncell[0] : 0);
            ey += (ey < 0) ? P.ncell[1] : ((ey >= P.ncell[1]) ? -P.ncell[1] : 0);
            ez += (ez < 0) ? P.ncell[2] : ((ez >= P.ncell[2]) ? -P.ncell[2] : 0);
            const int e = (ez * P.ncell[1] + ey) * P.ncell[0] + ex;
            e_start = B.cell_start[P.cs_off + e];
            e_cnt = B.cell_start[P.cs_off + e + 1] - e_start;
        }
        int incl = e_cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int excl = incl - e_cnt;
        const int a0 = B.cell_start[P.cs_off + c], na = B.cell_start[P.cs_off + c + 1] - a0;
        for (int base = 0; base < na; base += 32) {
            const int nb = min(32, na - base);
            if (lane < nb) W.cell_u[warp][lane] = sw[a0 + base + lane];
            int my_cnt = 0;
            __syncwarp();
            for (int m0 = 0; m0 < total; m0 += 32) {
                const int m = m0 + lane;
                int code = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int probe = min(code + step, 26);
                    const int off = __shfl_sync(0xffffffffu, excl, probe);
                    if (code + step <= 26 && off <= m) code = probe;
                }
                const int st0 = __shfl_sync(0xffffffffu, e_start, code);
                const int of0 = __shfl_sync(0xffffffffu, excl, code);
                const bool valid = m < total;
                const int q = st0 + (m - of0);
                float4 wq = make_float4(0.f, 0.f, 0.f, 0.f);
                if (valid) {
                    const float4 uq = sw[q];
                    const float4 shf = S.shift[code];
                    wq = make_float4(uq.x + shf.x, uq.y + shf.y, uq.z + shf.z, 0.f);
                }
                for (int a = 0; a < nb; ++a) {
                    const int p = a0 + base + a;
                    const float4 up = W.cell_u[warp][a];
                    bool in = false;
                    if (valid && q != p) {
                        const float dx = wq.x - up.x, dy = wq.y - up.y, dz = wq.z - up.z;
                        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        in = (r2 < P.screen_lo_f)
                                 ? true
                                 : ((r2 > P.screen_hi_f) ? false : rb_exact(B, P, set, P.atom_off + p, P.atom_off + q));
                    }
                    const unsigned mask = __ballot_sync(0xffffffffu, in);
                    const int cnt0 = __shfl_sync(0xffffffffu, my_cnt, a);
                    if (in) {
                        const int pos = cnt0 + __popc(mask & lt);
                        if (pos < cap)
                            B.list[P.list_off + (size_t)pos * P.ld + p] =
                                list_entry((uint32_t)q, code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1);
                    }
                    if (lane == a) my_cnt += __popc(mask);
                }
            }
            if (lane < nb) {
                B.nnb[P.atom_off + a0 + base + lane] = min(my_cnt, cap);
                if (my_cnt > cap) atomicOr(&st->error, ERR_LIST_OVERFLOW);
                my_max = max(my_max, my_cnt);
            }
            __syncwarp();
        }
    }
    const int m = block_max_i(my_max, W);
    if (threadIdx.x == 0) st->max_nnb = max(st->max_nnb, m);
}

// ---- one replica, all steps ----

__device__ void run_replica(const BatchBufs &B, Smem &S, int r, int mode, int nsteps, double dt)
{
    RepParam &P = S.P;
    RepState *st = B.st + r;
    const float4 *cf2 = B.coef2;
    const SplineDesc<float> g = B.fphi[P.pot];
    const SplineDesc<float> Fd = B.Fd[P.pot];
    const double hk = P.kick_per_dt * dt;  // F dt / (2m) per unit force
    const float hkf = (float)hk;
    const float hf[3] = {P.h_f[0], P.h_f[1], P.h_f[2]};
    int set = st->set, sp = st->sp, since = st->since_build;
    float maxd2 = st->maxdisp2;
    const int steps = (mode == BATCH_INIT) ? 1 : nsteps;
    if (mode == BATCH_RUN && nsteps > 0) {
        // opening kick and drift from the cached forces
        float dmax = 0.f;
        for (int i = threadIdx.x; i < P.n; i += blockDim.x) {
            const int gi = P.atom_off + i;
            float dd = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double v = fma((double)B.fcache[a][gi], hk, B.v[set][a][gi]);
                B.v[set][a][gi] = v;
                const double dn = fma(v, dt, B.d[a][gi]);
                B.d[a][gi] = dn;
                reinterpret_cast<float *>(B.shadow[sp ^ 1] + gi)[a] = B.uref[a][gi] + (float)dn;
                const float gc = (float)dn;
                dd += gc * gc;
            }
            dmax = fmaxf(dmax, dd);
        }
        maxd2 = block_max_f(dmax, S);
    }
    for (int it = 0; it < steps; ++it) {
        const bool last = (it == steps - 1);
        bool need;
        if (mode == BATCH_INIT) {
            need = true;
        } else {
            sp ^= 1;
            ++since;
            need = (since >= B.rebuild_every) || ((double)maxd2 > P.disp2_thr);
        }
        if (need) {
            rb_bin(B, P, set);
            __syncthreads();
            rb_scan(B, P, S);
            __syncthreads();
            rb_scatter(B, P);
            __syncthreads();
            rb_sort(B, P, set);
            __syncthreads();
            rb_permute(B, P, set, sp);
            __syncthreads();
            set = 1 - set;
            since = 0;
            rb_list(B, S, set, sp, B.cap, st);
            __syncthreads();
            if (threadIdx.x == 0) st->rebuilds += 1;
        }
        // density pass: rho, F'(rho) into the record's w; F(rho) on the last step
        float4 *sw = B.shadow[sp] + P.atom_off;
        float e_emb = 0.f;
        for (int i = threadIdx.x; i < P.n; i += blockDim.x) {
            const float4 ui = sw[i];
            const int nn = B.nnb[P.atom_off + i];
            const uint32_t *lp = B.list + P.list_off + i;
            float rho = 0.f;
            // kBatchDensityPairs pairs per round, all gathers issued before
            // any is used; the sum runs in column order
            constexpr int UQ = kBatchDensityPairs;
            for (int k = 0; k < nn; k += UQ) {
                uint32_t e[UQ];
                float4 u[UQ];
#pragma unroll
                for (int q = 0; q < UQ; ++q) e[q] = (k + q < nn) ? lp[(size_t)(k + q) * P.ld] : 0u;
#pragma unroll
                for (int q = 0; q < UQ; ++q) u[q] = sw[(q == 0 || k + q < nn ? e[q] : e[0]) & kIndexMask];
#pragma unroll
                for (int q = 0; q < UQ; ++q) {
                    const Shift<float> shf = entry_shift<float>(e[q], hf);
                    const float dx = (u[q].x - ui.x) + shf.x, dy = (u[q].y - ui.y) + shf.y,
                                dz = (u[q].z - ui.z) + shf.z;
                    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    if (k + q < nn && r2 < P.rc2_f) {
                        float rinv, rr;
                        inv_r(r2, rinv, rr);
                        float t;
                        const int kk = segment(g, rr, t);
                        const float4 c = B.coef_f[g.offset + kk];
                        rho += fmaf(t, fmaf(t, fmaf(t, c.w, c.z), c.y), c.x);
                    }
                }
            }
            float Fv, Fdv;
            spline_any(Fd, B.coef, rho, Fv, Fdv);
            reinterpret_cast<float *>(sw + i)[3] = Fdv;
            e_emb += Fv;
        }
        __syncthreads();
        // force pass fused with the kicks and the drift
        const bool energy = last;
        float e_pair = 0.f;
        double ke = 0.0;
        float dmax = 0.f;
        for (int i = threadIdx.x; i < P.n; i += blockDim.x) {
            const int gi = P.atom_off + i;
            const float4 ui = sw[i];
            const int nn = B.nnb[gi];
            const uint32_t *lp = B.list + P.list_off + i;
            float fx = 0.f, fy = 0.f, fz = 0.f;
            // two pairs per round; the next round's records and the columns
            // of the round after are in flight while a round is computed
            uint32_t e[2], en[2];
            float4 u[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) e[q] = (q < nn) ? lp[(size_t)q * P.ld] : 0u;
#pragma unroll
            for (int q = 0; q < 2; ++q) en[q] = (2 + q < nn) ? lp[(size_t)(2 + q) * P.ld] : 0u;
#pragma unroll
            for (int q = 0; q < 2; ++q) u[q] = (nn > 0) ? sw[(q == 0 || q < nn ? e[q] : e[0]) & kIndexMask] : ui;
            for (int k = 0; k < nn; k += 2) {
                float4 un[2];
                uint32_t e2[2];
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    un[q] = (k + 2 < nn) ? sw[(q == 0 || k + 2 + q < nn ? en[q] : en[0]) & kIndexMask] : ui;
#pragma unroll
                for (int q = 0; q < 2; ++q) e2[q] = (k + 4 + q < nn) ? lp[(size_t)(k + 4 + q) * P.ld] : 0u;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                const float4 uj = u[q];
                const Shift<float> shf = entry_shift<float>(e[q], hf);
                const float dx = (uj.x - ui.x) + shf.x, dy = (uj.y - ui.y) + shf.y, dz = (uj.z - ui.z) + shf.z;
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                if (k + q < nn && r2 < P.rc2_f) {
                    float rinv, rr;
                    inv_r(r2, rinv, rr);
                    float t;
                    const int kk = segment(g, rr, t);
                    const float4 cf = cf2[2 * (g.offset + kk)];
                    const float4 cp = cf2[2 * (g.offset + kk) + 1];
                    const float fd = fmaf(t, fmaf(t, 3.f * cf.w, 2.f * cf.z), cf.y);
                    const float pd = fmaf(t, fmaf(t, 3.f * cp.w, 2.f * cp.z), cp.y);
                    const float sij = fmaf(uj.w, fd, fmaf(ui.w, fd, pd));
                    const float sr = sij * rinv;
                    fx = fmaf(sr, dx, fx);
                    fy = fmaf(sr, dy, fy);
                    fz = fmaf(sr, dz, fz);
                    if (energy) e_pair += 0.5f * fmaf(t, fmaf(t, fmaf(t, cp.w, cp.z), cp.y), cp.x);
                }
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    e[q] = en[q];
                    en[q] = e2[q];
                    u[q] = un[q];
                }
            }
            if (!isfinite(fx + fy + fz)) atomicOr(&st->error, ERR_NONFINITE);
            const float f[3] = {fx, fy, fz};
            float dd = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double v = B.v[set][a][gi];
                if (mode == BATCH_INIT || last) B.fcache[a][gi] = f[a];
                if (mode == BATCH_RUN) {
                    if (last) {
                        v = fma((double)f[a], hk, v);  // closing half kick only
                    } else {
                        v += (double)(2.f * (f[a] * hkf));  // closing + opening half kicks
                        const double dn = fma(v, dt, B.d[a][gi]);
                        B.d[a][gi] = dn;
                        reinterpret_cast<float *>(B.shadow[sp ^ 1] + gi)[a] = B.uref[a][gi] + (float)dn;
                        const float gc = (float)dn;
                        dd += gc * gc;
                    }
                    B.v[set][a][gi] = v;
                }
                if (energy) ke += P.ke_factor * v * v;
            }
            dmax = fmaxf(dmax, dd);
        }
        maxd2 = block_max_f(dmax, S);
        if (energy) {
            const double eb = block_sum_ff(e_emb, 0.f, S);
            const double ep = block_sum_ff(e_pair, 0.f, S);
            const float kh = (float)ke;
            const double kt = block_sum_ff(kh, (float)(ke - (double)kh), S);
            if (threadIdx.x == 0) {
                st->e_embed = eb;
                st->e_pair = ep;
                st->ke = kt;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st->set = set;
        st->sp = sp;
        st->since_build = since;
        st->maxdisp2 = maxd2;
        if (mode == BATCH_RUN) st->step += nsteps;
    }
    __syncthreads();
}

template <int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) k_batch(BatchBufs B, int mode, int nsteps, double dt)
{
    __shared__ Smem S;
    for (;;) {
        if (threadIdx.x == 0) S.rep = atomicAdd(B.queue, 1);
        __syncthreads();
        const int k = S.rep;
        if (k >= B.nrep) return;
        const int r = B.order[k];
        if (threadIdx.x == 0) S.P = B.par[r];
        __syncthreads();
        for (int c = threadIdx.x; c < 27; c += blockDim.x) {
            const int dx = c % 3 - 1, dy = (c / 3) % 3 - 1, dz = c / 9 - 1;
            S.shift[c] = make_float4(dx * S.P.h_f[0], dy * S.P.h_f[1], dz * S.P.h_f[2], 0.f);
        }
        __syncthreads();
        run_replica(B, S, r, mode, nsteps, dt);
    }
}

// replica state to the caller's order (AoS): positions, velocities, forces
__global__ void k_batch_store(BatchBufs B, int r, double *pos, double *vel, double *force)
{
    const RepParam &P = B.par[r];
    const int s = B.st[r].set;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n) return;
    const int gp = P.atom_off + p;
    const size_t o = 3 * (size_t)B.id[s][gp];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (pos) pos[o + a] = __dadd_rn(B.xr[s][a][gp], B.d[a][gp]);
        if (vel) vel[o + a] = B.v[s][a][gp];
        if (force) force[o + a] = (double)B.fcache[a][gp];
    }
}



// ==========================================================================
// host side

SplineDesc<float> batch_desc(const md_spline &s, int offset, const double *row_last, const double *row0)
{
    SplineDesc<float> d;
    d.offset = offset;
    d.nint = s.n - 1;
    d.x0 = (float)s.x0;
    d.inv_h = (float)(1.0 / s.dx);
    d.h_hi = (float)s.dx;
    d.h_lo = (float)(s.dx - (double)d.h_hi);
    const double x_end = s.x0 + (double)(s.n - 1) * s.dx;
    d.x_end = (float)x_end;
    d.y_lo = (float)row0[0];
    d.s_lo = (float)row0[1];
    const double t = s.dx;
    d.y_end = (float)(row_last[0] + t * (row_last[1] + t * (row_last[2] + t * row_last[3])));
    d.s_end = (float)(row_last[1] + t * (2.0 * row_last[2] + 3.0 * t * row_last[3]));
    return d;
}

thread_local std::string g_batch_create_error;

}  // namespace
}  // namespace eammd

using namespace eammd;

struct md_batch {
    int nrep = 0;
    int64_t total = 0;
    std::vector<RepParam> par;
    std::vector<int> order;
    BatchBufs B{};
    RepState *st_host = nullptr;
    std::vector<void *> allocs;
    md_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int grid = 0;
    int schedule = 0;
    double *stage = nullptr;
    int max_n = 0;
    long long launches = 0;
    struct G { int nsteps; double dt; cudaGraph_t g; cudaGraphExec_t e; };
    std::vector<G> graphs;
    std::string err;
    md_status fail(md_status s, const std::string &m)
    {
        err = m;
        return s;
    }
};

namespace {

void *balloc(md_batch *b, size_t bytes)
{
    bytes = ((bytes ? bytes : 256) + 255) & ~size_t(255);
    void *p = nullptr;
    if (b->opt.alloc) {
        p = b->opt.alloc(bytes, b->opt.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) b->allocs.push_back(p);
    return p;
}

template <class T>
bool balloc_n(md_batch *b, T *&p, size_t count)
{
    p = (T *)balloc(b, count * sizeof(T));
    return p != nullptr;
}

#define BCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return b->fail(e_ == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA,             \
                           std::string(#call) + ": " + cudaGetErrorString(e_));                    \
    } while (0)

// schedules the autotuner chooses from: threads per block, blocks per SM
struct BatchSchedule {
    int block, min_blocks;
};
constexpr BatchSchedule kSchedules[5] = {{512, 1}, {256, 2}, {256, 3}, {1024, 1}, {512, 2}};
constexpr int kNumSchedules = 5;

md_status batch_launch(md_batch *b, int mode, int nsteps, double dt)
{
    BCK(cudaMemsetAsync(b->B.queue, 0, sizeof(int), b->stream));
    switch (b->schedule) {
    case 1: k_batch<256, 2><<<b->grid, 256, 0, b->stream>>>(b->B, mode, nsteps, dt); break;
    case 3: k_batch<1024, 1><<<b->grid, 1024, 0, b->stream>>>(b->B, mode, nsteps, dt); break;
    case 4: k_batch<512, 2><<<b->grid, 512, 0, b->stream>>>(b->B, mode, nsteps, dt); break;
    case 2: k_batch<256, 3><<<b->grid, 256, 0, b->stream>>>(b->B, mode, nsteps, dt); break;
    default: k_batch<512, 1><<<b->grid, 512, 0, b->stream>>>(b->B, mode, nsteps, dt); break;
    }
    b->launches += 1;
    BCK(cudaGetLastError());
    return MD_OK;
}

md_status batch_sync(md_batch *b)
{
    BCK(cudaStreamSynchronize(b->stream));
    BCK(cudaMemcpy(b->st_host, b->B.st, sizeof(RepState) * b->nrep, cudaMemcpyDeviceToHost));
    for (int r = 0; r < b->nrep; ++r) {
        const unsigned e = b->st_host[r].error;
        if (e & ERR_LIST_OVERFLOW)
            return b->fail(MD_ERR_LIST_OVERFLOW, "replica " + std::to_string(r) + ": list capacity exceeded (" +
                                                     std::to_string(b->st_host[r].max_nnb) + " > " +
                                                     std::to_string(b->B.cap) + ")");
        if (e & ERR_NONFINITE) return b->fail(MD_ERR_NONFINITE, "replica " + std::to_string(r) + ": non-finite force");
    }
    return MD_OK;
}

}  // namespace

extern "C" {

md_status md_batch_create(int32_t nrep, const md_replica *reps, int32_t npot, const md_potential *pots,
                          const md_options *opt, md_batch **out)
{
    g_batch_create_error.clear();
    auto bad = [](md_status s, const std::string &m) {
        g_batch_create_error = m;
        return s;
    };
    if (!out) return bad(MD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nrep < 1 || !reps || npot < 1 || !pots) return bad(MD_ERR_ARG, "need at least one replica and potential");
    md_options o;
    md_options_default(&o);
    if (opt) o = *opt;
    if (o.precision != MD_PRECISION_MIXED) return bad(MD_ERR_ARG, "batches run the mixed-precision path");
    if (o.open_axes != 0) return bad(MD_ERR_ARG, "batch replicas are periodic (open_axes must be 0)");
    if ((o.alloc == nullptr) != (o.free == nullptr)) return bad(MD_ERR_ARG, "alloc and free go together");
    if (o.rebuild_every < 1) o.rebuild_every = 10;
    if (o.batch_schedule < 0 || o.batch_schedule > kNumSchedules)
        return bad(MD_ERR_ARG, "batch_schedule must be 0 (tuned) or 1..5");
    // potentials: one type each, f and phi on one grid (fused rows)
    std::vector<double> rowsF, rows2, rowsf;
    std::vector<SplineDesc<float>> dF(npot), dfphi(npot);
    for (int q = 0; q < npot; ++q) {
        const md_potential &pt = pots[q];
        if (pt.ntypes != 1 || !pt.mass || !pt.F || !pt.f || !pt.phi || !(pt.mass[0] > 0.0) || !(pt.r_cut > 0.0) ||
            !(pt.skin >= 0.0))
            return bad(MD_ERR_ARG, "batch potentials have one atom type, mass > 0, r_cut > 0, skin >= 0");
        const md_spline &F = pt.F[0], &f = pt.f[0], &ph = pt.phi[0];
        for (const md_spline *sp : {&F, &f, &ph}) {
            if (sp->n < 2 || !(sp->dx > 0.0) || !sp->y) return bad(MD_ERR_ARG, "bad spline");
            for (int k = 0; k < sp->n; ++k)
                if (!std::isfinite(sp->y[k])) return bad(MD_ERR_ARG, "non-finite knot value");
        }
        if (f.n != ph.n || f.x0 != ph.x0 || f.dx != ph.dx || f.x0 > 0.0 || f.x0 + (f.n - 1) * f.dx < pt.r_cut)
            return bad(MD_ERR_ARG, "batch potentials need f and phi on one grid covering [0, r_cut]");
        std::vector<double> rf, rp;
        int offF = (int)(rowsF.size() / 4);
        if (!hermite_coefficients(F, rowsF)) return bad(MD_ERR_ARG, "singular spline");
        dF[q] = batch_desc(F, offF, &rowsF[rowsF.size() - 4], &rowsF[4 * (size_t)offF]);
        if (!hermite_coefficients(f, rf) || !hermite_coefficients(ph, rp)) return bad(MD_ERR_ARG, "singular spline");
        int off2 = (int)(rows2.size() / 8);
        for (int k = 0; k < f.n - 1; ++k) {
            for (int c = 0; c < 4; ++c) rows2.push_back(rf[4 * (size_t)k + c]);
            for (int c = 0; c < 4; ++c) rows2.push_back(rp[4 * (size_t)k + c]);
            for (int c = 0; c < 4; ++c) rowsf.push_back(rf[4 * (size_t)k + c]);
        }
        dfphi[q] = batch_desc(f, off2, &rf[rf.size() - 4], &rf[0]);
    }
    md_batch *b = new (std::nothrow) md_batch();
    if (!b) return bad(MD_ERR_OOM, "host allocation failed");
    b->opt = o;
    b->nrep = nrep;
    b->par.resize(nrep);
    int64_t atom_off = 0, cell_off = 0, cs_off = 0;
    double max_expect = 0.0;
    for (int r = 0; r < nrep; ++r) {
        const md_replica &R = reps[r];
        if (R.potential < 0 || R.potential >= npot || R.n < 1 || !R.pos) {
            delete b;
            return bad(MD_ERR_ARG, "replica " + std::to_string(r) + ": bad potential index, n or pos");
        }
        const md_potential &pt = pots[R.potential];
        const double r_list = pt.r_cut + pt.skin;
        RepParam &P = b->par[r];
        memset(&P, 0, sizeof(P));
        P.n = (int)R.n;
        P.atom_off = (int)atom_off;
        P.ld = (int)((R.n + 31) / 32 * 32);
        P.pot = R.potential;
        double hmax = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double L = R.box[a];
            if (!(L > 0.0) || std::floor(L / r_list) < 3.0) {
                delete b;
                return bad(MD_ERR_BOX, "replica " + std::to_string(r) + ": box edge shorter than 3 (r_cut + skin)");
            }
            P.box[a] = L;
            P.half_box[a] = 0.5 * L;
            P.ncell[a] = (int)std::floor(L / r_list);
            P.inv_cell[a] = (double)P.ncell[a] / L;
            P.h[a] = L / (double)P.ncell[a];
            P.h_f[a] = (float)P.h[a];
            hmax = std::max(hmax, P.h[a]);
        }
        P.ncells = P.ncell[0] * P.ncell[1] * P.ncell[2];
        P.cell_off = (int)cell_off;
        P.cs_off = (int)cs_off;
        P.rl2 = r_list * r_list;
        const double margin = 8.0 * (20.0 * hmax * r_list + 4.0 * r_list * r_list) * std::ldexp(1.0, -24);
        P.screen_lo_f = (float)(P.rl2 - margin);
        P.screen_hi_f = (float)(P.rl2 + margin);
        P.rc2_f = (float)(pt.r_cut * pt.r_cut);
        P.kick_per_dt = 0.5 * kAccel / pt.mass[0];
        P.ke_factor = 0.5 * pt.mass[0] / kAccel;
        P.disp2_thr = 0.25 * pt.skin * pt.skin;
        const double vol = R.box[0] * R.box[1] * R.box[2];
        max_expect = std::max(max_expect, (double)R.n / vol * 4.0 / 3.0 * M_PI * r_list * r_list * r_list);
        for (int64_t i = 0; i < 3 * R.n; ++i)
            if (!std::isfinite(R.pos[i]) || (R.vel && !std::isfinite(R.vel[i]))) {
                delete b;
                return bad(MD_ERR_NONFINITE, "replica " + std::to_string(r) + ": non-finite input");
            }
        atom_off += R.n;
        cell_off += P.ncells;
        cs_off += P.ncells + 1;
        b->max_n = std::max(b->max_n, (int)R.n);
    }
    if (atom_off >= (int64_t)kIndexMask) {
        delete b;
        return bad(MD_ERR_CAPACITY, "more than 2^26 atoms in all");
    }
    b->total = atom_off;
    const int cap = o.list_capacity > 0 ? o.list_capacity : std::max(16, ((int)std::ceil(1.25 * max_expect) + 8 + 3) & ~3);
    long long list_off = 0;
    for (auto &P : b->par) {
        P.list_off = list_off;
        list_off += (long long)cap * P.ld;
    }
    // order: largest first
    b->order.resize(nrep);
    for (int r = 0; r < nrep; ++r) b->order[r] = r;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return b->par[x].n > b->par[y].n; });
    if (o.cuda_stream) {
        b->stream = (cudaStream_t)o.cuda_stream;
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess) {
        b->own_stream = true;
    } else {
        delete b;
        return bad(MD_ERR_CUDA, "cannot create a stream");
    }
    BatchBufs &B = b->B;
    const size_t N = (size_t)atom_off;
    bool ok = true;
    for (int s = 0; s < 2; ++s)
        for (int a = 0; a < 3; ++a) ok = ok && balloc_n(b, B.xr[s][a], N) && balloc_n(b, B.v[s][a], N);
    for (int a = 0; a < 3; ++a)
        ok = ok && balloc_n(b, B.d[a], N) && balloc_n(b, B.xw[a], N) && balloc_n(b, B.uref[a], N) &&
             balloc_n(b, B.fcache[a], N);
    for (int s = 0; s < 2; ++s) ok = ok && balloc_n(b, B.id[s], N) && balloc_n(b, B.shadow[s], N);
    ok = ok && balloc_n(b, B.cell, N) && balloc_n(b, B.cell_old, N) && balloc_n(b, B.slot, N) &&
         balloc_n(b, B.cell_atoms, N) && balloc_n(b, B.nnb, N);
    ok = ok && balloc_n(b, B.count, (size_t)cell_off) && balloc_n(b, B.cell_start, (size_t)cs_off);
    ok = ok && balloc_n(b, B.list, (size_t)list_off);
    float4 *coef = nullptr, *coef2 = nullptr, *coef_f = nullptr;
    SplineDesc<float> *dfp = nullptr, *dFd = nullptr;
    RepParam *par = nullptr;
    int *order = nullptr;
    ok = ok && balloc_n(b, coef, rowsF.size() / 4) && balloc_n(b, coef2, rows2.size() / 4) &&
         balloc_n(b, coef_f, rowsf.size() / 4) &&
         balloc_n(b, dfp, (size_t)npot) && balloc_n(b, dFd, (size_t)npot) && balloc_n(b, par, (size_t)nrep) &&
         balloc_n(b, B.st, (size_t)nrep) && balloc_n(b, order, (size_t)nrep) && balloc_n(b, B.queue, 1) &&
         balloc_n(b, b->stage, 9 * (size_t)b->max_n);
    if (!ok) {
        md_batch_destroy(b);
        return bad(MD_ERR_OOM, "device allocation failed");
    }
    auto up4 = [](float4 *dst, const std::vector<double> &src) {
        std::vector<float4> t(src.size() / 4);
        for (size_t k = 0; k < t.size(); ++k)
            t[k] = make_float4((float)src[4 * k], (float)src[4 * k + 1], (float)src[4 * k + 2], (float)src[4 * k + 3]);
        return cudaMemcpy(dst, t.data(), t.size() * sizeof(float4), cudaMemcpyHostToDevice);
    };
    cudaError_t ce = up4(coef, rowsF);
    if (ce == cudaSuccess) ce = up4(coef2, rows2);
    if (ce == cudaSuccess) ce = up4(coef_f, rowsf);
    if (ce == cudaSuccess) ce = cudaMemcpy(dfp, dfphi.data(), sizeof(SplineDesc<float>) * npot, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(dFd, dF.data(), sizeof(SplineDesc<float>) * npot, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(par, b->par.data(), sizeof(RepParam) * nrep, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(order, b->order.data(), sizeof(int) * nrep, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemset(B.count, 0, sizeof(int) * (size_t)cell_off);
    if (ce == cudaSuccess) ce = cudaMemset(B.st, 0, sizeof(RepState) * (size_t)nrep);
    if (ce == cudaSuccess) ce = cudaMallocHost((void **)&b->st_host, sizeof(RepState) * nrep);
    // per-replica state, caller order within each replica
    for (int r = 0; r < nrep && ce == cudaSuccess; ++r) {
        const md_replica &R = reps[r];
        const RepParam &P = b->par[r];
        std::vector<double> x(R.n), v(R.n, 0.0);
        for (int a = 0; a < 3 && ce == cudaSuccess; ++a) {
            for (int64_t i = 0; i < R.n; ++i) {
                x[i] = R.pos[3 * i + a];
                v[i] = R.vel ? R.vel[3 * i + a] : 0.0;
            }
            ce = cudaMemcpy(B.xr[0][a] + P.atom_off, x.data(), sizeof(double) * R.n, cudaMemcpyHostToDevice);
            if (ce == cudaSuccess) ce = cudaMemcpy(B.v[0][a] + P.atom_off, v.data(), sizeof(double) * R.n, cudaMemcpyHostToDevice);
            if (ce == cudaSuccess) ce = cudaMemset(B.d[a] + P.atom_off, 0, sizeof(double) * R.n);
        }
        std::vector<int> id(R.n);
        for (int64_t i = 0; i < R.n; ++i) id[i] = (int)i;
        if (ce == cudaSuccess) ce = cudaMemcpy(B.id[0] + P.atom_off, id.data(), sizeof(int) * R.n, cudaMemcpyHostToDevice);
    }
    if (ce != cudaSuccess) {
        md_batch_destroy(b);
        return bad(MD_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(ce));
    }
    B.coef = coef;
    B.coef2 = coef2;
    B.coef_f = coef_f;
    B.fphi = dfp;
    B.Fd = dFd;
    B.par = par;
    B.order = order;
    B.nrep = nrep;
    B.cap = cap;
    B.rebuild_every = o.rebuild_every;
    int sms = 1, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto grid_for = [&](int sched) {
        int per_sm = 1;
        if (sched == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<256, 2>, 256, 0);
        else if (sched == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<256, 3>, 256, 0);
        else if (sched == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<1024, 1>, 1024, 0);
        else if (sched == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<512, 2>, 512, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<512, 1>, 512, 0);
        return std::max(1, std::min(nrep, std::max(per_sm, 1) * sms));
    };
    b->schedule = 0;
    b->grid = grid_for(0);
    md_status rc = batch_launch(b, BATCH_INIT, 1, 0.0);
    if (rc == MD_OK) rc = batch_sync(b);
    // schedule autotuner: right after the initial build every replica is
    // rebuild_every steps from its next build, so rebuild_every - 1 steps of
    // dt = 0 change nothing but the counters, which are restored afterwards
    if (rc == MD_OK && o.batch_schedule > 0) {
        b->schedule = o.batch_schedule - 1;
        b->grid = grid_for(b->schedule);
    } else if (rc == MD_OK && o.rebuild_every > 1 && o.lanes_per_atom == 0) {
        const int trial = std::min(o.rebuild_every - 1, 8);
        float best = 1e30f;
        int best_s = 0;
        cudaEvent_t t0, t1;
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        for (int round = 0; round < 2 && rc == MD_OK; ++round)
            for (int sc = 0; sc < kNumSchedules && rc == MD_OK; ++sc) {
                b->schedule = sc;
                b->grid = grid_for(sc);
                cudaEventRecord(t0, b->stream);
                rc = batch_launch(b, BATCH_RUN, trial, 0.0);
                cudaEventRecord(t1, b->stream);
                if (rc == MD_OK) rc = batch_sync(b);
                float ms = 0;
                cudaEventElapsedTime(&ms, t0, t1);
                if (round == 1 && ms < best) {
                    best = ms;
                    best_s = sc;
                }
                if (rc == MD_OK && cudaMemcpy(B.st, b->st_host, sizeof(RepState) * nrep, cudaMemcpyHostToDevice) != cudaSuccess)
                    rc = MD_ERR_CUDA;
                if (rc == MD_OK) {
                    // restore the counters of the state after the initial build
                    std::vector<RepState> restore(nrep);
                    memcpy(restore.data(), b->st_host, sizeof(RepState) * nrep);
                    for (int r = 0; r < nrep; ++r) {
                        restore[r].step -= trial;
                        restore[r].since_build -= trial;
                        if (trial & 1) restore[r].sp ^= 1;
                    }
                    if (cudaMemcpy(B.st, restore.data(), sizeof(RepState) * nrep, cudaMemcpyHostToDevice) != cudaSuccess)
                        rc = MD_ERR_CUDA;
                }
            }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        b->schedule = best_s;
        b->grid = grid_for(best_s);
        b->launches = 1;
    }
    if (rc == MD_OK) rc = batch_sync(b);
    if (rc != MD_OK) {
        g_batch_create_error = b->err;
        md_batch_destroy(b);
        return rc;
    }
    // rebuild counters start after the initial build
    for (int r = 0; r < nrep; ++r) b->st_host[r].rebuilds = 0;
    if (cudaMemcpy(B.st, b->st_host, sizeof(RepState) * nrep, cudaMemcpyHostToDevice) != cudaSuccess) {
        md_batch_destroy(b);
        return bad(MD_ERR_CUDA, "state upload failed");
    }
    *out = b;
    return MD_OK;
}

md_status md_batch_step(md_batch *b, int64_t nsteps, double dt)
{
    if (!b) return MD_ERR_ARG;
    if (nsteps < 0 || nsteps > (int64_t)1 << 30 || !std::isfinite(dt)) return b->fail(MD_ERR_ARG, "bad nsteps or dt");
    if (nsteps == 0) return MD_OK;
    if (!b->opt.use_graphs) return batch_launch(b, BATCH_RUN, (int)nsteps, dt);
    for (auto &g : b->graphs)
        if (g.nsteps == (int)nsteps && g.dt == dt) {
            BCK(cudaGraphLaunch(g.e, b->stream));
            b->launches += 1;
            return MD_OK;
        }
    cudaStream_t cs;
    BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t keep = b->stream;
    b->stream = cs;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    md_status rc = (e == cudaSuccess) ? batch_launch(b, BATCH_RUN, (int)nsteps, dt) : MD_ERR_CUDA;
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    b->stream = keep;
    b->launches -= 1;
    cudaStreamDestroy(cs);
    if (e != cudaSuccess || e2 != cudaSuccess || rc != MD_OK) return b->fail(MD_ERR_CUDA, "graph capture failed");
    cudaGraphExec_t ex;
    BCK(cudaGraphInstantiate(&ex, g, 0));
    b->graphs.push_back({(int)nsteps, dt, g, ex});
    BCK(cudaGraphLaunch(ex, b->stream));
    b->launches += 1;
    return MD_OK;
}

md_status md_batch_energy(md_batch *b, double *pe, double *ke)
{
    if (!b) return MD_ERR_ARG;
    md_status rc = batch_sync(b);
    if (rc != MD_OK) return rc;
    for (int r = 0; r < b->nrep; ++r) {
        if (pe) pe[r] = b->st_host[r].e_embed + b->st_host[r].e_pair;
        if (ke) ke[r] = b->st_host[r].ke;
    }
    return MD_OK;
}

md_status md_batch_get_state(md_batch *b, int32_t r, double *pos, double *vel, double *force)
{
    if (!b) return MD_ERR_ARG;
    if (r < 0 || r >= b->nrep) return b->fail(MD_ERR_ARG, "replica index out of range");
    md_status rc = batch_sync(b);
    if (rc != MD_OK) return rc;
    const int n = b->par[r].n;
    double *dp = b->stage, *dv = b->stage + 3 * (size_t)n, *df = b->stage + 6 * (size_t)n;
    k_batch_store<<<(n + 255) / 256, 256, 0, b->stream>>>(b->B, r, pos ? dp : nullptr, vel ? dv : nullptr,
                                                          force ? df : nullptr);
    b->launches += 1;
    BCK(cudaGetLastError());
    if (pos) BCK(cudaMemcpyAsync(pos, dp, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, b->stream));
    if (vel) BCK(cudaMemcpyAsync(vel, dv, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, b->stream));
    if (force) BCK(cudaMemcpyAsync(force, df, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return MD_OK;
}

md_status md_batch_info(md_batch *b, md_batch_info_t *out)
{
    if (!b || !out) return b ? b->fail(MD_ERR_ARG, "out is NULL") : MD_ERR_ARG;
    md_status rc = batch_sync(b);
    if (rc != MD_OK) return rc;
    memset(out, 0, sizeof(*out));
    out->replicas = b->nrep;
    out->atoms = b->total;
    out->blocks = b->grid;
    out->threads_per_block = kSchedules[b->schedule].block;
    out->list_capacity = b->B.cap;
    out->kernel_launches = b->launches;
    for (int r = 0; r < b->nrep; ++r) {
        out->rebuilds += b->st_host[r].rebuilds;
        out->max_neighbors = std::max(out->max_neighbors, b->st_host[r].max_nnb);
        out->steps = std::max<int64_t>(out->steps, b->st_host[r].step);
    }
    return MD_OK;
}

const char *md_batch_last_error(const md_batch *b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

void md_batch_destroy(md_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &g : b->graphs) {
        cudaGraphExecDestroy(g.e);
        cudaGraphDestroy(g.g);
    }
    for (void *p : b->allocs) {
        if (b->opt.free) b->opt.free(p, b->opt.alloc_ctx);
        else cudaFree(p);
    }
    if (b->st_host) cudaFreeHost(b->st_host);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
