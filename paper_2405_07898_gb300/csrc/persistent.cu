// persistent.cu -- md_step as one launch: every phase of every step (opening
// kick, rebuild decision, list rebuild, density, force with the kicks and the
// drift, energy sums) runs in one kernel, either a cooperative grid whose
// blocks meet at grid barriers (k_steps) or one thread-block cluster
// (k_steps_cluster, below).  For small systems, where a step is a few
// microseconds of work, this removes the per-kernel launch and scheduling
// gaps of the graph path.  The per-atom arithmetic is that of the graph path (same device
// functions, same lanes per atom), so positions, velocities and forces are
// bitwise equal; energy sums differ in rounding only (other block partition).
//
// Grid barriers: all blocks are resident (cooperative launch); a barrier is
// an arrival counter in device memory.  A wait gives up after the wait limit
// (md_options.wait_limit_us, 1 s by default) of %globaltimer, raises
// ERR_TIMEOUT and every later barrier of the launch returns at once, so the
// kernel ends within about the limit of a stuck block and the host reports
// MD_ERR_TIMEOUT.
#include "cluster.cuh"
#include "pair_kernels.cuh"
#include "rebuild_device.cuh"

#include <algorithm>

namespace eammd {
namespace {

__device__ __forceinline__ void prefetch_l1(const void *p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(__cvta_generic_to_global(p)));
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(__cvta_generic_to_global(p)) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(__cvta_generic_to_global(p)) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(__cvta_generic_to_global(p)) : "memory");
    return v;
}

// Grid barrier on a counter that only grows during a launch (zeroed by the
// host before it): barrier b of the launch is passed once the counter reaches
// (b + 1) x gridDim.x.  Arrival is a release add, the wait an acquire load, so
// every block sees the writes all blocks made before the barrier.  Returns
// false once any wait of the launch has timed out.
__device__ __forceinline__ bool grid_barrier(PersistScratch *ps, unsigned *err, uint64_t wait_ns)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        if (ld_acquire(err) & ERR_TIMEOUT) {
            good = 0;
        } else {
            unsigned long long a;
            asm volatile("atom.add.release.gpu.global.u64 %0, [%1], 1;"
                         : "=l"(a)
                         : "l"(__cvta_generic_to_global(&ps->arrive))
                         : "memory");
            const unsigned long long g = gridDim.x;
            const unsigned long long target = (a / g + 1) * g;
            if (a + 1 != target) {
                // relaxed polls, one acquire load once the count is reached;
                // the error word and the clock are read every 64th poll only
                const uint64_t t0 = global_ns();
                unsigned spins = 0;
                while (ld_relaxed(&ps->arrive) < target || ld_acquire(&ps->arrive) < target) {
                    if ((++spins & 63u) == 0 &&
                        ((ld_acquire(err) & ERR_TIMEOUT) || global_ns() - t0 > wait_ns)) {
                        atomicOr(err, ERR_TIMEOUT);
                        good = 0;
                        break;
                    }
                    __nanosleep(16);
                }
            }
        }
        ok = good;
    }
    __syncthreads();
    return ok;
}

// Lanes per atom of the list builds in the single-launch forms, taken when
// one pass of the grid (of the CTA, in the cluster form) covers all its
// atoms; otherwise one thread walks each atom's stencil.
constexpr int kListLanes = 8, kListLanesCluster = 4;

// One step loop of nsteps steps (nsteps >= 1).  The counters of DevState
// (set, record buffer, steps since the build) advance identically in every
// block; block 0 writes them back at the end.  The largest squared
// displacement alternates between two words: the force pass of step k writes
// word k & 1, the decision of step k + 1 reads it (the opening drift writes
// word 1 for the decision of step 0).
template <class R, bool MULTI, int TPA>
__global__ void __launch_bounds__(256) k_steps(Bufs<R> B, Geom G, Launch L, long long nsteps, PersistScratch *ps)
{
    using R4 = typename V4<R>::T;
    constexpr int UD = PairsInFlight<MULTI>::density, UF = PairsInFlight<MULTI>::force;
    DevState *st = B.st;
    unsigned *err = &st->error;
    int s = st->set, sp = st->sp, since = st->since_build;
    long long step = st->step, rebuilds = 0;
    int need = 0;
    const int n = L.n, nthreads = gridDim.x * blockDim.x, gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int width = blockDim.x / TPA, l = threadIdx.x % TPA;
    const int ntiles = (n + width - 1) / width;
    R h[3];
    load_h<R>(G, h);
    const R rc2 = g_rc2<R>(G);

    // opening kick and drift from the cached forces
    {
        float d2 = 0.f;
        for (int i = gtid; i < n; i += nthreads) d2 = fmaxf(d2, open_atom<R>(B, L, s, sp, i));
        block_max_disp(d2, &ps->maxdisp[1]);
    }
    if (!grid_barrier(ps, err, L.wait_ns)) return;

    for (long long k = 0; k < nsteps; ++k) {
        const bool last = k == nsteps - 1;
        // decision (as k_decide)
        sp ^= 1;
        step += 1;
        since += 1;
        const float md = __uint_as_float(ld_acquire(&ps->maxdisp[(k + 1) & 1]));
        need = (since >= L.rebuild_every) || ((double)md > L.disp2_thr);
        // word k & 1 was last read by the decision of step k - 1
        if (gtid == 0) ps->maxdisp[k & 1] = 0u;

        if (need) {
            for (int i = gtid; i < n; i += nthreads) bin_atom<R>(B, G, s, i);
            if (!grid_barrier(ps, err, L.wait_ns)) return;
            if (blockIdx.x == 0) scan_cells_block<R>(B, G.ncells);
            if (!grid_barrier(ps, err, L.wait_ns)) return;
            for (int i = gtid; i < n; i += nthreads) scatter_atom<R>(B, i);
            if (!grid_barrier(ps, err, L.wait_ns)) return;
            for (int c = gtid; c < G.ncells; c += nthreads) sort_cell<R>(B, s, c);
            if (!grid_barrier(ps, err, L.wait_ns)) return;
            for (int p = gtid; p < n; p += nthreads) permute_atom<R>(B, G, s, sp, p);
            if (gtid == 0) st->max_nnb = 0;
            s = 1 - s;
            since = 0;
            rebuilds += 1;
            if (!grid_barrier(ps, err, L.wait_ns)) return;
            if ((long long)n * kListLanes <= nthreads) {
                // kListLanes lanes per atom, all atoms in one pass
                const int p = blockIdx.x * (blockDim.x / kListLanes) + threadIdx.x / kListLanes;
                const int cnt =
                    (p < n) ? list_atom_lanes<R, kListLanes>(B, G, s, sp, p, L.ld, L.cap, threadIdx.x % kListLanes)
                            : 0;
                block_max_nnb(cnt, &st->max_nnb);
            } else {
                for (int base = blockIdx.x * blockDim.x; base < n; base += nthreads) {
                    const int p = base + threadIdx.x;
                    const int cnt = (p < n) ? list_atom<R>(B, G, s, sp, p, L.ld, L.cap) : 0;
                    block_max_nnb(cnt, &st->max_nnb);
                }
            }
            if (!grid_barrier(ps, err, L.wait_ns)) return;
        }

        // density pass
        {
            R4 *sw = B.shadow[sp];
            R e_embed = (R)0;
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
                const int i = tile * width + threadIdx.x / TPA;
                const bool active = i < n;
                const int ti = (MULTI && active) ? B.type[s][i] : 0;
                R rho = (R)0;
                if (active)
                    rho = density_lane<R, MULTI, TPA, UD>(B, h, rc2, s, B.nnb + i, L.cap, l, sw[i], ListGlobal{B.list + i, L.ld},
                                                          GlobalFetch<R>{sw}, TabGlobal<R>{B.coef2, B.coef_f});
                rho = lane_sum<TPA>(rho);
                if (active && l == 0) e_embed += embed<R>(B, sw, i, ti, rho);
            }
            if (last) {
                const R v[1] = {e_embed};
                block_sums_t<1, R>(v, B.partials, L.pstride, 0);
            }
        }
        if (!grid_barrier(ps, err, L.wait_ns)) return;

        // force pass with the closing kick (and, but for the last step, the
        // next opening kick and the drift)
        {
            const R4 *sw = B.shadow[sp];
            R e7[7] = {0, 0, 0, 0, 0, 0, 0};
            double ke = 0.0;
            float d2max = 0.f;
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
                const int i = tile * width + threadIdx.x / TPA;
                const bool active = i < n;
                const int ti = (MULTI && active) ? B.type[s][i] : 0;
                R f[3] = {0, 0, 0};
                float d2 = 0.f;
                const ListGlobal list{B.list + i, L.ld};
                // the integration's inputs into L1 while the pair loop runs
                if (active && l == 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        prefetch_l1(B.v[s][c] + i);
                        prefetch_l1(B.d[c] + i);
                        prefetch_l1(B.uref[c] + i);
                    }
                }
                if (last) {
                    if (active)
                        force_lane<R, MULTI, true, TPA, UF>(B, L, h, rc2, s, B.nnb + i, l, ti, sw[i], list,
                                                            GlobalFetch<R>{sw}, f, e7, TabGlobal<R>{B.coef2, B.coef_f});
#pragma unroll
                    for (int c = 0; c < 3; ++c) f[c] = lane_sum<TPA>(f[c]);
                    if (active) integrate<R, MODE_CLOSE, true, TPA>(B, L, s, sp, i, l, ti, f, ke, d2);
                } else {
                    if (active)
                        force_lane<R, MULTI, false, TPA, UF>(B, L, h, rc2, s, B.nnb + i, l, ti, sw[i], list,
                                                             GlobalFetch<R>{sw}, f, e7, TabGlobal<R>{B.coef2, B.coef_f});
#pragma unroll
                    for (int c = 0; c < 3; ++c) f[c] = lane_sum<TPA>(f[c]);
                    if (active) integrate<R, MODE_CLOSE_OPEN, false, TPA>(B, L, s, sp, i, l, ti, f, ke, d2);
                }
                d2max = fmaxf(d2max, lane_sum<TPA>(d2));
            }
            if (last) {
                const R ke_hi = (R)ke;
                const R ke_lo = (R)(ke - (double)ke_hi);
                const R v8[8] = {e7[0], ke_hi, e7[1], e7[2], e7[3], e7[4], e7[5], e7[6]};
                const R lo8[8] = {0, ke_lo, 0, 0, 0, 0, 0, 0};
                block_sums_t<8, R>(v8, B.partials, L.pstride, 1, lo8);
            } else {
                block_max_disp(d2max, &ps->maxdisp[k & 1]);
            }
        }
        if (!grid_barrier(ps, err, L.wait_ns)) return;
    }

    // energies of the last step, counters back to DevState
    for (int slot = blockIdx.x; slot < 9; slot += gridDim.x) reduce_slot(B.partials, st, slot, gridDim.x, L.pstride);
    if (gtid == 0) {
        st->set = s;
        st->sp = sp;
        st->since_build = since;
        st->step = step;
        st->rebuilds += rebuilds;
        st->need_rebuild = need;
        st->maxdisp2 = 0u;
        ps->maxdisp[0] = 0u;
        ps->maxdisp[1] = 0u;
    }
}

// ---- the same step loop in one thread-block cluster ----
//
// Up to a few thousand atoms a step is a few microseconds of latency-bound
// work.  In the cooperative grid every barrier is a device-memory round trip
// (arrival and release) whose release also waits for the block's stores to
// reach L2, and after its acquire every list column, count and neighbour
// record comes from L2 again.  Here the step loop runs in one cluster of at
// most 16 CTAs and, between list builds, reads device memory only for what
// does not fit or is type-dependent (the f and phi rows unless they are
// copied, the neighbour types and spline rows of several types) and writes it
// only for the cached forces of the last step:
//   * CTA r owns the atoms [r 2^shift, (r + 1) 2^shift) and holds their
//     state in shared memory: both record buffers, v and d (FP64), uref, the
//     list counts and the list columns (cluster_layout).  The device
//     functions of the graph path run unchanged on a view of Bufs whose
//     per-atom pointers are redirected there (offset by -r 2^shift);
//   * neighbour records are read from their owner's buffer through
//     distributed shared memory;
//   * the barrier is an mbarrier in every CTA on which each CTA arrives
//     remotely with release semantics at cluster scope; two alternate, so that
//     an arrival for the next barrier cannot land in the current phase, and a
//     wait is bounded as the grid barrier's is;
//   * an arrival can carry the CTA's largest squared displacement, stored
//     into every CTA's shared memory before the arrive, so that the rebuild
//     decision reads shared memory instead of a device word;
//   * a list build writes v and d back, runs the phases of the grid form on
//     device memory, and loads the new order's state; the launch ends by
//     writing v, d and the current records back;
//   * the spline descriptors and, where they fit, the rows of F sit in
//     shared memory, and optionally (FP32, one fused table) the f and phi
//     rows too.
// Owned atoms are walked in tiles of blockDim / TPA atoms, so the per-atom
// arithmetic is that of the graph path, bitwise.
struct ClusterSync {
    unsigned long long bar[2];
    float dmax[kMaxClusterCtas];  // slot r: CTA r's largest squared displacement
    float wmax[kPersistentBlock / 32];
    int ok;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// The address of the same shared-memory word in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_rank(uint32_t a, uint32_t rank)
{
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

template <class R>
__device__ __forceinline__ typename V4<R>::T ld_cluster(uint32_t a);
template <>
__device__ __forceinline__ float4 ld_cluster<float>(uint32_t a)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a));
    return v;
}
template <>
__device__ __forceinline__ double4_32a ld_cluster<double>(uint32_t a)
{
    double4_32a v;
    asm volatile("ld.shared::cluster.v2.f64 {%0,%1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
    asm volatile("ld.shared::cluster.v2.f64 {%0,%1}, [%2+16];" : "=d"(v.z), "=d"(v.w) : "r"(a));
    return v;
}

// Neighbour records from the owning CTA's buffer (the same shared-memory
// offset in every CTA).
template <class R>
struct ClusterFetch {
    uint32_t base;  // shared-window address of this CTA's copy of the buffer
    int shift;      // log2 of the atoms per CTA
    __device__ __forceinline__ typename V4<R>::T operator()(uint32_t e) const
    {
        const uint32_t j = e & kIndexMask;
        const uint32_t off = (j & ((1u << shift) - 1u)) * (uint32_t)sizeof(typename V4<R>::T);
        return ld_cluster<R>(map_rank(base + off, j >> shift));
    }
};

// Cluster barrier number b of the launch (every CTA counts its barriers
// alike).  With send, the block maximum of d2 goes into slot `rank` of every
// CTA's dmax ahead of the arrival.  Returns false once any wait of the launch
// has timed out.
__device__ __forceinline__ bool cluster_barrier(ClusterSync &cs, unsigned &b, int nct, uint32_t rank, bool send,
                                                float d2, unsigned *err, uint64_t wait_ns)
{
    if (send) {
        for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
        if ((threadIdx.x & 31) == 0) cs.wmax[threadIdx.x >> 5] = d2;
    }
    __syncthreads();
    const uint32_t k = b & 1u, parity = (b >> 1) & 1u;
    ++b;
    if ((int)threadIdx.x < nct) {
        const uint32_t t = threadIdx.x;
        if (send) {
            float m = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, cs.wmax[w]);
            asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(map_rank(smem_addr(&cs.dmax[rank]), t)), "f"(m)
                         : "memory");
        }
        asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(
                         map_rank(smem_addr(&cs.bar[k]), t))
                     : "memory");
    }
    if (threadIdx.x == 0) {
        int good = 1;
        const uint32_t a = smem_addr(&cs.bar[k]);
        const uint64_t t0 = global_ns();
        unsigned spins = 0;
        for (;;) {
            uint32_t done;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
                " selp.u32 %0, 1, 0, p;\n}"
                : "=r"(done)
                : "r"(a), "r"(parity)
                : "memory");
            if (done) break;
            if ((++spins & 15u) == 0 && ((ld_acquire(err) & ERR_TIMEOUT) || global_ns() - t0 > wait_ns)) {
                atomicOr(err, ERR_TIMEOUT);
                good = 0;
                break;
            }
        }
        cs.ok = good;
    }
    __syncthreads();
    return cs.ok;
}

// After a failed wait: leave only once every CTA has left or given up, since
// until then the others may still read this CTA's shared memory or arrive on
// its barriers.  They notice the timeout at their next barrier (the error
// word is polled there), so this wait is short; it is bounded by the larger
// of the wait limit and 1 s, so that a very small configured limit does not
// let a CTA leave early.  The count is ps->arrive, zeroed by the host before
// the launch; a CTA that finishes normally adds itself as it ends.
__device__ __forceinline__ void cluster_leave(PersistScratch *ps, int nct, unsigned *err, uint64_t wait_ns)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&ps->arrive, 1ull);
        const uint64_t t0 = global_ns(), limit = wait_ns > kWaitLimitNs ? wait_ns : kWaitLimitNs;
        while (ld_acquire(&ps->arrive) < (unsigned long long)nct) {
            if (global_ns() - t0 > limit) {
                atomicOr(err, ERR_TIMEOUT);
                break;
            }
            __nanosleep(256);
        }
    }
    __syncthreads();
}

template <class R, bool TABSM>
struct ClusterTab {
    using T = TabGlobal<R>;
    __device__ static T make(const Bufs<R> &B, const float4 *, const float4 *) { return T{B.coef2, B.coef_f}; }
};
template <>
struct ClusterTab<float, true> {
    using T = TabShared;
    __device__ static T make(const Bufs<float> &, const float4 *f_rows, const float4 *phi_rows)
    {
        return T{f_rows, phi_rows};
    }
};

template <class R, bool MULTI, int TPA, bool TABSM>
__global__ void __launch_bounds__(kPersistentBlock, 1)
    k_steps_cluster(Bufs<R> B, Geom G, Launch L, long long nsteps, PersistScratch *ps, ClusterPlan plan)
{
    using R4 = typename V4<R>::T;
    constexpr int UD = PairsInFlight<MULTI>::density, UF = PairsInFlight<MULTI>::force;
    __shared__ ClusterSync cs;
    __shared__ Tables<R> s_tab;
    DevState *st = B.st;
    unsigned *err = &st->error;
    int s = st->set, sp = st->sp, since = st->since_build;
    long long step = st->step, rebuilds = 0;
    int need = 0;
    const int n = L.n, nct = gridDim.x, nthreads = nct * blockDim.x, gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t rank = blockIdx.x;  // the grid is one cluster
    const int shift = plan.shift;
    const int chunk = 1 << shift, a0 = (int)rank << shift, a1 = min(n, a0 + chunk), m = a1 - a0;
    const int width = blockDim.x / TPA, l = threadIdx.x % TPA;
    const ClusterLayout lay = cluster_layout<R>(chunk, L.cap, plan.nF, TABSM ? L.nint_fused : 0);
    R4 *const rec0 = reinterpret_cast<R4 *>(dyn + lay.rec);  // buffers 0 and 1 of the owned atoms
    double *const sv = reinterpret_cast<double *>(dyn + lay.v);
    double *const sd = reinterpret_cast<double *>(dyn + lay.d);
    R *const su = reinterpret_cast<R *>(dyn + lay.uref);
    int *const snnb = reinterpret_cast<int *>(dyn + lay.nnb);
    uint32_t *const slist = reinterpret_cast<uint32_t *>(dyn + lay.list);
    const float4 *f_rows = nullptr, *phi_rows = nullptr;
    if constexpr (TABSM) {
        float4 *rows = reinterpret_cast<float4 *>(dyn + lay.tab);
        copy_rows(B.coef2, L.nint_fused, rows, rows + L.nint_fused);
        f_rows = rows;
        phi_rows = rows + L.nint_fused;
    }
    const auto tab = ClusterTab<R, TABSM>::make(B, f_rows, phi_rows);
    // The view the per-atom device functions run on: owned-atom arrays in
    // shared memory (indexed by the global atom index), buffer set 0 and
    // record buffer 0 always the current ones, so that the functions are
    // called with s = sp = 0 and index nothing dynamically.
    Bufs<R> V = B;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        V.v[0][c] = V.v[1][c] = sv + c * chunk - a0;
        V.d[c] = sd + c * chunk - a0;
        V.uref[c] = su + c * chunk - a0;
    }
    V.type[0] = V.type[1] = B.type[s];
    // the spline descriptors, and the rows of F, in shared memory
    {
        const int *src = reinterpret_cast<const int *>(B.tables);
        int *dst = reinterpret_cast<int *>(&s_tab);
        for (int w = threadIdx.x; w < (int)(sizeof(Tables<R>) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
        V.tables = &s_tab;
        if (plan.nF > 0) {
            R4 *frows = reinterpret_cast<R4 *>(dyn + lay.frows);
            const int off = B.tables->F[0].offset;
            for (int q = threadIdx.x; q < plan.nF; q += blockDim.x) frows[q] = B.coef[off + q];
            V.coef = frows - off;
        }
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&cs.bar[0])), "r"(nct) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&cs.bar[1])), "r"(nct) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // every CTA's barriers exist before any remote arrival, and the copies
    // above are complete (all CTAs of a cluster are resident together and
    // every thread passes here once)
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    unsigned nb = 0;
    auto sync = [&](bool send, float d2) {
        if (cluster_barrier(cs, nb, nct, rank, send, d2, err, L.wait_ns)) return true;
        cluster_leave(ps, nct, err, L.wait_ns);
        return false;
    };
    // owned state from device memory: v (set s), d, uref, list counts and
    // columns, and (after a build) the records of buffer sp
    auto load_owned = [&](bool records) {
        for (int o = threadIdx.x; o < m; o += blockDim.x) {
            const int i = a0 + o;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sv[c * chunk + o] = B.v[s][c][i];
                sd[c * chunk + o] = B.d[c][i];
                su[c * chunk + o] = B.uref[c][i];
            }
            snnb[o] = B.nnb[i];
            if (records) rec0[sp * chunk + o] = B.shadow[sp][i];
        }
        const int ncol = min(L.cap, st->max_nnb);
        for (int e = threadIdx.x; e < ncol * m; e += blockDim.x) {
            const int k = e / m, o = e - k * m;
            slist[k * chunk + o] = B.list[(size_t)k * L.ld + a0 + o];
        }
    };
    // v and d back to device memory (and the records of buffer sp)
    auto store_owned = [&](bool records) {
        for (int o = threadIdx.x; o < m; o += blockDim.x) {
            const int i = a0 + o;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                B.v[s][c][i] = sv[c * chunk + o];
                B.d[c][i] = sd[c * chunk + o];
            }
            if (records) B.shadow[sp][i] = rec0[sp * chunk + o];
        }
    };
    load_owned(false);
    __syncthreads();
    R h[3];
    load_h<R>(G, h);
    const R rc2 = g_rc2<R>(G);

    // opening kick and drift from the cached forces (record buffer sp ^ 1)
    {
        V.shadow[0] = rec0 + sp * chunk - a0;
        V.shadow[1] = rec0 + (sp ^ 1) * chunk - a0;
        float d2 = 0.f;
        for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) d2 = fmaxf(d2, open_atom<R>(V, L, 0, 0, i));
        if (!sync(true, d2)) return;
    }

    for (long long k = 0; k < nsteps; ++k) {
        const bool last = k == nsteps - 1;
        sp ^= 1;
        step += 1;
        since += 1;
        float md = 0.f;
        for (int r = 0; r < nct; ++r) md = fmaxf(md, cs.dmax[r]);
        need = (since >= L.rebuild_every) || ((double)md > L.disp2_thr);

        if (need) {
            store_owned(false);
            if (!sync(false, 0.f)) return;
            for (int i = gtid; i < n; i += nthreads) bin_atom<R>(B, G, s, i);
            if (!sync(false, 0.f)) return;
            if (rank == 0) scan_cells_block<R>(B, G.ncells);
            if (!sync(false, 0.f)) return;
            for (int i = gtid; i < n; i += nthreads) scatter_atom<R>(B, i);
            if (!sync(false, 0.f)) return;
            for (int c = gtid; c < G.ncells; c += nthreads) sort_cell<R>(B, s, c);
            if (!sync(false, 0.f)) return;
            for (int p = gtid; p < n; p += nthreads) permute_atom<R>(B, G, s, sp, p);
            if (gtid == 0) st->max_nnb = 0;
            s = 1 - s;
            since = 0;
            rebuilds += 1;
            V.type[0] = V.type[1] = B.type[s];
            if (!sync(false, 0.f)) return;
            if (m * kListLanesCluster <= (int)blockDim.x) {
                const int p = a0 + threadIdx.x / kListLanesCluster;
                const int cnt = (p < a1) ? list_atom_lanes<R, kListLanesCluster>(B, G, s, sp, p, L.ld, L.cap,
                                                                                 threadIdx.x % kListLanesCluster)
                                         : 0;
                block_max_nnb(cnt, &st->max_nnb);
            } else {
                for (int base = a0; base < a1; base += blockDim.x) {
                    const int p = base + threadIdx.x;
                    const int cnt = (p < a1) ? list_atom<R>(B, G, s, sp, p, L.ld, L.cap) : 0;
                    block_max_nnb(cnt, &st->max_nnb);
                }
            }
            if (!sync(false, 0.f)) return;
            // the other CTAs read these records in the density pass
            load_owned(true);
            if (!sync(false, 0.f)) return;
        }
        R4 *const cur = rec0 + sp * chunk;
        V.shadow[0] = cur - a0;
        V.shadow[1] = rec0 + (sp ^ 1) * chunk - a0;
        const ClusterFetch<R> fetch{smem_addr(cur), shift};

        // density pass
        {
            R e_embed = (R)0;
            for (int base = a0; base < a1; base += width) {
                const int i = base + threadIdx.x / TPA;
                const bool active = i < a1;
                const int ti = (MULTI && active) ? V.type[0][i] : 0;
                R rho = (R)0;
                if (active)
                    rho = density_lane<R, MULTI, TPA, UD>(V, h, rc2, 0, snnb + (i - a0), L.cap, l, cur[i - a0],
                                                          ListGlobal{slist + (i - a0), chunk}, fetch, tab);
                rho = lane_sum<TPA>(rho);
                if (active && l == 0) e_embed += embed<R>(V, V.shadow[0], i, ti, rho);
            }
            if (last) {
                const R v[1] = {e_embed};
                block_sums_t<1, R>(v, B.partials, L.pstride, 0);
            }
        }
        if (!sync(false, 0.f)) return;

        // force pass with the closing kick (and, but for the last step, the
        // next opening kick and the drift)
        {
            R e7[7] = {0, 0, 0, 0, 0, 0, 0};
            double ke = 0.0;
            float d2max = 0.f;
            for (int base = a0; base < a1; base += width) {
                const int i = base + threadIdx.x / TPA;
                const bool active = i < a1;
                const int ti = (MULTI && active) ? V.type[0][i] : 0;
                R f[3] = {0, 0, 0};
                float d2 = 0.f;
                const ListGlobal list{slist + (i - a0), chunk};
                if (last) {
                    if (active)
                        force_lane<R, MULTI, true, TPA, UF>(V, L, h, rc2, 0, snnb + (i - a0), l, ti, cur[i - a0],
                                                            list, fetch, f, e7, tab);
#pragma unroll
                    for (int c = 0; c < 3; ++c) f[c] = lane_sum<TPA>(f[c]);
                    if (active) integrate<R, MODE_CLOSE, true, TPA>(V, L, 0, 0, i, l, ti, f, ke, d2);
                } else {
                    if (active)
                        force_lane<R, MULTI, false, TPA, UF>(V, L, h, rc2, 0, snnb + (i - a0), l, ti, cur[i - a0],
                                                             list, fetch, f, e7, tab);
#pragma unroll
                    for (int c = 0; c < 3; ++c) f[c] = lane_sum<TPA>(f[c]);
                    if (active) integrate<R, MODE_CLOSE_OPEN, false, TPA>(V, L, 0, 0, i, l, ti, f, ke, d2);
                }
                d2max = fmaxf(d2max, lane_sum<TPA>(d2));
            }
            if (last) {
                const R ke_hi = (R)ke;
                const R ke_lo = (R)(ke - (double)ke_hi);
                const R v8[8] = {e7[0], ke_hi, e7[1], e7[2], e7[3], e7[4], e7[5], e7[6]};
                const R lo8[8] = {0, ke_lo, 0, 0, 0, 0, 0, 0};
                block_sums_t<8, R>(v8, B.partials, L.pstride, 1, lo8);
            }
            if (!sync(!last, d2max)) return;
        }
    }

    // owned state back to device memory; energies of the last step, counters
    // back to DevState
    store_owned(true);
    for (int slot = blockIdx.x; slot < 9; slot += gridDim.x) reduce_slot(B.partials, st, slot, gridDim.x, L.pstride);
    if (gtid == 0) {
        st->set = s;
        st->sp = sp;
        st->since_build = since;
        st->step = step;
        st->rebuilds += rebuilds;
        st->need_rebuild = need;
        st->maxdisp2 = 0u;
        ps->maxdisp[0] = 0u;
        ps->maxdisp[1] = 0u;
    }
    // the count a CTA that gave up waits for
    if (threadIdx.x == 0) atomicAdd(&ps->arrive, 1ull);
}

template <class R, bool MULTI, bool TABSM>
const void *cluster_kernel_t(int tpa)
{
    switch (tpa) {
    case 1: return (const void *)k_steps_cluster<R, MULTI, 1, TABSM>;
    case 2: return (const void *)k_steps_cluster<R, MULTI, 2, TABSM>;
    case 4: return (const void *)k_steps_cluster<R, MULTI, 4, TABSM>;
    default: return (const void *)k_steps_cluster<R, MULTI, 8, TABSM>;
    }
}

template <class R>
const void *cluster_kernel(bool multi, bool tabsm, int tpa)
{
    if (multi) return cluster_kernel_t<R, true, false>(tpa);
    if constexpr (std::is_same<R, float>::value) {
        if (tabsm) return cluster_kernel_t<float, false, true>(tpa);
    }
    return cluster_kernel_t<R, false, false>(tpa);
}

template <class R, bool MULTI>
const void *steps_kernel(int tpa)
{
    switch (tpa) {
    case 1: return (const void *)k_steps<R, MULTI, 1>;
    case 2: return (const void *)k_steps<R, MULTI, 2>;
    case 4: return (const void *)k_steps<R, MULTI, 4>;
    default: return (const void *)k_steps<R, MULTI, 8>;
    }
}

}  // namespace

template <class R>
int persistent_grid(const Launch &L, int tpa)
{
    const void *fn = L.multi ? steps_kernel<R, true>(tpa) : steps_kernel<R, false>(tpa);
    int per_sm = 0, dev = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPersistentBlock, 0) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm <= 0)
        return 0;
    const int width = kPersistentBlock / tpa;
    const int ntiles = (L.n + width - 1) / width;
    return std::max(1, std::min(ntiles, per_sm * nsm));
}

template <class R>
cudaError_t launch_steps(const Bufs<R> &B, const Geom &G, const Launch &L, long long nsteps, int tpa, int grid,
                         PersistScratch *ps)
{
    const void *fn = L.multi ? steps_kernel<R, true>(tpa) : steps_kernel<R, false>(tpa);
    Bufs<R> b = B;
    Geom g = G;
    Launch l = L;
    long long ns = nsteps;
    PersistScratch *p = ps;
    void *args[] = {&b, &g, &l, &ns, &p};
    cudaError_t e = cudaMemsetAsync(&ps->arrive, 0, sizeof(ps->arrive), L.stream);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPersistentBlock), args, 0, L.stream);
}

template <class R>
size_t cluster_smem_bytes(const Launch &L, int shift, int nF, bool tabsm)
{
    return cluster_layout<R>(1 << shift, L.cap, nF, tabsm ? L.nint_fused : 0).total;
}

namespace {
cudaLaunchConfig_t cluster_config(const Launch &L, const ClusterPlan &plan, size_t smem, cudaLaunchAttribute *attr)
{
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)plan.nct;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)plan.nct);
    cfg.blockDim = dim3(kPersistentBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = L.stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t allow_cluster(const void *fn, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}
}  // namespace

template <class R>
bool cluster_plan(const Launch &L, int tpa, bool tabsm, int nF, ClusterPlan &plan)
{
    if (L.n <= 0 || (tabsm && (!std::is_same<R, float>::value || L.multi || L.nint_fused <= 0))) return false;
    const void *fn = cluster_kernel<R>(L.multi, tabsm, tpa);
    int shift = 0;
    while ((1 << shift) < kPersistentBlock / tpa) ++shift;
    for (; shift <= kMaxClusterShift; ++shift) {
        const long long chunk = 1ll << shift;
        ClusterPlan p{shift, (int)((L.n + chunk - 1) / chunk), L.multi ? 0 : nF};
        if (p.nct > kMaxClusterCtas) continue;
        if (cluster_smem_bytes<R>(L, shift, p.nF, tabsm) > (size_t)kClusterSmemLimit) p.nF = 0;
        const size_t smem = cluster_smem_bytes<R>(L, shift, p.nF, tabsm);
        if (smem > (size_t)kClusterSmemLimit) return false;
        if (allow_cluster(fn, smem) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        cudaLaunchAttribute attr[1];
        const cudaLaunchConfig_t cfg = cluster_config(L, p, smem, attr);
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (nclusters >= 1) {
            plan = p;
            return true;
        }
    }
    return false;
}

template <class R>
cudaError_t launch_steps_cluster(const Bufs<R> &B, const Geom &G, const Launch &L, long long nsteps, int tpa,
                                 bool tabsm, const ClusterPlan &plan, PersistScratch *ps)
{
    const void *fn = cluster_kernel<R>(L.multi, tabsm, tpa);
    const size_t smem = cluster_smem_bytes<R>(L, plan.shift, plan.nF, tabsm);
    if (smem > (size_t)kClusterSmemLimit) return cudaErrorInvalidConfiguration;
    cudaError_t e = allow_cluster(fn, smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(&ps->arrive, 0, sizeof(ps->arrive), L.stream);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = cluster_config(L, plan, smem, attr);
    Bufs<R> b = B;
    Geom g = G;
    Launch l = L;
    long long ns = nsteps;
    PersistScratch *p = ps;
    ClusterPlan pl = plan;
    void *args[] = {&b, &g, &l, &ns, &p, &pl};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

template bool cluster_plan<float>(const Launch &, int, bool, int, ClusterPlan &);
template bool cluster_plan<double>(const Launch &, int, bool, int, ClusterPlan &);
template cudaError_t launch_steps_cluster<float>(const Bufs<float> &, const Geom &, const Launch &, long long, int,
                                                 bool, const ClusterPlan &, PersistScratch *);
template cudaError_t launch_steps_cluster<double>(const Bufs<double> &, const Geom &, const Launch &, long long, int,
                                                  bool, const ClusterPlan &, PersistScratch *);
template int persistent_grid<float>(const Launch &, int);
template int persistent_grid<double>(const Launch &, int);
template cudaError_t launch_steps<float>(const Bufs<float> &, const Geom &, const Launch &, long long, int, int,
                                         PersistScratch *);
template cudaError_t launch_steps<double>(const Bufs<double> &, const Geom &, const Launch &, long long, int, int,
                                          PersistScratch *);

}  // namespace eammd
