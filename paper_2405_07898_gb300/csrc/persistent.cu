// persistent.cu -- md_step as one launch: every phase of every step (opening
// kick, rebuild decision, list rebuild, density, force with the kicks and the
// drift, energy sums) runs in one cooperative-grid kernel whose blocks meet at
// grid barriers (k_steps).  For small systems, where a step is a few
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

// The list build of the single launch: a warp per atom (list_atom_warp)
// while the grid's warps cover the atoms in at most this many passes, else
// one thread per atom (list_atom).  Measured on the BCC sweep: 8 passes
// gains 5-14 % per step up to 18,522 atoms; 16 and 64 lose at 43,904 and
// 118,638 atoms.
constexpr int kListWarpPasses = 8;

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
            if ((long long)n * 32 <= (long long)nthreads * kListWarpPasses) {
                // a warp per atom, one lane per stencil cell; the grid's warps
                // take the atoms in at most kListWarpPasses passes
                const int nwarps = nthreads >> 5;
                const int w0 = gtid >> 5;
                int cmax = 0;
                for (int base = 0; base < n; base += nwarps) {
                    const int p = base + w0;
                    // the warp's lanes share p, so the whole warp takes this branch
                    if (p < n) cmax = max(cmax, list_atom_warp<R>(B, G, s, sp, p, L.ld, L.cap));
                }
                block_max_nnb(cmax, &st->max_nnb);
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

template int persistent_grid<float>(const Launch &, int);
template int persistent_grid<double>(const Launch &, int);
template cudaError_t launch_steps<float>(const Bufs<float> &, const Geom &, const Launch &, long long, int, int,
                                         PersistScratch *);
template cudaError_t launch_steps<double>(const Bufs<double> &, const Geom &, const Launch &, long long, int, int,
                                          PersistScratch *);

}  // namespace eammd
