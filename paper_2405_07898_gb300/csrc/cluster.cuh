// cluster.cuh -- the single-cluster form of the one-launch md_step
// (persistent.cu): its plan, its shared-memory layout and its launchers.
#pragma once

#include "md_internal.cuh"

namespace eammd {

constexpr int kMaxClusterCtas = 16;            // CTAs of the cluster form (a non-portable cluster size)
constexpr int kMaxClusterShift = 11;           // at most 2^11 atoms per CTA
constexpr int kClusterSmemLimit = 200 * 1024;  // dynamic shared memory of a cluster-form CTA

// CTA r owns atoms [r 2^shift, (r + 1) 2^shift); nct CTAs; nF > 0: the
// intervals of the (one-type) embedding function F, whose rows the CTAs hold
// in shared memory.
struct ClusterPlan {
    int shift, nct, nF;
};

// Byte offsets in a cluster-form CTA's dynamic shared memory for chunk owned
// atoms and cap list slots per atom: both record buffers, v[3] and d[3]
// (FP64), uref[3], the list counts, the list columns (column k of owned atom
// o at k chunk + o), the nF rows of F and, with nint_tab > 0, the f and phi
// rows of the fused FP32 table (16 B each).
struct ClusterLayout {
    size_t rec, v, d, uref, nnb, list, frows, tab, total;
};
template <class R>
__host__ __device__ inline ClusterLayout cluster_layout(int chunk, int cap, int nF, int nint_tab)
{
    const size_t m = (size_t)chunk;
    ClusterLayout o;
    size_t p = 0;
    o.rec = p;
    p += 2 * m * sizeof(typename V4<R>::T);
    o.v = p;
    p += 3 * m * sizeof(double);
    o.d = p;
    p += 3 * m * sizeof(double);
    o.uref = p;
    p += (3 * m * sizeof(R) + 31) & ~(size_t)31;
    o.nnb = p;
    p += m * sizeof(int);
    o.list = p;
    p += ((size_t)cap * m * sizeof(uint32_t) + 31) & ~(size_t)31;
    o.frows = p;
    p += (size_t)nF * sizeof(typename V4<R>::T);
    o.tab = p;
    p += (size_t)nint_tab * 32u;
    o.total = p;
    return o;
}

// md_step as one launch of a single thread-block cluster whose CTAs hold
// their atoms' state in shared memory; tabsm: the FP32 fused spline rows
// there too.  cluster_plan: the fewest atoms per CTA with which the system
// fits a resident cluster, with the nF rows of F in shared memory where they
// fit (false if no plan fits).
template <class R> bool cluster_plan(const Launch &L, int tpa, bool tabsm, int nF, ClusterPlan &plan);
template <class R>
cudaError_t launch_steps_cluster(const Bufs<R> &B, const Geom &G, const Launch &L, long long nsteps, int tpa,
                                 bool tabsm, const ClusterPlan &plan, PersistScratch *ps);

}  // namespace eammd
