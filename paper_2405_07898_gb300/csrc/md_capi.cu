// md_capi.cu -- host runtime behind the C ABI of include/eammd.h: spline
// tables, device memory, the step schedule (eager launches or CUDA graphs
// whose list rebuild sits in a device-side conditional node), and the
// marshalling of states between the caller's order and the sorted order.
#include "eammd.h"
#include "md_internal.cuh"
#include "spline_host.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

using namespace eammd;

namespace {

thread_local std::string g_create_error;

int blocks_for_host(int64_t n, int b) { return (int)((n + b - 1) / b); }

template <class R>
SplineDesc<R> make_desc(const md_spline &s, int offset, const double *row_last, const double *row0)
{
    SplineDesc<R> d;
    d.offset = offset;
    d.nint = s.n - 1;
    d.x0 = (R)s.x0;
    d.inv_h = (R)(1.0 / s.dx);
    d.h_hi = (R)s.dx;
    d.h_lo = (R)(s.dx - (double)d.h_hi);
    double x_end = s.x0 + (double)(s.n - 1) * s.dx;
    d.x_end = (R)x_end;
    d.y_lo = (R)row0[0];
    d.s_lo = (R)row0[1];
    double t = s.dx;
    d.y_end = (R)(row_last[0] + t * (row_last[1] + t * (row_last[2] + t * row_last[3])));
    d.s_end = (R)(row_last[1] + t * (2.0 * row_last[2] + 3.0 * t * row_last[3]));
    return d;
}

bool spline_ok(const md_spline &s)
{
    if (s.n < 2 || !(s.dx > 0.0) || !std::isfinite(s.dx) || !std::isfinite(s.x0) || !s.y) return false;
    for (int k = 0; k < s.n; ++k)
        if (!std::isfinite(s.y[k])) return false;
    if (s.bc_lo == 1 && !std::isfinite(s.d_lo)) return false;
    if (s.bc_hi == 1 && !std::isfinite(s.d_hi)) return false;
    return true;
}

struct GraphEntry {
    int kind;     // 0 = middle steps, 1 = closing step
    int nsteps;
    double dt;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

}  // namespace

struct md_ctx {
    int precision = MD_PRECISION_MIXED;
    int64_t n = 0;
    int ntypes = 1;
    double box[3] = {0, 0, 0};
    md_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr, body_stream = nullptr;
    Geom G{};
    Launch L{};
    double mass[kMaxTypes] = {0};
    std::vector<void *> allocs;
    Bufs<float> Bf{};
    Bufs<double> Bd{};
    DevState *st = nullptr;
    DevState *st_host = nullptr;  // pinned
    double *stage = nullptr;      // 9 n doubles: AoS pos, vel, force
    int *types_orig = nullptr;
    std::vector<GraphEntry> graphs;
    long long fixed_launches = 0;
    long long rebuilds_at_create = 0;
    int64_t host_steps = 0;       // step counter when n == 0
    std::vector<md_spline> shapes; // grids of F[t], f[t], phi[q] (values not kept)
    double r_cut = 0.0, skin = 0.0;
    int off_F0 = 0, off_f0 = 0, off_phi0 = 0;  // coefficient rows of the type-0 tables
    // force-matching adjoint workspace (FP64 path), allocated on first use
    double *adj_g = nullptr, *adj_rho = nullptr, *adj_drho = nullptr, *adj_bins = nullptr, *adj_pg = nullptr;
    double *adj_cg = nullptr, *adj_sq = nullptr, *adj_Mt = nullptr, *adj_kg = nullptr;
    int *adj_knot_func = nullptr, *adj_func_coef0 = nullptr, *adj_func_ncoef = nullptr;
    long long *adj_knot_mt0 = nullptr;
    int adj_nrows = 0, adj_nknots = 0;
    // persistent step launch (md_step as one cooperative kernel)
    PersistScratch *ps = nullptr;
    int persist_tpa = 0, persist_grid = 0;  // 0: graph path
    std::string err;

    md_status fail(md_status s, const std::string &m)
    {
        err = m;
        return s;
    }
};

namespace {

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            return ctx->fail(e_ == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA,           \
                             std::string(#call) + ": " + cudaGetErrorString(e_));                  \
        }                                                                                          \
    } while (0)

void *dalloc(md_ctx *ctx, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (ctx->opt.alloc) {
        p = ctx->opt.alloc(bytes, ctx->opt.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) ctx->allocs.push_back(p);
    return p;
}

void dfree_all(md_ctx *ctx)
{
    for (void *p : ctx->allocs) {
        if (ctx->opt.free) ctx->opt.free(p, ctx->opt.alloc_ctx);
        else cudaFree(p);
    }
    ctx->allocs.clear();
}

template <class T>
bool alloc_n(md_ctx *ctx, T *&p, size_t count)
{
    p = (T *)dalloc(ctx, count * sizeof(T));
    return p != nullptr;
}

template <class R>
Bufs<R> &bufs(md_ctx *ctx);
template <>
Bufs<float> &bufs<float>(md_ctx *ctx) { return ctx->Bf; }
template <>
Bufs<double> &bufs<double>(md_ctx *ctx) { return ctx->Bd; }

// Texture objects over the two FP32 record buffers, for the density pass's
// gathers.  Where the buffers do not meet the texture rules (alignment, the
// largest linear texture), none is made and the density pass gathers through
// the load path; both paths read the same words.
void make_record_textures(Bufs<float> &B, size_t n)
{
    int dev = 0, align = 0, maxw = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&align, cudaDevAttrTextureAlignment, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture1DLinearWidth, dev) != cudaSuccess)
        return;
    if (n > (size_t)maxw) return;
    unsigned long long t[2] = {0, 0};
    for (int s = 0; s < 2; ++s) {
        if (align <= 0 || (reinterpret_cast<uintptr_t>(B.shadow[s]) % (uintptr_t)align) != 0) break;
        cudaResourceDesc rd{};
        rd.resType = cudaResourceTypeLinear;
        rd.res.linear.devPtr = B.shadow[s];
        rd.res.linear.desc = cudaCreateChannelDesc<float4>();
        rd.res.linear.sizeInBytes = n * sizeof(float4);
        cudaTextureDesc td{};
        td.readMode = cudaReadModeElementType;
        td.filterMode = cudaFilterModePoint;
        td.normalizedCoords = 0;
        cudaTextureObject_t obj = 0;
        if (cudaCreateTextureObject(&obj, &rd, &td, nullptr) != cudaSuccess) break;
        t[s] = (unsigned long long)obj;
    }
    if (t[0] && t[1]) {
        B.tex_shadow[0] = t[0];
        B.tex_shadow[1] = t[1];
        return;
    }
    for (int s = 0; s < 2; ++s)
        if (t[s]) cudaDestroyTextureObject((cudaTextureObject_t)t[s]);
    (void)cudaGetLastError();  // a refused texture is not an error of this context
}

template <class R>
bool alloc_buffers(md_ctx *ctx, const std::vector<double> &rows, const std::vector<double> &rows2,
                   const Tables<R> &tables)
{
    using R4 = typename V4<R>::T;
    Bufs<R> &B = bufs<R>(ctx);
    const size_t n = (size_t)std::max<int64_t>(ctx->n, 1);
    const Geom &G = ctx->G;
    bool ok = true;
    for (int s = 0; s < 2; ++s)
        for (int a = 0; a < 3; ++a) {
            ok = ok && alloc_n(ctx, B.xr[s][a], n);
            ok = ok && alloc_n(ctx, B.v[s][a], n);
        }
    for (int a = 0; a < 3; ++a) {
        ok = ok && alloc_n(ctx, B.d[a], n);
        ok = ok && alloc_n(ctx, B.xw[a], n);
        ok = ok && alloc_n(ctx, B.uref[a], n);
        ok = ok && alloc_n(ctx, B.fcache[a], n);
        ok = ok && alloc_n(ctx, B.center[a], (size_t)G.ncell[a]);
    }
    for (int s = 0; s < 2; ++s) {
        ok = ok && alloc_n(ctx, B.id[s], n);
        ok = ok && alloc_n(ctx, B.type[s], n);
        ok = ok && alloc_n(ctx, B.shadow[s], n);
    }
    ok = ok && alloc_n(ctx, B.cell, n);
    ok = ok && alloc_n(ctx, B.cell_old, n);
    ok = ok && alloc_n(ctx, B.slot, n);
    ok = ok && alloc_n(ctx, B.cell_atoms, n);
    ok = ok && alloc_n(ctx, B.nnb, n);
    ok = ok && alloc_n(ctx, B.count, (size_t)G.ncells + 1);
    ok = ok && alloc_n(ctx, B.cell_start, (size_t)G.ncells + 1);
    ok = ok && alloc_n(ctx, B.block_sums, (size_t)(G.ncells + kScanBlock - 1) / kScanBlock + 1);
    ok = ok && alloc_n(ctx, B.partials, (size_t)kEnergySlots * std::max(ctx->L.pstride, 1));
    ok = ok && alloc_n(ctx, B.list, (size_t)ctx->L.cap * ctx->L.ld);
    if (ctx->opt.half_list) {
        ok = ok && alloc_n(ctx, B.acc_rho, n);
        ok = ok && alloc_n(ctx, B.acc_f, 3 * n);
        ok = ok && alloc_n(ctx, B.own, n);
    }
    R4 *coef = nullptr, *coef2 = nullptr;
    Tables<R> *tab = nullptr;
    ok = ok && alloc_n(ctx, coef, rows.size() / 4);
    ok = ok && alloc_n(ctx, coef2, std::max<size_t>(rows2.size() / 4, 2));
    ok = ok && alloc_n(ctx, tab, 1);
    if (!ok) return false;
    B.coef = coef;
    B.coef2 = coef2;
    B.coef_f = tables.fused ? coef2 + 2 * (size_t)tables.fphi.nint : coef2;
    B.tables = tab;
    B.st = ctx->st;
    auto upload = [](R4 *dst_dev, const std::vector<double> &src) -> bool {
        std::vector<R4> rr(src.size() / 4);
        for (size_t k = 0; k < rr.size(); ++k) {
            R *dst = reinterpret_cast<R *>(&rr[k]);
            for (int c = 0; c < 4; ++c) dst[c] = (R)src[4 * k + c];
        }
        return rr.empty() || cudaMemcpy(dst_dev, rr.data(), rr.size() * sizeof(R4), cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (!upload(coef, rows) || !upload(coef2, rows2)) return false;
    if (cudaMemcpy(tab, &tables, sizeof(Tables<R>), cudaMemcpyHostToDevice) != cudaSuccess) return false;
    for (int a = 0; a < 3; ++a) {
        std::vector<double> c(G.ncell[a]);
        for (int k = 0; k < G.ncell[a]; ++k) c[k] = ((double)k + 0.5) * G.h[a];
        if (cudaMemcpy(B.center[a], c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return false;
    }
    B.tex_shadow[0] = B.tex_shadow[1] = 0;
    if constexpr (std::is_same<R, float>::value) make_record_textures(B, n);
    if (cudaMemset(B.count, 0, sizeof(int) * ((size_t)G.ncells + 1)) != cudaSuccess) return false;
    if (cudaMemset(B.nnb, 0, sizeof(int) * n) != cudaSuccess) return false;
    if (ctx->opt.half_list && (cudaMemset(B.acc_rho, 0, sizeof(unsigned long long) * n) != cudaSuccess ||
                               cudaMemset(B.acc_f, 0, sizeof(unsigned long long) * 3 * n) != cudaSuccess))
        return false;
    for (int a = 0; a < 3; ++a)
        if (cudaMemset(B.fcache[a], 0, sizeof(R) * n) != cudaSuccess) return false;
    return true;
}

void drop_graphs(md_ctx *ctx)
{
    for (auto &g : ctx->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    ctx->graphs.clear();
}

template <class R>
bool grow_list(md_ctx *ctx, int cap)
{
    Bufs<R> &B = bufs<R>(ctx);
    drop_graphs(ctx);  // captured kernels hold the old list pointer
    uint32_t *nl = nullptr;
    if (!alloc_n(ctx, nl, (size_t)cap * ctx->L.ld)) return false;
    // the old block stays owned by the context until md_destroy
    B.list = nl;
    ctx->L.cap = cap;
    return true;
}

md_status read_state(md_ctx *ctx)
{
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(ctx->st_host, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost));
    return MD_OK;
}

// The error flags of the device state last read into st_host.
md_status state_errors(md_ctx *ctx)
{
    unsigned int e = ctx->st_host->error;
    if (e & ERR_LIST_OVERFLOW)
        return ctx->fail(MD_ERR_LIST_OVERFLOW, "an atom had more neighbours (" +
                                                   std::to_string(ctx->st_host->max_nnb) +
                                                   ") than the list capacity (" + std::to_string(ctx->L.cap) + ")");
    if (e & ERR_NONFINITE) return ctx->fail(MD_ERR_NONFINITE, "non-finite position or force");
    if (e & ERR_TIMEOUT) return ctx->fail(MD_ERR_TIMEOUT, "a bounded device wait gave up");
    return MD_OK;
}

md_status check_device_errors(md_ctx *ctx)
{
    md_status rc = read_state(ctx);
    if (rc != MD_OK) return rc;
    return state_errors(ctx);
}

// Rebuild + density + force (no integration) + reduction at the current
// positions: the state after md_create / md_set_state.
template <class R>
md_status measure(md_ctx *ctx)
{
    const Bufs<R> &B = bufs<R>(ctx);
    Launch L = ctx->L;
    L.use_cond = 0;
    L.cond = 0;
    ctx->fixed_launches += launch_rebuild<R>(B, ctx->G, L);
    ctx->fixed_launches += launch_density<R>(B, ctx->G, L, true);
    ctx->fixed_launches += launch_force<R>(B, ctx->G, L, MODE_MEASURE, true);
    ctx->fixed_launches += launch_reduce<R>(B, L);
    CK(cudaGetLastError());
    return MD_OK;
}

// Upload a state in the caller's order and evaluate it.  When the list
// overflows and the capacity was not fixed by the caller, grow and retry.
template <class R>
md_status load_and_measure(md_ctx *ctx, const double *pos, const double *vel, int64_t step)
{
    const Bufs<R> &B0 = bufs<R>(ctx);
    const size_t n = (size_t)ctx->n;
    // the permutation restarts from the caller's order in buffer set 0
    DevState h{};
    h.step = step;
    h.need_rebuild = 1;
    h.set = 0;
    h.sp = 0;
    CK(cudaMemcpyAsync(ctx->st, &h, sizeof(DevState), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->stage, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (vel) CK(cudaMemcpyAsync(ctx->stage + 3 * n, vel, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    Launch L = ctx->L;
    ctx->fixed_launches += launch_load_state<R>(B0, L, ctx->stage, vel ? ctx->stage + 3 * n : nullptr, ctx->types_orig);
    CK(cudaGetLastError());
    for (int attempt = 0; attempt < 4; ++attempt) {
        md_status rc = measure<R>(ctx);
        if (rc != MD_OK) return rc;
        rc = read_state(ctx);
        if (rc != MD_OK) return rc;
        const DevState &hs = *ctx->st_host;
        // automatic capacity: at least the longest list of this build with
        // room to grow (a density estimate from the box undercounts slabs
        // with vacuum)
        const int want = ((hs.max_nnb + hs.max_nnb / 4 + 8) + 3) & ~3;
        if (((hs.error & ERR_LIST_OVERFLOW) || want > ctx->L.cap) && ctx->opt.list_capacity <= 0) {
            int cap = std::max(want, ((hs.max_nnb + hs.max_nnb / 8 + 8) + 3) & ~3);
            if (!grow_list<R>(ctx, cap)) return ctx->fail(MD_ERR_OOM, "cannot grow the neighbour list");
            // the state is already sorted; rebuild from it with the larger capacity
            DevState again = hs;
            again.error &= ~ERR_LIST_OVERFLOW;
            again.need_rebuild = 1;
            again.rebuilds = 0;
            CK(cudaMemcpy(ctx->st, &again, sizeof(DevState), cudaMemcpyHostToDevice));
            continue;
        }
        break;
    }
    // the state read last in the loop is the current one
    md_status rc = state_errors(ctx);
    if (rc != MD_OK) return rc;
    // rebuilds are counted from here on
    DevState hs = *ctx->st_host;
    ctx->rebuilds_at_create = hs.rebuilds;
    return MD_OK;
}

template <class R>
void enqueue_step(md_ctx *ctx, const Launch &L, bool last)
{
    const Bufs<R> &B = bufs<R>(ctx);
    launch_decide<R>(B, L);
    if (L.use_cond) {
        // the rebuild kernels are captured into the conditional node body by the caller
    } else {
        launch_rebuild<R>(B, ctx->G, L);
    }
    launch_density<R>(B, ctx->G, L, last);
    launch_force<R>(B, ctx->G, L, last ? MODE_CLOSE : MODE_CLOSE_OPEN, last);
}

// Capture nsteps steps (the last one closing with energies when kind == 1)
// into a graph.  Each step is [decide -> IF(rebuild) -> density -> force];
// decide sets the IF node's condition on the device.
template <class R>
md_status build_graph(md_ctx *ctx, int kind, int nsteps, double dt, GraphEntry &out)
{
    const Bufs<R> &B = bufs<R>(ctx);
    cudaStream_t cs = ctx->cap_stream;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int s = 0; s < nsteps; ++s) {
        bool last = (kind == 1) && (s == nsteps - 1);
        cudaStreamCaptureStatus status;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, &deps, nullptr, &ndeps));
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
        Launch L = ctx->L;
        L.stream = cs;
        L.cond = h;
        L.use_cond = 1;
        launch_decide<R>(B, L);
        CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, &deps, nullptr, &ndeps));
        alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
        memset(raw, 0, sizeof(raw));
        cudaGraphNodeParams &p = *reinterpret_cast<cudaGraphNodeParams *>(raw);
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeIf;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &p));
        CK(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        cudaGraph_t body = p.conditional.phGraph_out[0];
        CK(cudaStreamBeginCaptureToGraph(ctx->body_stream, body, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal));
        Launch Lb = L;
        Lb.stream = ctx->body_stream;
        launch_rebuild<R>(B, ctx->G, Lb);
        CK(cudaStreamEndCapture(ctx->body_stream, &body));
        launch_density<R>(B, ctx->G, L, last);
        launch_force<R>(B, ctx->G, L, last ? MODE_CLOSE : MODE_CLOSE_OPEN, last);
        if (last) launch_reduce<R>(B, L);
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamEndCapture(cs, &graph));
    cudaGraphExec_t exec = nullptr;
    CK(cudaGraphInstantiate(&exec, graph, 0));
    out.kind = kind;
    out.nsteps = nsteps;
    out.dt = dt;
    out.graph = graph;
    out.exec = exec;
    return MD_OK;
}

template <class R>
md_status get_graph(md_ctx *ctx, int kind, int nsteps, double dt, cudaGraphExec_t &exec)
{
    for (auto &g : ctx->graphs)
        if (g.kind == kind && g.nsteps == nsteps && g.dt == dt) {
            exec = g.exec;
            return MD_OK;
        }
    GraphEntry e{};
    md_status rc = build_graph<R>(ctx, kind, nsteps, dt, e);
    if (rc != MD_OK) return rc;
    ctx->graphs.push_back(e);
    exec = e.exec;
    return MD_OK;
}

template <class R> md_status setup_persistent(md_ctx *ctx);

template <class R>
md_status step_impl(md_ctx *ctx, int64_t nsteps, double dt)
{
    const Bufs<R> &B = bufs<R>(ctx);
    ctx->L.dt = dt;
    for (int t = 0; t < ctx->ntypes; ++t) ctx->L.half_kick[t] = 0.5 * dt * kAccel / ctx->mass[t];
    Launch L = ctx->L;
    L.use_cond = 0;
    L.cond = 0;
    if (ctx->persist_grid > 0) {
        CK(launch_steps<R>(B, ctx->G, L, nsteps, ctx->persist_tpa, ctx->persist_grid, ctx->ps));
        ctx->fixed_launches += 1;
        return MD_OK;
    }
    ctx->fixed_launches += launch_open<R>(B, ctx->G, L);
    if (!ctx->opt.use_graphs) {
        for (int64_t s = 0; s < nsteps; ++s) {
            enqueue_step<R>(ctx, L, s == nsteps - 1);
            ctx->fixed_launches += 3 + 8;
        }
        ctx->fixed_launches += launch_reduce<R>(B, L);
        CK(cudaGetLastError());
        return MD_OK;
    }
    const int chunk = 10;
    int64_t mid = nsteps - 1;
    cudaGraphExec_t ex;
    if (mid >= chunk) {
        md_status rc = get_graph<R>(ctx, 0, chunk, dt, ex);
        if (rc != MD_OK) return rc;
        for (int64_t k = 0; k < mid / chunk; ++k) CK(cudaGraphLaunch(ex, ctx->stream));
    }
    if (mid % chunk) {
        md_status rc = get_graph<R>(ctx, 0, (int)(mid % chunk), dt, ex);
        if (rc != MD_OK) return rc;
        CK(cudaGraphLaunch(ex, ctx->stream));
    }
    md_status rc = get_graph<R>(ctx, 1, 1, dt, ex);
    if (rc != MD_OK) return rc;
    CK(cudaGraphLaunch(ex, ctx->stream));
    ctx->fixed_launches += 3 * nsteps + 1;
    return MD_OK;
}

// Eager steps with events around each kernel group (see md_profile).
template <class R>
md_status profile_impl(md_ctx *ctx, int64_t nsteps, double dt, md_profile_t *out)
{
    const Bufs<R> &B = bufs<R>(ctx);
    ctx->L.dt = dt;
    for (int t = 0; t < ctx->ntypes; ++t) ctx->L.half_kick[t] = 0.5 * dt * kAccel / ctx->mass[t];
    Launch L = ctx->L;
    L.use_cond = 0;
    L.cond = 0;
    md_status rc0 = read_state(ctx);
    if (rc0 != MD_OK) return rc0;
    const long long rebuilds0 = ctx->st_host->rebuilds;
    const int64_t ne = 4 * nsteps + 2;
    std::vector<cudaEvent_t> ev(ne);
    for (auto &e : ev) CK(cudaEventCreate(&e));
    int64_t k = 0;
    CK(cudaEventRecord(ev[k++], ctx->stream));
    ctx->fixed_launches += launch_open<R>(B, ctx->G, L);
    for (int64_t s = 0; s < nsteps; ++s) {
        bool last = s == nsteps - 1;
        ctx->fixed_launches += launch_decide<R>(B, L);
        CK(cudaEventRecord(ev[k++], ctx->stream));
        ctx->fixed_launches += launch_rebuild<R>(B, ctx->G, L);
        CK(cudaEventRecord(ev[k++], ctx->stream));
        ctx->fixed_launches += launch_density<R>(B, ctx->G, L, last);
        CK(cudaEventRecord(ev[k++], ctx->stream));
        ctx->fixed_launches += launch_force<R>(B, ctx->G, L, last ? MODE_CLOSE : MODE_CLOSE_OPEN, last);
        CK(cudaEventRecord(ev[k++], ctx->stream));
    }
    ctx->fixed_launches += launch_reduce<R>(B, L);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    double dens = 0, force = 0, reb = 0, total = 0;
    int64_t nreb = 0;
    std::vector<float> span(nsteps);
    for (int64_t s = 0; s < nsteps; ++s) {
        float a = 0, b = 0, c = 0;
        CK(cudaEventElapsedTime(&a, ev[1 + 4 * s], ev[2 + 4 * s]));
        CK(cudaEventElapsedTime(&b, ev[2 + 4 * s], ev[3 + 4 * s]));
        CK(cudaEventElapsedTime(&c, ev[3 + 4 * s], ev[4 + 4 * s]));
        span[s] = a;
        dens += b;
        force += c;
    }
    // the 8 guarded rebuild kernels exit at once when no build is due: the
    // device counted the builds, and they are the longest spans
    md_status rc = read_state(ctx);
    if (rc != MD_OK) return rc;
    nreb = std::min<int64_t>(std::max<int64_t>(ctx->st_host->rebuilds - rebuilds0, 0), nsteps);
    std::sort(span.begin(), span.end(), [](float x, float y) { return x > y; });
    for (int64_t s = 0; s < nreb; ++s) reb += span[s];
    float tot = 0;
    CK(cudaEventElapsedTime(&tot, ev[0], ev[4 * nsteps]));
    total = tot;
    for (auto &e : ev) cudaEventDestroy(e);
    memset(out, 0, sizeof(*out));
    out->density_ms = dens / (double)nsteps;
    out->force_ms = force / (double)nsteps;
    out->rebuild_ms = nreb ? reb / (double)nreb : 0.0;
    out->step_ms = total / (double)nsteps;
    out->density_launches = nsteps;
    out->force_launches = nsteps;
    out->rebuilds = nreb;
    return MD_OK;
}

template <class R>
md_status store_state(md_ctx *ctx, double *pos, double *vel, double *force)
{
    const size_t n = (size_t)ctx->n;
    if (n == 0) return MD_OK;
    Launch L = ctx->L;
    double *dp = pos ? ctx->stage : nullptr;
    double *dv = vel ? ctx->stage + 3 * n : nullptr;
    double *df = force ? ctx->stage + 6 * n : nullptr;
    ctx->fixed_launches += launch_store_state<R>(bufs<R>(ctx), L, dp, dv, df);
    CK(cudaGetLastError());
    if (pos) CK(cudaMemcpyAsync(pos, dp, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (vel) CK(cudaMemcpyAsync(vel, dv, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (force) CK(cudaMemcpyAsync(force, df, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MD_OK;
}

// Coefficient rows of all splines (F[t], f[t], phi[q] in that order), the
// fused f | phi rows of the single-type fast path, and their descriptors.
template <class R>
md_status build_tables(md_ctx *ctx, const md_potential *pot, std::vector<double> &rows, std::vector<double> &rows2,
                       Tables<R> &tab)
{
    rows.clear();
    rows2.clear();
    memset(&tab, 0, sizeof(tab));
    tab.ntypes = pot->ntypes;
    auto add = [&](const md_spline &s, SplineDesc<R> &d) -> bool {
        int off = (int)(rows.size() / 4);
        if (!hermite_coefficients(s, rows)) return false;
        d = make_desc<R>(s, off, &rows[rows.size() - 4], &rows[4 * (size_t)off]);
        return true;
    };
    int npair = pot->ntypes * (pot->ntypes + 1) / 2;
    for (int t = 0; t < pot->ntypes; ++t) {
        if (!add(pot->F[t], tab.F[t]) || !add(pot->f[t], tab.f[t]))
            return ctx->fail(MD_ERR_ARG, "spline system is singular");
    }
    for (int q = 0; q < npair; ++q)
        if (!add(pot->phi[q], tab.phi[q])) return ctx->fail(MD_ERR_ARG, "spline system is singular");
    // one type whose f and phi share a knot grid: interleave their rows so a
    // pair's f' and phi' come from one 32-byte (FP32) row
    const md_spline &f0 = pot->f[0], &p0 = pot->phi[0];
    if (pot->ntypes == 1 && f0.n == p0.n && f0.x0 == p0.x0 && f0.dx == p0.dx) {
        tab.fused = 1;
        tab.fphi = tab.f[0];
        tab.fphi.offset = 0;
        for (int k = 0; k < f0.n - 1; ++k) {
            for (int c = 0; c < 4; ++c) rows2.push_back(rows[4 * ((size_t)tab.f[0].offset + k) + c]);
            for (int c = 0; c < 4; ++c) rows2.push_back(rows[4 * ((size_t)tab.phi[0].offset + k) + c]);
        }
        // then the f rows alone, for the density pass: twice as many
        // intervals per cache line as in the interleaved rows
        for (int k = 0; k < f0.n - 1; ++k)
            for (int c = 0; c < 4; ++c) rows2.push_back(rows[4 * ((size_t)tab.f[0].offset + k) + c]);
    }
    return MD_OK;
}

// Schedule of one pass: lanes per atom and threads per block.
struct PassSched {
    int tpa, block;  // block 0: the context's block_size
};

void set_sched(md_ctx *ctx, PassSched d, PassSched f)
{
    Launch &L = ctx->L;
    L.tpa_d = d.tpa;
    L.tpa_f = f.tpa;
    L.block_d = d.block > 0 ? d.block : L.block;
    L.block_f = f.block > 0 ? f.block : L.block;
    L.nb_d = blocks_for_host((int64_t)L.n * d.tpa, L.block_d);
    L.nb_f = blocks_for_host((int64_t)L.n * f.tpa, L.block_f);
}

// Choices of the autotuner, per (precision, type path, size bucket), kept for
// the life of the process so that every context of the same shape runs the
// same schedule (and gives bitwise identical results).
struct TuneKey {
    int precision, multi, bucket;
};
struct TuneChoice {
    PassSched d, f;
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, TuneChoice>> g_tune_cache;

// Density and force (forces only, no integration) at the current state.
template <class R>
md_status reevaluate(md_ctx *ctx)
{
    const Bufs<R> &B = bufs<R>(ctx);
    Launch L = ctx->L;
    L.use_cond = 0;
    ctx->fixed_launches += launch_density<R>(B, ctx->G, L, true);
    ctx->fixed_launches += launch_force<R>(B, ctx->G, L, MODE_MEASURE, true);
    ctx->fixed_launches += launch_reduce<R>(B, L);
    CK(cudaGetLastError());
    return MD_OK;
}

// Schedule of the density and force passes: time, on the current state
// (density, and the force pass with its kicks and drift at dt = 0; neither
// changes positions or velocities), the atom-parallel passes with 1, 2, 4, 8
// lanes per atom and several block sizes; keep the fastest of each pass.
template <class R>
md_status autotune(md_ctx *ctx)
{
    int bucket = 0;
    for (int64_t m = ctx->n; m > 1; m >>= 1) ++bucket;
    TuneKey key{ctx->precision, ctx->L.multi, bucket};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (auto &e : g_tune_cache)
            if (e.first.precision == key.precision && e.first.multi == key.multi && e.first.bucket == key.bucket) {
                set_sched(ctx, e.second.d, e.second.f);
                return reevaluate<R>(ctx);
            }
    }
    const Bufs<R> &B = bufs<R>(ctx);
    // block sizes below 256 let the atom-parallel passes fill their last
    // wave of blocks on the GPU
    std::vector<PassSched> cand;
    for (int t : {1, 2})
        for (int b : {256, 224, 192, 160, 128, 96, 64}) cand.push_back({t, b});
    cand.push_back({4, 256});
    cand.push_back({8, 256});
    const int nc = (int)cand.size();
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // rounds over the candidates in turn (so clock and cache drift hit all
    // alike); each candidate keeps its fastest single launch
    std::vector<float> best_d(nc, 1e30f), best_f(nc, 1e30f);
    const int rounds = 6;
    // the force pass is timed as md_step runs it (kicks and drift fused), at
    // dt = 0: positions and velocities keep their values; the device state
    // words it touches are restored afterwards
    DevState saved;
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(&saved, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost));
    for (int round = 0; round < rounds; ++round) {
        for (int ci = 0; ci < nc; ++ci) {
            set_sched(ctx, cand[ci], cand[ci]);
            Launch L = ctx->L;
            L.use_cond = 0;
            L.dt = 0.0;
            for (int t = 0; t < ctx->ntypes; ++t) L.half_kick[t] = 0.0;
            float ms = 0;
            CK(cudaEventRecord(e0, ctx->stream));
            launch_density<R>(B, ctx->G, L, false);
            CK(cudaEventRecord(e1, ctx->stream));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (round > 0) best_d[ci] = std::min(best_d[ci], ms);
            CK(cudaEventRecord(e0, ctx->stream));
            launch_force<R>(B, ctx->G, L, MODE_CLOSE_OPEN, false);
            CK(cudaEventRecord(e1, ctx->stream));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (round > 0) best_f[ci] = std::min(best_f[ci], ms);
            ctx->fixed_launches += 2;
        }
    }
    CK(cudaMemcpy(ctx->st, &saved, sizeof(DevState), cudaMemcpyHostToDevice));
    // candidates in order of preference: a later one must win by 3%
    int cd = 0, cf = 0;
    for (int ci = 1; ci < nc; ++ci) {
        if (best_d[ci] < 0.97f * best_d[cd]) cd = ci;
        if (best_f[ci] < 0.97f * best_f[cf]) cf = ci;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const TuneChoice choice{cand[cd], cand[cf]};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache.push_back({key, choice});
    }
    set_sched(ctx, choice.d, choice.f);
    // forces and energies of the state under the chosen schedule
    md_status rc = reevaluate<R>(ctx);
    if (rc != MD_OK) return rc;
    return check_device_errors(ctx);
}

// Threshold of MD_PERSIST_AUTO: at and below this many atoms a step is a few
// microseconds of work and one cooperative launch per md_step call beats the
// graph replay (measured on GB300 over the BCC sweep).
constexpr int64_t kPersistentAutoAtoms = 65536;

// The persistent step launch: a cooperative grid of as many blocks as are
// resident.  Lanes per atom come from the options, else every feasible
// choice is timed over rebuild_every - 1 steps at dt = 0, which moves no atom
// and builds no list; the device state is restored after each trial.
template <class R>
md_status setup_persistent(md_ctx *ctx)
{
    ctx->persist_grid = 0;
    const md_options &o = ctx->opt;
    const bool want = o.persistent == MD_PERSIST_ON || (o.persistent == MD_PERSIST_AUTO && ctx->n <= kPersistentAutoAtoms);
    if (!want || ctx->n == 0) return MD_OK;
    const bool forced = o.persistent != MD_PERSIST_AUTO;
    if (!ctx->ps) {
        if (!alloc_n(ctx, ctx->ps, 1)) return ctx->fail(MD_ERR_OOM, "device allocation failed");
        CK(cudaMemsetAsync(ctx->ps, 0, sizeof(PersistScratch), ctx->stream));
    }
    int dev = 0, coop = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    const Bufs<R> &B = bufs<R>(ctx);
    std::vector<int> tpas;
    if (o.lanes_per_atom > 0) tpas.push_back(o.lanes_per_atom);
    else if (ctx->L.rebuild_every < 2) tpas.push_back(2);  // every step builds: no state-neutral trial
    else tpas = {1, 2, 4, 8};
    struct Cand {
        int tpa, grid;
    };
    std::vector<Cand> cand;
    for (int tpa : tpas) {
        if (!coop) break;
        const int grid = persistent_grid<R>(ctx->L, tpa);
        if (grid > 0) cand.push_back({tpa, grid});
    }
    if (cand.empty()) {
        if (forced) return ctx->fail(MD_ERR_CUDA, "the persistent step kernel cannot be resident");
        return MD_OK;
    }
    auto take = [&](const Cand &c) {
        ctx->persist_tpa = c.tpa;
        ctx->persist_grid = c.grid;
    };
    if (cand.size() == 1 || ctx->L.rebuild_every < 2) {
        take(cand[0]);
        return MD_OK;
    }
    const int trial_steps = ctx->L.rebuild_every - 1;
    DevState saved;
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(&saved, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost));
    Launch L = ctx->L;
    L.dt = 0.0;
    for (int t = 0; t < ctx->ntypes; ++t) L.half_kick[t] = 0.0;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_i = -1;
    for (int round = 0; round < 3; ++round) {
        for (size_t c = 0; c < cand.size(); ++c) {
            const Cand &k = cand[c];
            CK(cudaEventRecord(e0, ctx->stream));
            CK(launch_steps<R>(B, ctx->G, L, trial_steps, k.tpa, k.grid, ctx->ps));
            CK(cudaEventRecord(e1, ctx->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            CK(cudaMemcpy(ctx->st, &saved, sizeof(DevState), cudaMemcpyHostToDevice));
            ctx->fixed_launches += 1;
            // a later candidate must win by 3%
            if (ms < 0.97f * best) {
                best = ms;
                best_i = (int)c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (saved.error) return check_device_errors(ctx);
    take(cand[best_i]);
    return check_device_errors(ctx);
}

// Replace the spline values of a context (same grids, same r_cut and skin)
// and re-evaluate forces and energies at the current positions.
template <class R>
md_status set_potential_impl(md_ctx *ctx, const md_potential *pot)
{
    using R4 = typename V4<R>::T;
    std::vector<double> rows, rows2;
    Tables<R> tab;
    md_status rc = build_tables<R>(ctx, pot, rows, rows2, tab);
    if (rc != MD_OK) return rc;
    Bufs<R> &B = bufs<R>(ctx);
    auto upload = [&](const R4 *dst_dev, const std::vector<double> &src) -> cudaError_t {
        std::vector<R4> rr(src.size() / 4);
        for (size_t k = 0; k < rr.size(); ++k) {
            R *dst = reinterpret_cast<R *>(&rr[k]);
            for (int c = 0; c < 4; ++c) dst[c] = (R)src[4 * k + c];
        }
        if (rr.empty()) return cudaSuccess;
        return cudaMemcpyAsync((void *)dst_dev, rr.data(), rr.size() * sizeof(R4), cudaMemcpyHostToDevice,
                               ctx->stream);
    };
    CK(upload(B.coef, rows));
    CK(upload(B.coef2, rows2));
    CK(cudaMemcpyAsync((void *)B.tables, &tab, sizeof(Tables<R>), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // the host staging vectors go out of scope
    if (ctx->n == 0) return MD_OK;
    rc = reevaluate<R>(ctx);
    if (rc != MD_OK) return rc;
    return check_device_errors(ctx);
}

// Adjoint workspace and the transposed spline basis maps of phi, f, F.
md_status adjoint_setup(md_ctx *ctx)
{
    if (ctx->adj_g) return MD_OK;
    const size_t n = (size_t)ctx->n;
    const md_spline *fs[3] = {&ctx->shapes[2], &ctx->shapes[1], &ctx->shapes[0]};  // phi, f, F
    int nrows = 0, nknots = 0;
    for (auto *sp : fs) {
        nrows += sp->n - 1;
        nknots += sp->n;
    }
    if (adjoint_smem_bytes(nrows) > 200 * 1024) return ctx->fail(MD_ERR_CAPACITY, "too many spline intervals for the adjoint bins");
    CK(allow_adjoint_smem(adjoint_smem_bytes(nrows)));
    std::vector<double> Mt;
    std::vector<int> knot_func, coef0(3), ncoef(3);
    std::vector<long long> mt0;
    int coef_base = 0;
    for (int fn = 0; fn < 3; ++fn) {
        const md_spline &sp = *fs[fn];
        coef0[fn] = coef_base;
        ncoef[fn] = 4 * (sp.n - 1);
        coef_base += ncoef[fn];
        std::vector<double> y(sp.n, 0.0);
        for (int q = 0; q < sp.n; ++q) {
            std::fill(y.begin(), y.end(), 0.0);
            y[q] = 1.0;
            md_spline unit = sp;
            unit.y = y.data();
            unit.d_lo = 0.0;
            unit.d_hi = 0.0;
            std::vector<double> rows;
            if (!hermite_coefficients(unit, rows)) return ctx->fail(MD_ERR_ARG, "spline basis failed");
            knot_func.push_back(fn);
            mt0.push_back((long long)Mt.size());
            Mt.insert(Mt.end(), rows.begin(), rows.end());
        }
    }
    const int nw = (int)((n + 31) / 32), nb = (int)((n + 255) / 256);
    bool ok = alloc_n(ctx, ctx->adj_g, 3 * n) && alloc_n(ctx, ctx->adj_rho, n) && alloc_n(ctx, ctx->adj_drho, n) &&
              alloc_n(ctx, ctx->adj_bins, (size_t)nw * kAdjWarps * 4 * nrows) && alloc_n(ctx, ctx->adj_pg, (size_t)nb) &&
              alloc_n(ctx, ctx->adj_cg, (size_t)4 * nrows) && alloc_n(ctx, ctx->adj_sq, 1) &&
              alloc_n(ctx, ctx->adj_Mt, Mt.size()) && alloc_n(ctx, ctx->adj_kg, (size_t)nknots) &&
              alloc_n(ctx, ctx->adj_knot_func, (size_t)nknots) && alloc_n(ctx, ctx->adj_func_coef0, 3) &&
              alloc_n(ctx, ctx->adj_func_ncoef, 3) && alloc_n(ctx, ctx->adj_knot_mt0, (size_t)nknots);
    if (!ok) {
        ctx->adj_g = nullptr;
        return ctx->fail(MD_ERR_OOM, "adjoint workspace");
    }
    CK(cudaMemcpy(ctx->adj_Mt, Mt.data(), Mt.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->adj_knot_func, knot_func.data(), knot_func.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->adj_func_coef0, coef0.data(), 3 * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->adj_func_ncoef, ncoef.data(), 3 * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->adj_knot_mt0, mt0.data(), mt0.size() * sizeof(long long), cudaMemcpyHostToDevice));
    ctx->adj_nrows = nrows;
    ctx->adj_nknots = nknots;
    return MD_OK;
}

md_status force_match_impl(md_ctx *ctx, const double *f_ref, double e_ref, double w, double *loss, double *grad)
{
    md_status rc = check_device_errors(ctx);
    if (rc != MD_OK) return rc;
    const double E = ctx->st_host->e_embed + ctx->st_host->e_pair;
    rc = adjoint_setup(ctx);
    if (rc != MD_OK) return rc;
    const size_t n = (size_t)ctx->n;
    CK(cudaMemcpyAsync(ctx->stage, f_ref, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    const md_spline *fs[3] = {&ctx->shapes[2], &ctx->shapes[1], &ctx->shapes[0]};
    AdjointArgs a;
    memset(&a, 0, sizeof(a));
    for (int q = 0; q < 3; ++q) {
        a.x0[q] = fs[q]->x0;
        a.h[q] = fs[q]->dx;
        a.nint[q] = fs[q]->n - 1;
    }
    a.off_f = ctx->off_f0;
    a.off_F = ctx->off_F0;
    a.A = 2.0 * (E - e_ref) / (double)n;
    a.w = w;
    a.f_ref = ctx->stage;
    a.g = ctx->adj_g;
    a.rho = ctx->adj_rho;
    a.drho = ctx->adj_drho;
    a.block_bins = ctx->adj_bins;
    a.partials_g = ctx->adj_pg;
    a.coef_grad = ctx->adj_cg;
    a.sq = ctx->adj_sq;
    a.Mt = ctx->adj_Mt;
    a.nknots_total = ctx->adj_nknots;
    a.knot_func = ctx->adj_knot_func;
    a.func_coef0 = ctx->adj_func_coef0;
    a.func_ncoef = ctx->adj_func_ncoef;
    a.knot_mt0 = ctx->adj_knot_mt0;
    a.knot_grad = grad ? ctx->adj_kg : nullptr;
    Launch L = ctx->L;
    ctx->fixed_launches += launch_adjoint(ctx->Bd, ctx->G, L, a);
    CK(cudaGetLastError());
    double sq = 0.0;
    CK(cudaMemcpyAsync(&sq, ctx->adj_sq, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (grad)
        CK(cudaMemcpyAsync(grad, ctx->adj_kg, sizeof(double) * (size_t)ctx->adj_nknots, cudaMemcpyDeviceToHost,
                           ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (loss) *loss = (E - e_ref) * (E - e_ref) / (double)n + w * sq;
    return MD_OK;
}

template <class R>
md_status create_impl(md_ctx *ctx, const double *pos, const double *vel, const int32_t *types,
                      const md_potential *pot)
{
    std::vector<double> rows, rows2;
    Tables<R> tab;
    md_status trc = build_tables<R>(ctx, pot, rows, rows2, tab);
    if (trc != MD_OK) return trc;
    ctx->L.multi = tab.fused ? 0 : 1;
    ctx->L.nint_fused = tab.fused ? tab.fphi.nint : 0;
    if (ctx->opt.half_list && (ctx->precision != MD_PRECISION_MIXED || ctx->L.multi))
        return ctx->fail(MD_ERR_ARG, "half_list takes mixed precision and one atom type whose f and phi share a knot grid");
    ctx->L.half = ctx->opt.half_list ? 1 : 0;
    ctx->shapes.clear();
    for (int t = 0; t < pot->ntypes; ++t) ctx->shapes.push_back(pot->F[t]);
    for (int t = 0; t < pot->ntypes; ++t) ctx->shapes.push_back(pot->f[t]);
    for (int q = 0; q < pot->ntypes * (pot->ntypes + 1) / 2; ++q) ctx->shapes.push_back(pot->phi[q]);
    for (auto &sh : ctx->shapes) sh.y = nullptr;
    ctx->off_F0 = tab.F[0].offset;
    ctx->off_f0 = tab.f[0].offset;
    ctx->off_phi0 = tab.phi[0].offset;
    ctx->r_cut = pot->r_cut;
    ctx->skin = pot->skin;

    CK(cudaMallocHost((void **)&ctx->st_host, sizeof(DevState)));
    if (!alloc_n(ctx, ctx->st, 1) || !alloc_n(ctx, ctx->stage, 9 * (size_t)std::max<int64_t>(ctx->n, 1)) ||
        !alloc_n(ctx, ctx->types_orig, (size_t)std::max<int64_t>(ctx->n, 1)))
        return ctx->fail(MD_ERR_OOM, "device allocation failed");
    if (!alloc_buffers<R>(ctx, rows, rows2, tab)) return ctx->fail(MD_ERR_OOM, "device allocation failed");
    DevState h{};
    CK(cudaMemcpy(ctx->st, &h, sizeof(DevState), cudaMemcpyHostToDevice));
    if (ctx->n == 0) return MD_OK;
    CK(cudaMemcpy(ctx->types_orig, types, sizeof(int32_t) * (size_t)ctx->n, cudaMemcpyHostToDevice));
    md_status rc = load_and_measure<R>(ctx, pos, vel, 0);
    if (rc != MD_OK) return rc;
    const md_options &o = ctx->opt;
    if (ctx->L.half) {
        // one lane per atom, the context's block size; the graph path only
        set_sched(ctx, PassSched{1, 0}, PassSched{1, 0});
        rc = reevaluate<R>(ctx);
        if (rc != MD_OK) return rc;
        return check_device_errors(ctx);
    }
    if (o.lanes_per_atom == 0) {
        rc = autotune<R>(ctx);
        if (rc != MD_OK) return rc;
    }
    return setup_persistent<R>(ctx);
}

}  // namespace

// ==========================================================================
// C ABI

extern "C" {

void md_options_default(md_options *opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->precision = MD_PRECISION_MIXED;
    opt->rebuild_every = 10;
    opt->list_capacity = 0;
    opt->use_graphs = 1;
    opt->block_size = 256;
}

md_status md_create(const double box[3], int64_t n, const double *pos, const double *vel,
                    const int32_t *types, const md_potential *pot, const md_options *opt, md_ctx **out)
{
    g_create_error.clear();
    auto bad = [](md_status s, const char *m) {
        g_create_error = m;
        return s;
    };
    if (!out) return bad(MD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!box || !pot || n < 0 || (n > 0 && (!pos || !types))) return bad(MD_ERR_ARG, "null argument or n < 0");
    if (n >= (int64_t)kIndexMask) return bad(MD_ERR_CAPACITY, "n must be below 2^26");
    if (pot->ntypes < 1 || pot->ntypes > kMaxTypes || !pot->mass || !pot->F || !pot->f || !pot->phi)
        return bad(MD_ERR_ARG, "potential: ntypes must be 1..8 and all tables given");
    if (!(pot->r_cut > 0.0) || !(pot->skin >= 0.0) || !std::isfinite(pot->r_cut) || !std::isfinite(pot->skin))
        return bad(MD_ERR_ARG, "r_cut must be > 0 and skin >= 0");
    const double r_list = pot->r_cut + pot->skin;
    for (int t = 0; t < pot->ntypes; ++t) {
        if (!(pot->mass[t] > 0.0) || !std::isfinite(pot->mass[t])) return bad(MD_ERR_ARG, "masses must be > 0");
        if (!spline_ok(pot->F[t]) || !spline_ok(pot->f[t])) return bad(MD_ERR_ARG, "bad F or f spline");
        const md_spline &f = pot->f[t];
        if (f.x0 > 0.0 || f.x0 + (f.n - 1) * f.dx < pot->r_cut)
            return bad(MD_ERR_ARG, "f tables must cover [0, r_cut]");
    }
    for (int q = 0; q < pot->ntypes * (pot->ntypes + 1) / 2; ++q) {
        const md_spline &s = pot->phi[q];
        if (!spline_ok(s)) return bad(MD_ERR_ARG, "bad phi spline");
        if (s.x0 > 0.0 || s.x0 + (s.n - 1) * s.dx < pot->r_cut)
            return bad(MD_ERR_ARG, "phi tables must cover [0, r_cut]");
    }
    const int open_mask = opt ? opt->open_axes : 0;
    if (open_mask < 0 || open_mask > 7) return bad(MD_ERR_ARG, "open_axes must be a mask of bits 1 (x), 2 (y), 4 (z)");
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0.0) || !std::isfinite(box[a])) return bad(MD_ERR_ARG, "box edges must be > 0");
        const bool open_axis = (open_mask >> a) & 1;
        if (std::floor(box[a] / r_list) < (open_axis ? 1.0 : 3.0))
            return bad(MD_ERR_BOX, open_axis ? "open box edge shorter than r_cut + skin"
                                             : "periodic box edge shorter than 3 (r_cut + skin)");
    }
    for (int64_t i = 0; i < 3 * n; ++i) {
        if (!std::isfinite(pos[i]) || (vel && !std::isfinite(vel[i])))
            return bad(MD_ERR_NONFINITE, "non-finite position or velocity");
    }
    for (int64_t i = 0; i < n; ++i)
        if (types[i] < 0 || types[i] >= pot->ntypes) return bad(MD_ERR_ARG, "atom type out of range");
    md_options o;
    md_options_default(&o);
    if (opt) o = *opt;
    if (o.precision != MD_PRECISION_FP64 && o.precision != MD_PRECISION_MIXED)
        return bad(MD_ERR_ARG, "precision must be 0 (FP64) or 1 (mixed)");
    if (o.rebuild_every < 1) o.rebuild_every = 10;
    if (o.block_size <= 0) o.block_size = 256;
    if (o.block_size > 256 || (o.block_size & 31)) return bad(MD_ERR_ARG, "block_size must be a multiple of 32, <= 256");
    if ((o.alloc == nullptr) != (o.free == nullptr)) return bad(MD_ERR_ARG, "alloc and free go together");
    if (!(o.lanes_per_atom == 0 || o.lanes_per_atom == 1 || o.lanes_per_atom == 2 || o.lanes_per_atom == 4 ||
          o.lanes_per_atom == 8))
        return bad(MD_ERR_ARG, "lanes_per_atom must be 0 (tune), 1, 2, 4 or 8");
    if (o.persistent < MD_PERSIST_AUTO || o.persistent > MD_PERSIST_ON)
        return bad(MD_ERR_ARG, "persistent must be MD_PERSIST_AUTO, _OFF or _ON");
    if (o.wait_limit_us < 0) return bad(MD_ERR_ARG, "wait_limit_us must be >= 0");
    if (o.half_list != 0 && o.half_list != 1) return bad(MD_ERR_ARG, "half_list must be 0 or 1");
    if (o.half_list && (o.persistent == MD_PERSIST_ON || o.lanes_per_atom > 1))
        return bad(MD_ERR_ARG, "half_list runs as graphs with one lane per atom");

    md_ctx *ctx = new (std::nothrow) md_ctx();
    if (!ctx) return bad(MD_ERR_OOM, "host allocation failed");
    ctx->opt = o;
    ctx->precision = o.precision;
    ctx->n = n;
    ctx->ntypes = pot->ntypes;
    for (int t = 0; t < pot->ntypes; ++t) ctx->mass[t] = pot->mass[t];
    memcpy(ctx->box, box, sizeof(ctx->box));
    if (o.cuda_stream) {
        ctx->stream = (cudaStream_t)o.cuda_stream;
    } else if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) == cudaSuccess) {
        ctx->own_stream = true;
    } else {
        delete ctx;
        return bad(MD_ERR_CUDA, "cannot create a CUDA stream");
    }
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->body_stream, cudaStreamNonBlocking) != cudaSuccess) {
        md_destroy(ctx);
        return bad(MD_ERR_CUDA, "cannot create a CUDA stream");
    }

    // geometry: cells of edge >= r_list, at least 3 per axis
    Geom &G = ctx->G;
    double hmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        G.box[a] = box[a];
        G.half_box[a] = 0.5 * box[a];
        G.ncell[a] = (int)std::floor(box[a] / r_list);
        G.inv_cell[a] = (double)G.ncell[a] / box[a];
        G.h[a] = box[a] / (double)G.ncell[a];
        hmax = std::max(hmax, G.h[a]);
    }
    G.ncells = G.ncell[0] * G.ncell[1] * G.ncell[2];
    G.open_mask = o.open_axes;
    G.rl2 = r_list * r_list;
    G.rc2 = pot->r_cut * pot->r_cut;
    // rounding bound of the screened r^2 (cell-relative coordinates, |u| <= h)
    const double eps = (o.precision == MD_PRECISION_MIXED) ? std::ldexp(1.0, -24) : std::ldexp(1.0, -53);
    const double margin = 8.0 * (20.0 * hmax * r_list + 4.0 * r_list * r_list) * eps;
    G.screen_lo = G.rl2 - margin;
    G.screen_hi = G.rl2 + margin;
    for (int a = 0; a < 3; ++a) {
        G.h_f[a] = (float)G.h[a];
        G.inv_cell_f[a] = (float)G.inv_cell[a];
    }
    G.rc2_f = (float)G.rc2;
    G.screen_lo_f = (float)G.screen_lo;
    G.screen_hi_f = (float)G.screen_hi;

    Launch &L = ctx->L;
    L.n = (int)n;
    L.ld = (int)((n + 31) / 32 * 32);
    L.block = o.block_size;
    L.nblocks = (int)((n + L.block - 1) / L.block);
    {
        // the list build of a small system: blocks as small as it takes to
        // give every SM two (down to one warp)
        int dev = 0, nsm = 152;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            nsm = 152;
        L.list_block = L.block;
        while (L.list_block > 32 && (n + L.list_block - 1) / L.list_block < 2 * (int64_t)nsm) L.list_block /= 2;
        L.list_block = std::max(32, L.list_block / 32 * 32);
    }
    L.pstride = std::max(1, blocks_for_host(8 * n, std::min(L.block, 128)));
    {
        int lanes = o.lanes_per_atom > 0 ? o.lanes_per_atom : (o.half_list ? 1 : 4);
        L.tpa_d = L.tpa_f = lanes;
        L.block_d = L.block_f = L.block;
        L.nb_d = L.nb_f = blocks_for_host(n * lanes, L.block);
    }
    L.ntypes = pot->ntypes;
    L.rebuild_every = o.rebuild_every;
    L.disp2_thr = 0.25 * pot->skin * pot->skin;
    L.stream = ctx->stream;
    L.wait_ns = 1000ull * (unsigned long long)(o.wait_limit_us > 0 ? o.wait_limit_us : 1000000);
    for (int t = 0; t < pot->ntypes; ++t) L.ke_factor[t] = 0.5 * pot->mass[t] / kAccel;
    if (o.list_capacity > 0) {
        L.cap = o.list_capacity;
    } else {
        double vol = box[0] * box[1] * box[2];
        double expect = (double)n / vol * 4.0 / 3.0 * M_PI * r_list * r_list * r_list;
        L.cap = std::max(16, ((int)std::ceil(1.25 * expect) + 8 + 3) & ~3);
    }

    md_status rc = (o.precision == MD_PRECISION_MIXED) ? create_impl<float>(ctx, pos, vel, types, pot)
                                                       : create_impl<double>(ctx, pos, vel, types, pot);
    if (rc != MD_OK) {
        g_create_error = ctx->err;
        md_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return MD_OK;
}

md_status md_step(md_ctx *ctx, int64_t nsteps, double dt)
{
    if (!ctx) return MD_ERR_ARG;
    if (nsteps < 0 || !std::isfinite(dt)) return ctx->fail(MD_ERR_ARG, "nsteps must be >= 0 and dt finite");
    if (nsteps == 0) return MD_OK;
    if (ctx->n == 0) {
        ctx->host_steps += nsteps;
        return MD_OK;
    }
    return ctx->precision == MD_PRECISION_MIXED ? step_impl<float>(ctx, nsteps, dt)
                                                : step_impl<double>(ctx, nsteps, dt);
}

md_status md_sync(md_ctx *ctx)
{
    if (!ctx) return MD_ERR_ARG;
    if (ctx->n == 0) return MD_OK;
    return check_device_errors(ctx);
}

md_status md_energy(md_ctx *ctx, double *pe, double *ke)
{
    if (!ctx) return MD_ERR_ARG;
    if (ctx->n == 0) {
        if (pe) *pe = 0.0;
        if (ke) *ke = 0.0;
        return MD_OK;
    }
    md_status rc = check_device_errors(ctx);
    if (rc != MD_OK) return rc;
    if (pe) *pe = ctx->st_host->e_embed + ctx->st_host->e_pair;
    if (ke) *ke = ctx->st_host->ke;
    return MD_OK;
}

md_status md_virial(md_ctx *ctx, double w[6])
{
    if (!ctx || !w) return ctx ? ctx->fail(MD_ERR_ARG, "w is NULL") : MD_ERR_ARG;
    if (ctx->n == 0) {
        for (int k = 0; k < 6; ++k) w[k] = 0.0;
        return MD_OK;
    }
    md_status rc = check_device_errors(ctx);
    if (rc != MD_OK) return rc;
    for (int k = 0; k < 6; ++k) w[k] = ctx->st_host->virial[k];
    return MD_OK;
}

md_status md_forces(md_ctx *ctx, double *f)
{
    if (!ctx || !f) return ctx ? ctx->fail(MD_ERR_ARG, "f is NULL") : MD_ERR_ARG;
    md_status rc = md_sync(ctx);
    if (rc != MD_OK) return rc;
    return ctx->precision == MD_PRECISION_MIXED ? store_state<float>(ctx, nullptr, nullptr, f)
                                                : store_state<double>(ctx, nullptr, nullptr, f);
}

md_status md_get_state(md_ctx *ctx, double *pos, double *vel, int64_t *step)
{
    if (!ctx) return MD_ERR_ARG;
    md_status rc = md_sync(ctx);
    if (rc != MD_OK) return rc;
    if (step) *step = ctx->n == 0 ? ctx->host_steps : (int64_t)ctx->st_host->step;
    if (!pos && !vel) return MD_OK;
    return ctx->precision == MD_PRECISION_MIXED ? store_state<float>(ctx, pos, vel, nullptr)
                                                : store_state<double>(ctx, pos, vel, nullptr);
}

md_status md_set_state(md_ctx *ctx, const double *pos, const double *vel, int64_t step)
{
    if (!ctx) return MD_ERR_ARG;
    if (ctx->n == 0) {
        ctx->host_steps = step;
        return MD_OK;
    }
    if (!pos) return ctx->fail(MD_ERR_ARG, "pos is NULL");
    // finiteness is checked on the device as the state is loaded
    return ctx->precision == MD_PRECISION_MIXED ? load_and_measure<float>(ctx, pos, vel, step)
                                                : load_and_measure<double>(ctx, pos, vel, step);
}

md_status md_neighbors(md_ctx *ctx, int64_t *offsets, int32_t *js, int64_t cap)
{
    if (!ctx || !offsets) return ctx ? ctx->fail(MD_ERR_ARG, "offsets is NULL") : MD_ERR_ARG;
    const int64_t n = ctx->n;
    if (n == 0) {
        offsets[0] = 0;
        return MD_OK;
    }
    md_status rc = md_sync(ctx);
    if (rc != MD_OK) return rc;
    const int set = ctx->st_host->set;
    std::vector<int> nnb(n), id(n);
    std::vector<uint32_t> list((size_t)ctx->L.cap * ctx->L.ld);
    const int *idp = ctx->precision == MD_PRECISION_MIXED ? ctx->Bf.id[set] : ctx->Bd.id[set];
    const int *nnbp = ctx->precision == MD_PRECISION_MIXED ? ctx->Bf.nnb : ctx->Bd.nnb;
    const uint32_t *lp = ctx->precision == MD_PRECISION_MIXED ? ctx->Bf.list : ctx->Bd.list;
    CK(cudaMemcpy(nnb.data(), nnbp, sizeof(int) * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(id.data(), idp, sizeof(int) * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(list.data(), lp, sizeof(uint32_t) * list.size(), cudaMemcpyDeviceToHost));
    const size_t ld = (size_t)ctx->L.ld;
    if (ctx->L.half) {
        // each pair is listed once, by one of its atoms: give it to both
        // ends (the other end's stencil code is the mirrored one, t -> 2 - t
        // per axis), then order every list as the full-list build does,
        // which is ascending entry value (stencil code in the high bits,
        // sorted index below)
        std::vector<std::vector<uint32_t>> full(n);
        for (int64_t p = 0; p < n; ++p)
            for (int k = 0; k < nnb[p]; ++k) {
                const uint32_t e = list[(size_t)k * ld + p];
                const uint32_t q = e & kIndexMask, c = e >> kCodeShift;
                const uint32_t mc = (2u - (c & 3u)) | ((2u - ((c >> 2) & 3u)) << 2) | ((2u - (c >> 4)) << 4);
                full[p].push_back(e);
                full[q].push_back((uint32_t)p | (mc << kCodeShift));
            }
        std::vector<int64_t> cnt(n + 1, 0);
        for (int64_t p = 0; p < n; ++p) {
            std::sort(full[p].begin(), full[p].end());
            cnt[id[p]] = (int64_t)full[p].size();
        }
        offsets[0] = 0;
        for (int64_t i = 0; i < n; ++i) offsets[i + 1] = offsets[i] + cnt[i];
        if (js && offsets[n] <= cap) {
            for (int64_t p = 0; p < n; ++p) {
                int64_t o = offsets[id[p]];
                for (uint32_t e : full[p]) js[o++] = id[e & kIndexMask];
            }
        }
        return MD_OK;
    }
    std::vector<int64_t> cnt(n + 1, 0);
    for (int64_t p = 0; p < n; ++p) cnt[id[p]] = nnb[p];
    offsets[0] = 0;
    for (int64_t i = 0; i < n; ++i) offsets[i + 1] = offsets[i] + cnt[i];
    if (js && offsets[n] <= cap) {
        for (int64_t p = 0; p < n; ++p) {
            int64_t o = offsets[id[p]];
            for (int k = 0; k < nnb[p]; ++k) js[o + k] = id[list[(size_t)k * ld + p] & kIndexMask];
        }
    }
    return MD_OK;
}

md_status md_cells(md_ctx *ctx, int32_t ncell[3], int32_t *cell_start, int32_t *cell_atoms)
{
    if (!ctx) return MD_ERR_ARG;
    if (ncell)
        for (int a = 0; a < 3; ++a) ncell[a] = ctx->G.ncell[a];
    if (!cell_start && !cell_atoms) return MD_OK;
    if (ctx->n == 0) {
        if (cell_start) memset(cell_start, 0, sizeof(int32_t) * ((size_t)ctx->G.ncells + 1));
        return MD_OK;
    }
    md_status rc = md_sync(ctx);
    if (rc != MD_OK) return rc;
    const int set = ctx->st_host->set;
    const int *csp = ctx->precision == MD_PRECISION_MIXED ? ctx->Bf.cell_start : ctx->Bd.cell_start;
    const int *idp = ctx->precision == MD_PRECISION_MIXED ? ctx->Bf.id[set] : ctx->Bd.id[set];
    if (cell_start) CK(cudaMemcpy(cell_start, csp, sizeof(int) * ((size_t)ctx->G.ncells + 1), cudaMemcpyDeviceToHost));
    if (cell_atoms) CK(cudaMemcpy(cell_atoms, idp, sizeof(int) * (size_t)ctx->n, cudaMemcpyDeviceToHost));
    return MD_OK;
}

md_status md_stats(md_ctx *ctx, md_stats_t *out)
{
    if (!ctx || !out) return ctx ? ctx->fail(MD_ERR_ARG, "out is NULL") : MD_ERR_ARG;
    memset(out, 0, sizeof(*out));
    out->list_capacity = ctx->L.cap;
    if (ctx->n == 0) {
        out->steps = ctx->host_steps;
        return MD_OK;
    }
    md_status rc = read_state(ctx);
    if (rc != MD_OK) return rc;
    const DevState &h = *ctx->st_host;
    out->steps = h.step;
    out->rebuilds = h.rebuilds - ctx->rebuilds_at_create;
    out->max_neighbors = h.max_nnb;
    out->table_out_of_range = (int64_t)h.table_oor;
    out->kernel_launches = ctx->fixed_launches + 8 * h.graph_rebuilds;
    out->lanes_density = ctx->L.tpa_d;
    out->lanes_force = ctx->L.tpa_f;
    out->threads_density = ctx->L.block_d;
    out->threads_force = ctx->L.block_f;
    out->persistent_blocks = ctx->persist_grid;
    out->persistent_lanes = ctx->persist_grid ? ctx->persist_tpa : 0;
    out->half_list = ctx->L.half;
    out->record_textures = (ctx->precision == MD_PRECISION_MIXED && ctx->Bf.tex_shadow[0] && ctx->Bf.tex_shadow[1]) ? 1 : 0;
    return MD_OK;
}

md_status md_profile(md_ctx *ctx, int64_t nsteps, double dt, md_profile_t *out)
{
    if (!ctx || !out) return ctx ? ctx->fail(MD_ERR_ARG, "out is NULL") : MD_ERR_ARG;
    if (nsteps < 1 || !std::isfinite(dt)) return ctx->fail(MD_ERR_ARG, "nsteps must be >= 1 and dt finite");
    memset(out, 0, sizeof(*out));
    if (ctx->n == 0) return MD_OK;
    md_status rc = ctx->precision == MD_PRECISION_MIXED ? profile_impl<float>(ctx, nsteps, dt, out)
                                                        : profile_impl<double>(ctx, nsteps, dt, out);
    if (rc != MD_OK) return rc;
    return check_device_errors(ctx);
}

md_status md_set_potential(md_ctx *ctx, const md_potential *pot)
{
    if (!ctx || !pot) return ctx ? ctx->fail(MD_ERR_ARG, "pot is NULL") : MD_ERR_ARG;
    if (pot->ntypes != ctx->ntypes || pot->r_cut != ctx->r_cut || pot->skin != ctx->skin || !pot->mass ||
        !pot->F || !pot->f || !pot->phi)
        return ctx->fail(MD_ERR_ARG, "md_set_potential keeps ntypes, r_cut and skin");
    std::vector<const md_spline *> given;
    for (int t = 0; t < pot->ntypes; ++t) given.push_back(&pot->F[t]);
    for (int t = 0; t < pot->ntypes; ++t) given.push_back(&pot->f[t]);
    for (int q = 0; q < pot->ntypes * (pot->ntypes + 1) / 2; ++q) given.push_back(&pot->phi[q]);
    for (size_t k = 0; k < given.size(); ++k) {
        const md_spline &a = *given[k], &b = ctx->shapes[k];
        if (!spline_ok(a) || a.n != b.n || a.x0 != b.x0 || a.dx != b.dx || a.bc_lo != b.bc_lo || a.bc_hi != b.bc_hi)
            return ctx->fail(MD_ERR_ARG, "md_set_potential keeps every knot grid and end condition");
    }
    for (int t = 0; t < pot->ntypes; ++t)
        if (pot->mass[t] != ctx->mass[t]) return ctx->fail(MD_ERR_ARG, "md_set_potential keeps the masses");
    return ctx->precision == MD_PRECISION_MIXED ? set_potential_impl<float>(ctx, pot)
                                                : set_potential_impl<double>(ctx, pot);
}

md_status md_force_match(md_ctx *ctx, const double *f_ref, double e_ref, double w, double *loss, double *grad)
{
    if (!ctx || !f_ref) return ctx ? ctx->fail(MD_ERR_ARG, "f_ref is NULL") : MD_ERR_ARG;
    if (ctx->precision != MD_PRECISION_FP64 || ctx->ntypes != 1 || ctx->n < 1)
        return ctx->fail(MD_ERR_ARG, "md_force_match needs an FP64 context with one atom type and n >= 1");
    if (!std::isfinite(e_ref) || !std::isfinite(w)) return ctx->fail(MD_ERR_ARG, "e_ref and w must be finite");
    return force_match_impl(ctx, f_ref, e_ref, w, loss, grad);
}

const char *md_last_error(const md_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

void md_destroy(md_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    for (int s = 0; s < 2; ++s)
        if (ctx->Bf.tex_shadow[s]) cudaDestroyTextureObject((cudaTextureObject_t)ctx->Bf.tex_shadow[s]);
    dfree_all(ctx);
    if (ctx->st_host) cudaFreeHost(ctx->st_host);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->body_stream) cudaStreamDestroy(ctx->body_stream);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

}  // extern "C"
