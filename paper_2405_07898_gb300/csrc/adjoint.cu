// adjoint.cu -- gradient of the force-matching loss with respect to the
// spline coefficients of phi, f and F (single atom type, FP64 path).
//
// For one configuration with energy E (Eq. 3) and forces F (Eq. 4):
//   L = (E - E_ref)^2 / N + w sum_i |F_i - F_ref,i|^2.
// With A = 2 (E - E_ref)/N and g = F - F_ref, and since F = -dE/dx,
//   dL/dtheta = A dE/dtheta - 2 w D_g[dE/dtheta],
// D_g the derivative along the position perturbation dx = g:
//   dr_ij = (x_j - x_i)/r . (g_j - g_i),   drho_i = sum_j f'(r_ij) dr_ij.
// Per interval row (a, b, c, d) of the spline that holds x, with
// B = (1, t, t^2, t^3) and B' = (0, 1, 2t, 3t^2):
//   phi row of r_ij (each ordered pair):  1/2 A B - w B' dr_ij
//   f   row of r_ij (each ordered pair):  A F'_i B - 2w (F''_i drho_i B + F'_i B' dr_ij)
//   F   row of rho_i (each atom):         A B - 2w B' drho_i
// rho is recomputed here from the neighbour list (no per-pair term is
// stored).  Each warp owns shared-memory bins for all rows; its lanes add in
// lane order, blocks are summed in block order: the gradient is bitwise
// reproducible.
#include "device_common.cuh"

#include <cuda_runtime.h>

namespace eammd {
namespace {

struct AdjDesc {
    // spline grids (FP64) of phi, f, F
    double x0[3], h[3];
    int nint[3];       // intervals
    int row0[3];       // first bin row of each function in the bin array
    int nrows;         // total rows (sum of nint)
    double A, w;
};

__device__ __forceinline__ int adj_seg(const AdjDesc &D, int q, double x, double &t)
{
    int k;
    if (x < D.x0[q]) k = 0;
    else k = min((int)floor((x - D.x0[q]) / D.h[q]), D.nint[q] - 1);
    t = x - (D.x0[q] + (double)k * D.h[q]);
    return k;
}

// value and slope rows of the coefficient derivative at x (inside: the
// cubic; beyond an end: the tangent line used by the spline evaluation)
__device__ __forceinline__ int adj_rows(const AdjDesc &D, int q, double x, double bv[4], double bd[4])
{
    double t;
    int k = adj_seg(D, q, x, t);
    double x_end = D.x0[q] + (double)D.nint[q] * D.h[q];
    if (x < D.x0[q]) {
        bv[0] = 1.0; bv[1] = x - D.x0[q]; bv[2] = 0.0; bv[3] = 0.0;
        bd[0] = 0.0; bd[1] = 1.0; bd[2] = 0.0; bd[3] = 0.0;
    } else if (x > x_end) {
        double hh = D.h[q], e = x - x_end;
        bv[0] = 1.0; bv[1] = hh + e; bv[2] = hh * hh + 2.0 * hh * e; bv[3] = hh * hh * hh + 3.0 * hh * hh * e;
        bd[0] = 0.0; bd[1] = 1.0; bd[2] = 2.0 * hh; bd[3] = 3.0 * hh * hh;
    } else {
        bv[0] = 1.0; bv[1] = t; bv[2] = t * t; bv[3] = t * t * t;
        bd[0] = 0.0; bd[1] = 1.0; bd[2] = 2.0 * t; bd[3] = 3.0 * t * t;
    }
    return D.row0[q] + k;
}

// spline value, first and second derivative from a coefficient row
__device__ __forceinline__ double adj_eval(const double4_32a *coef, int offset, const AdjDesc &D, int q, double x,
                                           double &d1, double &d2)
{
    double t;
    int k = adj_seg(D, q, x, t);
    double x_end = D.x0[q] + (double)D.nint[q] * D.h[q];
    if (x < D.x0[q]) {
        double4_32a c = coef[offset];
        d1 = c.y; d2 = 0.0;
        return c.x + c.y * (x - D.x0[q]);
    }
    if (x > x_end) {
        double4_32a c = coef[offset + D.nint[q] - 1];
        double hh = D.h[q];
        double ye = c.x + hh * (c.y + hh * (c.z + hh * c.w));
        double se = c.y + hh * (2.0 * c.z + 3.0 * hh * c.w);
        d1 = se; d2 = 0.0;
        return ye + se * (x - x_end);
    }
    double4_32a c = coef[offset + k];
    d1 = c.y + t * (2.0 * c.z + 3.0 * t * c.w);
    d2 = 2.0 * c.z + 6.0 * t * c.w;
    return c.x + t * (c.y + t * (c.z + t * c.w));
}

// g = F - F_ref in sorted order; block partial sums of |g|^2
__global__ void k_adj_g(Bufs<double> B, const double *f_ref, double *g, int n, double *partials)
{
    const int s = B.st->set;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (p < n) {
        size_t o = 3 * (size_t)B.id[s][p];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double v = B.fcache[c][p] - f_ref[o + c];
            g[(size_t)c * n + p] = v;
            sq += v * v;
        }
    }
    double v1[1] = {sq};
    block_sums_t<1, double>(v1, partials, gridDim.x, 0);
}

// rho_i recomputed from the list, F'(rho_i), F''(rho_i), drho_i
__global__ void k_adj_rho(Bufs<double> B, Geom G, int n, int ld, AdjDesc D, int off_f, int off_F, const double *g,
                          double *rho_out, double *drho_out)
{
    double h[3];
    load_h<double>(G, h);
    const int sp = B.st->sp;
    const double4_32a *sw = B.shadow[sp];
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double4_32a ui = sw[p];
    const int nn = B.nnb[p];
    double rho = 0.0, drho = 0.0;
    const double gx = g[p], gy = g[(size_t)n + p], gz = g[2 * (size_t)n + p];
    for (int k = 0; k < nn; ++k) {
        uint32_t e = B.list[(size_t)k * ld + p];
        int j = (int)(e & kIndexMask);
        double4_32a uj = sw[j];
        const Shift<double> s = entry_shift<double>(e, h);
        double dx = (uj.x - ui.x) + s.x, dy = (uj.y - ui.y) + s.y, dz = (uj.z - ui.z) + s.z;
        double r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < G.rc2)) continue;
        double r = sqrt(r2), d1, d2;
        rho += adj_eval(B.coef, off_f, D, 1, r, d1, d2);
        double dr = (dx * (g[j] - gx) + dy * (g[(size_t)n + j] - gy) + dz * (g[2 * (size_t)n + j] - gz)) / r;
        drho += d1 * dr;
    }
    rho_out[p] = rho;
    drho_out[p] = drho;
    (void)off_F;
}

// Contributions of 32 atoms to the coefficient bins.  Block = kAdjWarps
// warps over the same 32 atoms: warp w takes list columns w, w + kAdjWarps,
// ... (and warp 0 the F rows), each into bins of its own in dynamic shared
// memory (4 * nrows doubles per warp), added in column then lane order; the
// block writes its warps' bins in warp order.
__global__ void k_adj_accum(Bufs<double> B, Geom G, int n, int ld, AdjDesc D, int off_f, int off_F, const double *g,
                            const double *rho_in, const double *drho_in, double *block_bins)
{
    extern __shared__ double bins_all[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *bins = bins_all + (size_t)warp * 4 * D.nrows;
    for (int r = lane; r < 4 * D.nrows; r += 32) bins[r] = 0.0;
    double h[3];
    load_h<double>(G, h);
    __syncwarp();
    const int sp = B.st->sp;
    const double4_32a *sw = B.shadow[sp];
    const int p = blockIdx.x * 32 + lane;
    const bool active = p < n;
    double4_32a ui = make_double4_32a(0, 0, 0, 0);
    double gx = 0, gy = 0, gz = 0, dF = 0, d2F = 0, drho = 0;
    int nn = 0;
    double contrib[8];
    int row_a = -1, row_b = -1;
    if (active) {
        ui = sw[p];
        nn = B.nnb[p];
        gx = g[p]; gy = g[(size_t)n + p]; gz = g[2 * (size_t)n + p];
        drho = drho_in[p];
        adj_eval(B.coef, off_F, D, 2, rho_in[p], dF, d2F);
        // F row of rho_p (warp 0)
        if (warp == 0) {
            double bv[4], bd[4];
            row_a = adj_rows(D, 2, rho_in[p], bv, bd);
#pragma unroll
            for (int c = 0; c < 4; ++c) contrib[c] = D.A * bv[c] - 2.0 * D.w * bd[c] * drho;
        }
    }
    for (int L = 0; L < 32; ++L) {
        if (lane == L && row_a >= 0)
#pragma unroll
            for (int c = 0; c < 4; ++c) bins[4 * row_a + c] += contrib[c];
        __syncwarp();
    }
    int kmax = nn;
    for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    for (int k = warp; k < kmax; k += kAdjWarps) {
        row_a = row_b = -1;
        if (active && k < nn) {
            uint32_t e = B.list[(size_t)k * ld + p];
            int j = (int)(e & kIndexMask);
            double4_32a uj = sw[j];
            const Shift<double> s = entry_shift<double>(e, h);
            double dx = (uj.x - ui.x) + s.x, dy = (uj.y - ui.y) + s.y, dz = (uj.z - ui.z) + s.z;
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < G.rc2) {
                double r = sqrt(r2);
                double dr = (dx * (g[j] - gx) + dy * (g[(size_t)n + j] - gy) + dz * (g[2 * (size_t)n + j] - gz)) / r;
                double bv[4], bd[4];
                row_a = adj_rows(D, 0, r, bv, bd);  // phi
#pragma unroll
                for (int c = 0; c < 4; ++c) contrib[c] = 0.5 * D.A * bv[c] - D.w * bd[c] * dr;
                row_b = adj_rows(D, 1, r, bv, bd);  // f
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    contrib[4 + c] = D.A * dF * bv[c] - 2.0 * D.w * (d2F * drho * bv[c] + dF * bd[c] * dr);
            }
        }
        for (int L = 0; L < 32; ++L) {
            if (lane == L && row_a >= 0) {
#pragma unroll
                for (int c = 0; c < 4; ++c) bins[4 * row_a + c] += contrib[c];
#pragma unroll
                for (int c = 0; c < 4; ++c) bins[4 * row_b + c] += contrib[4 + c];
            }
            __syncwarp();
        }
    }
    for (int r = lane; r < 4 * D.nrows; r += 32)
        block_bins[((size_t)blockIdx.x * kAdjWarps + warp) * 4 * D.nrows + r] = bins[r];
}

// Sum the block bins in block order (one thread per coefficient), and the
// |g|^2 block partials.
__global__ void k_adj_finish(const double *block_bins, int nblocks, int nrows, const double *partials_g, int nb_g,
                             double *coef_grad, double *sq_out)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < 4 * nrows; r += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += block_bins[(size_t)b * 4 * nrows + r];
        coef_grad[r] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb_g; ++b) s += partials_g[b];
        *sq_out = s;
    }
}

// knot gradient: for knot q of function fn, sum over that function's
// coefficient rows of M[row][q] * coef_grad[row] (M stored transposed:
// Mt[q][row] over the function's 4*nint coefficients, fixed order).
__global__ void k_adj_knots(const double *coef_grad, const double *Mt, int nknots_total, const int *knot_func,
                            const int *func_coef0, const int *func_ncoef, const long long *knot_mt0,
                            double *knot_grad)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nknots_total) return;
    int fn = knot_func[q];
    const double *m = Mt + knot_mt0[q];
    const double *cg = coef_grad + func_coef0[fn];
    double s = 0.0;
    for (int r = 0; r < func_ncoef[fn]; ++r) s += m[r] * cg[r];
    knot_grad[q] = s;
}

}  // namespace

int launch_adjoint(const Bufs<double> &B, const Geom &G, const Launch &L, const AdjointArgs &a)
{
    AdjDesc D;
    int row = 0;
    for (int q = 0; q < 3; ++q) {
        D.x0[q] = a.x0[q];
        D.h[q] = a.h[q];
        D.nint[q] = a.nint[q];
        D.row0[q] = row;
        row += a.nint[q];
    }
    D.nrows = row;
    D.A = a.A;
    D.w = a.w;
    const int n = L.n;
    const int nb = blocks_for(n, 256);
    k_adj_g<<<nb, 256, 0, L.stream>>>(B, a.f_ref, a.g, n, a.partials_g);
    // one warp per block: the few atoms of a force-matching configuration
    // spread over as many SMs' FP64 pipes as they can fill
    k_adj_rho<<<blocks_for(n, 32), 32, 0, L.stream>>>(B, G, n, L.ld, D, a.off_f, a.off_F, a.g, a.rho, a.drho);
    const int nw = blocks_for(n, 32);
    const size_t smem = adjoint_smem_bytes(D.nrows);
    k_adj_accum<<<nw, 32 * kAdjWarps, smem, L.stream>>>(B, G, n, L.ld, D, a.off_f, a.off_F, a.g, a.rho, a.drho,
                                                        a.block_bins);
    k_adj_finish<<<blocks_for(4 * D.nrows, 256), 256, 0, L.stream>>>(a.block_bins, nw * kAdjWarps, D.nrows,
                                                                      a.partials_g, nb, a.coef_grad, a.sq);
    int launched = 4;
    if (a.knot_grad) {
        k_adj_knots<<<blocks_for(a.nknots_total, 128), 128, 0, L.stream>>>(
            a.coef_grad, a.Mt, a.nknots_total, a.knot_func, a.func_coef0, a.func_ncoef, a.knot_mt0, a.knot_grad);
        ++launched;
    }
    return launched;
}

size_t adjoint_smem_bytes(int nrows) { return sizeof(double) * 4 * (size_t)nrows * kAdjWarps; }

cudaError_t allow_adjoint_smem(size_t bytes)
{
    return cudaFuncSetAttribute(k_adj_accum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace eammd
