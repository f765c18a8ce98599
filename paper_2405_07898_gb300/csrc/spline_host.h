// spline_host.h -- host construction of the cubic spline tables used by the
// kernels (single-system and batched paths).
#pragma once

#include "eammd.h"

#include <cmath>
#include <vector>

namespace eammd {

// Spline tables.  The C2 cubic through uniform knots is parametrised by its
// knot slopes m_k: continuity of the second derivative at interior knots gives
//   m_{k-1} + 4 m_k + m_{k+1} = 3 (y_{k+1} - y_{k-1}) / h,
// a natural end gives 2 m_0 + m_1 = 3 (y_1 - y_0) / h (and its mirror), a
// clamped end fixes the slope.  Each interval is the Hermite cubic through
// (y_k, m_k) and (y_{k+1}, m_{k+1}).
inline bool hermite_coefficients(const md_spline &s, std::vector<double> &rows)
{
    const int n = s.n;
    const double h = s.dx;
    const double *y = s.y;
    std::vector<double> lo(n, 0.0), di(n, 0.0), up(n, 0.0), rhs(n, 0.0), m(n, 0.0);
    if (s.bc_lo == 1) {
        di[0] = 1.0; rhs[0] = s.d_lo;
    } else {
        di[0] = 2.0; up[0] = 1.0; rhs[0] = 3.0 * (y[1] - y[0]) / h;
    }
    for (int k = 1; k < n - 1; ++k) {
        lo[k] = 1.0; di[k] = 4.0; up[k] = 1.0;
        rhs[k] = 3.0 * (y[k + 1] - y[k - 1]) / h;
    }
    if (s.bc_hi == 1) {
        di[n - 1] = 1.0; rhs[n - 1] = s.d_hi;
    } else {
        lo[n - 1] = 1.0; di[n - 1] = 2.0; rhs[n - 1] = 3.0 * (y[n - 1] - y[n - 2]) / h;
    }
    // tridiagonal solve (forward sweep, back substitution)
    for (int k = 1; k < n; ++k) {
        double w = lo[k] / di[k - 1];
        di[k] -= w * up[k - 1];
        rhs[k] -= w * rhs[k - 1];
    }
    m[n - 1] = rhs[n - 1] / di[n - 1];
    for (int k = n - 2; k >= 0; --k) m[k] = (rhs[k] - up[k] * m[k + 1]) / di[k];
    for (int k = 0; k < n - 1; ++k) {
        double dy = (y[k + 1] - y[k]) / h;
        rows.push_back(y[k]);
        rows.push_back(m[k]);
        rows.push_back((3.0 * dy - 2.0 * m[k] - m[k + 1]) / h);
        rows.push_back((m[k] + m[k + 1] - 2.0 * dy) / (h * h));
    }
    for (double v : m)
        if (!std::isfinite(v)) return false;
    return true;
}

}  // namespace eammd
