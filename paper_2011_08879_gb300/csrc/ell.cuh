// ELL row pairs shared by the ELL SpMV and the CG product that fuses p.q:
// rows (r, r+1) with their slot k at k * n_pad + r (column-major, n_pad
// even), one 128-bit value load and one 64-bit index load per slot,
// padding (col < 0) skipped.
#pragma once

#include "common.cuh"
#include "segmented.cuh"

namespace gko {

__device__ __forceinline__ void ell_pair_sum(int64_t r, int64_t n_pad, int64_t K, const int32_t* __restrict__ col,
                                             const double* __restrict__ val, const double* __restrict__ x,
                                             double& a0_out, double& a1_out)
{
    double a0 = 0.0, a1 = 0.0;
    const int2* c2 = reinterpret_cast<const int2*>(col + r);
    const double2* v2 = reinterpret_cast<const double2*>(val + r);
    const int64_t step = n_pad / 2;
    int64_t k = 0;
    for (; k + 4 <= K; k += 4) {
        int2 c[4];
        double2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = __ldcs(c2 + (k + u) * step);
            v[u] = __ldcs(v2 + (k + u) * step);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u].x >= 0) a0 = fma(v[u].x, ldg(x + c[u].x), a0);
            if (c[u].y >= 0) a1 = fma(v[u].y, ldg(x + c[u].y), a1);
        }
    }
    for (; k < K; ++k) {
        const int2 c = __ldcs(c2 + k * step);
        const double2 v = __ldcs(v2 + k * step);
        if (c.x >= 0) a0 = fma(v.x, ldg(x + c.x), a0);
        if (c.y >= 0) a1 = fma(v.y, ldg(x + c.y), a1);
    }
    a0_out = a0;
    a1_out = a1;
}

template <bool kAlpha, bool kBeta>
__device__ __forceinline__ void store_pair(double* y, int64_t r, int64_t n, double a0, double a1, double alpha,
                                           double beta)
{
    if (r + 1 < n) {
        // y is caller-owned: vector access only when y + r is 16-byte aligned
        const bool vec = (reinterpret_cast<uintptr_t>(y + r) & 15) == 0;
        double2 o;
        o.x = kAlpha ? alpha * a0 : a0;
        o.y = kAlpha ? alpha * a1 : a1;
        if (kBeta) {
            double2 yo;
            if (vec)
                yo = *reinterpret_cast<const double2*>(y + r);
            else
                yo = make_double2(y[r], y[r + 1]);
            o.x = fma(beta, yo.x, o.x);
            o.y = fma(beta, yo.y, o.y);
        }
        if (vec)
            *reinterpret_cast<double2*>(y + r) = o;
        else {
            y[r] = o.x;
            y[r + 1] = o.y;
        }
    } else if (r < n) {
        seg_store<kAlpha, kBeta>(y, r, a0, alpha, beta);
    }
}

}  // namespace gko
