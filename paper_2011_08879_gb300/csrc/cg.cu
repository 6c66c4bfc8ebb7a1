// Conjugate gradients (Hestenes-Stiefel 1952), the Krylov solver the
// paper's Sec. 6.2 runs on SpMV, plus mixed-precision CG with FP64
// iterative refinement.
//
// One CG step is four launches (three on ELL, whose product carries p.q):
//   q = A p                                  (format kernel of choice)
//   alpha = rho / (p.q)                      (dot with grid reduction)
//   r -= alpha q, rho' = r.r                 (fused update + grid reduction)
//   x += alpha p, p = r + beta p             (beta = rho'/rho)
// Each dot is one grid-wide reduction: every block writes its partial, the
// last block to finish (atomic ticket) sums the partials in index order, so
// results do not depend on block scheduling.  Scalars stay on the device.
// The loop body is captured once into a CUDA graph under a conditional
// WHILE node; the reduction epilogue clears the condition when the solve
// stops, so the host waits once per solve (plus once per true-residual
// confirmation) instead of once per step.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "ell.cuh"
#include "segmented.cuh"
#include "solver.cuh"

namespace gko {

int launch_seg(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* row_ptr, const int32_t* rows, const int32_t* col,
               const double* val, const int32_t* thr_row, const SegArrays& sa, const double* x, double* y,
               double alpha, double beta, uint32_t* err, bool coo, cudaStream_t st, bool accumulate, int coo_p);

enum { kDotStore = 0, kDotRhoInit = 1, kDotPQ = 2 };

// Scalar step after p.q: alpha = rho / p.q, iteration count, breakdown and
// timeout tests; step_ok tells the x update of this step whether alpha
// was formed.
__device__ __forceinline__ void pq_step(SolverState* s, double tot, cudaGraphConditionalHandle h,
                                        const uint32_t* err)
{
    s->step_ok = 0;
    if (s->done || s->iter >= s->maxit) {
        // already stopped (e.g. converged before the first step):
        // clear the loop condition so the WHILE node always ends
        stop_loop(s, h);
        return;
    }
    s->pq = tot;
    s->iter += 1;
    // a product whose bulk copies did not land leaves q undefined and
    // sets the timeout bit of the handle's error word
    if (err && (*reinterpret_cast<const volatile uint32_t*>(err) & 1u)) {
        s->status = GKO_ERR_TIMEOUT;
        stop_loop(s, h);
    } else if (!(tot > 0.0)) {
        s->status = GKO_ERR_BREAKDOWN;
        stop_loop(s, h);
    } else {
        s->alpha = s->rho / tot;
        s->step_ok = 1;
    }
}

// Scalar step after rho' = r.r: beta = rho'/rho, rho = rho', stop tests.
__device__ __forceinline__ void rr_step(SolverState* s, double rho_new, cudaGraphConditionalHandle h)
{
    if (!(rho_new == rho_new)) {
        s->status = GKO_ERR_BREAKDOWN;
        stop_loop(s, h);
        return;
    }
    s->beta = rho_new / s->rho;
    s->rho = rho_new;
    if (sqrt(rho_new) <= s->tol * s->stop_ref) {
        s->conv = 1;
        s->status = GKO_OK;
        stop_loop(s, h);
    } else if (s->iter >= s->maxit) {
        s->status = GKO_ERR_NOT_CONVERGED;
        stop_loop(s, h);
    }
}

// dot(a, b) with per-thread accumulation in T, cross-thread in FP64
template <typename T, int kMode>
__global__ void __launch_bounds__(kRedThreads)
    dot_kernel(int64_t n, const T* __restrict__ a, const T* __restrict__ b, SolverState* s, double* part,
               cudaGraphConditionalHandle h, const uint32_t* err = nullptr)
{
    T acc = T(0);
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads)
        acc = fma(a[i], b[i], acc);
    grid_sum(static_cast<double>(acc), part, &s->ticket, [&](double tot) {
        if (kMode == kDotStore) {
            s->dot_out = tot;
        } else if (kMode == kDotRhoInit) {
            s->rho = tot;
            s->rho0 = tot;
            if (s->rel_inner) s->stop_ref = sqrt(tot);
            if (sqrt(tot) <= s->tol * s->stop_ref) {
                s->conv = 1;
                s->status = GKO_OK;
                s->done = 1;
            }
        } else {  // p.q -> alpha
            pq_step(s, tot, h, err);
        }
    });
}

// p = r + beta p
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    pupdate_kernel(int64_t n, T* __restrict__ p, const T* __restrict__ r, const SolverState* s, int force)
{
    if (s->done && !force) return;
    const T beta = static_cast<T>(s->beta);
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads)
        p[i] = fma(beta, p[i], r[i]);
}

// --------------------------------- FP64 CG step with regrouped updates
//
// The plain FP64 step runs as
//   q = A p and p.q -> alpha       (ELL: one kernel, the dot fused)
//   r -= alpha q, rho' = r.r -> beta, stop tests
//   x += alpha p, p = r + beta p   (one pass over x, p, r)
// which moves two vector passes fewer than product, dot, (x, r) update and
// p update as separate kernels.  When the solve stops at the r update, the
// last kernel still applies x += alpha p (step_ok) but leaves p.

// q = A p for ELL with p.q in the same pass (persistent grid; one grid
// reduction, partials summed in block order)
__global__ void __launch_bounds__(256)
    ell_pq_kernel(int64_t n, int64_t n_pad, int64_t K, const int32_t* __restrict__ col,
                  const double* __restrict__ val, const double* __restrict__ p, double* __restrict__ q,
                  SolverState* s, double* part, cudaGraphConditionalHandle h)
{
    double acc = 0.0;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; 2 * t < n;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = 2 * t;
        double a0, a1;
        ell_pair_sum(r, n_pad, K, col, val, p, a0, a1);
        store_pair<false, false>(q, r, n, a0, a1, 1.0, 0.0);
        acc = fma(p[r], a0, acc);
        if (r + 1 < n) acc = fma(p[r + 1], a1, acc);
    }
    grid_sum(acc, part, &s->ticket, [&](double tot) { pq_step(s, tot, h, nullptr); });
}

// r -= alpha q; rho' = r.r; beta; stop tests (kVec: 128-bit accesses, the
// vectors 16-byte aligned)
template <bool kVec>
__global__ void __launch_bounds__(kRedThreads)
    r_update_kernel(int64_t n, double* __restrict__ r, const double* __restrict__ q, SolverState* s, double* part,
                    cudaGraphConditionalHandle h)
{
    if (s->done) return;  // only the last block of the previous kernel can set it
    const double alpha = s->alpha;
    const int64_t tid = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x;
    const int64_t nth = static_cast<int64_t>(gridDim.x) * kRedThreads;
    double acc = 0.0;
    int64_t i0 = 0;
    if (kVec) {
        const int64_t nv = n / 2;
        for (int64_t i = tid; i < nv; i += nth) {
            double2 rv = reinterpret_cast<const double2*>(r)[i];
            const double2 qv = reinterpret_cast<const double2*>(q)[i];
            rv.x = fma(-alpha, qv.x, rv.x);
            rv.y = fma(-alpha, qv.y, rv.y);
            reinterpret_cast<double2*>(r)[i] = rv;
            acc = fma(rv.x, rv.x, acc);
            acc = fma(rv.y, rv.y, acc);
        }
        i0 = 2 * nv;
    }
    for (int64_t i = i0 + tid; i < n; i += nth) {
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    grid_sum(acc, part, &s->ticket, [&](double rho_new) { rr_step(s, rho_new, h); });
}

// x += alpha p; then p = r + beta p unless the solve stopped at this step
template <bool kVec>
__global__ void __launch_bounds__(kRedThreads)
    px_update_kernel(int64_t n, double* __restrict__ x, double* __restrict__ p, const double* __restrict__ r,
                     const SolverState* s)
{
    if (!s->step_ok) return;
    const double alpha = s->alpha, beta = s->beta;
    const bool more = !s->done;
    const int64_t tid = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x;
    const int64_t nth = static_cast<int64_t>(gridDim.x) * kRedThreads;
    int64_t i0 = 0;
    if (kVec) {
        const int64_t nv = n / 2;
        for (int64_t i = tid; i < nv; i += nth) {
            const double2 pv = reinterpret_cast<const double2*>(p)[i];
            double2 xv = reinterpret_cast<const double2*>(x)[i];
            xv.x = fma(alpha, pv.x, xv.x);
            xv.y = fma(alpha, pv.y, xv.y);
            reinterpret_cast<double2*>(x)[i] = xv;
            if (more) {
                const double2 rv = reinterpret_cast<const double2*>(r)[i];
                reinterpret_cast<double2*>(p)[i] = make_double2(fma(beta, pv.x, rv.x), fma(beta, pv.y, rv.y));
            }
        }
        i0 = 2 * nv;
    }
    for (int64_t i = i0 + tid; i < n; i += nth) {
        const double pi = p[i];
        x[i] = fma(alpha, pi, x[i]);
        if (more) p[i] = fma(beta, pi, r[i]);
    }
}

static bool aligned16(const void* a) { return (reinterpret_cast<uintptr_t>(a) & 15) == 0; }

// ------------------------------------------------ Jacobi preconditioning

// dinv[i] = 1 / a_ii (rows sorted by column: the first entry >= i); a zero
// or missing diagonal sets *bad (the preconditioner does not exist)
__global__ void diag_inv_kernel(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const double* __restrict__ val, double* __restrict__ dinv, int32_t* bad)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double d = 0.0;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            if (col[k] >= i) {
                if (col[k] == i) d = val[k];
                break;
            }
        dinv[i] = d != 0.0 ? 1.0 / d : 0.0;
        if (!(d != 0.0)) atomicOr(bad, 1);
    }
}

// p = D^-1 r + beta p (beta_mode 0: the state's beta; 1: beta = 0, the
// initial direction)
__global__ void __launch_bounds__(kRedThreads)
    pcg_pupdate_kernel(int64_t n, double* __restrict__ p, const double* __restrict__ r,
                       const double* __restrict__ dinv, const SolverState* s, int force, int initial)
{
    if (s->done && !force) return;
    const double beta = initial ? 0.0 : s->beta;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads)
        p[i] = initial ? r[i] * dinv[i] : fma(beta, p[i], r[i] * dinv[i]);
}

// rho = r.D^-1 r and the initial stop test on ||r|| (state: rho, dot_out = r.r)
__global__ void __launch_bounds__(kRedThreads)
    pcg_init_dots_kernel(int64_t n, const double* __restrict__ r, const double* __restrict__ dinv, SolverState* s,
                         double* part)
{
    double rr = 0.0, rz = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads) {
        const double ri = r[i];
        rr = fma(ri, ri, rr);
        rz = fma(ri, ri * dinv[i], rz);
    }
    grid_sum2(rr, rz, part, &s->ticket, [&](double rr0, double rz0) {
        s->rho = rz0;
        s->rho0 = rz0;
        s->dot_out = rr0;
        if (sqrt(rr0) <= s->tol * s->stop_ref) {
            s->conv = 1;
            s->status = GKO_OK;
            s->done = 1;
        }
    });
}

// Block-Jacobi PCG step, first half: x += alpha p; r -= alpha q; ||r||^2 and
// the stop tests (rho' = r.M^-1 r and beta come from the z kernel that
// follows, which needs the whole updated r)
__global__ void __launch_bounds__(kRedThreads)
    xr_update_kernel(int64_t n, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                     const double* __restrict__ q, SolverState* s, double* part, cudaGraphConditionalHandle h)
{
    if (s->done) return;
    const double alpha = s->alpha;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    grid_sum(acc, part, &s->ticket, [&](double rr) {
        if (!(rr == rr)) {
            s->status = GKO_ERR_BREAKDOWN;
            stop_loop(s, h);
            return;
        }
        s->dot_out = rr;
        if (sqrt(rr) <= s->tol * s->stop_ref) {
            s->conv = 1;
            s->status = GKO_OK;
            stop_loop(s, h);
        } else if (s->iter >= s->maxit) {
            s->status = GKO_ERR_NOT_CONVERGED;
            stop_loop(s, h);
        }
    });
}

// p = z + beta p (initial: p = z)
__global__ void __launch_bounds__(kRedThreads)
    zupdate_kernel(int64_t n, double* __restrict__ p, const double* __restrict__ z, const SolverState* s, int force,
                   int initial)
{
    if (s->done && !force) return;
    const double beta = initial ? 0.0 : s->beta;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads)
        p[i] = initial ? z[i] : fma(beta, p[i], z[i]);
}

// Jacobi PCG step regrouped like the plain one: r -= alpha q with
// ||r||^2 (stop tests) and rho' = r.D^-1 r (beta); then x += alpha p and
// p = D^-1 r + beta p in one pass (pcg_px_update_kernel)
__global__ void __launch_bounds__(kRedThreads)
    pcg_r_update_kernel(int64_t n, double* __restrict__ r, const double* __restrict__ q,
                        const double* __restrict__ dinv, SolverState* s, double* part, cudaGraphConditionalHandle h)
{
    if (s->done) return;
    const double alpha = s->alpha;
    double rr = 0.0, rz = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads) {
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        rr = fma(ri, ri, rr);
        rz = fma(ri, ri * dinv[i], rz);
    }
    grid_sum2(rr, rz, part, &s->ticket, [&](double rr_new, double rho_new) {
        if (!(rr_new == rr_new) || !(rho_new == rho_new)) {
            s->status = GKO_ERR_BREAKDOWN;
            stop_loop(s, h);
            return;
        }
        s->beta = rho_new / s->rho;
        s->rho = rho_new;
        s->dot_out = rr_new;
        if (sqrt(rr_new) <= s->tol * s->stop_ref) {
            s->conv = 1;
            s->status = GKO_OK;
            stop_loop(s, h);
        } else if (s->iter >= s->maxit) {
            s->status = GKO_ERR_NOT_CONVERGED;
            stop_loop(s, h);
        }
    });
}

// x += alpha p; then p = D^-1 r + beta p unless the solve stopped here
__global__ void __launch_bounds__(kRedThreads)
    pcg_px_update_kernel(int64_t n, double* __restrict__ x, double* __restrict__ p, const double* __restrict__ r,
                         const double* __restrict__ dinv, const SolverState* s)
{
    if (!s->step_ok) return;
    const double alpha = s->alpha, beta = s->beta;
    const bool more = !s->done;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads) {
        const double pi = p[i];
        x[i] = fma(alpha, pi, x[i]);
        if (more) p[i] = fma(beta, pi, r[i] * dinv[i]);
    }
}

static int red_grid(int64_t n)
{
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(kRedBlocks, (n + kRedThreads - 1) / kRedThreads)));
}

// ------------------------------------------- single-reduction CG kernels

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
};
template <>
struct Vec16<double> {
    using type = double2;
};

// One vector step of the single-reduction CG (Chronopoulos and Gear 1989):
//   p = r + beta p;  s = w + beta s;  x += alpha p;  r -= alpha s
// with alpha, beta from the product kernel's scalar step (s = A p is carried
// by recurrence, so no second product or reduction is needed).  kVec: all
// vectors 16-byte aligned, moved as 128-bit words.
// kPrec: preconditioned by a diagonal (dinv = its inverse): p = u + beta p
// with u = dinv r the preconditioned residual, and u is refreshed from the
// updated r.
template <typename T, bool kVec, bool kPrec = false>
__global__ void __launch_bounds__(kRedThreads)
    cg1_update_kernel(int64_t n, T* __restrict__ x, T* __restrict__ r, T* __restrict__ p, T* __restrict__ s,
                      const T* __restrict__ w, const SolverState* st, const T* __restrict__ dinv = nullptr,
                      T* __restrict__ u = nullptr)
{
    if (st->done) return;
    const T alpha = static_cast<T>(st->alpha), beta = static_cast<T>(st->beta);
    const int64_t tid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const int64_t nth = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int64_t i0 = 0;
    if (kVec) {
        using V = typename Vec16<T>::type;
        constexpr int W = 16 / sizeof(T);
        union U {
            V v;
            T a[W];
        };
        const int64_t nv = n / W;
        for (int64_t i = tid; i < nv; i += nth) {
            U rv, wv, pv, sv, xv, uv, dv;
            rv.v = reinterpret_cast<const V*>(r)[i];
            wv.v = reinterpret_cast<const V*>(w)[i];
            pv.v = reinterpret_cast<const V*>(p)[i];
            sv.v = reinterpret_cast<const V*>(s)[i];
            xv.v = reinterpret_cast<const V*>(x)[i];
            if (kPrec) {
                uv.v = reinterpret_cast<const V*>(u)[i];
                dv.v = reinterpret_cast<const V*>(dinv)[i];
            }
#pragma unroll
            for (int k = 0; k < W; ++k) {
                pv.a[k] = fma(beta, pv.a[k], kPrec ? uv.a[k] : rv.a[k]);
                sv.a[k] = fma(beta, sv.a[k], wv.a[k]);
                xv.a[k] = fma(alpha, pv.a[k], xv.a[k]);
                rv.a[k] = fma(-alpha, sv.a[k], rv.a[k]);
                if (kPrec) uv.a[k] = dv.a[k] * rv.a[k];
            }
            reinterpret_cast<V*>(p)[i] = pv.v;
            reinterpret_cast<V*>(s)[i] = sv.v;
            reinterpret_cast<V*>(x)[i] = xv.v;
            reinterpret_cast<V*>(r)[i] = rv.v;
            if (kPrec) reinterpret_cast<V*>(u)[i] = uv.v;
        }
        i0 = nv * W;
    }
    for (int64_t i = i0 + tid; i < n; i += nth) {
        const T pi = fma(beta, p[i], kPrec ? u[i] : r[i]);
        const T si = fma(beta, s[i], w[i]);
        p[i] = pi;
        s[i] = si;
        x[i] = fma(alpha, pi, x[i]);
        const T ri = fma(-alpha, si, r[i]);
        r[i] = ri;
        if (kPrec) u[i] = dinv[i] * ri;
    }
}

// gamma = r.r and delta = w.r with one grid reduction ending in the scalar
// step (for products by kernels that do not fuse the dots themselves)
// (with a preconditioner: gamma = rd.u and delta = w.u for u = M^-1 rd; here
// u is passed as r and the residual as rd; rd = r without one)
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    cg1_dots_kernel(int64_t n, const T* __restrict__ r, const T* __restrict__ rd, const T* __restrict__ w,
                    Cg1Reduce red)
{
    T g = T(0), d = T(0);
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads) {
        const T ri = r[i];
        g = fma(rd[i], ri, g);
        d = fma(w[i], ri, d);
    }
    SolverState* s = red.s;
    grid_sum2(static_cast<double>(g), static_cast<double>(d), red.part, &s->ticket,
              [&](double gamma, double delta) { cg1_scalars(s, gamma, delta, red.err, red.h); });
}

static int upd_grid(int64_t n)
{
    const int64_t v = (n + 3) / 4;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(152 * 8, (v + kRedThreads - 1) / kRedThreads)));
}

template <typename T>
static void launch_cg1_update(int64_t n, T* x, T* r, T* p, T* s, const T* w, const SolverState* st,
                              cudaStream_t cs, const T* dinv = nullptr, T* u = nullptr)
{
    const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(r) |
                       reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(s) |
                       reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(dinv) |
                       reinterpret_cast<uintptr_t>(u)) & 15) == 0;
    if (dinv) {
        if (vec)
            cg1_update_kernel<T, true, true><<<upd_grid(n), kRedThreads, 0, cs>>>(n, x, r, p, s, w, st, dinv, u);
        else
            cg1_update_kernel<T, false, true><<<upd_grid(n), kRedThreads, 0, cs>>>(n, x, r, p, s, w, st, dinv, u);
    } else if (vec) {
        cg1_update_kernel<T, true><<<upd_grid(n), kRedThreads, 0, cs>>>(n, x, r, p, s, w, st);
    } else {
        cg1_update_kernel<T, false><<<upd_grid(n), kRedThreads, 0, cs>>>(n, x, r, p, s, w, st);
    }
}

// dinv[i] = 1 / (diagonal of the rounded matrix A_lo) in FP32 (values in CSR
// order: float, or bf16 bits); a zero or missing diagonal sets *bad
template <int kBf16>
__global__ void diag_lo_inv_kernel(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                   const float* __restrict__ v32, const uint16_t* __restrict__ v16,
                                   float* __restrict__ dinv, int32_t* bad)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float d = 0.0f;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            if (col[k] >= i) {
                if (col[k] == i) d = kBf16 ? __uint_as_float(static_cast<uint32_t>(v16[k]) << 16) : v32[k];
                break;
            }
        dinv[i] = d != 0.0f ? 1.0f / d : 0.0f;
        if (!(d != 0.0f)) atomicOr(bad, 1);
    }
}

// ------------------------------------------------ host <-> device state

static int read_state(SolverState* h, const SolverState* d, cudaStream_t st)
{
    GKO_CUDA(cudaMemcpyAsync(h, d, sizeof(SolverState), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    return GKO_OK;
}

static int write_state(SolverState* d, const SolverState* h, cudaStream_t st)
{
    GKO_CUDA(cudaMemcpyAsync(d, h, sizeof(SolverState), cudaMemcpyHostToDevice, st));
    return GKO_OK;
}

static int spmv_fmt(const gko_matrix* A, int fmt, const double* x, double* y, double alpha, double beta,
                    cudaStream_t st)
{
    switch (fmt) {
        case GKO_FMT_CSR: return spmv_csr(A, GKO_CFG_DEFAULT, x, y, alpha, beta, st);
        case GKO_FMT_COO: return spmv_coo(A, A->coo, x, y, alpha, beta, st);
        case GKO_FMT_ELL: return spmv_ell(A, A->ell, x, y, alpha, beta, st);
        case GKO_FMT_SELLP: return spmv_sellp(A, x, y, alpha, beta, st);
        case GKO_FMT_HYBRID: return spmv_hybrid(A, x, y, alpha, beta, st);
    }
    return fail(GKO_ERR_INVALID_ARG, "unknown format");
}

// ||b - A x|| / ||b|| with the residual in FP64 (t is scratch of n)
static int true_residual(const gko_matrix* A, int fmt, const double* b, const double* x, double* t,
                         SolverState* ds, double* part, double bnorm, cudaStream_t st, double* out)
{
    const int64_t n = A->n_rows;
    GKO_CUDA(cudaMemcpyAsync(t, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    GKO_TRY(spmv_fmt(A, fmt, x, t, -1.0, 1.0, st));
    dot_kernel<double, kDotStore><<<red_grid(n), kRedThreads, 0, st>>>(n, t, t, ds, part, 0);
    GKO_CUDA(cudaGetLastError());
    double d = 0.0;
    GKO_CUDA(cudaMemcpyAsync(&d, &ds->dot_out, sizeof(double), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    *out = bnorm > 0.0 ? std::sqrt(d) / bnorm : std::sqrt(d);
    return GKO_OK;
}

static void fill_info(gko_solve_info* info, int iters, int outer, double res, int status)
{
    if (!info) return;
    info->iterations = iters;
    info->outer_iterations = outer;
    info->rel_residual = res;
    info->status = status;
    info->aux = 0;
}

// -------------------------------------------------------------- FP64 CG

// Hestenes-Stiefel CG; jacobi: preconditioned by the diagonal of A (the
// matrix's CSR part supplies the diagonal); bj: preconditioned by a
// block-Jacobi M (z = M^-1 r stored, two more launches per step).
static int cg_solve_impl(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit,
                         cudaStream_t st, gko_solve_info* info, bool jacobi, const gko_block_jacobi* bj = nullptr)
{
    const int64_t n = A->n_rows;
    if (n == 0) {
        fill_info(info, 0, 0, 0.0, GKO_OK);
        return GKO_OK;
    }
    Workspace ws(st);
    double *r, *p, *q, *part, *dinv = nullptr, *z = nullptr;
    SolverState* ds;
    GKO_TRY(ws.get(&r, n));
    GKO_TRY(ws.get(&p, n));
    GKO_TRY(ws.get(&q, n));
    GKO_TRY(ws.get(&part, 2 * kRedBlocks));
    GKO_TRY(ws.get(&ds, 1));
    const int grid = red_grid(n);
    if (bj) GKO_TRY(ws.get(&z, n));
    if (jacobi) {
        int32_t* bad;
        GKO_TRY(ws.get(&dinv, n));
        GKO_TRY(ws.get(&bad, 1));
        GKO_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), st));
        diag_inv_kernel<<<grid, kRedThreads, 0, st>>>(n, A->csr.row_ptr, A->csr.col, A->csr.val, dinv, bad);
        int32_t hbad = 0;
        GKO_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        GKO_CUDA(cudaStreamSynchronize(st));
        if (hbad) {
            fill_info(info, 0, 0, -1.0, GKO_ERR_BREAKDOWN);
            set_error("Jacobi preconditioner: a diagonal entry is zero or not stored");
            return GKO_ERR_BREAKDOWN;
        }
    }

    SolverState hs = {};
    GKO_TRY(write_state(ds, &hs, st));
    dot_kernel<double, kDotStore><<<grid, kRedThreads, 0, st>>>(n, b, b, ds, part, 0);
    GKO_TRY(read_state(&hs, ds, st));
    const double bnorm = std::sqrt(hs.dot_out);
    if (bnorm == 0.0) {
        GKO_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st));
        GKO_CUDA(cudaStreamSynchronize(st));
        fill_info(info, 0, 0, 0.0, GKO_OK);
        return GKO_OK;
    }
    // r = b - A x, p = r (D^-1 r), rho = r.r (r.D^-1 r)
    GKO_CUDA(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    GKO_TRY(spmv_fmt(A, fmt, x, r, -1.0, 1.0, st));
    hs = {};
    hs.tol = tol;
    hs.stop_ref = bnorm;
    hs.maxit = maxit;
    hs.status = GKO_ERR_NOT_CONVERGED;
    GKO_TRY(write_state(ds, &hs, st));
    if (bj) {
        bj_z_launch(bj, r, z, ds, part, grid, 0, kBjInit, 1, st);
        zupdate_kernel<<<grid, kRedThreads, 0, st>>>(n, p, z, ds, 1, 1);
    } else if (jacobi) {
        pcg_pupdate_kernel<<<grid, kRedThreads, 0, st>>>(n, p, r, dinv, ds, 1, 1);
        pcg_init_dots_kernel<<<grid, kRedThreads, 0, st>>>(n, r, dinv, ds, part);
    } else {
        GKO_CUDA(cudaMemcpyAsync(p, r, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        dot_kernel<double, kDotRhoInit><<<grid, kRedThreads, 0, st>>>(n, r, r, ds, part, 0);
    }
    GKO_TRY(read_state(&hs, ds, st));
    if (hs.conv) {  // r is the true residual here
        double res;
        GKO_TRY(true_residual(A, fmt, b, x, q, ds, part, bnorm, st, &res));
        fill_info(info, 0, 0, res, GKO_OK);
        return GKO_OK;
    }
    if (maxit == 0) {
        double res;
        GKO_TRY(true_residual(A, fmt, b, x, q, ds, part, bnorm, st, &res));
        fill_info(info, 0, 0, res, GKO_ERR_NOT_CONVERGED);
        return GKO_ERR_NOT_CONVERGED;
    }

    // plain CG on ELL: the product carries p.q (persistent grid, its own partials)
    const bool fused_pq = !bj && fmt == GKO_FMT_ELL && A->ell.K > 0;
    int pq_grid = 0;
    double* pq_part = part;
    if (fused_pq) {
        pq_grid = static_cast<int>(std::max<int64_t>(
            1, std::min<int64_t>((n + 511) / 512, static_cast<int64_t>(device_sm_count()) * 5)));
        if (pq_grid > 2 * kRedBlocks) GKO_TRY(ws.get(&pq_part, pq_grid));
    }
    GraphHolder gh;
    GKO_TRY(build_while_graph(&gh, [&](cudaGraphConditionalHandle h, cudaStream_t cs) -> int {
        if (fused_pq) {
            ell_pq_kernel<<<pq_grid, 256, 0, cs>>>(n, A->ell.n_pad, A->ell.K, A->ell.col, A->ell.val, p, q, ds,
                                                   pq_part, h);
        } else {
            GKO_TRY(spmv_fmt(A, fmt, p, q, 1.0, 0.0, cs));
            dot_kernel<double, kDotPQ><<<grid, kRedThreads, 0, cs>>>(n, p, q, ds, part, h, A->d_err);
        }
        if (bj) {
            xr_update_kernel<<<grid, kRedThreads, 0, cs>>>(n, x, r, p, q, ds, part, h);
            bj_z_launch(bj, r, z, ds, part, grid, h, kBjStep, 0, cs);
            zupdate_kernel<<<grid, kRedThreads, 0, cs>>>(n, p, z, ds, 0, 0);
        } else if (jacobi) {
            pcg_r_update_kernel<<<grid, kRedThreads, 0, cs>>>(n, r, q, dinv, ds, part, h);
            pcg_px_update_kernel<<<grid, kRedThreads, 0, cs>>>(n, x, p, r, dinv, ds);
        } else {
            // 2 * kRedBlocks partials fit the wider grid of the vector kernels
            const int vgrid = static_cast<int>(
                std::max<int64_t>(1, std::min<int64_t>(2 * kRedBlocks, (n / 2 + kRedThreads - 1) / kRedThreads)));
            if (aligned16(x)) {
                r_update_kernel<true><<<vgrid, kRedThreads, 0, cs>>>(n, r, q, ds, part, h);
                px_update_kernel<true><<<vgrid, kRedThreads, 0, cs>>>(n, x, p, r, ds);
            } else {
                r_update_kernel<false><<<grid, kRedThreads, 0, cs>>>(n, r, q, ds, part, h);
                px_update_kernel<false><<<grid, kRedThreads, 0, cs>>>(n, x, p, r, ds);
            }
        }
        GKO_CUDA(cudaGetLastError());
        return GKO_OK;
    }));

    int status = GKO_ERR_NOT_CONVERGED, checks = 0;
    double res = -1.0;
    while (true) {
        GKO_CUDA(cudaGraphLaunch(gh.exec, st));
        GKO_TRY(read_state(&hs, ds, st));
        if (hs.status == GKO_ERR_BREAKDOWN || hs.status == GKO_ERR_TIMEOUT) {
            status = hs.status;
            break;
        }
        if (hs.conv) {
            GKO_TRY(true_residual(A, fmt, b, x, q, ds, part, bnorm, st, &res));
            ++checks;
            if (res <= tol) {
                status = GKO_OK;
                break;
            }
            if (checks >= 4 || hs.iter >= maxit) {
                status = GKO_ERR_NOT_CONVERGED;
                break;
            }
            // not confirmed: finish this step (p = r + beta p) and go on
            hs.conv = 0;
            hs.done = 0;
            hs.status = GKO_ERR_NOT_CONVERGED;
            GKO_CUDA(cudaMemcpyAsync(ds, &hs, sizeof(SolverState), cudaMemcpyHostToDevice, st));
            if (bj) {
                bj_z_launch(bj, r, z, ds, part, grid, 0, kBjStep, 1, st);
                zupdate_kernel<<<grid, kRedThreads, 0, st>>>(n, p, z, ds, 1, 0);
            } else if (jacobi)
                pcg_pupdate_kernel<<<grid, kRedThreads, 0, st>>>(n, p, r, dinv, ds, 1, 0);
            else
                pupdate_kernel<double><<<grid, kRedThreads, 0, st>>>(n, p, r, ds, 1);
            res = -1.0;
            continue;
        }
        status = GKO_ERR_NOT_CONVERGED;  // maxit
        break;
    }
    if (res < 0.0) GKO_TRY(true_residual(A, fmt, b, x, q, ds, part, bnorm, st, &res));
    fill_info(info, hs.iter, 0, res, status);
    if (status != GKO_OK)
        set_error(status == GKO_ERR_BREAKDOWN ? "CG breakdown (p.q <= 0 or NaN)"
                  : status == GKO_ERR_TIMEOUT  ? "CG product: a bounded wait for a bulk copy gave up"
                                               : "CG reached maxit");
    return status;
}

int cg_solve(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit, cudaStream_t st,
             gko_solve_info* info)
{
    return cg_solve_impl(A, fmt, b, x, tol, maxit, st, info, false);
}

int pcg_jacobi_solve(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit,
                     cudaStream_t st, gko_solve_info* info)
{
    return cg_solve_impl(A, fmt, b, x, tol, maxit, st, info, true);
}

int pcg_block_jacobi_solve(const gko_matrix* A, int fmt, const gko_block_jacobi* M, const double* b, double* x,
                           double tol, int maxit, cudaStream_t st, gko_solve_info* info)
{
    return cg_solve_impl(A, fmt, b, x, tol, maxit, st, info, false, M);
}

// ------------------------------------------------ single-reduction CG

// The step's product w = A r with the dots and scalar step fused where the
// kernel allows it (row-block CSR), else the format's SpMV + one dot kernel.
static int cg1_product_f64(const gko_matrix* A, int fmt, const double* r, double* w, Cg1Reduce red, int grid,
                           cudaStream_t cs)
{
    const int64_t n = A->n_rows;
    if (fmt == GKO_FMT_CSR && A->nnz > 0 && default_csr_config(A) == GKO_CFG_CSR_ROWBLOCK) {
        const cudaError_t e = rowblock_cg1_f64(A, r, w, red, cs);
        return e == cudaSuccess ? GKO_OK : cuda_fail(e, "single-reduction CG product");
    }
    GKO_TRY(spmv_fmt(A, fmt, r, w, 1.0, 0.0, cs));
    cg1_dots_kernel<double><<<grid, kRedThreads, 0, cs>>>(n, r, r, w, red);
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

// CG in the single-reduction form of Chronopoulos and Gear (1989): per step
// one product w = A r fused with gamma = r.r, delta = w.r and the scalar
// step, then one vector update of p, s = A p, x and r.  Two launches and one
// grid reduction per step instead of four launches and two reductions.
// Stopping, confirmation by the true residual and breakdown as in cg_solve.
int cg1_solve(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit, cudaStream_t st,
              gko_solve_info* info)
{
    const int64_t n = A->n_rows;
    if (n == 0) {
        fill_info(info, 0, 0, 0.0, GKO_OK);
        return GKO_OK;
    }
    Workspace ws(st);
    double *r, *w, *p, *sv, *part;
    SolverState* ds;
    GKO_TRY(ws.get(&r, n));
    GKO_TRY(ws.get(&w, n));
    GKO_TRY(ws.get(&p, n));
    GKO_TRY(ws.get(&sv, n));
    GKO_TRY(ws.get(&part, 2 * kRedBlocks));
    GKO_TRY(ws.get(&ds, 1));
    const int grid = red_grid(n);

    SolverState hs = {};
    GKO_TRY(write_state(ds, &hs, st));
    dot_kernel<double, kDotStore><<<grid, kRedThreads, 0, st>>>(n, b, b, ds, part, 0);
    GKO_TRY(read_state(&hs, ds, st));
    const double bnorm = std::sqrt(hs.dot_out);
    if (bnorm == 0.0) {
        GKO_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st));
        GKO_CUDA(cudaStreamSynchronize(st));
        fill_info(info, 0, 0, 0.0, GKO_OK);
        return GKO_OK;
    }
    // r = b - A x; p = s = 0 (beta = 0 at the first step)
    GKO_CUDA(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    GKO_TRY(spmv_fmt(A, fmt, x, r, -1.0, 1.0, st));
    GKO_CUDA(cudaMemsetAsync(p, 0, n * sizeof(double), st));
    GKO_CUDA(cudaMemsetAsync(sv, 0, n * sizeof(double), st));
    hs = {};
    hs.tol = tol;
    hs.stop_ref = bnorm;
    hs.maxit = maxit;
    hs.status = GKO_ERR_NOT_CONVERGED;
    GKO_TRY(write_state(ds, &hs, st));

    GraphHolder gh;
    GKO_TRY(build_while_graph(&gh, [&](cudaGraphConditionalHandle h, cudaStream_t cs) -> int {
        const Cg1Reduce red{ds, part, A->d_err, h};
        GKO_TRY(cg1_product_f64(A, fmt, r, w, red, grid, cs));
        launch_cg1_update<double>(n, x, r, p, sv, w, ds, cs);
        GKO_CUDA(cudaGetLastError());
        return GKO_OK;
    }));

    int status = GKO_ERR_NOT_CONVERGED, checks = 0;
    double res = -1.0;
    while (true) {
        GKO_CUDA(cudaGraphLaunch(gh.exec, st));
        GKO_TRY(read_state(&hs, ds, st));
        if (hs.status == GKO_ERR_BREAKDOWN || hs.status == GKO_ERR_TIMEOUT) {
            status = hs.status;
            break;
        }
        if (hs.conv) {
            GKO_TRY(true_residual(A, fmt, b, x, w, ds, part, bnorm, st, &res));
            ++checks;
            if (res <= tol) {
                status = GKO_OK;
                break;
            }
            if (checks >= 4 || hs.iter >= maxit) {
                status = GKO_ERR_NOT_CONVERGED;
                break;
            }
            // not confirmed: take the step the test stopped and go on
            GKO_TRY(read_state(&hs, ds, st));  // true_residual used dot_out only
            hs.conv = 0;
            hs.done = 0;
            hs.skip_test = 1;
            hs.status = GKO_ERR_NOT_CONVERGED;
            GKO_TRY(write_state(ds, &hs, st));
            res = -1.0;
            continue;
        }
        status = GKO_ERR_NOT_CONVERGED;  // maxit
        break;
    }
    if (res < 0.0) GKO_TRY(true_residual(A, fmt, b, x, w, ds, part, bnorm, st, &res));
    fill_info(info, hs.iter, 0, res, status);
    if (status != GKO_OK)
        set_error(status == GKO_ERR_BREAKDOWN ? "CG breakdown (non-positive curvature or NaN)"
                  : status == GKO_ERR_TIMEOUT  ? "CG product: a bounded wait for a bulk copy gave up"
                                               : "CG reached maxit");
    return status;
}

// ------------------------------------------------------------ BiCGSTAB

// Device-resident scalars of BiCGSTAB (van der Vorst 1992).
struct BicgState {
    double rho;       // r^.r of the current residual (rho' of the coming step)
    double alpha, omega, beta;
    double rv, ss, tt, ts, rr;
    double stop_ref, tol;
    int32_t iter, maxit, done, status, conv, half;
    uint32_t ticket;
};

__device__ __forceinline__ void bicg_stop(BicgState* s, cudaGraphConditionalHandle h)
{
    s->done = 1;
    if (h) cudaGraphSetConditional(h, 0);
}

// p = r + beta (p - omega v)
__global__ void __launch_bounds__(kRedThreads)
    bicg_p_kernel(int64_t n, double* __restrict__ p, const double* __restrict__ r, const double* __restrict__ v,
                  const BicgState* s)
{
    if (s->done) return;
    const double beta = s->beta, omega = s->omega;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads)
        p[i] = fma(beta, fma(-omega, v[i], p[i]), r[i]);
}

// alpha = rho / (r^.v)
__global__ void __launch_bounds__(kRedThreads)
    bicg_alpha_kernel(int64_t n, const double* __restrict__ rh, const double* __restrict__ v, BicgState* s,
                      double* part, cudaGraphConditionalHandle h)
{
    if (s->done) return;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads)
        acc = fma(rh[i], v[i], acc);
    grid_sum(acc, part, &s->ticket, [&](double rv) {
        s->rv = rv;
        if (!(rv != 0.0) || !(rv == rv)) {
            s->status = GKO_ERR_BREAKDOWN;
            bicg_stop(s, h);
            return;
        }
        s->alpha = s->rho / rv;
    });
}

// s = r - alpha v, ss = s.s; a small s ends the step half way (x += alpha p
// is then taken by the host-side finish)
__global__ void __launch_bounds__(kRedThreads)
    bicg_s_kernel(int64_t n, double* __restrict__ sv, const double* __restrict__ r, const double* __restrict__ v,
                  BicgState* s, double* part, cudaGraphConditionalHandle h)
{
    if (s->done) return;
    const double alpha = s->alpha;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads) {
        const double si = fma(-alpha, v[i], r[i]);
        sv[i] = si;
        acc = fma(si, si, acc);
    }
    grid_sum(acc, part, &s->ticket, [&](double ss) {
        s->ss = ss;
        if (!(ss == ss)) {
            s->status = GKO_ERR_BREAKDOWN;
            bicg_stop(s, h);
        } else if (sqrt(ss) <= s->tol * s->stop_ref) {
            s->half = 1;
            s->conv = 1;
            s->status = GKO_OK;
            bicg_stop(s, h);
        }
    });
}

// omega = (t.s) / (t.t)
__global__ void __launch_bounds__(kRedThreads)
    bicg_omega_kernel(int64_t n, const double* __restrict__ t, const double* __restrict__ sv, BicgState* s,
                      double* part, cudaGraphConditionalHandle h)
{
    if (s->done) return;
    double tt = 0.0, ts = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads) {
        const double ti = t[i];
        tt = fma(ti, ti, tt);
        ts = fma(ti, sv[i], ts);
    }
    grid_sum2(tt, ts, part, &s->ticket, [&](double tt_, double ts_) {
        s->tt = tt_;
        s->ts = ts_;
        const double omega = ts_ / tt_;
        if (!(tt_ > 0.0) || !(omega != 0.0) || !(omega == omega)) {
            s->status = GKO_ERR_BREAKDOWN;
            bicg_stop(s, h);
            return;
        }
        s->omega = omega;
    });
}

// x += alpha p + omega s; r = s - omega t; rho' = r^.r, rr = r.r; then the
// next step's beta and the stop tests
__global__ void __launch_bounds__(kRedThreads)
    bicg_xr_kernel(int64_t n, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                   const double* __restrict__ sv, const double* __restrict__ t, const double* __restrict__ rh,
                   BicgState* s, double* part, cudaGraphConditionalHandle h)
{
    if (s->done) return;
    const double alpha = s->alpha, omega = s->omega;
    double rho = 0.0, rr = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads) {
        x[i] = fma(omega, sv[i], fma(alpha, p[i], x[i]));
        const double ri = fma(-omega, t[i], sv[i]);
        r[i] = ri;
        rho = fma(rh[i], ri, rho);
        rr = fma(ri, ri, rr);
    }
    grid_sum2(rho, rr, part, &s->ticket, [&](double rho_next, double rr_) {
        s->iter += 1;
        s->rr = rr_;
        if (!(rr_ == rr_) || !(rho_next == rho_next)) {
            s->status = GKO_ERR_BREAKDOWN;
            bicg_stop(s, h);
            return;
        }
        s->beta = (rho_next / s->rho) * (s->alpha / s->omega);
        s->rho = rho_next;
        if (sqrt(rr_) <= s->tol * s->stop_ref) {
            s->conv = 1;
            s->status = GKO_OK;
            bicg_stop(s, h);
        } else if (s->iter >= s->maxit) {
            s->status = GKO_ERR_NOT_CONVERGED;
            bicg_stop(s, h);
        } else if (!(rho_next != 0.0)) {
            s->status = GKO_ERR_BREAKDOWN;
            bicg_stop(s, h);
        }
    });
}

// x += alpha p (the half step)
__global__ void bicg_half_kernel(int64_t n, double* __restrict__ x, const double* __restrict__ p,
                                 const BicgState* s)
{
    const double alpha = s->alpha;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        x[i] = fma(alpha, p[i], x[i]);
}

// r^ = r; p = v = 0; rho = r^.r (and rr); used at the start and to restart
// from a true residual that did not confirm a half step
__global__ void __launch_bounds__(kRedThreads)
    bicg_restart_kernel(int64_t n, const double* __restrict__ r, double* __restrict__ rh, double* __restrict__ p,
                        double* __restrict__ v, BicgState* s, double* part)
{
    double acc = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads) {
        const double ri = r[i];
        rh[i] = ri;
        p[i] = 0.0;
        v[i] = 0.0;
        acc = fma(ri, ri, acc);
    }
    grid_sum(acc, part, &s->ticket, [&](double rr) {
        s->rho = rr;
        s->rr = rr;
        s->alpha = s->omega = 1.0;
        s->beta = 0.0;
        s->conv = s->half = s->done = 0;
        s->status = GKO_ERR_NOT_CONVERGED;
        if (sqrt(rr) <= s->tol * s->stop_ref) {
            s->conv = 1;
            s->status = GKO_OK;
            s->done = 1;
        } else if (!(rr == rr)) {
            s->status = GKO_ERR_BREAKDOWN;
            s->done = 1;
        }
    });
}

// BiCGSTAB on A x = b (general square A).  Steps: p update, v = A p,
// alpha, s = r - alpha v (+ ||s||), t = A s, omega, x/r update (+ r^.r,
// ||r||): seven launches per step inside the graph's WHILE node.  A step
// that ends half way (||s|| small) or a converged step is confirmed by the
// FP64 true residual; an unconfirmed half step restarts from the true
// residual (r^ = r), an unconfirmed full step continues (up to four checks).
int bicgstab_solve(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit,
                   cudaStream_t st, gko_solve_info* info)
{
    const int64_t n = A->n_rows;
    if (n == 0) {
        fill_info(info, 0, 0, 0.0, GKO_OK);
        return GKO_OK;
    }
    Workspace ws(st);
    double *r, *rh, *p, *v, *sv, *t, *part;
    SolverState* ds;
    BicgState* bs;
    GKO_TRY(ws.get(&r, n));
    GKO_TRY(ws.get(&rh, n));
    GKO_TRY(ws.get(&p, n));
    GKO_TRY(ws.get(&v, n));
    GKO_TRY(ws.get(&sv, n));
    GKO_TRY(ws.get(&t, n));
    GKO_TRY(ws.get(&part, 2 * kRedBlocks));
    GKO_TRY(ws.get(&ds, 1));
    GKO_TRY(ws.get(&bs, 1));
    const int grid = red_grid(n);

    SolverState hs = {};
    GKO_TRY(write_state(ds, &hs, st));
    dot_kernel<double, kDotStore><<<grid, kRedThreads, 0, st>>>(n, b, b, ds, part, 0);
    GKO_TRY(read_state(&hs, ds, st));
    const double bnorm = std::sqrt(hs.dot_out);
    if (bnorm == 0.0) {
        GKO_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st));
        GKO_CUDA(cudaStreamSynchronize(st));
        fill_info(info, 0, 0, 0.0, GKO_OK);
        return GKO_OK;
    }
    BicgState hb = {};
    hb.tol = tol;
    hb.stop_ref = bnorm;
    hb.maxit = maxit;
    hb.status = GKO_ERR_NOT_CONVERGED;
    auto put = [&]() -> int {
        GKO_CUDA(cudaMemcpyAsync(bs, &hb, sizeof(BicgState), cudaMemcpyHostToDevice, st));
        return GKO_OK;
    };
    auto get = [&]() -> int {
        GKO_CUDA(cudaMemcpyAsync(&hb, bs, sizeof(BicgState), cudaMemcpyDeviceToHost, st));
        GKO_CUDA(cudaStreamSynchronize(st));
        return GKO_OK;
    };
    auto restart = [&]() -> int {  // r = b - A x, r^ = r, p = v = 0
        GKO_CUDA(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        GKO_TRY(spmv_fmt(A, fmt, x, r, -1.0, 1.0, st));
        bicg_restart_kernel<<<grid, kRedThreads, 0, st>>>(n, r, rh, p, v, bs, part);
        GKO_CUDA(cudaGetLastError());
        return get();
    };
    GKO_TRY(put());
    GKO_TRY(restart());
    double res = -1.0;
    if (hb.conv || maxit == 0 || hb.status == GKO_ERR_BREAKDOWN) {
        GKO_TRY(true_residual(A, fmt, b, x, t, ds, part, bnorm, st, &res));
        const int st0 = hb.conv ? GKO_OK : hb.status;
        fill_info(info, 0, 0, res, st0);
        return st0;
    }

    GraphHolder gh;
    GKO_TRY(build_while_graph(&gh, [&](cudaGraphConditionalHandle h, cudaStream_t cs) -> int {
        bicg_p_kernel<<<grid, kRedThreads, 0, cs>>>(n, p, r, v, bs);
        GKO_TRY(spmv_fmt(A, fmt, p, v, 1.0, 0.0, cs));
        bicg_alpha_kernel<<<grid, kRedThreads, 0, cs>>>(n, rh, v, bs, part, h);
        bicg_s_kernel<<<grid, kRedThreads, 0, cs>>>(n, sv, r, v, bs, part, h);
        GKO_TRY(spmv_fmt(A, fmt, sv, t, 1.0, 0.0, cs));
        bicg_omega_kernel<<<grid, kRedThreads, 0, cs>>>(n, t, sv, bs, part, h);
        bicg_xr_kernel<<<grid, kRedThreads, 0, cs>>>(n, x, r, p, sv, t, rh, bs, part, h);
        GKO_CUDA(cudaGetLastError());
        return GKO_OK;
    }));

    int status = GKO_ERR_NOT_CONVERGED, checks = 0, steps = 0;
    while (true) {
        GKO_CUDA(cudaGraphLaunch(gh.exec, st));
        GKO_TRY(get());
        steps = hb.iter + (hb.half ? 1 : 0);
        if (hb.status == GKO_ERR_BREAKDOWN) {
            status = GKO_ERR_BREAKDOWN;
            break;
        }
        if (hb.conv) {
            if (hb.half) {
                bicg_half_kernel<<<grid, kRedThreads, 0, st>>>(n, x, p, bs);
                GKO_CUDA(cudaGetLastError());
            }
            GKO_TRY(true_residual(A, fmt, b, x, t, ds, part, bnorm, st, &res));
            ++checks;
            if (res <= tol) {
                status = GKO_OK;
                break;
            }
            if (checks >= 4 || steps >= maxit) {
                status = GKO_ERR_NOT_CONVERGED;
                break;
            }
            const int it_done = steps;
            if (hb.half) {  // restart from the true residual of the half-step iterate
                GKO_TRY(restart());
                hb.iter = it_done;
                hb.half = 0;
                GKO_TRY(put());
            } else {  // continue from the recursive residual
                hb.conv = 0;
                hb.done = 0;
                hb.status = GKO_ERR_NOT_CONVERGED;
                GKO_TRY(put());
            }
            res = -1.0;
            continue;
        }
        status = GKO_ERR_NOT_CONVERGED;  // maxit
        break;
    }
    if (res < 0.0) GKO_TRY(true_residual(A, fmt, b, x, t, ds, part, bnorm, st, &res));
    fill_info(info, steps, 0, res, status);
    if (status != GKO_OK)
        set_error(status == GKO_ERR_BREAKDOWN ? "BiCGSTAB breakdown (r^.v, t.t or omega zero, or NaN)"
                                              : "BiCGSTAB reached maxit");
    return status;
}

// --------------------------------------------------------------- GMRES


// Device-resident state of one GMRES(m) cycle.  H is (m + 1) x m row-major;
// g the rotated right-hand side of the least-squares problem.
struct GmState {
    double bnorm, tol;  // stop when |g[j]| <= tol * bnorm
    double hn;          // norm of the vector just orthogonalised
    double hn_inv;      // 1 / hn
    int32_t j;          // Arnoldi steps done in this cycle (columns of H)
    int32_t m, total, maxit;
    int32_t stop, broke;
    int32_t low_steps;  // steps whose second Gram-Schmidt update ran in FP32
    int32_t next_col;   // column of v_{j+1}
    uint32_t ticket;
    // second update of this step (set by the last block of the second
    // coefficient sums): low = FP32 path, its coefficients hf * sc, and hn
    // from ||w1||^2 - ||h2||^2
    int32_t low;
    uint32_t coef_ticket;
    double sc;
    float hf[128];
    double beta0;        // ||r|| of the residual the cycle starts from
    int32_t restart_ok;  // the cycle runs (no convergence, breakdown or maxit yet)
};

// The block's share of V_c . w for the CNT columns c0 .. c0+CNT-1 into
// part[blk * ldp + c]; CNT is exact, so no FP64 slot is spent on a
// predicated-off column (they cost the FP64 pipe as much as live ones).
template <int CNT>
__device__ __forceinline__ void gm_chunk_dots(int64_t n, const double* __restrict__ V, int c0,
                                              const double* __restrict__ w, double* __restrict__ part, int ldp,
                                              double (*sh)[kRedThreads / 32])
{
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const double* Vc = V + static_cast<int64_t>(c0) * n;
    double acc[CNT];
#pragma unroll
    for (int c = 0; c < CNT; ++c) acc[c] = 0.0;
    const int64_t nth = static_cast<int64_t>(gridDim.x) * kRedThreads;
    int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x;
    for (; i + nth < n; i += 2 * nth) {  // two rows per pass: twice the loads in flight
        const double w0 = w[i], w1 = w[i + nth];
        double v0[CNT], v1[CNT];
#pragma unroll
        for (int c = 0; c < CNT; ++c) {
            v0[c] = Vc[c * n + i];
            v1[c] = Vc[c * n + i + nth];
        }
#pragma unroll
        for (int c = 0; c < CNT; ++c) acc[c] = fma(v1[c], w1, fma(v0[c], w0, acc[c]));
    }
    if (i < n) {
        const double wi = w[i];
#pragma unroll
        for (int c = 0; c < CNT; ++c) acc[c] = fma(Vc[c * n + i], wi, acc[c]);
    }
    // warp sums by reduce-scatter: P (CNT rounded up to a power of two)
    // partial sums per lane; at distance d = 16, 8, ... each lane keeps the
    // half of its columns picked by bit d of its lane and adds the partner's
    // partials of them (P - 1 FP64 adds), then plain butterfly steps finish
    // the sum: P - 1 + 5 - log2(P) adds per lane instead of 5 CNT.
    constexpr int P = CNT > 4 ? 8 : CNT > 2 ? 4 : CNT;
    constexpr int LOG_P = P == 8 ? 3 : P == 4 ? 2 : P == 2 ? 1 : 0;
    double v[P];
#pragma unroll
    for (int c = 0; c < P; ++c) v[c] = c < CNT ? acc[c] : 0.0;
    int col = 0;
#pragma unroll
    for (int step = 0, K = P; step < LOG_P; ++step, K /= 2) {
        const int d = 16 >> step;
        const bool upper = (lane & d) != 0;
#pragma unroll
        for (int q = 0; q < K / 2; ++q) {
            const double send = upper ? v[q] : v[q + K / 2];
            const double keep = upper ? v[q + K / 2] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, d);
        }
        if (upper) col += K / 2;
    }
#pragma unroll
    for (int d = 16 >> LOG_P; d; d >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], d);
    // lanes whose bits below the reduce-scatter distances are zero hold column col
    if ((lane & ((16 >> LOG_P) * 2 - 1)) == 0 && col < CNT) sh[col][wp] = v[0];
    __syncthreads();
    if (threadIdx.x < CNT) {
        double t = 0.0;
        for (int k = 0; k < kRedThreads / 32; ++k) t += sh[threadIdx.x][k];
        part[blockIdx.x * static_cast<int64_t>(ldp) + c0 + threadIdx.x] = t;
    }
    __syncthreads();
}

constexpr int kGmChunk = 8;  // basis vectors per pass of the multi-dot loops

// part[blk * ldp + c] = the block's share of V_c . w for every c < ncols,
// in chunks of kGmChunk columns (ncols block-uniform).
__device__ __forceinline__ void gm_partial_dots(int64_t n, const double* __restrict__ V, int ncols,
                                                const double* __restrict__ w, double* __restrict__ part, int ldp)
{
    __shared__ double sh[kGmChunk][kRedThreads / 32];
    for (int c0 = 0; c0 < ncols; c0 += kGmChunk) {
        switch (min(kGmChunk, ncols - c0)) {
            case 8: gm_chunk_dots<8>(n, V, c0, w, part, ldp, sh); break;
            case 7: gm_chunk_dots<7>(n, V, c0, w, part, ldp, sh); break;
            case 6: gm_chunk_dots<6>(n, V, c0, w, part, ldp, sh); break;
            case 5: gm_chunk_dots<5>(n, V, c0, w, part, ldp, sh); break;
            case 4: gm_chunk_dots<4>(n, V, c0, w, part, ldp, sh); break;
            case 3: gm_chunk_dots<3>(n, V, c0, w, part, ldp, sh); break;
            case 2: gm_chunk_dots<2>(n, V, c0, w, part, ldp, sh); break;
            default: gm_chunk_dots<1>(n, V, c0, w, part, ldp, sh); break;
        }
    }
}

// w[i] -= sum_{c < nc} h[c] V_c[i] (in column order) for this thread's
// grid-stride rows, two rows per pass (two independent FMA chains, loads
// unrolled ahead of them); *sq, when given, accumulates the squares of the
// new entries.
__device__ __forceinline__ void gm_project_rows(const double* __restrict__ V, int64_t n, const double* hs, int nc,
                                                double* __restrict__ w, double* sq)
{
    const int64_t nth = static_cast<int64_t>(gridDim.x) * kRedThreads;
    int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x;
    double acc = 0.0;
    for (; i + nth < n; i += 2 * nth) {
        double t0 = w[i], t1 = w[i + nth];
#pragma unroll 8
        for (int c = 0; c < nc; ++c) {
            const double h = -hs[c];
            t0 = fma(h, V[c * n + i], t0);
            t1 = fma(h, V[c * n + i + nth], t1);
        }
        w[i] = t0;
        w[i + nth] = t1;
        if (sq) acc = fma(t1, t1, fma(t0, t0, acc));
    }
    if (i < n) {
        double t = w[i];
        for (int c = 0; c < nc; ++c) t = fma(-hs[c], V[c * n + i], t);
        w[i] = t;
        if (sq) acc = fma(t, t, acc);
    }
    if (sq) *sq = acc;
}

// First Gram-Schmidt pass: partial dots of V_0..V_j with w = A v_j.
__global__ void __launch_bounds__(kRedThreads, 4)
    gm_dots_kernel(int64_t n, const double* __restrict__ V, const double* __restrict__ w, double* __restrict__ part,
                   int ldp, const GmState* s)
{
    gm_partial_dots(n, V, s->j + 1, w, part, ldp);
}

// coef[c] = sum over blocks of part[b * ldp + c] (block c of the grid sums
// column c in a fixed tree order) for c <= j; hh[c] = coef[c] on the first
// pass, hh[c] += coef[c] on the second, whose column j + 1 holds ||w1||^2
// (no Hessenberg entry).
__global__ void __launch_bounds__(kRedThreads)
    gm_coef_kernel(int nblocks, const double* __restrict__ part, int ldp, double* __restrict__ coef,
                   double* __restrict__ hh, int second, GmState* s)
{
    __shared__ double sh[32];
    __shared__ bool last;
    const int c = blockIdx.x, j = s->j;
    if (c > j + (second ? 1 : 0)) return;  // block-uniform
    double t = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kRedThreads) t += part[b * static_cast<int64_t>(ldp) + c];
    t = block_sum(t, sh);
    if (threadIdx.x == 0) {
        coef[c] = t;
        if (c <= j) hh[c] = second ? hh[c] + t : t;
    }
    if (!second) return;
    // the second pass: the last of its j + 2 blocks decides the update's
    // precision once for the step (see gm_combine_norm_kernel)
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&s->coef_ticket, 1u) == static_cast<unsigned>(j + 1);
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    const int ncols = j + 1;
    double hm = 0.0, h2 = 0.0;
    for (int q = threadIdx.x; q < ncols; q += 32) {
        const double h = __ldcg(coef + q);
        hm = fmax(hm, fabs(h));
        h2 = fma(h, h, h2);
    }
    for (int o = 16; o; o >>= 1) {
        hm = fmax(hm, __shfl_xor_sync(0xffffffffu, hm, o));
        h2 += __shfl_xor_sync(0xffffffffu, h2, o);
    }
    const double w1n2 = __ldcg(coef + ncols);
    const double hn2 = w1n2 - h2;  // ||w2||^2: w1 is orthogonal to the basis up to rounding
    const bool low = hm <= ldexp(sqrt(w1n2), -33) && hn2 > 0.0 && hn2 < INFINITY;  // false on NaN
    int e = 0;
    if (low && hm > 0.0) frexp(hm, &e);  // hm < 2^e <= 2 hm
    const double isc = ldexp(1.0, -e);   // scaling by a power of two is exact
    if (low)
        for (int q = threadIdx.x; q < ncols; q += 32) s->hf[q] = static_cast<float>(__ldcg(coef + q) * isc);
    if (threadIdx.x == 0) {
        s->low = low;
        s->sc = ldexp(1.0, e);
        s->coef_ticket = 0;
        if (low) {
            const double hn = sqrt(hn2);
            s->hn = hn;
            s->hn_inv = 1.0 / hn;
            s->next_col = j + 1;
            s->low_steps += 1;
        }
    }
}

// w -= sum_{c <= j} coef[c] V_c, then the partial dots of V_0..V_j with the
// updated w1 (the second Gram-Schmidt pass; its dots re-read the V entries
// this thread has just read, mostly from L2) and the partial ||w1||^2 as
// column j + 1.
__global__ void __launch_bounds__(kRedThreads, 4)
    gm_combine_dots_kernel(int64_t n, const double* __restrict__ V, double* __restrict__ w,
                           const double* __restrict__ coef, double* __restrict__ part, int ldp, const GmState* s)
{
    __shared__ double hs[128];
    const int ncols = s->j + 1;
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) hs[c] = coef[c];
    __syncthreads();
    double sq;
    gm_project_rows(V, n, hs, ncols, w, &sq);
    {
        __shared__ double shq[32];
        sq = block_sum(sq, shq);
        if (threadIdx.x == 0) part[blockIdx.x * static_cast<int64_t>(ldp) + ncols] = sq;  // ||w1||^2
    }
    // each thread reads back only the w entries it wrote: no grid barrier needed
    gm_partial_dots(n, V, ncols, w, part, ldp);
}

// Column j of the Hessenberg matrix: hh[0..j] and hn; the earlier Givens
// rotations applied to it, a new rotation zeroing its subdiagonal, the
// least-squares right-hand side g rotated, the cycle's stop decided (residual
// estimate |g[j+1]| <= tol ||b||, m columns, maxit steps in all, a zero hn,
// or a breakdown: NaN or a zero rotation).  The block stages the column and
// the rotations in shared memory; thread 0 applies them.
__device__ __forceinline__ void gm_givens_block(double* __restrict__ H, double* __restrict__ cs,
                                                double* __restrict__ sn, double* __restrict__ g,
                                                const double* __restrict__ hh, GmState* s,
                                                cudaGraphConditionalHandle h, int j)
{
    __shared__ double col[129], c_s[128], s_s[128];
    const int m = s->m;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        col[i] = hh[i];
        c_s[i] = cs[i];
        s_s[i] = sn[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double hn = s->hn;
        s->total += 1;
        bool stop = false;
        if (!(hn == hn)) {
            s->broke = 1;
            stop = true;
        } else {
            col[j + 1] = hn;
            for (int i = 0; i < j; ++i) {  // earlier rotations on the new column
                const double a = col[i], c = col[i + 1];
                col[i] = c_s[i] * a + s_s[i] * c;
                col[i + 1] = -s_s[i] * a + c_s[i] * c;
            }
            const double a = col[j], c = col[j + 1];
            const double d = sqrt(a * a + c * c);
            if (!(d > 0.0)) {
                s->broke = 1;
                stop = true;
            } else {
                cs[j] = a / d;
                sn[j] = c / d;
                col[j] = d;
                col[j + 1] = 0.0;
                const double gj = g[j];
                g[j + 1] = -(c / d) * gj;
                g[j] = (a / d) * gj;
                s->j = j + 1;
                stop = fabs(g[j + 1]) <= s->tol * s->bnorm || !(hn > 0.0) || j + 1 >= m || s->total >= s->maxit;
            }
        }
        if (stop) {
            s->stop = 1;
            cudaGraphSetConditional(h, 0);
        }
    }
    __syncthreads();
    if (!s->broke)
        for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) H[i * m + j] = col[i];
}

// v = (w1 - sum_{c < nc} h[c] V_c[i]) / hn with the sum formed in FP32 from
// the float copy of the basis: h[c] = hf[c] * sc (sc a power of two,
// |hf| < 1), the float sum converted exactly and applied by one FP64 FMA;
// v goes to the next basis column, its float copy and vcur.  Two rows per
// pass.
__device__ __forceinline__ void gm_correct_rows_f32(const float* __restrict__ Vf, int64_t n, const float* hf, int nc,
                                                    double sc, const double* __restrict__ w, double inv_hn,
                                                    double* __restrict__ vnext, float* __restrict__ vnextf,
                                                    double* __restrict__ vcur)
{
    const int64_t nth = static_cast<int64_t>(gridDim.x) * kRedThreads;
    int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x;
    for (; i + nth < n; i += 2 * nth) {
        const double w0 = w[i], w1 = w[i + nth];  // issued before the column loop
        float c0 = 0.0f, c1 = 0.0f;
#pragma unroll 8
        for (int c = 0; c < nc; ++c) {
            c0 = fmaf(hf[c], Vf[c * n + i], c0);
            c1 = fmaf(hf[c], Vf[c * n + i + nth], c1);
        }
        const double v0 = fma(-sc, static_cast<double>(c0), w0) * inv_hn;
        const double v1 = fma(-sc, static_cast<double>(c1), w1) * inv_hn;
        vnext[i] = v0;
        vnext[i + nth] = v1;
        vnextf[i] = static_cast<float>(v0);
        vnextf[i + nth] = static_cast<float>(v1);
        vcur[i] = v0;
        vcur[i + nth] = v1;
    }
    if (i < n) {
        float c0 = 0.0f;
        for (int c = 0; c < nc; ++c) c0 = fmaf(hf[c], Vf[c * n + i], c0);
        const double v = fma(-sc, static_cast<double>(c0), w[i]) * inv_hn;
        vnext[i] = v;
        vnextf[i] = static_cast<float>(v);
        vcur[i] = v;
    }
}

// Second Gram-Schmidt update w2 = w1 - sum_{c <= j} coef[c] V_c and the
// next basis vector v = w2 / ||w2||.  The second pass's coefficients are
// rounding-level corrections: when max |coef| <= 2^-33 ||w1|| (decided once
// by gm_coef_kernel, s->low) the update runs in FP32 on the float copy of
// the basis, whose error (below 2^-23 sqrt(j + 1) max |coef|) then stays
// under the FP64 rounding of w1 itself; ||w2|| is then known beforehand
// (||w1||^2 - ||coef||^2, no cancellation at that size) and v is written
// here.  Otherwise the update runs in FP64, ||w2|| is reduced over the grid
// (the last block stores it) and gm_next_vector_kernel normalises.
__global__ void __launch_bounds__(kRedThreads, 4)
    gm_combine_norm_kernel(int64_t n, double* __restrict__ V, float* __restrict__ Vf, double* __restrict__ w,
                           double* __restrict__ vcur, const double* __restrict__ coef, double* __restrict__ part,
                           GmState* s)
{
    __shared__ double hs[128];
    __shared__ float hf[128];
    const int j = s->j, ncols = j + 1;
    if (s->low) {  // the same for every block
        for (int c = threadIdx.x; c < ncols; c += blockDim.x) hf[c] = s->hf[c];
        __syncthreads();
        gm_correct_rows_f32(Vf, n, hf, ncols, s->sc, w, s->hn_inv, V + (j + 1) * n, Vf + (j + 1) * n, vcur);
        return;
    }
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) hs[c] = coef[c];
    __syncthreads();
    double acc;
    gm_project_rows(V, n, hs, ncols, w, &acc);
    grid_sum(acc, part, &s->ticket, [&](double tot) {
        s->hn = sqrt(tot);
        s->hn_inv = 1.0 / s->hn;
        s->next_col = j + 1;
    });
}

// The Givens step of column j = s->j.
__global__ void __launch_bounds__(128)
    gm_givens_kernel(double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                     double* __restrict__ g, const double* __restrict__ hh, GmState* s, cudaGraphConditionalHandle h)
{
    gm_givens_block(H, cs, sn, g, hh, s, h, s->j);
}

// After an FP64 second update: v_{j+1} = w / hn (as w * (1 / hn): one FP64
// division per step instead of one per entry) into basis column
// s->next_col, its float copy and vcur (the next product's input); nothing
// when hn is zero or not finite (the cycle stops there).
__global__ void gm_next_vector_kernel(int64_t n, double* __restrict__ V, float* __restrict__ Vf,
                                      double* __restrict__ vcur, const double* __restrict__ w, const GmState* s)
{
    const double hn = s->hn;
    if (s->low || !(hn > 0.0) || !(hn < INFINITY)) return;  // s->low: written by the norm kernel
    const double inv = s->hn_inv;
    double* dst = V + static_cast<int64_t>(s->next_col) * n;
    float* dstf = Vf + static_cast<int64_t>(s->next_col) * n;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double v = w[i] * inv;
        dst[i] = v;
        dstf[i] = static_cast<float>(v);
        vcur[i] = v;
    }
}

// y = H(0:j, 0:j)^-1 g(0:j) by back substitution (H and g staged in shared
// memory by the block, solved by thread 0).
__global__ void __launch_bounds__(128)
    gm_backsub_kernel(const double* __restrict__ H, const double* __restrict__ g, double* __restrict__ y,
                      const GmState* s)
{
    extern __shared__ double hs[];
    if (s->broke) return;  // x stays as it was
    const int j = s->j, m = s->m;
    double* gs = hs + static_cast<size_t>(j) * j;
    for (int t = threadIdx.x; t < j * j; t += blockDim.x) hs[t] = H[(t / j) * m + t % j];
    for (int t = threadIdx.x; t < j; t += blockDim.x) gs[t] = g[t];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = j - 1; i >= 0; --i) {
            double acc = gs[i];
            for (int k = i + 1; k < j; ++k) acc -= hs[i * j + k] * gs[k];
            gs[i] = acc / hs[i * j + i];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < j; t += blockDim.x) y[t] = gs[t];
}

// x += sum_{c < j} y[c] V_c
__global__ void __launch_bounds__(kRedThreads)
    gm_update_x_kernel(int64_t n, double* __restrict__ x, const double* __restrict__ V, const double* __restrict__ y,
                       const GmState* s)
{
    __shared__ double ys[128];
    if (s->broke) return;
    const int ncols = s->j;
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) ys[c] = y[c];
    __syncthreads();
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads) {
        double t = x[i];
        for (int c = 0; c < ncols; ++c) t = fma(ys[c], V[c * n + i], t);
        x[i] = t;
    }
}

// Start of a cycle, from beta^2 = ||r||^2 of the residual r = b - A x
// (in V_0): the cycle runs unless ||r|| <= tol ||b||, beta is not a number,
// the previous cycle broke down or maxit steps are spent; if it runs, the
// cycle's state is reset and g = (beta, 0, ..., 0).  One thread.
__global__ void gm_restart_kernel(const SolverState* ds, GmState* s, double* __restrict__ g)
{
    const double beta = sqrt(ds->dot_out);
    s->beta0 = beta;
    const bool run = !s->broke && beta == beta && !(beta <= s->tol * s->bnorm) && s->total < s->maxit;
    s->restart_ok = run;
    if (!run) return;
    s->j = 0;
    s->stop = 0;
    s->hn = 0.0;
    s->ticket = 0;
    s->coef_ticket = 0;
    g[0] = beta;
    for (int i = 1; i <= s->m; ++i) g[i] = 0.0;
}

// V_0 = r / beta in place (with its float copy) and into vcur, when the
// cycle runs
__global__ void gm_scale_kernel(int64_t n, double* __restrict__ V, float* __restrict__ Vf, double* __restrict__ vcur,
                                const GmState* s)
{
    if (!s->restart_ok) return;
    const double inv = 1.0 / s->beta0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double v = V[i] * inv;
        V[i] = v;
        Vf[i] = static_cast<float>(v);
        vcur[i] = v;
    }
}

// Restarted GMRES(m) (Saad and Schultz 1986) for general square A.  The
// Arnoldi basis V (m + 1 vectors of n) lives in device memory.  One cycle is
// a CUDA graph whose WHILE node runs the Arnoldi steps: the product
// w = A v_j, classical Gram-Schmidt applied twice (partial dots of the
// basis with w, their fixed-order sums, the combination fused with the
// second pass's dots, the second combination fused with ||w||), the next
// basis vector, and the Givens step on the new Hessenberg column, all on the
// device; the Givens kernel ends the loop when the residual estimate is
// <= tol ||b||, at m steps or at maxit.  The host synchronises once per
// cycle: x += V y (back substitution on the device), and the next cycle
// starts from the FP64 true residual, which decides convergence.
int gmres_solve(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int m, int maxit,
                cudaStream_t st, gko_solve_info* info)
{
    const int64_t n = A->n_rows;
    if (n == 0) {
        fill_info(info, 0, 0, 0.0, GKO_OK);
        return GKO_OK;
    }
    Workspace ws(st);
    double *V, *w, *vcur, *part, *H, *cs, *sn, *g, *hh, *coef, *yv;
    SolverState* ds;
    GmState* gs;
    // 3 CTAs per SM: 1-3 % faster than 4 on the 1024^2 convection-diffusion
    // operator in three measurements (the Arnoldi kernels run 2 rows per
    // thread per pass)
    const int grid = static_cast<int>(
        std::max<int64_t>(1, std::min<int64_t>(3 * device_sm_count(), (n + kRedThreads - 1) / kRedThreads)));
    const int ldp = m + 1;
    float* Vf;
    GKO_TRY(ws.get(&V, n * (m + 1)));
    GKO_TRY(ws.get(&Vf, n * (m + 1)));
    GKO_TRY(ws.get(&w, n));
    GKO_TRY(ws.get(&vcur, n));
    GKO_TRY(ws.get(&part, static_cast<int64_t>(std::max(grid, kRedBlocks)) * ldp + 2 * std::max(grid, kRedBlocks)));
    GKO_TRY(ws.get(&H, static_cast<int64_t>(m + 1) * m));
    GKO_TRY(ws.get(&cs, m));
    GKO_TRY(ws.get(&sn, m));
    GKO_TRY(ws.get(&g, m + 1));
    GKO_TRY(ws.get(&hh, m + 1));
    GKO_TRY(ws.get(&coef, m + 1));
    double* coef2;  // second pass, and ||w1||^2 at index j + 1
    GKO_TRY(ws.get(&coef2, m + 2));
    GKO_TRY(ws.get(&yv, m));
    GKO_TRY(ws.get(&ds, 1));
    GKO_TRY(ws.get(&gs, 1));
    SolverState hs = {};
    GKO_TRY(write_state(ds, &hs, st));
    auto norm = [&](const double* v, double* out) -> int {
        dot_kernel<double, kDotStore><<<grid, kRedThreads, 0, st>>>(n, v, v, ds, part, 0);
        GKO_TRY(read_state(&hs, ds, st));
        *out = std::sqrt(hs.dot_out);
        return GKO_OK;
    };
    double bnorm;
    GKO_TRY(norm(b, &bnorm));
    if (bnorm == 0.0) {
        GKO_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st));
        GKO_CUDA(cudaStreamSynchronize(st));
        fill_info(info, 0, 0, 0.0, GKO_OK);
        return GKO_OK;
    }
    GmState hg = {};
    hg.bnorm = bnorm;
    hg.tol = tol;
    hg.m = m;
    hg.maxit = maxit;
    GKO_CUDA(cudaMemsetAsync(part, 0, (static_cast<int64_t>(kRedBlocks) * ldp + 2 * kRedBlocks) * sizeof(double), st));

    GraphHolder gh;
    GKO_TRY(build_while_graph(&gh, [&](cudaGraphConditionalHandle h, cudaStream_t cs_) -> int {
        GKO_TRY(spmv_fmt(A, fmt, vcur, w, 1.0, 0.0, cs_));
        gm_dots_kernel<<<grid, kRedThreads, 0, cs_>>>(n, V, w, part, ldp, gs);
        gm_coef_kernel<<<m + 2, kRedThreads, 0, cs_>>>(grid, part, ldp, coef, hh, 0, gs);
        gm_combine_dots_kernel<<<grid, kRedThreads, 0, cs_>>>(n, V, w, coef, part, ldp, gs);
        gm_coef_kernel<<<m + 2, kRedThreads, 0, cs_>>>(grid, part, ldp, coef2, hh, 1, gs);
        gm_combine_norm_kernel<<<grid, kRedThreads, 0, cs_>>>(
            n, V, Vf, w, vcur, coef2, part + static_cast<int64_t>(std::max(grid, kRedBlocks)) * ldp, gs);
        gm_next_vector_kernel<<<grid, kRedThreads, 0, cs_>>>(n, V, Vf, vcur, w, gs);
        gm_givens_kernel<<<1, 128, 0, cs_>>>(H, cs, sn, g, hh, gs, h);
        GKO_CUDA(cudaGetLastError());
        return GKO_OK;
    }));

    // The host synchronises once per cycle: after the cycle's graph, x += V y
    // and the next cycle's start (residual, its norm, the restart decision,
    // V_0 and g) are queued behind it and the state is read once.
    const int bs_smem = m * (m + 1) * static_cast<int>(sizeof(double));
    GKO_CUDA(smem_limit_once(reinterpret_cast<const void*>(gm_backsub_kernel), bs_smem));
    auto start_cycle = [&]() -> int {
        // r = b - A x into V_0, ||r||^2, then the decision and V_0 = r / ||r||
        GKO_CUDA(cudaMemcpyAsync(V, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        GKO_TRY(spmv_fmt(A, fmt, x, V, -1.0, 1.0, st));
        dot_kernel<double, kDotStore><<<grid, kRedThreads, 0, st>>>(n, V, V, ds, part, 0);
        gm_restart_kernel<<<1, 1, 0, st>>>(ds, gs, g);
        gm_scale_kernel<<<grid, kRedThreads, 0, st>>>(n, V, Vf, vcur, gs);
        GKO_CUDA(cudaGetLastError());
        GKO_CUDA(cudaMemcpyAsync(&hg, gs, sizeof(GmState), cudaMemcpyDeviceToHost, st));
        GKO_CUDA(cudaStreamSynchronize(st));
        return GKO_OK;
    };
    GKO_CUDA(cudaMemcpyAsync(gs, &hg, sizeof(GmState), cudaMemcpyHostToDevice, st));
    GKO_TRY(start_cycle());
    int status = GKO_ERR_NOT_CONVERGED, total = 0;
    double res = -1.0;
    while (true) {
        total = hg.total;
        res = hg.beta0 / bnorm;
        if (hg.broke || !(hg.beta0 == hg.beta0)) {
            status = GKO_ERR_BREAKDOWN;
            break;
        }
        if (hg.beta0 <= tol * bnorm) {
            status = GKO_OK;
            break;
        }
        if (!hg.restart_ok) break;  // maxit
        GKO_CUDA(cudaGraphLaunch(gh.exec, st));
        gm_backsub_kernel<<<1, 128, bs_smem, st>>>(H, g, yv, gs);
        gm_update_x_kernel<<<grid, kRedThreads, 0, st>>>(n, x, V, yv, gs);
        GKO_CUDA(cudaGetLastError());
        GKO_TRY(start_cycle());
    }
    GKO_CUDA(cudaStreamSynchronize(st));
    fill_info(info, total, 0, res, status);
    if (info) info->aux = hg.low_steps;
    if (status != GKO_OK)
        set_error(status == GKO_ERR_BREAKDOWN ? "GMRES breakdown (NaN or zero rotation)" : "GMRES reached maxit");
    return status;
}

// ------------------------------------------- mixed precision refinement

// IEEE binary64 -> bfloat16, round to nearest, ties to even, from the bit
// pattern (values in the normal range of bfloat16).
__device__ __forceinline__ uint16_t f64_to_bf16_rn(double v)
{
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(v));
    const uint64_t sign = b >> 63;
    int64_t exp = static_cast<int64_t>((b >> 52) & 0x7ff);
    uint64_t mant = b & ((1ull << 52) - 1);
    if (exp == 0 && mant == 0) return static_cast<uint16_t>(sign << 15);
    uint64_t keep = mant >> 45;                    // top 7 stored bits
    const uint64_t rem = mant & ((1ull << 45) - 1);
    const uint64_t half = 1ull << 44;
    if (rem > half || (rem == half && (keep & 1))) {
        ++keep;
        if (keep == 128) {
            keep = 0;
            ++exp;
        }
    }
    const uint64_t e8 = static_cast<uint64_t>(exp - 1023 + 127);
    return static_cast<uint16_t>((sign << 15) | (e8 << 7) | keep);
}

template <int kBf16>
__device__ __forceinline__ double round_lo(double v)
{
    if (kBf16) {
        const uint32_t bits = static_cast<uint32_t>(f64_to_bf16_rn(v)) << 16;
        return static_cast<double>(__uint_as_float(bits));
    }
    return static_cast<double>(__double2float_rn(v));
}

// Low-precision copy, one row per thread: off-diagonals rounded to
// nearest-even; the diagonal target a_ii + sum_j(|rn(a_ij)| - |a_ij|)
// formed in FP64 (row sums preserved) and rounded to nearest-even.
template <int kBf16>
__global__ void lowprec_kernel(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                               const double* __restrict__ val, float* __restrict__ out32,
                               uint16_t* __restrict__ out16)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    double shift = 0.0;
    int64_t kd = -1;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
        if (col[k] == i) {
            kd = k;
            continue;
        }
        const double r = round_lo<kBf16>(val[k]);
        const double d = fabs(r) - fabs(val[k]);
        shift = shift + d;
        if (kBf16)
            out16[k] = f64_to_bf16_rn(val[k]);
        else
            out32[k] = __double2float_rn(val[k]);
    }
    if (kd >= 0) {
        const double d = __dadd_rn(val[kd], shift);
        if (kBf16)
            out16[kd] = f64_to_bf16_rn(d);
        else
            out32[kd] = __double2float_rn(d);
    }
}

// rl = float(r / nr); d = p = s = 0; with a preconditioner u = dinv rl
__global__ void inner_init_kernel(int64_t n, const double* __restrict__ r, double nr, float* __restrict__ rl,
                                  float* __restrict__ d, float* __restrict__ p, float* __restrict__ s,
                                  const float* __restrict__ dinv, float* __restrict__ u)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float v = __double2float_rn(r[i] / nr);
        rl[i] = v;
        d[i] = 0.0f;
        p[i] = 0.0f;
        s[i] = 0.0f;
        if (dinv) u[i] = dinv[i] * v;
    }
}

// x += nr * d in FP64
__global__ void correct_kernel(int64_t n, double* __restrict__ x, const float* __restrict__ d, double nr)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        x[i] = fma(nr, static_cast<double>(d[i]), x[i]);
}

template <typename V>
static cudaError_t inner_spmv(const gko_matrix* A, const V* val, SegScratchT<float> sc, const float* p, float* q,
                              cudaStream_t st)
{
    if (A->nnz == 0) {
        return cudaMemsetAsync(q, 0, A->n_rows * sizeof(float), st);
    }
    if (rowblock_preferred(A)) {  // rows of similar length: one thread per row
        if constexpr (sizeof(V) == 2)
            return rowblock_lowprec_bf16(A, val, p, q, st);
        else
            return rowblock_lowprec_f32(A, val, p, q, st);
    }
    return seg_launch<kSegP, V, float, false, false, false, false>(A->n_rows, A->n_cols, A->nnz, A->csr.row_ptr, nullptr,
                                                                   A->csr.col, val, A->csr.thr_row, sc, p, q, 1.0f,
                                                                   0.0f, A->d_err, st);
}

int cg_mixed_solve(gko_matrix* A, int inner, const double* b, double* x, double tol, int maxit_outer,
                   double inner_tol, int inner_maxit, cudaStream_t st, gko_solve_info* info, int precond)
{
    const int64_t n = A->n_rows, nnz = A->nnz;
    if (n == 0) {
        fill_info(info, 0, 0, 0.0, GKO_OK);
        return GKO_OK;
    }
    const bool bf16 = inner == GKO_BF16;
    // cached low-precision copy of the values (CSR order)
    if (bf16 && !A->val_bf16) {
        GKO_TRY(dev_alloc(&A->val_bf16, padded_len(nnz)));
        GKO_CUDA(cudaMemsetAsync(A->val_bf16, 0, padded_len(nnz) * sizeof(uint16_t), st));
        lowprec_kernel<1><<<ceil_div(n, 256), 256, 0, st>>>(n, A->csr.row_ptr, A->csr.col, A->csr.val, nullptr,
                                                             A->val_bf16);
    }
    if (!bf16 && !A->val_f32) {
        GKO_TRY(dev_alloc(&A->val_f32, padded_len(nnz)));
        GKO_CUDA(cudaMemsetAsync(A->val_f32, 0, padded_len(nnz) * sizeof(float), st));
        lowprec_kernel<0><<<ceil_div(n, 256), 256, 0, st>>>(n, A->csr.row_ptr, A->csr.col, A->csr.val, A->val_f32,
                                                             nullptr);
    }
    GKO_CUDA(cudaGetLastError());
    bool use_ell = false;
    GKO_TRY(lp_ell_prepare(A, bf16, st, &use_ell));

    Workspace ws(st);
    double *r, *part;
    float *rl, *d, *p, *sv, *w, *dinv = nullptr, *u = nullptr;
    SolverState *ds, *di;
    GKO_TRY(ws.get(&r, n));
    GKO_TRY(ws.get(&part, 2 * std::max(kRedBlocks, use_ell ? lp_ell_grid(A) : 0)));
    GKO_TRY(ws.get(&rl, n));
    GKO_TRY(ws.get(&d, n));
    GKO_TRY(ws.get(&p, n));
    GKO_TRY(ws.get(&sv, n));
    GKO_TRY(ws.get(&w, n));
    GKO_TRY(ws.get(&ds, 1));
    GKO_TRY(ws.get(&di, 1));
    const bool jac = precond == GKO_PRECOND_JACOBI;
    if (jac) {  // M = diag(A_lo)
        int32_t* bad;
        GKO_TRY(ws.get(&dinv, n));
        GKO_TRY(ws.get(&u, n));
        GKO_TRY(ws.get(&bad, 1));
        GKO_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), st));
        if (bf16)
            diag_lo_inv_kernel<1><<<red_grid(n), kRedThreads, 0, st>>>(n, A->csr.row_ptr, A->csr.col, nullptr,
                                                                        A->val_bf16, dinv, bad);
        else
            diag_lo_inv_kernel<0><<<red_grid(n), kRedThreads, 0, st>>>(n, A->csr.row_ptr, A->csr.col, A->val_f32,
                                                                        nullptr, dinv, bad);
        int32_t hbad = 0;
        GKO_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        GKO_CUDA(cudaStreamSynchronize(st));
        if (hbad) {
            fill_info(info, 0, 0, -1.0, GKO_ERR_BREAKDOWN);
            set_error("Jacobi preconditioner: a diagonal entry of the rounded matrix is zero or not stored");
            return GKO_ERR_BREAKDOWN;
        }
    }
    float* ux = jac ? u : rl;  // the vector the product gathers (u = M^-1 rl, or rl itself)
    const int64_t tiles = std::max<int64_t>(1, (nnz + SegShape<kSegP>::kTile - 1) / SegShape<kSegP>::kTile);
    SegScratchT<float> sc;
    GKO_TRY(ws.get(&sc.tail_val, tiles));
    GKO_TRY(ws.get(&sc.tail_row, tiles));
    GKO_TRY(ws.get(&sc.tail_pass, tiles));
    GKO_TRY(ws.get(&sc.head_val, tiles));
    GKO_TRY(ws.get(&sc.head_row, tiles));
    const int grid = red_grid(n);

    SolverState hs = {};
    GKO_TRY(write_state(ds, &hs, st));
    dot_kernel<double, kDotStore><<<grid, kRedThreads, 0, st>>>(n, b, b, ds, part, 0);
    GKO_TRY(read_state(&hs, ds, st));
    const double bnorm = std::sqrt(hs.dot_out);
    if (bnorm == 0.0) {
        GKO_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st));
        GKO_CUDA(cudaStreamSynchronize(st));
        fill_info(info, 0, 0, 0.0, GKO_OK);
        return GKO_OK;
    }

    // inner CG on A_lo d = rl in the single-reduction form (Chronopoulos and
    // Gear): w = A_lo rl fused with the dots and the scalar step (ELL copy of
    // A_lo when its padding is small, else row-block CSR; otherwise the
    // load-balanced product + one dot kernel), then
    // p = rl + beta p, s = w + beta s, d += alpha p, rl -= alpha s
    const bool fused = nnz > 0 && rowblock_preferred(A) && !jac;
    GraphHolder gh;
    GKO_TRY(build_while_graph(&gh, [&](cudaGraphConditionalHandle h, cudaStream_t cs) -> int {
        const Cg1Reduce red{di, part, A->d_err, h};
        cudaError_t e;
        if (use_ell) {
            e = lp_ell_cg1(A, bf16, ux, rl, w, red, cs);
        } else if (fused) {
            e = bf16 ? rowblock_cg1_bf16(A, A->val_bf16, rl, w, red, cs) : rowblock_cg1_f32(A, A->val_f32, rl, w, red, cs);
        } else {
            e = bf16 ? inner_spmv<__nv_bfloat16>(A, reinterpret_cast<const __nv_bfloat16*>(A->val_bf16), sc, ux, w, cs)
                     : inner_spmv<float>(A, A->val_f32, sc, ux, w, cs);
            if (e == cudaSuccess) {
                cg1_dots_kernel<float><<<grid, kRedThreads, 0, cs>>>(n, ux, rl, w, red);
                e = cudaGetLastError();
            }
        }
        if (e != cudaSuccess) return cuda_fail(e, "inner CG product launch");
        launch_cg1_update<float>(n, d, rl, p, sv, w, di, cs, dinv, u);
        GKO_CUDA(cudaGetLastError());
        return GKO_OK;
    }));

    int status = GKO_ERR_NOT_CONVERGED, outer = 0, inner_total = 0;
    double res = -1.0;
    for (int o = 0; o <= maxit_outer; ++o) {
        // r = b - A x (FP64), ||r||
        GKO_CUDA(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        GKO_TRY(spmv_csr(A, GKO_CFG_DEFAULT, x, r, -1.0, 1.0, st));
        dot_kernel<double, kDotStore><<<grid, kRedThreads, 0, st>>>(n, r, r, ds, part, 0);
        GKO_TRY(read_state(&hs, ds, st));
        const double nr = std::sqrt(hs.dot_out);
        res = nr / bnorm;
        if (!(nr == nr)) {
            status = GKO_ERR_BREAKDOWN;
            break;
        }
        if (res <= tol) {
            status = GKO_OK;
            break;
        }
        if (o == maxit_outer) break;
        outer = o + 1;
        inner_init_kernel<<<grid, kRedThreads, 0, st>>>(n, r, nr, rl, d, p, sv, dinv, u);
        SolverState is = {};
        is.tol = inner_tol;
        is.rel_inner = 1;
        is.maxit = inner_maxit;
        is.status = GKO_ERR_NOT_CONVERGED;
        GKO_TRY(write_state(di, &is, st));
        GKO_CUDA(cudaGraphLaunch(gh.exec, st));
        correct_kernel<<<grid, kRedThreads, 0, st>>>(n, x, d, nr);
        GKO_TRY(read_state(&is, di, st));
        inner_total += is.iter;
        if (is.status == GKO_ERR_TIMEOUT) {
            status = GKO_ERR_TIMEOUT;
            break;
        }
    }
    GKO_CUDA(cudaGetLastError());
    fill_info(info, inner_total, outer, res, status);
    if (status != GKO_OK) set_error("mixed-precision CG did not reach the tolerance");
    return status;
}

}  // namespace gko
