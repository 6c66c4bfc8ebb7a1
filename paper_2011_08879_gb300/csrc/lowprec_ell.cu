// Low-precision ELL copy for the inner solve of mixed-precision CG, and its
// product fused with the dots and scalar step of the single-reduction CG.
//
// The inner solve only ever multiplies by the rounded matrix A_lo, so it
// keeps A_lo in the layout that streams best: ELL (column-major slots, row i
// slot k at k * n_pad + i) whenever padding adds at most a quarter to the
// stored entries.  Column indices are int32, or int16 offsets c - i when
// every |c - i| <= 32767 (stencil and banded operators): with FP32 values an
// entry moves 6 bytes instead of the 8 of CSR plus row pointers, with BF16
// values 4.  Padding slots point at their own row with the value +0.0.
//
// One thread owns four consecutive rows and moves each slot's four values
// and indices with one vector load each (128-bit for FP32 values / int32
// indices, 64-bit for BF16 / int16), marked evict-first (the matrix is read
// once per step; the solver's vectors stay in L2).  The thread then adds
// rd_i r_i and w_i r_i of its rows to the step's two dots (rd = r without a
// preconditioner; with one, r is the preconditioned residual u = M^-1 rd
// and rd the residual); one grid reduction
// (block partials, then a one-block kernel that sums them in block order)
// ends in the CG scalar step.  A ticket atomic and fence at the end of every
// block of this short kernel would cost more than that extra launch.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "segmented.cuh"
#include "solver.cuh"

namespace gko {

constexpr int kLpThreads = 256;


// ------------------------------------------------------------ building

// slot k of row i: column (int32) or offset c - i (int16).  A padding slot
// points at the row itself (column i, offset 0) and holds the value +0.0,
// so the product needs no test per slot; rows i >= n (the tail up to n_pad,
// fewer than 32) point at row n - 1, within int16 reach.  The inner solve's vectors are finite (a NaN or Inf
// residual already stops it as a breakdown), so 0 * r_i adds nothing.
template <typename I>
__global__ void lp_ell_cols_kernel(int64_t n, int64_t n_pad, int K, const int32_t* __restrict__ row_ptr,
                                   const int32_t* __restrict__ col, I* __restrict__ out)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= n_pad) return;
    const int64_t k0 = i < n ? row_ptr[i] : 0;
    const int len = i < n ? row_ptr[i + 1] - static_cast<int32_t>(k0) : 0;
    const int64_t self = i < n ? i : n - 1;
    for (int k = 0; k < K; ++k) {
        const int64_t c = k < len ? col[k0 + k] : self;
        out[k * n_pad + i] = static_cast<I>(sizeof(I) == 2 ? c - i : c);
    }
}

template <typename V>
__global__ void lp_ell_vals_kernel(int64_t n, int64_t n_pad, int K, const int32_t* __restrict__ row_ptr,
                                   const V* __restrict__ val, V* __restrict__ out)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= n_pad) return;
    const int64_t k0 = i < n ? row_ptr[i] : 0;
    const int len = i < n ? row_ptr[i + 1] - static_cast<int32_t>(k0) : 0;
    for (int k = 0; k < K; ++k) out[k * n_pad + i] = k < len ? val[k0 + k] : V(0);
}

// Build (once) the ELL copy of the rounded values in CSR order val_lo
// (float or bf16 bits).  Returns GKO_OK and sets *usable when the layout
// applies to this matrix (padding <= 25 % of nnz).
int lp_ell_prepare(gko_matrix* A, bool bf16, cudaStream_t st, bool* usable)
{
    LowPrecEll& E = A->lp_ell;
    *usable = false;
    const int64_t n = A->n_rows, nnz = A->nnz;
    if (!E.tried) {
        E.tried = true;
        const int64_t K = A->csr.max_len;
        const int64_t n_pad = (n + 31) / 32 * 32;
        E.ok = nnz > 0 && K >= 1 && K <= 1024 && K * n_pad <= nnz + nnz / 4 + 4096;
        if (E.ok) {
            E.K = K;
            E.n_pad = n_pad;
            E.idx16 = A->csr.band >= 0 && A->csr.band <= 32767;
            const int64_t slots = K * n_pad;
            if (E.idx16) {
                int16_t* c;
                GKO_TRY(dev_alloc(&c, slots));
                E.col = c;
                lp_ell_cols_kernel<int16_t><<<ceil_div(n_pad, 256), 256, 0, st>>>(n, n_pad, static_cast<int>(K),
                                                                                   A->csr.row_ptr, A->csr.col, c);
            } else {
                int32_t* c;
                GKO_TRY(dev_alloc(&c, slots));
                E.col = c;
                lp_ell_cols_kernel<int32_t><<<ceil_div(n_pad, 256), 256, 0, st>>>(n, n_pad, static_cast<int>(K),
                                                                                   A->csr.row_ptr, A->csr.col, c);
            }
            GKO_CUDA(cudaGetLastError());
        }
    }
    if (!E.ok) return GKO_OK;
    const int64_t slots = E.K * E.n_pad;
    if (bf16 && !E.val_bf16) {
        GKO_TRY(dev_alloc(&E.val_bf16, slots));
        lp_ell_vals_kernel<uint16_t><<<ceil_div(E.n_pad, 256), 256, 0, st>>>(
            n, E.n_pad, static_cast<int>(E.K), A->csr.row_ptr, A->val_bf16, E.val_bf16);
    }
    if (!bf16 && !E.val_f32) {
        GKO_TRY(dev_alloc(&E.val_f32, slots));
        lp_ell_vals_kernel<float><<<ceil_div(E.n_pad, 256), 256, 0, st>>>(n, E.n_pad, static_cast<int>(E.K),
                                                                           A->csr.row_ptr, A->val_f32, E.val_f32);
    }
    GKO_CUDA(cudaGetLastError());
    *usable = true;
    return GKO_OK;
}

void lp_ell_free(gko_matrix* A)
{
    LowPrecEll& E = A->lp_ell;
    if (E.col) cudaFree(E.col);
    dev_free(E.val_f32);
    dev_free(E.val_bf16);
    E = LowPrecEll{};
}

// ------------------------------------------------------------- product

// G consecutive slots (rows row0 .. row0 + G - 1) of one ELL column of
// element type T, loaded as raw 32-bit words (one or two 64/128-bit loads,
// streaming: evict-first) and unpacked at use.
template <typename T, int G>
struct Slots {
    static constexpr int kBytes = G * static_cast<int>(sizeof(T));
    static constexpr int kWords = kBytes / 4;
    static_assert(kBytes == 8 || kBytes % 16 == 0, "8 bytes or whole 16-byte words");
    uint32_t w[kWords];
    __device__ __forceinline__ void load(const T* p)
    {
        if (kBytes == 8) {
            const uint2 t = __ldcs(reinterpret_cast<const uint2*>(p));
            w[0] = t.x;
            w[1] = t.y;
        } else {
#pragma unroll
            for (int i = 0; i < kWords / 4; ++i) {
                const uint4 t = __ldcs(reinterpret_cast<const uint4*>(p) + i);
                w[4 * i] = t.x;
                w[4 * i + 1] = t.y;
                w[4 * i + 2] = t.z;
                w[4 * i + 3] = t.w;
            }
        }
    }
    __device__ __forceinline__ void fill(uint32_t v)
    {
#pragma unroll
        for (int i = 0; i < kWords; ++i) w[i] = v;
    }
    // 16-bit element u (int16 offsets, bf16 bits) or 32-bit element u
    __device__ __forceinline__ uint32_t half(int u) const { return u & 1 ? w[u >> 1] >> 16 : w[u >> 1] & 0xffffu; }
};

// column of row row0 + u, -1 for padding
template <int G>
__device__ __forceinline__ int column(const Slots<int32_t, G>& c, int u, int64_t /*row0*/)
{
    return static_cast<int>(c.w[u]);
}
template <int G>
__device__ __forceinline__ int column(const Slots<int16_t, G>& c, int u, int64_t row0)
{
    return static_cast<int>(row0) + u + static_cast<int16_t>(c.half(u));
}
template <int G>
__device__ __forceinline__ float value(const Slots<float, G>& v, int u)
{
    return __uint_as_float(v.w[u]);
}
template <int G>
__device__ __forceinline__ float value(const Slots<uint16_t, G>& v, int u)  // bf16 bits
{
    return __uint_as_float(v.half(u) << 16);
}

// rows per thread: one 16-byte load of values per slot (FP32: 4, BF16: 8)
template <typename V>
constexpr int lp_rows() { return 16 / static_cast<int>(sizeof(V)); }

// w = A_lo r on the ELL copy, with the block partials of gamma = r.r and
// delta = w.r written to part[2 b], part[2 b + 1] (no atomics, no fences:
// cg1_finish_kernel reduces them).  V: float or bf16 bits; I: int32
// columns or int16 offsets.  Each thread owns G = lp_rows<V>() consecutive
// rows, so every warp reads at least 512 contiguous bytes of each array per
// slot; n_pad is a multiple of 32, so every group is aligned.  Slots go in
// chunks of eight whose loads are all issued before their gathers and FMAs
// (a 7-point operator is one chunk).
// KC = K when K <= 8 (every slot's load unconditional, all in flight
// together), 0 for wider matrices (chunks of eight, the last one masked).
template <typename V, typename I, int KC>
__global__ void __launch_bounds__(kLpThreads)
    lp_ell_cg1_kernel(int64_t n, int64_t n_pad, int K, const I* __restrict__ col, const V* __restrict__ val,
                      const float* __restrict__ r, const float* __restrict__ rd, float* __restrict__ w,
                      double* __restrict__ part)
{
    constexpr int G = lp_rows<V>();
    if (KC > 0) K = KC;
    const int64_t groups = n_pad / G;
    float g = 0.0f, d = 0.0f;
    const int64_t q = blockIdx.x * static_cast<int64_t>(kLpThreads) + threadIdx.x;
    if (q < groups) {
        const int64_t row0 = G * q;
        float a[G];
#pragma unroll
        for (int u = 0; u < G; ++u) a[u] = 0.0f;
        for (int k = 0; k < K; k += 8) {
            Slots<I, G> c[8];
            Slots<V, G> v[8];
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                if (KC > 0 ? s < KC : k + s < K) {
                    c[s].load(col + (k + s) * n_pad + row0);
                    v[s].load(val + (k + s) * n_pad + row0);
                }
            }
#pragma unroll
            for (int s = 0; s < (KC > 0 ? KC : 8); ++s)
                if (KC > 0 || k + s < K) {
#pragma unroll
                    for (int u = 0; u < G; ++u) a[u] = fmaf(value(v[s], u), ldg(r + column(c[s], u, row0)), a[u]);
                }
        }
        if (row0 + G <= n) {
#pragma unroll
            for (int h = 0; h < G; h += 4) {
                const float4 rr = *reinterpret_cast<const float4*>(r + row0 + h);
                const float4 rv = *reinterpret_cast<const float4*>(rd + row0 + h);
                *reinterpret_cast<float4*>(w + row0 + h) = make_float4(a[h], a[h + 1], a[h + 2], a[h + 3]);
                g = fmaf(rv.x, rr.x, fmaf(rv.y, rr.y, fmaf(rv.z, rr.z, fmaf(rv.w, rr.w, g))));
                d = fmaf(a[h], rr.x, fmaf(a[h + 1], rr.y, fmaf(a[h + 2], rr.z, fmaf(a[h + 3], rr.w, d))));
            }
        } else {
#pragma unroll
            for (int u = 0; u < G; ++u)
                if (row0 + u < n) {
                    const float ri = r[row0 + u];
                    w[row0 + u] = a[u];
                    g = fmaf(rd[row0 + u], ri, g);
                    d = fmaf(a[u], ri, d);
                }
        }
    }
    __shared__ double sh[32];
    const double bg = block_sum(static_cast<double>(g), sh);
    const double bd = block_sum(static_cast<double>(d), sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = bg;
        part[2 * blockIdx.x + 1] = bd;
    }
}

// Sum the product kernel's block partials in a fixed order (thread t takes
// partials t, t + 1024, ... with four loads in flight) and take the CG
// scalar step; one block of 1024 threads.
constexpr int kFinishThreads = 1024;
__global__ void __launch_bounds__(kFinishThreads) cg1_finish_kernel(int nparts, const double* __restrict__ part,
                                                                    Cg1Reduce red)
{
    __shared__ double sh[32];
    double a0[4] = {0.0, 0.0, 0.0, 0.0}, a1[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i0 = threadIdx.x; i0 < nparts; i0 += 4 * kFinishThreads) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * kFinishThreads;
            if (i < nparts) {
                a0[u] += part[2 * i];
                a1[u] += part[2 * i + 1];
            }
        }
    }
    const double g = block_sum((a0[0] + a0[1]) + (a0[2] + a0[3]), sh);
    const double d = block_sum((a1[0] + a1[1]) + (a1[2] + a1[3]), sh);
    if (threadIdx.x == 0) cg1_scalars(red.s, g, d, red.err, red.h);
}

// ------------------------------------------------ TMA-staged product

// Shape of the staged kernel for a matrix of width K: R rows per stage (a
// multiple of 1024 = 256 threads x 4 rows, stage <= 48 KB), 0 if K is too
// wide for that (such matrices take the direct-load kernel).
template <typename V, typename I>
constexpr int lp_stage_rows(int K)
{
    const int per_row = K * static_cast<int>(sizeof(V) + sizeof(I));
    const int r = (48 * 1024 / per_row) / 1024 * 1024;
    return r > 2048 ? 2048 : r;
}
constexpr int kLpStageBytes = 48 * 1024;

// w = A_lo r on the ELL copy, the slots streamed into shared memory by 1-D
// bulk copies (TMA) completing on an mbarrier, two stages per CTA, two CTAs
// per SM, persistent over stages of R rows: while one stage is summed the
// next one's K index runs and K value runs (each R entries long, contiguous
// in the column-major layout) land.  Thread t sums rows t, t + 256, ... of
// the stage four at a time (rows 4t .. 4t + 3, then + 1024, ...), reading
// each slot's four indices and four values with one vector load each from
// shared memory (consecutive threads read consecutive words: no bank
// conflicts) and gathering r through L1/L2.
// The dots go through one grid reduction per launch (last-block ticket, once
// per CTA) into the CG scalar step.
template <typename V, typename I, int KC>
__global__ void __launch_bounds__(kLpThreads, 2)
    lp_ell_tma_cg1_kernel(int64_t n, int64_t n_pad, int K, int R, const I* __restrict__ col,
                          const V* __restrict__ val, const float* __restrict__ r, const float* __restrict__ rd,
                          float* __restrict__ w, uint32_t* err, Cg1Reduce red, uint32_t polls)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar[2];
    if (KC > 0) K = KC;
    const int tid = threadIdx.x;
    const int64_t n_stages = (n_pad + R - 1) / R;
    const int64_t stride = gridDim.x;
    const size_t idx_bytes = static_cast<size_t>(K) * R * sizeof(I);
    auto s_col = [&](int st) { return reinterpret_cast<I*>(smem + st * kLpStageBytes); };
    auto s_val = [&](int st) { return reinterpret_cast<V*>(smem + st * kLpStageBytes + idx_bytes); };
    auto rows_of = [&](int64_t b) { return static_cast<int>(min(static_cast<int64_t>(R), n_pad - b * R)); };
    auto issue = [&](int64_t b, int st) {
        const int rows = rows_of(b);  // a multiple of 32
        const int64_t r0 = b * R;
        mbar_arrive_expect_tx(&bar[st], static_cast<uint32_t>(K * rows * (sizeof(I) + sizeof(V))));
        const uint64_t pol = l2_evict_first_policy();
        for (int k = 0; k < K; ++k) {
            bulk_g2s_hint(s_col(st) + k * R, col + k * n_pad + r0, rows * sizeof(I), &bar[st], pol);
            bulk_g2s_hint(s_val(st) + k * R, val + k * n_pad + r0, rows * sizeof(V), &bar[st], pol);
        }
    };
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < 2; ++k) {
            const int64_t b = blockIdx.x + k * stride;
            if (b < n_stages) issue(b, k);
        }
    float g = 0.0f, d = 0.0f;
    bool failed = false;
    for (int it = 0;; ++it) {
        const int64_t b = blockIdx.x + it * stride;
        if (b >= n_stages) break;
        const int st = it & 1;
        const uint32_t parity = (it >> 1) & 1;
        const bool landed = mbar_wait_bounded(&bar[st], parity, err, polls);
        if (!__syncthreads_and(landed)) {  // CTA-uniform: give up on the rest
            // wait (default limit) for the copies still in flight into this
            // stage and the next one, so none lands after the CTA has exited
            if (tid == 0) {
                mbar_wait_bounded(&bar[st], parity, err);
                if (b + stride < n_stages) mbar_wait_bounded(&bar[st ^ 1], ((it + 1) >> 1) & 1, err);
            }
            __syncthreads();
            failed = true;
            break;
        }
        const int rows = rows_of(b);
        const int64_t r0 = b * R;
        const I* sc = s_col(st);
        const V* sv = s_val(st);
        // four consecutive rows per thread: per slot one 64/128-bit shared
        // load of their indices and one of their values, four gathers
        for (int l = 4 * tid; l < rows; l += 4 * kLpThreads) {
            const int64_t i0 = r0 + l;
            const float* rb = r + (sizeof(I) == 2 ? i0 : 0);  // gathers: rb[c_u + u] (offsets) or r[c_u]
            float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll(KC > 0 ? KC : 4)
            for (int k = 0; k < K; ++k) {
                int c[4];
                if (sizeof(I) == 2) {
                    const uint2 t = *reinterpret_cast<const uint2*>(sc + k * R + l);
                    c[0] = static_cast<int16_t>(t.x & 0xffffu);
                    c[1] = static_cast<int16_t>(t.x >> 16) + 1;
                    c[2] = static_cast<int16_t>(t.y & 0xffffu) + 2;
                    c[3] = static_cast<int16_t>(t.y >> 16) + 3;
                } else {
                    const int4 t = *reinterpret_cast<const int4*>(sc + k * R + l);
                    c[0] = t.x;
                    c[1] = t.y;
                    c[2] = t.z;
                    c[3] = t.w;
                }
                float v[4];
                if (sizeof(V) == 2) {
                    const uint2 t = *reinterpret_cast<const uint2*>(sv + k * R + l);
                    v[0] = __uint_as_float(t.x << 16);
                    v[1] = __uint_as_float(t.x & 0xffff0000u);
                    v[2] = __uint_as_float(t.y << 16);
                    v[3] = __uint_as_float(t.y & 0xffff0000u);
                } else {
                    const float4 t = *reinterpret_cast<const float4*>(sv + k * R + l);
                    v[0] = t.x;
                    v[1] = t.y;
                    v[2] = t.z;
                    v[3] = t.w;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) a[u] = fmaf(v[u], ldg(rb + c[u]), a[u]);
            }
            if (i0 + 4 <= n) {
                const float4 rr = *reinterpret_cast<const float4*>(r + i0);
                const float4 rv = *reinterpret_cast<const float4*>(rd + i0);
                *reinterpret_cast<float4*>(w + i0) = make_float4(a[0], a[1], a[2], a[3]);
                g = fmaf(rv.x, rr.x, fmaf(rv.y, rr.y, fmaf(rv.z, rr.z, fmaf(rv.w, rr.w, g))));
                d = fmaf(a[0], rr.x, fmaf(a[1], rr.y, fmaf(a[2], rr.z, fmaf(a[3], rr.w, d))));
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (i0 + u < n) {
                        const float ri = r[i0 + u];
                        w[i0 + u] = a[u];
                        g = fmaf(rd[i0 + u], ri, g);
                        d = fmaf(a[u], ri, d);
                    }
            }
        }
        __syncthreads();  // the stage is free again
        const int64_t b_issue = b + 2 * stride;
        if (tid == 0 && b_issue < n_stages) {
            fence_proxy_async_smem();
            issue(b_issue, st);
        }
    }
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    SolverState* s = red.s;
    grid_sum2(failed ? nan : static_cast<double>(g), failed ? nan : static_cast<double>(d), red.part, &s->ticket,
              [&](double gamma, double delta) { cg1_scalars(s, gamma, delta, red.err, red.h); });
}

template <typename V, typename I, int KC>
static cudaError_t launch_lp_tma_k(const gko_matrix* A, const V* val, const float* r, const float* rd, float* w,
                                   Cg1Reduce red, int R, int grid, cudaStream_t st)
{
    const LowPrecEll& E = A->lp_ell;
    const cudaError_t e =
        smem_limit_once(reinterpret_cast<const void*>(lp_ell_tma_cg1_kernel<V, I, KC>), 2 * kLpStageBytes);
    if (e != cudaSuccess) return e;
    lp_ell_tma_cg1_kernel<V, I, KC><<<grid, kLpThreads, 2 * kLpStageBytes, st>>>(
        A->n_rows, E.n_pad, static_cast<int>(E.K), R, static_cast<const I*>(E.col), val, r, rd, w, A->d_err, red,
        first_wait_polls());
    return cudaGetLastError();
}

template <typename V, typename I>
static cudaError_t launch_lp_tma(const gko_matrix* A, const V* val, const float* r, const float* rd, float* w,
                                 Cg1Reduce red, cudaStream_t st)
{
    const LowPrecEll& E = A->lp_ell;
    const int K = static_cast<int>(E.K);
    const int R = lp_stage_rows<V, I>(K);
    const int64_t n_stages = (E.n_pad + R - 1) / R;
    const int grid = static_cast<int>(std::min<int64_t>(n_stages, 2 * device_sm_count()));
    switch (K) {
        case 5: return launch_lp_tma_k<V, I, 5>(A, val, r, rd, w, red, R, grid, st);
        case 7: return launch_lp_tma_k<V, I, 7>(A, val, r, rd, w, red, R, grid, st);
        default: return launch_lp_tma_k<V, I, 0>(A, val, r, rd, w, red, R, grid, st);
    }
}

int lp_ell_grid(const gko_matrix* A);

template <typename V, typename I>
static cudaError_t launch_lp(const gko_matrix* A, const V* val, const float* r, const float* rd, float* w,
                             Cg1Reduce red, cudaStream_t st)
{
    const LowPrecEll& E = A->lp_ell;
    const int64_t groups = E.n_pad / lp_rows<V>();
    const int grid = static_cast<int>(std::max<int64_t>(1, (groups + kLpThreads - 1) / kLpThreads));
    const int K = static_cast<int>(E.K);
    const I* c = static_cast<const I*>(E.col);
    switch (K) {
#define GKO_LP(KC)                                                                                         \
    case KC:                                                                                               \
        lp_ell_cg1_kernel<V, I, KC><<<grid, kLpThreads, 0, st>>>(A->n_rows, E.n_pad, K, c, val, r, rd, w, red.part); \
        break
        GKO_LP(1);
        GKO_LP(2);
        GKO_LP(3);
        GKO_LP(4);
        GKO_LP(5);
        GKO_LP(6);
        GKO_LP(7);
        GKO_LP(8);
#undef GKO_LP
        default:
            lp_ell_cg1_kernel<V, I, 0><<<grid, kLpThreads, 0, st>>>(A->n_rows, E.n_pad, K, c, val, r, rd, w, red.part);
    }
    cg1_finish_kernel<<<1, kFinishThreads, 0, st>>>(grid, red.part, red);
    return cudaGetLastError();
}

cudaError_t lp_ell_cg1(const gko_matrix* A, bool bf16, const float* r, const float* rd, float* w, Cg1Reduce red,
                       cudaStream_t st)
{
    const LowPrecEll& E = A->lp_ell;
    const int K = static_cast<int>(E.K);
    const bool tma = bf16 ? (E.idx16 ? lp_stage_rows<uint16_t, int16_t>(K) : lp_stage_rows<uint16_t, int32_t>(K)) >= 1024
                          : (E.idx16 ? lp_stage_rows<float, int16_t>(K) : lp_stage_rows<float, int32_t>(K)) >= 1024;
    if (tma) {
        if (bf16)
            return E.idx16 ? launch_lp_tma<uint16_t, int16_t>(A, E.val_bf16, r, rd, w, red, st)
                           : launch_lp_tma<uint16_t, int32_t>(A, E.val_bf16, r, rd, w, red, st);
        return E.idx16 ? launch_lp_tma<float, int16_t>(A, E.val_f32, r, rd, w, red, st)
                       : launch_lp_tma<float, int32_t>(A, E.val_f32, r, rd, w, red, st);
    }
    if (bf16)
        return E.idx16 ? launch_lp<uint16_t, int16_t>(A, E.val_bf16, r, rd, w, red, st)
                       : launch_lp<uint16_t, int32_t>(A, E.val_bf16, r, rd, w, red, st);
    return E.idx16 ? launch_lp<float, int16_t>(A, E.val_f32, r, rd, w, red, st)
                   : launch_lp<float, int32_t>(A, E.val_f32, r, rd, w, red, st);
}

// blocks of the product kernel (its reduction needs 2 doubles per block)
int lp_ell_grid(const gko_matrix* A)
{
    const int64_t groups = A->lp_ell.n_pad / lp_rows<float>();  // the most blocks (FP32 values)
    return static_cast<int>(std::max<int64_t>(1, (groups + kLpThreads - 1) / kLpThreads));
}

}  // namespace gko
