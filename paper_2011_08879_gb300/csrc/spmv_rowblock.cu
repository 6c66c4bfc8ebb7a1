// CSR SpMV for matrices with rows of similar length: one thread per row,
// rows read from shared memory (paper Sec. 6.1: CSR moves 12 bytes per
// entry; at GB300's bandwidth that is one FP64 FMA per entry at ~97 % of
// the FP64 pipe, so the kernel spends nothing but that FMA per entry).
//
// Rows are cut into blocks of R = min(512, 4096 / max_row_length) rows, so
// a block holds at most 4096 entries; each of the 256 threads of a CTA sums
// rows r0 + t, r0 + t + 256, ...  A persistent grid (2 CTAs per SM) walks
// the blocks with two shared-memory stages: while one block is summed, the
// next block's values, column indices and row pointers stream in by 1-D
// bulk copies (TMA) on an mbarrier.  Each thread sums its row from shared
// memory with the x entries gathered through the read-only path: all
// gathers of a chunk are issued before its FMAs, two accumulator chains, no
// shuffles, no partial sums, one FMA per entry.  Rows of one warp run in
// lockstep, so the kernel suits rows of close length; by measurement it is
// the default for such rows 9 to 20 entries long (shorter and longer ones go
// to the subwarp kernel with 1 or 4 lanes per row, skewed rows to the binned
// kernel).
//
// Banded variant: for matrices with max |i - j| <= 1024 the x window
// [r0 - band, r1 + band) of each block is staged by one more bulk copy and
// the gathers read shared memory instead of L1/L2.
//
// V is the stored value type (double, float, bf16) and T the arithmetic
// and vector type (double, or float for the mixed-precision inner solve).
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "segmented.cuh"
#include "solver.cuh"

namespace gko {

constexpr int kRbThreads = 256;
constexpr int kRbEntries = 4096;             // entries staged per block
constexpr int kRbMaxRows = 512;              // rows per block at most
constexpr int kRbBuf = kRbEntries + 16;      // + alignment slack of the bulk copies
constexpr int kRbRowBuf = kRbMaxRows + 8;    // row_ptr entries staged per block
constexpr int kRbMaxBand = 1024;

template <typename V>
struct RbStage {
    static constexpr int kAlign = 16 / sizeof(V) > 4 ? static_cast<int>(16 / sizeof(V)) : 4;  // entries per group
    static constexpr size_t kVal = kRbBuf * sizeof(V);
    static constexpr size_t kCol = kRbBuf * sizeof(int32_t);
    static constexpr size_t kRp = kRbRowBuf * sizeof(int32_t);
    static constexpr size_t kBase = kVal + kCol + kRp;
    static_assert(kVal % 16 == 0 && kCol % 16 == 0 && kRp % 16 == 0, "16-byte aligned stage parts");
};

// entries of the staged x window for R rows and a band (0 without staging);
// a multiple of 16 bytes
template <typename T>
static int rb_xbuf(int R, int band)
{
    if (band < 0) return 0;
    const int per16 = 16 / static_cast<int>(sizeof(T));
    return (R + 2 * band + 2 * per16 + per16 - 1) / per16 * per16;
}

struct RbInfo {
    int32_t r0, r1;  // rows of the block
    int32_t a0;      // first staged entry (multiple of the alignment group)
    int32_t ra0;     // first staged row_ptr index (multiple of 4)
    int32_t w0, wl;  // staged x window: x[w0 .. w0 + wl)
};

// rows per block for this matrix (0: the kernel does not apply)
int rowblock_rows(const gko_matrix* A)
{
    const int32_t L = A->csr.max_len;
    if (L < 1 || L > kRbEntries / 32) return 0;
    return std::min(kRbMaxRows, kRbEntries / L);
}

bool rowblock_preferred(const gko_matrix* A)
{
    // lockstep rows: the longest row costs the whole warp; require rows of
    // similar length (max <= 2 * mean + 16)
    return rowblock_rows(A) > 0 && A->csr.max_len <= 2.0 * A->csr.mean_len + 16.0;
}

// kDots: the product of a single-reduction CG step (x = r, y = w = A r);
// every thread also sums r_i^2 and w_i r_i over its rows and the grid
// reduction ends in the solver's scalar step (alpha = 1, beta = 0).
// kHint: the matrix streams carry an L2 evict-first policy.
template <typename V, typename T, bool kAlpha, bool kBeta, bool kX, int CH, bool kDots = false, bool kHint = false>
__global__ void __launch_bounds__(kRbThreads, 2)
    csr_rowblock_kernel(int64_t n_rows, int64_t n_cols, int R, int band, int xbuf, const int32_t* __restrict__ row_ptr,
                        const int32_t* __restrict__ col, const V* __restrict__ val, const T* __restrict__ x,
                        T* __restrict__ y, T alpha, T beta, uint32_t* err, Cg1Reduce red, uint32_t polls)
{
    using G = RbStage<V>;
    constexpr int kXAl = 16 / static_cast<int>(sizeof(T));
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar[2];
    __shared__ RbInfo info[2];
    const int tid = threadIdx.x;
    const int64_t n_blocks = (n_rows + R - 1) / R;
    const int64_t stride = gridDim.x;
    const size_t stage_bytes = G::kBase + (kX ? static_cast<size_t>(xbuf) * sizeof(T) : 0);
    auto base = [&](int st) { return smem + st * stage_bytes; };
    auto s_val = [&](int st) { return reinterpret_cast<V*>(base(st)); };
    auto s_col = [&](int st) { return reinterpret_cast<int32_t*>(base(st) + G::kVal); };
    auto s_rp = [&](int st) { return reinterpret_cast<int32_t*>(base(st) + G::kVal + G::kCol); };
    auto s_x = [&](int st) { return reinterpret_cast<T*>(base(st) + G::kBase); };
    // e0 = row_ptr[r0], e1 = row_ptr[r1] (prefetched by the caller)
    auto issue = [&](int64_t b, int st, int32_t e0, int32_t e1) {
        RbInfo ti;
        ti.r0 = static_cast<int32_t>(b * R);
        ti.r1 = static_cast<int32_t>(min(static_cast<int64_t>(ti.r0) + R, n_rows));
        ti.a0 = e0 / G::kAlign * G::kAlign;
        ti.ra0 = ti.r0 & ~3;
        const int cnt = max(G::kAlign, (e1 - ti.a0 + G::kAlign - 1) / G::kAlign * G::kAlign);
        const int rcnt = (ti.r1 + 1 - ti.ra0 + 3) & ~3;
        uint32_t bytes = cnt * static_cast<uint32_t>(sizeof(V) + sizeof(int32_t)) + rcnt * 4;
        ti.w0 = 0;
        ti.wl = 0;
        if (kX) {
            ti.w0 = max(0, ti.r0 - band) / kXAl * kXAl;
            const int64_t w1 = min(n_cols, static_cast<int64_t>(ti.r1) + band);
            ti.wl = static_cast<int32_t>(w1 - ti.w0) / kXAl * kXAl;  // a ragged last part is read from x
            bytes += ti.wl * sizeof(T);
        }
        info[st] = ti;
        mbar_arrive_expect_tx(&bar[st], bytes);
        if (kHint) {
            const uint64_t pol = l2_evict_first_policy();
            bulk_g2s_hint(s_val(st), val + ti.a0, cnt * sizeof(V), &bar[st], pol);
            bulk_g2s_hint(s_col(st), col + ti.a0, cnt * sizeof(int32_t), &bar[st], pol);
            bulk_g2s_hint(s_rp(st), row_ptr + ti.ra0, rcnt * sizeof(int32_t), &bar[st], pol);
        } else {
            bulk_g2s(s_val(st), val + ti.a0, cnt * sizeof(V), &bar[st]);
            bulk_g2s(s_col(st), col + ti.a0, cnt * sizeof(int32_t), &bar[st]);
            bulk_g2s(s_rp(st), row_ptr + ti.ra0, rcnt * sizeof(int32_t), &bar[st]);
        }
        if (kX && ti.wl > 0) bulk_g2s(s_x(st), x + ti.w0, ti.wl * sizeof(T), &bar[st]);
    };
    auto meta0 = [&](int64_t b) { return row_ptr[b * R]; };
    auto meta1 = [&](int64_t b) { return row_ptr[min((b + 1) * R, n_rows)]; };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < 2; ++k) {
            const int64_t b = blockIdx.x + k * stride;
            if (b < n_blocks) issue(b, k, meta0(b), meta1(b));
        }

    T dot_rr = T(0), dot_wr = T(0);
    bool failed = false;
    for (int it = 0;; ++it) {
        const int64_t b = blockIdx.x + it * stride;
        if (b >= n_blocks) break;
        const int st = it & 1;
        const uint32_t parity = (it >> 1) & 1;
        const bool landed = mbar_wait_bounded(&bar[st], parity, err, polls);
        if (!__syncthreads_and(landed)) {  // CTA-uniform: give up on the rest
            // wait (default limit) for the copies still in flight into this
            // stage and the next one, so none lands after the CTA has exited
            if (tid == 0) {
                mbar_wait_bounded(&bar[st], parity, err);
                if (b + stride < n_blocks) mbar_wait_bounded(&bar[st ^ 1], ((it + 1) >> 1) & 1, err);
            }
            __syncthreads();
            failed = true;
            break;
        }
        const int64_t b_issue = b + 2 * stride;
        int32_t pe0 = 0, pe1 = 0;
        if (tid == 0 && b_issue < n_blocks) {
            pe0 = meta0(b_issue);
            pe1 = meta1(b_issue);
        }
        const RbInfo ti = info[st];
        const int32_t* rp = s_rp(st);
        const V* sv = s_val(st);
        const int32_t* sc = s_col(st);
        const T* sx = s_x(st);
        auto xat = [&](int c) -> T {
            if (kX) {
                const unsigned o = static_cast<unsigned>(c - ti.w0);
                return o < static_cast<unsigned>(ti.wl) ? sx[o] : ldg(x + c);
            }
            return ldg(x + c);
        };
        for (int r = ti.r0 + tid; r < ti.r1; r += kRbThreads) {
            const int kb = rp[r - ti.ra0] - ti.a0;
            const int len = rp[r + 1 - ti.ra0] - ti.a0 - kb;
            // Rows of equal even length L sit L entries apart, so their lanes
            // would meet in the same shared-memory banks (all of them when L
            // is a multiple of 16).  Such rows are walked starting at entry
            // (tid mod L), wrapping around, which spreads the lanes over the
            // banks.  Odd lengths are conflict-free and keep the natural order
            // (neighbouring rows then gather neighbouring x entries).
            int k = (len > 0 && (len & 1) == 0) ? kb + tid % len : kb;
            const int kend = kb + len;
            T acc0 = T(0), acc1 = T(0);  // two chains: more arithmetic in flight
            for (int j0 = 0; j0 < len; j0 += CH) {
                T xv[CH];
                int kk[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {  // all gathers of the chunk first
                    kk[u] = k;
                    xv[u] = (j0 + u < len) ? xat(sc[k]) : T(0);
                    k = (k + 1 == kend) ? kb : k + 1;
                }
#pragma unroll
                for (int u = 0; u < CH; u += 2) {
                    if (j0 + u < len) acc0 = fma(to_t<V, T>(sv[kk[u]]), xv[u], acc0);
                    if (u + 1 < CH && j0 + u + 1 < len) acc1 = fma(to_t<V, T>(sv[kk[u + 1]]), xv[u + 1], acc1);
                }
            }
            const T w = acc0 + acc1;
            seg_store<kAlpha, kBeta>(y, r, w, alpha, beta);
            if (kDots) {
                const T xr = ldg(x + r);
                dot_rr = fma(xr, xr, dot_rr);
                dot_wr = fma(w, xr, dot_wr);
            }
        }
        __syncthreads();  // the stage is free again
        if (tid == 0 && b_issue < n_blocks) {
            fence_proxy_async_smem();
            issue(b_issue, st, pe0, pe1);
        }
    }
    if (kDots) {
        // every block takes part in the reduction (a failed one with NaN),
        // so the scalar step always runs and the solver loop always ends
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        const double g = failed ? nan : static_cast<double>(dot_rr);
        const double d = failed ? nan : static_cast<double>(dot_wr);
        SolverState* s = red.s;
        grid_sum2(g, d, red.part, &s->ticket,
                  [&](double gamma, double delta) { cg1_scalars(s, gamma, delta, red.err, red.h); });
    }
}

template <typename V, typename T, bool kX, int CH, bool kDots = false, bool kHint = false>
static cudaError_t launch_rowblock_ch(const gko_matrix* A, const V* val, const T* x, T* y, T alpha, T beta,
                                      cudaStream_t st, Cg1Reduce red = Cg1Reduce{})
{
    const int R = rowblock_rows(A);
    const int band = kX ? A->csr.band : -1;
    const int xbuf = kX ? rb_xbuf<T>(R, band) : 0;
    const int64_t n_blocks = (A->n_rows + R - 1) / R;
    const int64_t grid = std::min<int64_t>(n_blocks, seg_grid_ctas());
    const size_t smem = 2 * (RbStage<V>::kBase + static_cast<size_t>(xbuf) * sizeof(T));
    const bool a = alpha != T(1), b = beta != T(0);
    cudaError_t e = cudaSuccess;
#define GKO_RB(KA, KB)                                                                                    \
    do {                                                                                                  \
        e = smem_limit_once(                                                                              \
            reinterpret_cast<const void*>(csr_rowblock_kernel<V, T, KA, KB, kX, CH, kDots, kHint>),       \
            static_cast<int>(smem));                                                                      \
        if (e != cudaSuccess) return e;                                                                   \
        csr_rowblock_kernel<V, T, KA, KB, kX, CH, kDots, kHint>                                           \
            <<<static_cast<unsigned>(grid), kRbThreads, smem, st>>>(A->n_rows, A->n_cols, R, band, xbuf,  \
                                                                    A->csr.row_ptr, A->csr.col, val, x, y, \
                                                                    alpha, beta, A->d_err, red,           \
                                                                    first_wait_polls());                  \
    } while (0)
    if (kDots)
        GKO_RB(false, false);
    else if (a && b)
        GKO_RB(true, true);
    else if (a)
        GKO_RB(true, false);
    else if (b)
        GKO_RB(false, true);
    else
        GKO_RB(false, false);
#undef GKO_RB
    return cudaGetLastError();
}

// chunk of 8 gathers for short rows, 16 otherwise
template <typename V, typename T, bool kX, bool kDots = false, bool kHint = false>
static cudaError_t launch_rowblock_t(const gko_matrix* A, const V* val, const T* x, T* y, T alpha, T beta,
                                     cudaStream_t st, Cg1Reduce red = Cg1Reduce{})
{
    if (A->csr.max_len <= 8) return launch_rowblock_ch<V, T, kX, 8, kDots, kHint>(A, val, x, y, alpha, beta, st, red);
    return launch_rowblock_ch<V, T, kX, 16, kDots, kHint>(A, val, x, y, alpha, beta, st, red);
}

int spmv_csr_rowblock(const gko_matrix* A, const double* x, double* y, double alpha, double beta, cudaStream_t st)
{
    if (rowblock_rows(A) <= 0) return fail(GKO_ERR_INVALID_ARG, "row-block CSR needs 1 <= max row length <= 128");
    const cudaError_t e = launch_rowblock_t<double, double, false>(A, A->csr.val, x, y, alpha, beta, st);
    return e == cudaSuccess ? GKO_OK : cuda_fail(e, "row-block CSR launch");
}

int spmv_csr_banded(const gko_matrix* A, const double* x, double* y, double alpha, double beta, cudaStream_t st)
{
    if (rowblock_rows(A) <= 0 || A->csr.band < 0 || A->csr.band > kRbMaxBand)
        return fail(GKO_ERR_INVALID_ARG, "banded CSR needs max row length <= 128 and max |i - j| <= 1024");
    cudaError_t e;
    if (reinterpret_cast<uintptr_t>(x) % 16 != 0)  // bulk copies need a 16-byte aligned x
        e = launch_rowblock_t<double, double, false>(A, A->csr.val, x, y, alpha, beta, st);
    else
        e = launch_rowblock_t<double, double, true>(A, A->csr.val, x, y, alpha, beta, st);
    return e == cudaSuccess ? GKO_OK : cuda_fail(e, "banded CSR launch");
}

// y = A_lo x in FP32 for the mixed-precision inner solve (values float or bf16)
cudaError_t rowblock_lowprec_f32(const gko_matrix* A, const float* val, const float* x, float* y, cudaStream_t st)
{
    return launch_rowblock_t<float, float, false>(A, val, x, y, 1.0f, 0.0f, st);
}
cudaError_t rowblock_lowprec_bf16(const gko_matrix* A, const void* val, const float* x, float* y, cudaStream_t st)
{
    return launch_rowblock_t<__nv_bfloat16, float, false>(A, static_cast<const __nv_bfloat16*>(val), x, y, 1.0f,
                                                          0.0f, st);
}

// Product of a single-reduction CG step: w = A r with the step's dots and
// scalars fused (double, float or bf16 values; FP64 or FP32 vectors).  The
// matrix streams are marked evict-first in L2 so the solver's vectors stay
// cached between the steps.
cudaError_t rowblock_cg1_f64(const gko_matrix* A, const double* r, double* w, Cg1Reduce red, cudaStream_t st)
{
    return launch_rowblock_t<double, double, false, true, true>(A, A->csr.val, r, w, 1.0, 0.0, st, red);
}
cudaError_t rowblock_cg1_f32(const gko_matrix* A, const float* val, const float* r, float* w, Cg1Reduce red,
                             cudaStream_t st)
{
    return launch_rowblock_t<float, float, false, true, true>(A, val, r, w, 1.0f, 0.0f, st, red);
}
cudaError_t rowblock_cg1_bf16(const gko_matrix* A, const void* val, const float* r, float* w, Cg1Reduce red,
                              cudaStream_t st)
{
    return launch_rowblock_t<__nv_bfloat16, float, false, true, true>(A, static_cast<const __nv_bfloat16*>(val), r,
                                                                      w, 1.0f, 0.0f, st, red);
}

}  // namespace gko
