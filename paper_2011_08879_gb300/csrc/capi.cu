// The C ABI (include/gko_gb300.h): argument checking, the matrix handle's
// lifetime, format dispatch.  Every entry point returns a status and
// records a message; none aborts.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "common.cuh"
#include "internal.h"

namespace gko {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int status, const std::string& msg)
{
    g_last_error = msg;
    return status;
}

int cuda_fail(cudaError_t e, const char* what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();  // clear non-sticky errors
    return e == cudaErrorMemoryAllocation ? GKO_ERR_OUT_OF_MEMORY : GKO_ERR_CUDA;
}

// ------------------------------------------------------ per-device state

namespace {
constexpr int kDevCache = 64;  // devices with cached state (others query every time)
std::mutex g_dev_mu;
int g_sm_count[kDevCache] = {0};
std::unordered_map<const void*, std::array<int, kDevCache>> g_smem_set;  // limit set per kernel and device
std::atomic<uint32_t> g_first_wait_polls{1u << 22};
}  // namespace

int device_sm_count()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < kDevCache) {
        std::lock_guard<std::mutex> lk(g_dev_mu);
        if (g_sm_count[dev] > 0) return g_sm_count[dev];
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    if (dev >= 0 && dev < kDevCache) {
        std::lock_guard<std::mutex> lk(g_dev_mu);
        g_sm_count[dev] = sms;
    }
    return sms;
}

cudaError_t smem_limit_once(const void* kernel, int bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kDevCache)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    auto it = g_smem_set.find(kernel);
    if (it == g_smem_set.end()) {
        std::array<int, kDevCache> z{};
        it = g_smem_set.emplace(kernel, z).first;
    }
    if (it->second[dev] >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) it->second[dev] = bytes;
    return e;
}

uint32_t first_wait_polls() { return g_first_wait_polls.load(std::memory_order_relaxed); }

static bool valid_fmt(int f) { return f >= GKO_FMT_CSR && f <= GKO_FMT_HYBRID; }

static int check_device(const gko_matrix* A)
{
    int dev = -1;
    GKO_CUDA(cudaGetDevice(&dev));
    if (dev != A->device) return fail(GKO_ERR_INVALID_ARG, "handle used on another device than it was created on");
    return GKO_OK;
}

}  // namespace gko

using namespace gko;

extern "C" {

const char* gko_last_error(void) { return g_last_error.c_str(); }

const char* gko_version(void) { return "gko-gb300 1.0 (sm_103a)"; }

int gko_set_wait_limit(uint32_t polls)
{
    g_first_wait_polls.store(polls == UINT32_MAX ? (1u << 22) : polls, std::memory_order_relaxed);
    return GKO_OK;
}

const char* gko_status_string(int s)
{
    switch (s) {
        case GKO_OK: return "GKO_OK";
        case GKO_ERR_INVALID_ARG: return "GKO_ERR_INVALID_ARG";
        case GKO_ERR_DIM_MISMATCH: return "GKO_ERR_DIM_MISMATCH";
        case GKO_ERR_FORMAT_UNAVAILABLE: return "GKO_ERR_FORMAT_UNAVAILABLE";
        case GKO_ERR_FORMAT_TOO_LARGE: return "GKO_ERR_FORMAT_TOO_LARGE";
        case GKO_ERR_OUT_OF_MEMORY: return "GKO_ERR_OUT_OF_MEMORY";
        case GKO_ERR_NOT_CONVERGED: return "GKO_ERR_NOT_CONVERGED";
        case GKO_ERR_BREAKDOWN: return "GKO_ERR_BREAKDOWN";
        case GKO_ERR_INVALID_MATRIX: return "GKO_ERR_INVALID_MATRIX";
        case GKO_ERR_TIMEOUT: return "GKO_ERR_TIMEOUT";
        case GKO_ERR_CUDA: return "GKO_ERR_CUDA";
        default: return "GKO_ERR_UNKNOWN";
    }
}

int gko_matrix_create_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                          const double* val, int on_device, void* stream, gko_matrix** out)
{
    if (!out) return fail(GKO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_rows < 0 || n_cols < 0 || nnz < 0) return fail(GKO_ERR_INVALID_ARG, "negative size");
    // int32 indices; a margin of 2^16 keeps tile arithmetic in int32
    if (n_rows >= INT32_MAX - 65536 || n_cols >= INT32_MAX - 65536 || nnz >= INT32_MAX - 65536)
        return fail(GKO_ERR_INVALID_ARG, "sizes must be below 2^31 - 2^16 (int32 indices)");
    if (!row_ptr || (nnz > 0 && (!col || !val))) return fail(GKO_ERR_INVALID_ARG, "NULL array");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    gko_matrix* A = new gko_matrix();
    GKO_CUDA(cudaGetDevice(&A->device));
    A->n_rows = n_rows;
    A->n_cols = n_cols;
    A->nnz = nnz;
    auto cleanup = [&](int s) {
        gko_matrix_destroy(A);
        return s;
    };
    const int64_t alloc = padded_len(nnz);
    int s;
    if ((s = dev_alloc(&A->d_err, 1)) != GKO_OK) return cleanup(s);
    if ((s = dev_alloc(&A->csr.row_ptr, padded_len(n_rows + 1))) != GKO_OK) return cleanup(s);
    if ((s = dev_alloc(&A->csr.col, alloc)) != GKO_OK) return cleanup(s);
    if ((s = dev_alloc(&A->csr.val, alloc)) != GKO_OK) return cleanup(s);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemsetAsync(A->d_err, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(A->csr.row_ptr, row_ptr, (n_rows + 1) * sizeof(int32_t), kind, st);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(A->csr.col, col, nnz * sizeof(int32_t), kind, st);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(A->csr.val, val, nnz * sizeof(double), kind, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(A->csr.row_ptr + n_rows + 1, 0, (padded_len(n_rows + 1) - n_rows - 1) * sizeof(int32_t),
                            st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(A->csr.col + nnz, 0, (alloc - nnz) * sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(A->csr.val + nnz, 0, (alloc - nnz) * sizeof(double), st);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "copying the CSR input"));
    if ((s = validate_csr(n_rows, n_cols, nnz, A->csr.row_ptr, A->csr.col, st)) != GKO_OK) return cleanup(s);
    if ((s = csr_analyse(A, st)) != GKO_OK) return cleanup(s);
    A->has[GKO_FMT_CSR] = true;
    *out = A;
    return GKO_OK;
}

int gko_matrix_destroy(gko_matrix* A)
{
    if (!A) return GKO_OK;
    for (int f = 0; f < 5; ++f) free_format(A, f);
    dev_free(A->d_err);
    dev_free(A->stage_x);
    dev_free(A->stage_y);
    dev_free(A->val_f32);
    dev_free(A->val_bf16);
    lp_ell_free(A);
    delete A;
    return GKO_OK;
}

int gko_matrix_set_params(gko_matrix* A, int sellp_slice, int sellp_stride, double ell_factor)
{
    if (!A) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (sellp_slice > 0) {
        if (sellp_slice > 128 || (sellp_slice & (sellp_slice - 1)))
            return fail(GKO_ERR_INVALID_ARG, "SELL-P slice size must be a power of two <= 128");
        A->sellp_S = sellp_slice;
    }
    if (sellp_stride > 0) A->sellp_f = sellp_stride;
    if (ell_factor > 0) A->ell_factor = ell_factor;
    return GKO_OK;
}

int gko_convert(gko_matrix* A, int src, int dst, void* stream)
{
    if (!A) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (!valid_fmt(src) || !valid_fmt(dst)) return fail(GKO_ERR_INVALID_ARG, "unknown format");
    GKO_TRY(check_device(A));
    if (!A->has[src]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "source format not materialised");
    if (src == dst) return GKO_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (src == GKO_FMT_CSR) {
        switch (dst) {
            case GKO_FMT_COO: return convert_csr_to_coo(A, st);
            case GKO_FMT_ELL: return convert_csr_to_ell(A, st);
            case GKO_FMT_SELLP: return convert_csr_to_sellp(A, st);
            case GKO_FMT_HYBRID: return convert_csr_to_hybrid(A, st);
        }
    }
    if (dst == GKO_FMT_CSR) {
        switch (src) {
            case GKO_FMT_COO: return convert_coo_to_csr(A, st);
            case GKO_FMT_ELL: return convert_ell_to_csr(A, st);
            case GKO_FMT_SELLP: return convert_sellp_to_csr(A, st);
            case GKO_FMT_HYBRID: return convert_hybrid_to_csr(A, st);
        }
    }
    // other pairs go through CSR
    if (!A->has[GKO_FMT_CSR]) GKO_TRY(gko_convert(A, src, GKO_FMT_CSR, stream));
    return gko_convert(A, GKO_FMT_CSR, dst, stream);
}

int gko_matrix_release(gko_matrix* A, int fmt)
{
    if (!A) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (!valid_fmt(fmt)) return fail(GKO_ERR_INVALID_ARG, "unknown format");
    if (!A->has[fmt]) return GKO_OK;
    int others = 0;
    for (int f = 0; f < 5; ++f) others += (f != fmt) && A->has[f];
    if (!others) return fail(GKO_ERR_INVALID_ARG, "cannot release the only materialised format");
    cudaDeviceSynchronize();
    free_format(A, fmt);
    return GKO_OK;
}

int gko_matrix_info(const gko_matrix* A, int fmt, int64_t* info)
{
    if (!A || !info) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    if (!valid_fmt(fmt)) return fail(GKO_ERR_INVALID_ARG, "unknown format");
    for (int i = 0; i < 8; ++i) info[i] = 0;
    info[0] = A->has[fmt];
    info[1] = A->n_rows;
    info[2] = A->n_cols;
    info[3] = A->nnz;
    if (!A->has[fmt]) return GKO_OK;
    switch (fmt) {
        case GKO_FMT_CSR: info[4] = A->csr.max_len; break;
        case GKO_FMT_COO: break;
        case GKO_FMT_ELL:
            info[4] = A->ell.K;
            info[5] = A->ell.n_pad;
            info[6] = A->ell.K * A->ell.n_pad;
            break;
        case GKO_FMT_SELLP:
            info[4] = A->sellp.S;
            info[5] = A->sellp.n_slices;
            info[6] = A->sellp.slots;
            info[7] = A->sellp.f;
            break;
        case GKO_FMT_HYBRID:
            info[4] = A->hyb.ell.K;
            info[5] = A->hyb.ell.n_pad;
            info[6] = A->hyb.coo.nnz;
            break;
    }
    return GKO_OK;
}

int gko_matrix_export(const gko_matrix* A, int fmt, int array, void* dst, int64_t bytes, int to_host, void* stream)
{
    if (!A || (!dst && bytes > 0)) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    if (!valid_fmt(fmt)) return fail(GKO_ERR_INVALID_ARG, "unknown format");
    if (!A->has[fmt]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "format not materialised");
    const void* src = nullptr;
    int64_t size = -1;
    const int64_t n = A->n_rows, nnz = A->nnz;
    switch (fmt) {
        case GKO_FMT_CSR:
            if (array == 0) src = A->csr.row_ptr, size = (n + 1) * 4;
            if (array == 1) src = A->csr.col, size = nnz * 4;
            if (array == 2) src = A->csr.val, size = nnz * 8;
            break;
        case GKO_FMT_COO:
            if (array == 0) src = A->coo.row, size = nnz * 4;
            if (array == 1) src = A->coo.col, size = nnz * 4;
            if (array == 2) src = A->coo.val, size = nnz * 8;
            break;
        case GKO_FMT_ELL: {
            const int64_t slots = A->ell.K * A->ell.n_pad;
            if (array == 0) src = A->ell.col, size = slots * 4;
            if (array == 1) src = A->ell.val, size = slots * 8;
            break;
        }
        case GKO_FMT_SELLP:
            if (array == 0) src = A->sellp.slice_len, size = A->sellp.n_slices * 4;
            if (array == 1) src = A->sellp.slice_set, size = (A->sellp.n_slices + 1) * 4;
            if (array == 2) src = A->sellp.col, size = A->sellp.slots * 4;
            if (array == 3) src = A->sellp.val, size = A->sellp.slots * 8;
            break;
        case GKO_FMT_HYBRID: {
            const int64_t slots = A->hyb.ell.K * A->hyb.ell.n_pad, c = A->hyb.coo.nnz;
            if (array == 0) src = A->hyb.ell.col, size = slots * 4;
            if (array == 1) src = A->hyb.ell.val, size = slots * 8;
            if (array == 2) src = A->hyb.coo.row, size = c * 4;
            if (array == 3) src = A->hyb.coo.col, size = c * 4;
            if (array == 4) src = A->hyb.coo.val, size = c * 8;
            break;
        }
    }
    if (size < 0) return fail(GKO_ERR_INVALID_ARG, "unknown array index for this format");
    if (bytes != size) return fail(GKO_ERR_DIM_MISMATCH, "bytes does not match the array size");
    if (size == 0) return GKO_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GKO_CUDA(cudaMemcpyAsync(dst, src, size, to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    return GKO_OK;
}

int gko_matrix_errors(gko_matrix* A, uint32_t* bits, int clear, void* stream)
{
    if (!A || !bits) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GKO_CUDA(cudaMemcpyAsync(bits, A->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    if (clear) GKO_CUDA(cudaMemsetAsync(A->d_err, 0, sizeof(uint32_t), st));
    return GKO_OK;
}

int gko_select_format(gko_matrix* A, int* fmt, int* config, void* stream);

}  // extern "C"

namespace gko {

const int kCandFmt[GKO_N_CANDIDATES] = {GKO_FMT_CSR, GKO_FMT_CSR, GKO_FMT_CSR,   GKO_FMT_CSR,    GKO_FMT_COO,
                                        GKO_FMT_ELL, GKO_FMT_SELLP, GKO_FMT_HYBRID, GKO_FMT_CSR, GKO_FMT_CSR};
const int kCandCfg[GKO_N_CANDIDATES] = {GKO_CFG_CSR_ROWBLOCK,  GKO_CFG_CSR_NNZSPLIT, GKO_CFG_CSR_SUBWARP_4,
                                        GKO_CFG_CSR_SUBWARP_32, 0, 0, 0, 0, GKO_CFG_CSR_BINNED,
                                        GKO_CFG_CSR_SUBWARP_1};

static int spmv_dispatch(int fmt, int config, const gko_matrix* A, const double* x, double* y, double alpha,
                         double beta, cudaStream_t st);

// Key of the AUTO choice: the selector generation and the materialised
// formats (a new selector or a converted/released format invalidates it).
static uint64_t auto_key(const gko_matrix* A)
{
    uint64_t mask = 0;
    for (int f = 0; f < 5; ++f) mask |= static_cast<uint64_t>(A->has[f]) << f;
    return (selector_generation() << 8) | (1u << 7) | mask;
}

// Exhaustive autotuning: every candidate the handle can run, one warm-up
// and five timed launches each (CUDA events on the stream, on the handle's
// staging vectors, alpha = 1, beta = 0), median per candidate, fastest wins.
static int autotune(gko_matrix* A, int* fmt, int* cfg, double* times_us, cudaStream_t st)
{
    constexpr int kReps = 5;
    if (!A->stage_x) {
        GKO_TRY(dev_alloc(&A->stage_x, std::max<int64_t>(A->n_cols, 1)));
        GKO_TRY(dev_alloc(&A->stage_y, std::max<int64_t>(A->n_rows, 1)));
    }
    GKO_CUDA(cudaMemsetAsync(A->stage_x, 0, std::max<int64_t>(A->n_cols, 1) * sizeof(double), st));
    cudaEvent_t ev[GKO_N_CANDIDATES][kReps + 1] = {};
    bool live[GKO_N_CANDIDATES] = {};
    int status = GKO_OK;
    for (int c = 0; c < GKO_N_CANDIDATES && status == GKO_OK; ++c) {
        if (!A->has[kCandFmt[c]]) continue;
        const std::string keep = gko_last_error();
        if (spmv_dispatch(kCandFmt[c], kCandCfg[c], A, A->stage_x, A->stage_y, 1.0, 0.0, st) != GKO_OK) {
            set_error(keep);  // configuration does not apply to this matrix
            continue;
        }
        live[c] = true;
        for (int k = 0; k <= kReps && status == GKO_OK; ++k) {
            cudaError_t e = cudaEventCreate(&ev[c][k]);
            if (e == cudaSuccess) e = cudaEventRecord(ev[c][k], st);
            if (e != cudaSuccess) status = cuda_fail(e, "autotuner events");
            if (status == GKO_OK && k < kReps)
                status = spmv_dispatch(kCandFmt[c], kCandCfg[c], A, A->stage_x, A->stage_y, 1.0, 0.0, st);
        }
    }
    if (status == GKO_OK) {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) status = cuda_fail(e, "autotuner timing");
    }
    int best = -1;
    double best_t = 0.0;
    for (int c = 0; c < GKO_N_CANDIDATES; ++c) {
        double med = NAN;
        if (live[c] && status == GKO_OK) {
            float ms[kReps];
            for (int k = 0; k < kReps; ++k) cudaEventElapsedTime(&ms[k], ev[c][k], ev[c][k + 1]);
            std::sort(ms, ms + kReps);
            med = 1e3 * ms[kReps / 2];
            if (best < 0 || med < best_t) best = c, best_t = med;
        }
        if (times_us) times_us[c] = med;
        for (int k = 0; k <= kReps; ++k)
            if (ev[c][k]) cudaEventDestroy(ev[c][k]);
    }
    if (status != GKO_OK) return status;
    *fmt = best >= 0 ? kCandFmt[best] : GKO_FMT_CSR;
    *cfg = best >= 0 ? kCandCfg[best] : GKO_CFG_DEFAULT;
    return GKO_OK;
}

static int spmv_dispatch(int fmt, int config, const gko_matrix* A, const double* x, double* y, double alpha,
                         double beta, cudaStream_t st)
{
    if (fmt == GKO_FMT_AUTO) {
        gko_matrix* M = const_cast<gko_matrix*>(A);
        const uint64_t key = auto_key(M);
        if (M->auto_fmt < 0 || M->auto_key != key) {
            int f = GKO_FMT_CSR, c = GKO_CFG_DEFAULT;
            if (selector_generation() != 0)
                GKO_TRY(gko_select_format(M, &f, &c, st));
            else
                GKO_TRY(autotune(M, &f, &c, nullptr, st));
            if (!M->has[f]) f = GKO_FMT_CSR, c = GKO_CFG_DEFAULT;
            M->auto_fmt = f;
            M->auto_cfg = c;
            M->auto_key = key;
        }
        return spmv_dispatch(M->auto_fmt, M->auto_cfg, A, x, y, alpha, beta, st);
    }
    if (!A->has[fmt]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "format not materialised (call gko_convert first)");
    if (fmt != GKO_FMT_CSR && config != GKO_CFG_DEFAULT)
        return fail(GKO_ERR_INVALID_ARG, "kernel configurations apply to CSR only");
    switch (fmt) {
        case GKO_FMT_CSR: return spmv_csr(A, config, x, y, alpha, beta, st);
        case GKO_FMT_COO: return spmv_coo(A, A->coo, x, y, alpha, beta, st);
        case GKO_FMT_ELL: return spmv_ell(A, A->ell, x, y, alpha, beta, st);
        case GKO_FMT_SELLP: return spmv_sellp(A, x, y, alpha, beta, st);
        case GKO_FMT_HYBRID: return spmv_hybrid(A, x, y, alpha, beta, st);
    }
    return fail(GKO_ERR_INVALID_ARG, "unknown format");
}

}  // namespace gko

extern "C" {

int gko_autotune_format(gko_matrix* A, int* fmt, int* config, double* times_us, void* stream)
{
    if (!A || !fmt || !config) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    GKO_TRY(check_device(A));
    *fmt = GKO_FMT_CSR;
    *config = GKO_CFG_DEFAULT;
    if (A->n_rows == 0) {
        if (times_us)
            for (int c = 0; c < GKO_N_CANDIDATES; ++c) times_us[c] = NAN;
        return GKO_OK;
    }
    GKO_TRY(autotune(A, fmt, config, times_us, static_cast<cudaStream_t>(stream)));
    if (selector_generation() == 0) {  // the choice GKO_FMT_AUTO uses without a selector
        A->auto_fmt = *fmt;
        A->auto_cfg = *config;
        A->auto_key = auto_key(A);
    }
    return GKO_OK;
}

static int spmv_checks(int fmt, const gko_matrix* A, const double* x, const double* y)
{
    if (!A) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (!(valid_fmt(fmt) || fmt == GKO_FMT_AUTO)) return fail(GKO_ERR_INVALID_ARG, "unknown format");
    if ((!x && A->n_cols > 0) || (!y && A->n_rows > 0)) return fail(GKO_ERR_INVALID_ARG, "NULL vector");
    if (x && y && static_cast<const void*>(x) == static_cast<const void*>(y) && A->n_rows > 0)
        return fail(GKO_ERR_INVALID_ARG, "x and y must not alias");
    return check_device(A);
}

int gko_spmv(int fmt, const gko_matrix* A, const double* x, double* y, double alpha, double beta, void* stream)
{
    GKO_TRY(spmv_checks(fmt, A, x, y));
    return spmv_dispatch(fmt, GKO_CFG_DEFAULT, A, x, y, alpha, beta, static_cast<cudaStream_t>(stream));
}

int gko_spmv_config(int fmt, int config, const gko_matrix* A, const double* x, double* y, double alpha,
                    double beta, void* stream)
{
    GKO_TRY(spmv_checks(fmt, A, x, y));
    if (config < GKO_CFG_DEFAULT || config > GKO_CFG_CSR_BINNED)
        return fail(GKO_ERR_INVALID_ARG, "unknown kernel configuration");
    if (fmt == GKO_FMT_AUTO) return fail(GKO_ERR_INVALID_ARG, "AUTO takes no explicit configuration");
    return spmv_dispatch(fmt, config, A, x, y, alpha, beta, static_cast<cudaStream_t>(stream));
}

int gko_spmm(const gko_matrix* A, int64_t k, const double* x, int64_t ldx, double* y, int64_t ldy, double alpha,
             double beta, void* stream)
{
    if (!A) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (!A->has[GKO_FMT_CSR]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "SpMM reads the CSR format");
    if (k < 0 || ldx < k || ldy < k || ldx < 1 || ldy < 1)
        return fail(GKO_ERR_INVALID_ARG, "k >= 0 and leading dimensions >= max(k, 1) required");
    if (k > 0 && ((A->n_cols > 0 && !x) || (A->n_rows > 0 && !y))) return fail(GKO_ERR_INVALID_ARG, "NULL block");
    GKO_TRY(check_device(A));
    return spmm_csr(A, k, x, ldx, y, ldy, alpha, beta, static_cast<cudaStream_t>(stream));
}

int gko_spmv_host(int fmt, const gko_matrix* A, const double* x_host, double* y_host, double alpha, double beta,
                  void* stream)
{
    GKO_TRY(spmv_checks(fmt, A, x_host, y_host));
    gko_matrix* M = const_cast<gko_matrix*>(A);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!M->stage_x) {
        GKO_TRY(dev_alloc(&M->stage_x, std::max<int64_t>(A->n_cols, 1)));
        GKO_TRY(dev_alloc(&M->stage_y, std::max<int64_t>(A->n_rows, 1)));
    }
    if (A->n_cols > 0)
        GKO_CUDA(cudaMemcpyAsync(M->stage_x, x_host, A->n_cols * sizeof(double), cudaMemcpyHostToDevice, st));
    if (beta != 0.0 && A->n_rows > 0)
        GKO_CUDA(cudaMemcpyAsync(M->stage_y, y_host, A->n_rows * sizeof(double), cudaMemcpyHostToDevice, st));
    GKO_TRY(spmv_dispatch(fmt, GKO_CFG_DEFAULT, A, M->stage_x, M->stage_y, alpha, beta, st));
    if (A->n_rows > 0)
        GKO_CUDA(cudaMemcpyAsync(y_host, M->stage_y, A->n_rows * sizeof(double), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    return GKO_OK;
}

int gko_cg(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit, void* stream,
           gko_solve_info* info)
{
    if (!A) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (A->n_rows != A->n_cols) return fail(GKO_ERR_DIM_MISMATCH, "CG needs a square matrix");
    if (!valid_fmt(fmt)) return fail(GKO_ERR_INVALID_ARG, "unknown format");
    if (!A->has[fmt]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "format not materialised");
    if (A->n_rows > 0 && (!b || !x)) return fail(GKO_ERR_INVALID_ARG, "NULL vector");
    if (!(tol >= 0.0) || maxit < 0) return fail(GKO_ERR_INVALID_ARG, "tol must be >= 0 and maxit >= 0");
    GKO_TRY(check_device(A));
    return cg_solve(A, fmt, b, x, tol, maxit, static_cast<cudaStream_t>(stream), info);
}

int gko_cg_single_reduction(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit,
                            void* stream, gko_solve_info* info)
{
    if (!A) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (A->n_rows != A->n_cols) return fail(GKO_ERR_DIM_MISMATCH, "CG needs a square matrix");
    if (!valid_fmt(fmt)) return fail(GKO_ERR_INVALID_ARG, "unknown format");
    if (!A->has[fmt]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "format not materialised");
    if (A->n_rows > 0 && (!b || !x)) return fail(GKO_ERR_INVALID_ARG, "NULL vector");
    if (!(tol >= 0.0) || maxit < 0) return fail(GKO_ERR_INVALID_ARG, "tol must be >= 0 and maxit >= 0");
    GKO_TRY(check_device(A));
    return cg1_solve(A, fmt, b, x, tol, maxit, static_cast<cudaStream_t>(stream), info);
}

int gko_pcg_jacobi(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit, void* stream,
                   gko_solve_info* info)
{
    if (!A) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (A->n_rows != A->n_cols) return fail(GKO_ERR_DIM_MISMATCH, "CG needs a square matrix");
    if (!valid_fmt(fmt)) return fail(GKO_ERR_INVALID_ARG, "unknown format");
    if (!A->has[fmt]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "format not materialised");
    if (!A->has[GKO_FMT_CSR]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "the preconditioner reads the CSR diagonal");
    if (A->n_rows > 0 && (!b || !x)) return fail(GKO_ERR_INVALID_ARG, "NULL vector");
    if (!(tol >= 0.0) || maxit < 0) return fail(GKO_ERR_INVALID_ARG, "tol must be >= 0 and maxit >= 0");
    GKO_TRY(check_device(A));
    return pcg_jacobi_solve(A, fmt, b, x, tol, maxit, static_cast<cudaStream_t>(stream), info);
}

int gko_bicgstab(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit, void* stream,
                 gko_solve_info* info)
{
    if (!A) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (A->n_rows != A->n_cols) return fail(GKO_ERR_DIM_MISMATCH, "BiCGSTAB needs a square matrix");
    if (!valid_fmt(fmt)) return fail(GKO_ERR_INVALID_ARG, "unknown format");
    if (!A->has[fmt]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "format not materialised");
    if (A->n_rows > 0 && (!b || !x)) return fail(GKO_ERR_INVALID_ARG, "NULL vector");
    if (!(tol >= 0.0) || maxit < 0) return fail(GKO_ERR_INVALID_ARG, "tol must be >= 0 and maxit >= 0");
    GKO_TRY(check_device(A));
    return bicgstab_solve(A, fmt, b, x, tol, maxit, static_cast<cudaStream_t>(stream), info);
}

int gko_gmres(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int restart, int maxit,
              void* stream, gko_solve_info* info)
{
    if (!A) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (A->n_rows != A->n_cols) return fail(GKO_ERR_DIM_MISMATCH, "GMRES needs a square matrix");
    if (!valid_fmt(fmt)) return fail(GKO_ERR_INVALID_ARG, "unknown format");
    if (!A->has[fmt]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "format not materialised");
    if (A->n_rows > 0 && (!b || !x)) return fail(GKO_ERR_INVALID_ARG, "NULL vector");
    if (!(tol >= 0.0) || maxit < 0 || restart < 1 || restart > 127)
        return fail(GKO_ERR_INVALID_ARG, "tol >= 0, maxit >= 0 and 1 <= restart <= 127 required");
    GKO_TRY(check_device(A));
    return gmres_solve(A, fmt, b, x, tol, restart, maxit, static_cast<cudaStream_t>(stream), info);
}

int gko_cg_mixed(gko_matrix* A, int inner_dtype, const double* b, double* x, double tol, int maxit_outer,
                 double inner_tol, int inner_maxit, void* stream, gko_solve_info* info)
{
    return gko_cg_mixed_precond(A, inner_dtype, GKO_PRECOND_NONE, b, x, tol, maxit_outer, inner_tol, inner_maxit,
                                stream, info);
}

int gko_cg_mixed_precond(gko_matrix* A, int inner_dtype, int precond, const double* b, double* x, double tol,
                         int maxit_outer, double inner_tol, int inner_maxit, void* stream, gko_solve_info* info)
{
    if (!A) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (precond != GKO_PRECOND_NONE && precond != GKO_PRECOND_JACOBI)
        return fail(GKO_ERR_INVALID_ARG, "precond must be GKO_PRECOND_NONE or GKO_PRECOND_JACOBI");
    if (A->n_rows != A->n_cols) return fail(GKO_ERR_DIM_MISMATCH, "CG needs a square matrix");
    if (inner_dtype != GKO_F32 && inner_dtype != GKO_BF16)
        return fail(GKO_ERR_INVALID_ARG, "inner_dtype must be GKO_F32 or GKO_BF16");
    if (!A->has[GKO_FMT_CSR]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "mixed CG needs the CSR format");
    if (A->n_rows > 0 && (!b || !x)) return fail(GKO_ERR_INVALID_ARG, "NULL vector");
    if (!(tol >= 0.0) || maxit_outer < 0 || !(inner_tol > 0.0) || inner_maxit < 1)
        return fail(GKO_ERR_INVALID_ARG, "bad tolerance or iteration limit");
    GKO_TRY(check_device(A));
    return cg_mixed_solve(A, inner_dtype, b, x, tol, maxit_outer, inner_tol, inner_maxit,
                          static_cast<cudaStream_t>(stream), info, precond);
}

int gko_features(const gko_matrix* A, double* out, void* stream)
{
    if (!A || !out) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    if (!A->has[GKO_FMT_CSR]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "features need the CSR format");
    if (A->n_rows == 0) return fail(GKO_ERR_INVALID_ARG, "features need at least one row");
    GKO_TRY(check_device(A));
    return features_compute(A, out, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
