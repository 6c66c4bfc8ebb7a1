// COO SpMV that allocates nothing: the load-balanced COO kernel with its
// per-tile carry arrays in a file-scope device array instead of memory
// owned by a matrix handle.  For callers that must not call cudaMalloc (or
// any allocator) once they are running: code that is captured into CUDA
// graphs or replayed under a fixed memory footprint, real-time loops that
// cannot afford an allocation's latency or failure, and hosts whose device
// memory belongs to another allocator (a framework's caching pool) that a
// library-side cudaMalloc would bypass and fragment.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "segmented.cuh"

namespace gko {

// Tiles of the COO kernel: 256 threads x kSegPCoo entries.
constexpr int64_t kNoAllocTile = static_cast<int64_t>(kSegThreads) * kSegPCoo;

// Carries of rows crossing tile boundaries for at most GKO_NOALLOC_MAX_TILES
// tiles (28 bytes per tile, 896 KiB in all).  Every GPU that loads the
// library holds this array until the process exits.
struct NoAllocScratch {
    double tail_val[GKO_NOALLOC_MAX_TILES];
    double head_val[GKO_NOALLOC_MAX_TILES];
    int32_t tail_row[GKO_NOALLOC_MAX_TILES];
    int32_t tail_pass[GKO_NOALLOC_MAX_TILES];
    int32_t head_row[GKO_NOALLOC_MAX_TILES];
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch, looked up once per device.  In host
// code the symbol's name only stands for the array; the kernel must get the
// address that cudaGetSymbolAddress returns for the current device.
constexpr int kNoAllocMaxDevices = 64;
static NoAllocScratch* g_scratch_addr[kNoAllocMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

static int noalloc_scratch(NoAllocScratch** out)
{
    int dev = 0;
    GKO_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(GKO_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_scratch_addr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_scratch_addr[dev];
    return GKO_OK;
}

}  // namespace gko

using namespace gko;

extern "C" int gko_spmv_coo_noalloc(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* row, const int32_t* col,
                                    const double* val, const double* x, double* y, double alpha, double beta,
                                    uint32_t* err_flags, void* stream)
{
    if (n_rows < 0 || n_cols < 0 || nnz < 0) return fail(GKO_ERR_INVALID_ARG, "negative size");
    if (n_rows >= INT32_MAX - 65536 || n_cols >= INT32_MAX - 65536)
        return fail(GKO_ERR_INVALID_ARG, "sizes must be below 2^31 - 2^16 (int32 indices)");
    if (nnz > GKO_NOALLOC_MAX_TILES * kNoAllocTile)
        return fail(GKO_ERR_INVALID_ARG,
                    "gko_spmv_coo_noalloc: nnz exceeds the fixed scratch (GKO_NOALLOC_MAX_TILES * 2816 entries)");
    if (nnz > 0 && n_cols == 0) return fail(GKO_ERR_DIM_MISMATCH, "entries in a matrix without columns");
    if ((nnz > 0 && (!row || !col || !val || !x)) || (n_rows > 0 && !y))
        return fail(GKO_ERR_INVALID_ARG, "NULL array");
    if (nnz > 0 && ((reinterpret_cast<uintptr_t>(row) | reinterpret_cast<uintptr_t>(col) |
                     reinterpret_cast<uintptr_t>(val)) & 15))
        return fail(GKO_ERR_INVALID_ARG, "gko_spmv_coo_noalloc: row, col and val must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_rows == 0) return GKO_OK;
    if (nnz == 0) return scale_vector(n_rows, y, beta, st);
    NoAllocScratch* s = nullptr;
    GKO_TRY(noalloc_scratch(&s));
    // every carry the fix-up reads is written earlier in the same call, so
    // the scratch needs no clearing between calls
    const SegScratch sc{s->tail_val, s->tail_row, s->tail_pass, s->head_val, s->head_row};
    const bool a = alpha != 1.0, b = beta != 0.0;
    cudaError_t e;
#define GKO_NA(KA, KB)                                                                                        \
    e = seg_launch<kSegPCoo, double, double, KA, KB, true, false, true>(n_rows, n_cols, nnz, nullptr, row, col, \
                                                                        val, nullptr, sc, x, y, alpha, beta, \
                                                                        err_flags, st)
    if (a && b)
        GKO_NA(true, true);
    else if (a)
        GKO_NA(true, false);
    else if (b)
        GKO_NA(false, true);
    else
        GKO_NA(false, false);
#undef GKO_NA
    if (e != cudaSuccess) return cuda_fail(e, "gko_spmv_coo_noalloc launch");
    return GKO_OK;
}
