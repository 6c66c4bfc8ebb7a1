// Host-side internals shared by the library's translation units: the
// matrix handle, error reporting and the kernel launchers each .cu exports.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gko_gb300.h"

namespace gko {

// --------------------------------------------------------------- errors

void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define GKO_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) return ::gko::cuda_fail(_e, #call);       \
    } while (0)

#define GKO_TRY(call)                    \
    do {                                 \
        int _s = (call);                 \
        if (_s != GKO_OK) return _s;     \
    } while (0)

// Owned device allocation helpers (stream-ordered frees are not used:
// handle arrays live as long as the handle).
template <typename T>
int dev_alloc(T** p, int64_t count)
{
    *p = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), static_cast<size_t>(count) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(GKO_ERR_OUT_OF_MEMORY, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    return GKO_OK;
}
template <typename T>
void dev_free(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

// Entries of value/index arrays are allocated rounded up to a multiple of
// 16 plus 16 so that 1-D bulk copies may move whole 16-byte groups past the
// last entry; the pad is zero-filled.
inline int64_t padded_len(int64_t n) { return (n + 15) / 16 * 16 + 16; }

constexpr int kSegP = 15;     // entries per thread of the load-balanced CSR kernel (and thr_row)
constexpr int kSegPCoo = 11;       // entries per thread of the load-balanced COO kernel (scattered columns;
                                   // also the allocation-free entry's tile)
constexpr int kSegPCooLocal = 13;  // ... for matrices whose columns stay near the diagonal
constexpr int kSegThreadsCoo = 64;  // threads per CTA (and per tile) of the load-balanced COO kernel

// ------------------------------------------------------------ the handle

struct SegArrays {
    double* tail_val = nullptr;
    int32_t* tail_row = nullptr;
    int32_t* tail_pass = nullptr;
    double* head_val = nullptr;
    int32_t* head_row = nullptr;
    int64_t n_tiles = 0;
};

struct CsrPart {
    int32_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
    int32_t* thr_row = nullptr;  // load-balanced analysis: row of entry g*P
    SegArrays seg;
    int32_t max_len = 0;
    double mean_len = 0.0;
    int32_t band = -1;  // max |i - j| (computed at analysis), -1 unknown
    int32_t* bin_rows = nullptr;  // rows grouped by length bin (binned kernel)
    int64_t bin_off[7] = {0, 0, 0, 0, 0, 0, 0};
    int4* bin_tasks = nullptr;    // (start, count, bin, 0) chunks of bin_rows in row order
    int64_t n_bin_tasks = 0;
};
constexpr int kCsrBins = 6;

struct CooPart {
    int32_t* row = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
    int64_t nnz = 0;
    int P = kSegPCoo;  // entries per thread of its load-balanced kernel (coo_entries_per_thread)
    SegArrays seg;
};

struct EllPart {
    int64_t K = 0, n_pad = 0;
    int32_t* col = nullptr;
    double* val = nullptr;
};

struct SellpPart {
    int64_t S = 64, f = 1, n_slices = 0, slots = 0;
    int32_t* slice_len = nullptr;
    int32_t* slice_set = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
};

struct HybridPart {
    EllPart ell;
    CooPart coo;
};

// ELL copy of the rounded matrix for the mixed-precision inner solve
// (lowprec_ell.cu): col holds int16 offsets c - i when idx16, else int32
// columns; K * n_pad slots.
struct LowPrecEll {
    bool tried = false, ok = false;
    int idx16 = 0;
    int64_t K = 0, n_pad = 0;
    void* col = nullptr;
    float* val_f32 = nullptr;
    uint16_t* val_bf16 = nullptr;
};

}  // namespace gko

struct gko_matrix {
    int device = 0;
    int64_t n_rows = 0, n_cols = 0, nnz = 0;
    bool has[5] = {false, false, false, false, false};
    gko::CsrPart csr;
    gko::CooPart coo;
    gko::EllPart ell;
    gko::SellpPart sellp;
    gko::HybridPart hyb;
    int sellp_S = 64, sellp_f = 1;
    double ell_factor = 4.0;
    uint32_t* d_err = nullptr;       // sticky device error bits
    double* stage_x = nullptr;       // gko_spmv_host staging
    double* stage_y = nullptr;
    float* val_f32 = nullptr;        // mixed-precision copies (CSR order)
    uint16_t* val_bf16 = nullptr;
    gko::LowPrecEll lp_ell;          // ELL layout of those copies (when padding is small)
    bool feats_valid = false;
    double feats[12] = {0};
    int auto_fmt = -1, auto_cfg = 0;  // cached GKO_FMT_AUTO choice (-1: not made yet)
    uint64_t auto_key = 0;            // selector generation and format mask it was made for
};

struct gko_batch {
    int device = 0;
    int64_t count = 0, n_rows = 0, nnz = 0;
    int64_t* row_off = nullptr;   // device, count + 1
    int32_t* row_ptr = nullptr;   // device, n_rows + 1 (global)
    int32_t* col = nullptr;       // device, local column indices
    double* val = nullptr;
    int32_t* order = nullptr;     // systems sorted by decreasing size (work queue order)
    int32_t* perm = nullptr;      // per system: the caller's row of each stored (renumbered) row
    int32_t* queue = nullptr;     // device work-queue counter
    double* res = nullptr;        // per system: relative residual
    int32_t* iters = nullptr;     // per system: iterations
    int32_t* status = nullptr;    // per system: status
    int32_t max_rows = 0;
    int best_block = 0;           // autotuned block size (0 = not tuned)
    uint32_t* d_err = nullptr;
    double* scratch = nullptr;    // split layout: x, r (, A p) of each resident block
    int64_t scratch_len = 0;      // doubles
    // instantiated graph of the last solve [queue reset + kernel], relaunched
    // while the launch arguments stay the same
    cudaGraphExec_t graph = nullptr;
    int graph_bs = 0, graph_maxit = 0;
    const double* graph_b = nullptr;
    double* graph_x = nullptr;
    double graph_tol = 0.0;
};

// Block-Jacobi preconditioner (block_jacobi.cu): boundaries of the diagonal
// blocks, the block of every row, and the inverses (entry (i, j) of the
// block starting at row o with s rows at inv[o * max_bs + j * s + i]).
struct gko_block_jacobi {
    int device = 0;
    int64_t n_rows = 0, n_blocks = 0;
    int max_bs = 1;
    int32_t* block_ptr = nullptr;  // device, n_blocks + 1
    int32_t* row_block = nullptr;  // device, n_rows
    double* inv = nullptr;         // device, n_rows * max_bs
};

namespace gko {

struct SolverState;

// z = M^-1 r fused with rho' = r.z (block_jacobi.cu).  mode kBjInit: also
// ||r||^2 and the initial stop test, rho = rho0 = r.z; kBjStep: beta = rho'/rho,
// rho = rho'.  Skipped when the state says done, unless force.  h: the loop's
// conditional handle (0 outside a graph).
enum { kBjInit = 0, kBjStep = 1 };
void bj_z_launch(const gko_block_jacobi* M, const double* r, double* z, SolverState* s, double* part, int grid,
                 cudaGraphConditionalHandle h, int mode, int force, cudaStream_t st);

// Launchers exported by the kernel translation units.  All asynchronous on
// the given stream; they validate nothing (the C-ABI layer does).
int csr_analyse(gko_matrix* A, cudaStream_t st);
int seg_alloc(SegArrays* s, int64_t nnz, int P, int threads);
// Entries per thread of the COO kernel for this matrix: 13 when its columns
// stay near the diagonal (max |i - j| <= max(4096, n / 16): the gathers of x
// hit L1), else 11 (scattered columns: the smaller shared-memory stages
// leave L1 room for more gathers in flight, and the gathers bypass L1).
// Measured on GB300.
int coo_entries_per_thread(const gko_matrix* A);
void seg_free(SegArrays* s);
int spmv_csr(const gko_matrix* A, int config, const double* x, double* y, double alpha, double beta,
             cudaStream_t st);
int spmv_coo(const gko_matrix* A, const CooPart& coo, const double* x, double* y, double alpha,
             double beta, cudaStream_t st);
int spmv_ell(const gko_matrix* A, const EllPart& ell, const double* x, double* y, double alpha,
             double beta, cudaStream_t st);
int spmv_sellp(const gko_matrix* A, const double* x, double* y, double alpha, double beta,
               cudaStream_t st);
int spmv_hybrid(const gko_matrix* A, const double* x, double* y, double alpha, double beta,
                cudaStream_t st);
int scale_vector(int64_t n, double* y, double beta, cudaStream_t st);  // y = beta * y (beta 0: zero)
int spmv_csr_rowblock(const gko_matrix* A, const double* x, double* y, double alpha, double beta,
                      cudaStream_t st);
int spmv_csr_banded(const gko_matrix* A, const double* x, double* y, double alpha, double beta,
                    cudaStream_t st);
int rowblock_rows(const gko_matrix* A);
bool rowblock_preferred(const gko_matrix* A);
int default_csr_config(const gko_matrix* A);  // kernel behind GKO_CFG_DEFAULT for CSR
cudaError_t rowblock_lowprec_f32(const gko_matrix* A, const float* val, const float* x, float* y, cudaStream_t st);
cudaError_t rowblock_lowprec_bf16(const gko_matrix* A, const void* val, const float* x, float* y, cudaStream_t st);
struct Cg1Reduce;  // solver.cuh
cudaError_t rowblock_cg1_f64(const gko_matrix* A, const double* r, double* w, Cg1Reduce red, cudaStream_t st);
cudaError_t rowblock_cg1_f32(const gko_matrix* A, const float* val, const float* r, float* w, Cg1Reduce red,
                             cudaStream_t st);
cudaError_t rowblock_cg1_bf16(const gko_matrix* A, const void* val, const float* r, float* w, Cg1Reduce red,
                              cudaStream_t st);

// conversions (convert.cu); all synchronise the stream where sizes are read
int convert_csr_to_coo(gko_matrix* A, cudaStream_t st);
int convert_coo_to_csr(gko_matrix* A, cudaStream_t st);
int convert_csr_to_ell(gko_matrix* A, cudaStream_t st);
int convert_ell_to_csr(gko_matrix* A, cudaStream_t st);
int convert_csr_to_sellp(gko_matrix* A, cudaStream_t st);
int convert_sellp_to_csr(gko_matrix* A, cudaStream_t st);
int convert_csr_to_hybrid(gko_matrix* A, cudaStream_t st);
int convert_hybrid_to_csr(gko_matrix* A, cudaStream_t st);
int validate_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* row_ptr,
                 const int32_t* col, cudaStream_t st);
void free_format(gko_matrix* A, int fmt);

// out[0..n] = exclusive scan of in[0..n-1] on the device (out[n] = total)
int exclusive_scan(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st);

// BLAS-1 and solvers (blas1.cu, cg.cu)
int cg_solve(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit,
             cudaStream_t st, gko_solve_info* info);
int lp_ell_prepare(gko_matrix* A, bool bf16, cudaStream_t st, bool* usable);
void lp_ell_free(gko_matrix* A);
cudaError_t lp_ell_cg1(const gko_matrix* A, bool bf16, const float* r, const float* rd, float* w, Cg1Reduce red,
                       cudaStream_t st);
int lp_ell_grid(const gko_matrix* A);
int pcg_jacobi_solve(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit,
                     cudaStream_t st, gko_solve_info* info);
int pcg_block_jacobi_solve(const gko_matrix* A, int fmt, const gko_block_jacobi* M, const double* b, double* x,
                           double tol, int maxit, cudaStream_t st, gko_solve_info* info);
int cg_multi_solve(const gko_matrix* A, int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx, double tol,
                   int maxit, cudaStream_t st, gko_solve_info* infos);
int bicgstab_solve(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit,
                   cudaStream_t st, gko_solve_info* info);
int spmm_csr(const gko_matrix* A, int64_t k, const double* x, int64_t ldx, double* y, int64_t ldy, double alpha,
             double beta, cudaStream_t st);
int gmres_solve(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int m, int maxit,
                cudaStream_t st, gko_solve_info* info);
int cg1_solve(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit,
              cudaStream_t st, gko_solve_info* info);
int cg_mixed_solve(gko_matrix* A, int inner, const double* b, double* x, double tol, int maxit_outer,
                   double inner_tol, int inner_maxit, cudaStream_t st, gko_solve_info* info, int precond);

// selector (selector.cu)
int features_compute(const gko_matrix* A, double* out_host, cudaStream_t st);
uint64_t selector_generation();  // 0: no selector installed; changes with every gko_selector_load/clear

// the (format, configuration) candidates of the exhaustive autotuner, in the
// order of the public table (GKO_N_CANDIDATES)
extern const int kCandFmt[GKO_N_CANDIDATES];
extern const int kCandCfg[GKO_N_CANDIDATES];

}  // namespace gko
