/*
 * gko_gb300.h -- C ABI of the GB300 (sm_103a) sparse hot path: SpMV in the
 * CSR, COO, ELL, SELL-P and hybrid ELL+COO formats, bit-exact conversions
 * between them, conjugate gradients (FP64; mixed FP32/BF16 storage with FP64
 * iterative refinement; batched over many small systems) and the learned
 * format selector.
 *
 * The operations follow Cojean, Tsai and Anzt, "Ginkgo - A Math Library
 * designed for Platform Portability": Sec. 6.1 (SpMV y = A x on sparse
 * formats, whose COO and CSR byte bounds it states) and Sec. 6.2 (Krylov
 * solvers built on SpMV).  Formats the paper names only through its
 * citations follow their standard definitions (ELL and hybrid: Bell and
 * Garland, SC'09; SELL-P: Anzt, Tomov and Dongarra, 2014).
 *
 * Conventions for every call:
 *  - Return value: a gko_status code (GKO_OK == 0).  No call aborts, traps
 *    or exits the process.  gko_last_error() gives a message for the last
 *    failing call of the calling thread.
 *  - Indices are int32, values IEEE binary64 unless stated.  Matrices are
 *    square or rectangular (n_rows x n_cols).
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless documented as
 *    synchronising (the solvers and the query/export calls).
 *  - Vectors passed to compute calls are caller-owned DEVICE pointers
 *    (except gko_spmv_host), 16-byte aligned is fastest but 8 suffices.
 *  - A gko_matrix handle owns device copies of every format materialised
 *    in it; the caller's input arrays are copied and may be freed after
 *    the creating call returns.
 *  - Every entry point needs a current CUDA device (the one of the stream);
 *    a handle must be used on the device it was created on.
 */
#ifndef GKO_GB300_H
#define GKO_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Storage formats. */
enum {
    GKO_FMT_CSR = 0,    /* row_ptr[n+1], col[nnz], val[nnz]; columns ascending per row */
    GKO_FMT_COO = 1,    /* row[nnz], col[nnz], val[nnz]; sorted by (row, col) */
    GKO_FMT_ELL = 2,    /* col[K*n_pad], val[K*n_pad]; slot (i,k) at k*n_pad+i; n_pad = n rounded up to 32;
                           K = max row length; padding col = -1, val = +0.0 */
    GKO_FMT_SELLP = 3,  /* slices of S rows; slice_len[n_slices] = slice width (max row length in the
                           slice rounded up to the stride factor f); slice_set[n_slices+1] = exclusive
                           prefix sum of widths; slot k of row s*S+l at (slice_set[s]+k)*S+l; padding
                           col = -1, val = +0.0 */
    GKO_FMT_HYBRID = 4, /* ELL part of width K_h (row i's first min(len_i, K_h) entries) + COO part
                           (the remaining entries, sorted by (row, col)).  K_h minimises
                           n_pad*K*(s_v+4) + overflow(K)*(s_v+8) bytes, s_v = 8, ties to smaller K */
    GKO_FMT_AUTO = 5    /* learned selector's choice, else the exhaustive autotuner's (gko_spmv only) */
};

/* Status codes. */
enum {
    GKO_OK = 0,
    GKO_ERR_INVALID_ARG = 1,        /* null pointer, negative size, unknown enum value */
    GKO_ERR_DIM_MISMATCH = 2,       /* sizes of the operands disagree */
    GKO_ERR_FORMAT_UNAVAILABLE = 3, /* the format is not materialised in the handle */
    GKO_ERR_FORMAT_TOO_LARGE = 4,   /* padded format would exceed its size limit */
    GKO_ERR_OUT_OF_MEMORY = 5,      /* a device allocation failed */
    GKO_ERR_NOT_CONVERGED = 6,      /* solver stopped at its iteration limit */
    GKO_ERR_BREAKDOWN = 7,          /* p.q <= 0 or NaN in CG: matrix not SPD or data not finite */
    GKO_ERR_INVALID_MATRIX = 8,     /* CSR input not valid (row_ptr not monotone, column out of range or
                                       columns not strictly ascending within a row) */
    GKO_ERR_TIMEOUT = 9,            /* a bounded device wait gave up (see gko_matrix_errors) */
    GKO_ERR_CUDA = 10               /* a CUDA runtime call failed (message in gko_last_error) */
};

/* Value types. */
enum { GKO_F64 = 0, GKO_F32 = 1, GKO_BF16 = 2 };

/* Preconditioners of the mixed-precision inner solve. */
enum { GKO_PRECOND_NONE = 0, GKO_PRECOND_JACOBI = 1 };

/* Kernel configurations accepted by gko_spmv_config (the candidates of the
 * exhaustive sweep / selector).  GKO_CFG_DEFAULT lets the library choose;
 * for CSR it picks, from the row-length statistics of the handle: rows of
 * close length (max <= 2 mean + 16 and max <= 128) one lane per row when at
 * most 8 long, the staged row blocks up to 20, four lanes per row beyond;
 * skewed rows the binned kernel. */
enum {
    GKO_CFG_DEFAULT = 0,
    GKO_CFG_CSR_SUBWARP_1 = 1,  /* CSR, classical: subwarp of 1,2,4,8,16,32 lanes per row */
    GKO_CFG_CSR_SUBWARP_2 = 2,
    GKO_CFG_CSR_SUBWARP_4 = 3,
    GKO_CFG_CSR_SUBWARP_8 = 4,
    GKO_CFG_CSR_SUBWARP_16 = 5,
    GKO_CFG_CSR_SUBWARP_32 = 6,
    GKO_CFG_CSR_NNZSPLIT = 7,   /* CSR, load-balanced equal-nnz split with segmented reduction */
    GKO_CFG_CSR_BANDED = 8,     /* CSR row blocks with the x window staged in shared memory (banded
                                   matrices: max |i - j| <= 1024 and max row length <= 128) */
    GKO_CFG_CSR_ROWBLOCK = 9,   /* CSR row blocks staged in shared memory, one thread per row (max row
                                   length <= 128) */
    GKO_CFG_CSR_BINNED = 10     /* CSR rows grouped by length (bins up to 8, 20, 48, 128, 512, longer; built
                                   when the handle is created): each bin by subwarps of 1, 2, 4, 8, 32
                                   lanes per row, the longest rows one thread block each */
};

typedef struct gko_matrix gko_matrix;
typedef struct gko_batch gko_batch;

/* Result of a solve.  status repeats the call's return code. */
typedef struct {
    int32_t iterations;       /* CG steps (products with A); for mixed CG: inner steps in total */
    int32_t outer_iterations; /* mixed CG: refinement corrections; 0 otherwise */
    double rel_residual;      /* true ||b - A x||_2 / ||b||_2 formed in FP64 at exit */
    int32_t status;
    int32_t aux;              /* GMRES: Arnoldi steps whose second Gram-Schmidt update ran in FP32; 0 otherwise */
} gko_solve_info;

/* Message of the last failing call on this thread ("" if none). */
const char* gko_last_error(void);
/* Name of a status code. */
const char* gko_status_string(int status);
/* Library version string. */
const char* gko_version(void);

/* Ceilings of the running GPU that the sparse kernels are judged against,
 * measured the way Sec. 6 characterises each platform before its SpMV
 * results (a stream benchmark for bandwidth, mixbench for arithmetic):
 * *fp64_tfma and *fp32_tfma receive the FMA rates (10^12 FMA/s; eight
 * independent chains per thread, 8 blocks of 256 threads per SM) and
 * *gathers_g the rate of random 8-byte loads (10^9/s) from a zeroed array
 * of gather_span doubles (a power of two >= 1024; indices from a counter
 * hash, so no index array is read).  Best of five timed runs after a
 * warm-up (CUDA events on stream).  Allocates and frees its scratch
 * stream-ordered; synchronises the stream. */
int gko_measure_ceilings(double* fp64_tfma, double* fp32_tfma, double* gathers_g, int64_t gather_span,
                         void* stream);

/* Failure-injection hook for tests of the timeout path (the paper has no
 * counterpart).  The staged kernels (load-balanced CSR/COO SpMV, the CSR
 * row-block kernel, the mixed-precision inner product) wait for each tile's
 * bulk copy with a bounded poll loop; polls sets the limit of that wait for
 * launches made after the call (default 2^22 polls, restored by UINT32_MAX;
 * CUDA graphs keep the value they were captured with).  polls = 0 makes
 * every such wait give up at once: the kernel ORs bit 0 into the handle's
 * error word (gko_matrix_errors), waits with the default limit for the copies
 * it has in flight, and its CTAs exit, leaving y undefined; solvers return
 * GKO_ERR_TIMEOUT.  Process-wide; not for concurrent use with other calls. */
int gko_set_wait_limit(uint32_t polls);

/* ----------------------------------------------------------- matrices */

/* Create a handle from a CSR matrix (Sec. 6.1).  row_ptr[n_rows+1],
 * col[nnz], val[nnz] are host pointers (on_device = 0) or device pointers
 * (on_device = 1); they are copied.  The input is validated on the device
 * (GKO_ERR_INVALID_MATRIX).  nnz == row_ptr[n_rows] must hold and fit int32.
 * Synchronises the stream.  On success *out owns the CSR copy and the
 * analysis data of the load-balanced kernels. */
int gko_matrix_create_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* row_ptr,
                          const int32_t* col, const double* val, int on_device, void* stream,
                          gko_matrix** out);

/* Free a handle and every device array it owns (NULL is a no-op). */
int gko_matrix_destroy(gko_matrix* A);

/* Set SELL-P parameters used by the next conversion to SELL-P: slice size
 * S in {1,2,4,8,16,32,64,128} (default 64) and stride factor f >= 1
 * (default 1).  Also sets the padding limit of the padded formats: ELL
 * (K*n_pad slots) and SELL-P (total slots) are refused with
 * GKO_ERR_FORMAT_TOO_LARGE when their slots exceed
 * max(ell_factor * nnz, 2^22) (ell_factor default 4; <= 0 keeps it).  The
 * hybrid format chooses its ELL width itself and is never refused. */
int gko_matrix_set_params(gko_matrix* A, int sellp_slice, int sellp_stride, double ell_factor);

/* Materialise format dst from format src inside the handle (src must be
 * materialised; one of them is CSR).  Indices and values are moved bit for
 * bit; padding follows the format definitions above.  Runs on the device;
 * synchronises the stream (sizes are read back). */
int gko_convert(gko_matrix* A, int src, int dst, void* stream);

/* Drop a materialised format (frees its arrays).  Dropping CSR is allowed
 * only if another format remains; gko_convert(A, X, GKO_FMT_CSR) rebuilds
 * it bit-exactly. */
int gko_matrix_release(gko_matrix* A, int fmt);

/* Sizes of a format: info[0] = 1 if materialised else 0, info[1] = n_rows,
 * info[2] = n_cols, info[3] = nnz (stored entries, padding excluded),
 * info[4] = K (ELL width; hybrid ELL width; SELL-P slice size S),
 * info[5] = n_pad (ELL, hybrid) or n_slices (SELL-P), info[6] = total
 * padded slots (ELL, SELL-P) or COO-part nnz (hybrid), info[7] = SELL-P
 * stride factor.  info must hold 8 int64. */
int gko_matrix_info(const gko_matrix* A, int fmt, int64_t* info);

/* Copy one array of a materialised format into dst (host if to_host,
 * else device), bytes = exact array size.  Arrays: CSR 0 row_ptr, 1 col,
 * 2 val; COO 0 row, 1 col, 2 val; ELL 0 col, 1 val; SELL-P 0 slice_len,
 * 1 slice_set, 2 col, 3 val; HYBRID 0 ell_col, 1 ell_val, 2 coo_row,
 * 3 coo_col, 4 coo_val.  Synchronises the stream. */
int gko_matrix_export(const gko_matrix* A, int fmt, int array, void* dst, int64_t bytes,
                      int to_host, void* stream);

/* Sticky device error bits of the handle's kernels (bit 0 bounded wait
 * timed out, bit 1 bad index, bit 2 int32 overflow); clears them when
 * clear != 0.  A call during which bit 0 was set left its output undefined
 * (not merely incomplete).  Synchronises the stream. */
int gko_matrix_errors(gko_matrix* A, uint32_t* bits, int clear, void* stream);

/* ---------------------------------------------------------------- SpMV */

/* y = alpha * A * x + beta * y with the named format (Sec. 6.1).  x has
 * n_cols entries, y n_rows (device pointers, caller-owned, not aliased).
 * beta == 0 means y is not read (NaN/Inf in y are overwritten).  FP64
 * arithmetic throughout; each y_i is within 1e-12 * (|alpha||A||x| +
 * |beta||y|)_i of the exact result.  GKO_FMT_AUTO runs the candidate (see
 * GKO_N_CANDIDATES) that the selector loaded with gko_selector_load predicts
 * fastest, or, with no selector loaded, the one gko_autotune_format measures
 * fastest; the choice is made on the first AUTO call (which then
 * synchronises the stream) and cached in the handle until another selector
 * is loaded or a format is materialised or released.  Asynchronous
 * otherwise.  AUTO calls on one handle must not run concurrently. */
int gko_spmv(int fmt, const gko_matrix* A, const double* x, double* y, double alpha, double beta,
             void* stream);

/* gko_spmv with an explicit kernel configuration (GKO_CFG_*); used by the
 * exhaustive sweep.  A configuration that does not apply to fmt returns
 * GKO_ERR_INVALID_ARG. */
int gko_spmv_config(int fmt, int config, const gko_matrix* A, const double* x, double* y,
                    double alpha, double beta, void* stream);

/* gko_spmv on HOST vectors: copies x (and y if beta != 0) host -> device,
 * runs the product, copies y back.  x_host/y_host should be pinned for
 * speed.  Device staging buffers are owned by the handle (allocated on first
 * use).  Synchronises the stream. */
int gko_spmv_host(int fmt, const gko_matrix* A, const double* x_host, double* y_host, double alpha,
                  double beta, void* stream);

/* Several right-hand sides at once (Sec. 6.1's product applied to a block
 * of k vectors): Y = alpha * A * X + beta * Y with X (n_cols x k) and Y
 * (n_rows x k) dense, row-major (element (i, c) at i*ld + c), leading
 * dimensions ldx, ldy >= max(k, 1); device pointers, caller-owned, not
 * aliased.  Reads the CSR format (must be materialised).  Each Y column is
 * the product with the same X column, within the accuracy stated for
 * gko_spmv; beta == 0: Y is not read.  k = 0 does nothing.  Asynchronous. */
int gko_spmm(const gko_matrix* A, int64_t k, const double* x, int64_t ldx, double* y, int64_t ldy, double alpha,
             double beta, void* stream);

/* COO SpMV that allocates no memory at all.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc (or any
 * allocator) while they run -- code captured into CUDA graphs or replayed
 * with a fixed memory footprint, real-time loops that cannot take an
 * allocation's latency or failure, and applications whose device memory
 * belongs to another allocator (a framework's caching pool) that a
 * library-side cudaMalloc would bypass.
 *
 * y = alpha * A * x + beta * y with A given directly by caller-owned device
 * arrays row[nnz], col[nnz], val[nnz] (COO sorted by (row, col), indices in
 * range; not validated), x[n_cols], y[n_rows].  row, col and val must be
 * 16-byte aligned; they are not read past nnz.  beta == 0: y is not read.
 * Same load-balanced kernel and accuracy as gko_spmv(GKO_FMT_COO, ...), run
 * with tiles of 256 threads x 11 entries (gko_spmv: 64 x 11).
 *
 * Scratch: the carries of rows that cross tiles live in a fixed device
 * array inside the library (GKO_NOALLOC_MAX_TILES tiles of 2816 entries,
 * 896 KiB, held by every GPU that loads the library until exit), so nnz
 * may not exceed GKO_NOALLOC_MAX_TILES * 2816 (GKO_ERR_INVALID_ARG beyond).
 * All calls share that array: calls that can overlap on the GPU (different
 * streams, or different host threads on one device) race and must be
 * serialised by the caller.  Nothing needs clearing between calls (each
 * call writes every carry it reads).
 *
 * The first call on a device looks up the device address of the array
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before capturing a stream.  Later calls only launch kernels.
 *
 * err_flags: optional caller-owned device word; bit 0 is ORed in if a
 * bounded wait for a bulk copy gave up (y is then undefined), bit 1 in the
 * bounds-checked build (libgkogb_checked.so) if an index was out of range
 * (that entry is skipped; a bad row index leaves y undefined).  NULL: not
 * reported.  Asynchronous on stream. */
#define GKO_NOALLOC_MAX_TILES 32768
int gko_spmv_coo_noalloc(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* row, const int32_t* col,
                         const double* val, const double* x, double* y, double alpha, double beta,
                         uint32_t* err_flags, void* stream);

/* ----------------------------------------------------------- solvers */

/* Conjugate gradients (Hestenes-Stiefel; the Krylov solvers of Sec. 6.2)
 * on A x = b using format fmt for the products.  b, x device vectors of
 * n_rows (square A).  x holds the initial guess on entry and the solution
 * on exit.  Stops when the recursive residual satisfies ||r|| <= tol ||b||
 * and the FP64 true residual confirms it (up to four confirmations), at
 * maxit (GKO_ERR_NOT_CONVERGED) or on breakdown (GKO_ERR_BREAKDOWN).
 * ||b|| = 0 returns x = 0.  A product whose bounded wait for a bulk copy
 * gave up (bit 0 of the handle's error word, see gko_matrix_errors; the bit
 * is sticky until cleared) stops the solve with GKO_ERR_TIMEOUT.  Work
 * vectors are allocated stream-ordered for the call.  Synchronises the
 * stream; info (host) may be NULL. */
int gko_cg(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit,
           void* stream, gko_solve_info* info);

/* CG in the single-reduction form of Chronopoulos and Gear (J. Comput.
 * Appl. Math. 25, 1989), the same Krylov method as gko_cg (Sec. 6.2) with
 * its two dot products merged: each step computes w = A r, gamma = r.r and
 * delta = w.r in one pass and one grid reduction, then
 *   beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old),
 *   p = r + beta p, s = w + beta s (s = A p), x += alpha p, r -= alpha s
 * in one vector pass: two kernel launches per step (for CSR matrices with
 * rows of similar length the dots run inside the SpMV kernel; other formats
 * add one dot launch).  Arguments, stopping (recursive residual, then the
 * FP64 true residual, up to four confirmations), breakdown (non-positive
 * delta - beta gamma / alpha_old, or NaN), errors and synchronisation are
 * those of gko_cg; info->iterations counts steps taken (updates of x).
 * Iterates equal gko_cg's up to rounding. */
int gko_cg_single_reduction(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit,
                            void* stream, gko_solve_info* info);

/* Conjugate gradients preconditioned by the diagonal of A (Jacobi
 * preconditioner M = diag(A)): the Krylov solver of Sec. 6.2 with the
 * simplest preconditioner, the textbook preconditioned CG
 *   r = b - A x0, z = M^-1 r, p = z, rho = r.z;
 *   q = A p, alpha = rho / p.q, x += alpha p, r -= alpha q, z = M^-1 r,
 *   rho' = r.z, beta = rho' / rho, p = z + beta p
 * (z is never stored: the update kernel forms r.M^-1 r and ||r||^2 in one
 * pass, the direction update reads r and the inverted diagonal).  Products
 * with format fmt; the diagonal is read from the CSR part, which must be
 * materialised.  Stops on the unpreconditioned recursive residual
 * ||r|| <= tol ||b|| confirmed by the FP64 true residual (up to four
 * times), at maxit or on breakdown; a zero or missing diagonal entry
 * returns GKO_ERR_BREAKDOWN before any step.  Otherwise as gko_cg. */
int gko_pcg_jacobi(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit, void* stream,
                   gko_solve_info* info);

/* ------------------------------------------ block-Jacobi preconditioner
 * M = blockdiag(A_11, ..., A_kk): the diagonal blocks of A on runs of
 * consecutive rows, each inverted once in FP64, applied as z = M^-1 r.  A
 * companion of the Krylov solvers of Sec. 6.2 (which the paper benchmarks
 * without defining a preconditioner): the textbook block-Jacobi of Saad,
 * Iterative Methods for Sparse Linear Systems, Sec. 10.2.  Blocks:
 * supervariables (maximal runs of consecutive rows whose stored column
 * lists are identical) are cut into pieces of at most max_block_size rows,
 * then merged greedily in row order while a block stays at most
 * max_block_size rows.  An opaque, device-resident object. */
typedef struct gko_block_jacobi gko_block_jacobi;

/* Builds M for A (square, CSR part materialised) with blocks of 1..32
 * rows.  The supervariable flags and the inversions (Gauss-Jordan with
 * partial pivoting, one warp per block, duplicates in A summed) run on the
 * device; the greedy merge scans the flags on the host (one copy of n_rows
 * bytes).  Device memory: n_rows * (8 * max_block_size + 4) bytes plus the
 * block boundaries.  Synchronises the stream.  Errors: GKO_ERR_INVALID_ARG
 * (NULL, max_block_size outside 1..32, wrong device), GKO_ERR_DIM_MISMATCH
 * (not square), GKO_ERR_FORMAT_UNAVAILABLE (no CSR part), GKO_ERR_BREAKDOWN
 * (a diagonal block is singular: a zero pivot), GKO_ERR_OUT_OF_MEMORY.  On
 * error *out is NULL.  M does not reference A after it is built. */
int gko_block_jacobi_create(const gko_matrix* A, int max_block_size, void* stream, gko_block_jacobi** out);
int gko_block_jacobi_destroy(gko_block_jacobi* M);

/* Copies M to host buffers: *n_blocks; block_ptr (n_blocks + 1 row
 * offsets, or NULL); inv (n_rows * max_block_size doubles, or NULL): entry
 * (i, j) of the inverse of the block that starts at row o and has s rows
 * at inv[o * max_block_size + j * s + i] (column-major within the block;
 * the slots past each block's s * s entries are zero).  Synchronises. */
int gko_block_jacobi_export(const gko_block_jacobi* M, int64_t* n_blocks, int32_t* block_ptr, double* inv,
                            void* stream);

/* z = M^-1 r (device vectors of n_rows doubles, not overlapping).
 * Asynchronous on the stream. */
int gko_block_jacobi_apply(const gko_block_jacobi* M, const double* r, double* z, void* stream);

/* Conjugate gradients preconditioned by M (built from the same A): the
 * preconditioned CG of gko_pcg_jacobi with z = M^-1 r stored, five launches
 * per step (product; p.q; x += alpha p, r -= alpha q with ||r||^2 and the
 * stop tests; z = M^-1 r with rho' = r.z; p = z + beta p).  Stopping,
 * breakdown, errors and synchronisation as gko_pcg_jacobi; M must have as
 * many rows as A (GKO_ERR_DIM_MISMATCH) and live on the same device. */
int gko_pcg_block_jacobi(const gko_matrix* A, int fmt, const gko_block_jacobi* M, const double* b, double* x,
                         double tol, int maxit, void* stream, gko_solve_info* info);

/* CG for several right-hand sides at once, A X = B with k = 1..32 columns:
 * k independent Hestenes-Stiefel recurrences (gko_cg per column, each with
 * its own alpha, beta, stop test and iteration count) sharing one product
 * per step, the SpMM of gko_spmm applied to the k search directions, so
 * the matrix is read once per step for all columns.  B (n x k) and X
 * (n x k, the initial guess on entry) are row-major device blocks (element
 * (i, c) at i * ld + c), ldb, ldx >= k, not aliased; the CSR part must be
 * materialised.  A column stops on ||r_c|| <= tol ||b_c|| confirmed by the
 * FP64 true residual (up to four times), at maxit steps of its own, or on a
 * breakdown of its own (p.q <= 0 or NaN); the others go on.  A zero column
 * of B gives a zero column of X.  infos (k entries, or NULL) receives each
 * column's steps, true relative residual and status; the return value is
 * GKO_OK when every column converged, else the first failing column's
 * status.  Workspace 3 n k doubles, stream-ordered; the loop runs in a CUDA
 * graph with one host synchronisation per confirmation.  Synchronises the
 * stream. */
int gko_cg_multi(const gko_matrix* A, int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx, double tol,
                 int maxit, void* stream, gko_solve_info* infos);

/* BiCGSTAB (van der Vorst, SIAM J. Sci. Stat. Comput. 13, 1992) on A x = b
 * for a general (nonsymmetric) square A, a Krylov solver of Sec. 6.2 for
 * systems CG does not cover.  Shadow residual r^ = r0; per step
 *   rho' = r^.r, beta = (rho'/rho)(alpha/omega), p = r + beta (p - omega v),
 *   v = A p, alpha = rho' / r^.v, s = r - alpha v,
 *   t = A s, omega = t.s / t.t, x += alpha p + omega s, r = s - omega t
 * (two products with format fmt, FP64 throughout, scalars on the device,
 * the loop inside a CUDA graph).  When ||s|| <= tol ||b|| the step ends
 * half way (x += alpha p).  Converged steps are confirmed by the FP64 true
 * residual (up to four times): an unconfirmed half step restarts from the
 * true residual, an unconfirmed full step continues.  r^.v = 0, t.t = 0,
 * omega = 0, rho' = 0 or a NaN is GKO_ERR_BREAKDOWN; maxit steps
 * GKO_ERR_NOT_CONVERGED.  info->iterations counts steps (half or full).
 * ||b|| = 0 returns x = 0.  Synchronises the stream. */
int gko_bicgstab(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int maxit, void* stream,
                 gko_solve_info* info);

/* Restarted GMRES(restart) (Saad and Schultz, SIAM J. Sci. Stat. Comput.
 * 7, 1986) on A x = b for a general square A, the minimal-residual Krylov
 * solver of Sec. 6.2's family: each cycle builds an Arnoldi basis from the
 * true residual, orthogonalised by classical Gram-Schmidt applied twice,
 * reduces the
 * Hessenberg matrix by Givens rotations and ends after restart steps
 * (1..127) or when the least-squares residual estimate is <= tol ||b||;
 * x += V y; the next cycle's FP64 true residual decides convergence.  The
 * Arnoldi steps, rotations and back substitution run on the device (one
 * CUDA graph per cycle, one host synchronisation per cycle).  Products with
 * format fmt; the basis ((restart + 1) n doubles) is allocated
 * stream-ordered for the call, with a float copy of it: the second
 * Gram-Schmidt update, whose coefficients are rounding-level corrections,
 * runs in FP32 on that copy when they are at most 2^-33 of ||w1|| (its
 * error then stays below the FP64 rounding of w1), else in FP64;
 * info->aux counts the steps that took FP32.  maxit bounds the Arnoldi steps
 * (info->iterations counts them): GKO_ERR_NOT_CONVERGED; a NaN or a zero
 * rotation before convergence: GKO_ERR_BREAKDOWN.  ||b|| = 0 returns x = 0.
 * Synchronises the stream. */
int gko_gmres(const gko_matrix* A, int fmt, const double* b, double* x, double tol, int restart, int maxit,
              void* stream, gko_solve_info* info);

/* Mixed-precision CG with FP64 iterative refinement.  The inner CG runs on
 * a copy of A stored in inner_dtype (GKO_F32 or GKO_BF16; off-diagonals
 * rounded to nearest-even, the diagonal a_ii + sum_j(|rn(a_ij)| - |a_ij|)
 * formed in FP64 and rounded to nearest-even, which keeps the row sums of
 * matrices with non-positive off-diagonals) with FP32 vectors and FP32
 * accumulation, in the single-reduction form above, from d = 0 to relative
 * recursive residual inner_tol or inner_maxit steps.  The outer loop forms
 * r = b - A x, x += correction and the norms in FP64 and stops at
 * ||r|| <= tol ||b||.  The low-precision copy is cached in the handle.
 * info->iterations = inner steps in total, outer_iterations = corrections.
 * Synchronises the stream. */
int gko_cg_mixed(gko_matrix* A, int inner_dtype, const double* b, double* x, double tol,
                 int maxit_outer, double inner_tol, int inner_maxit, void* stream,
                 gko_solve_info* info);

/* gko_cg_mixed with a preconditioner for the inner solve: precond
 * GKO_PRECOND_JACOBI preconditions the inner CG by M = diag(A_lo), the
 * rounded matrix's diagonal (its inverse kept in FP32): u = M^-1 r is what
 * the inner product gathers, gamma = r.u and delta = (A_lo u).u drive the
 * single-reduction step, and the inner stop is relative in the M^-1 norm
 * (sqrt(r.u)).  The outer FP64 residual still decides convergence.  A zero
 * or missing diagonal entry of A_lo returns GKO_ERR_BREAKDOWN before any
 * step.  GKO_PRECOND_NONE is gko_cg_mixed. */
int gko_cg_mixed_precond(gko_matrix* A, int inner_dtype, int precond, const double* b, double* x, double tol,
                         int maxit_outer, double inner_tol, int inner_maxit, void* stream,
                         gko_solve_info* info);

/* ------------------------------------------------------------- batched */

/* Create a batch of count independent square systems: rows of system s
 * are [row_off[s], row_off[s+1]) of one concatenated CSR (global row_ptr of
 * row_off[count]+1 entries, column indices local to the system).  Host or
 * device inputs as for gko_matrix_create_csr; copied.  Systems may have
 * 1..4096 rows; row_ptr must be non-decreasing and every column index lie in
 * 0..n_s - 1 of its system (GKO_ERR_INVALID_MATRIX otherwise).  Each system
 * is stored renumbered, its rows in order of decreasing length (so that a
 * warp's rows have like lengths); b and x of the solves stay in the
 * caller's order. */
int gko_batch_create(int64_t count, const int64_t* row_off, const int32_t* row_ptr,
                     const int32_t* col, const double* val, int on_device, void* stream,
                     gko_batch** out);
int gko_batch_destroy(gko_batch* B);

/* Layout flags of gko_cg_batched's block_size (OR'ed with the block size). */
#define GKO_BATCH_SHARED_P 0x10000
#define GKO_BATCH_SHARED_PQ 0x20000

/* Solve all systems of the batch by CG, one thread block per system taken
 * from a device work queue (largest systems first), launched as one
 * persistent kernel inside a CUDA graph (the instantiated graph is kept in
 * the batch and relaunched by later calls with the same block size, b, x,
 * tol and maxit).  block_size 64, 128, 256, 512 or 1024: x, r, p and A p
 * of the system in shared memory; -128, -256, -512 or -1024: that many
 * threads with 1024 / |block_size| rows each, x, r and A p of a thread's
 * rows in registers and only p in shared memory (systems of at most 1024
 * rows); GKO_BATCH_SHARED_P | bs or GKO_BATCH_SHARED_PQ | bs (bs = 32, 64,
 * 128 or 256): bs threads with only p (or p and A p) in shared memory and
 * the rest of the system's vectors in a device scratch the batch allocates
 * and keeps (4 - 1 or 4 - 2 vectors of max_rows doubles per resident
 * block), so that more systems share an SM; 0 = the autotuned choice, or
 * GKO_BATCH_SHARED_P | 128 before gko_batch_autotune has run.
 * b, x device vectors of row_off[count]
 * entries (x: initial guess in, solution out).  infos: host array of count
 * entries or NULL.  Returns the worst status.  Synchronises the stream. */
int gko_cg_batched(gko_batch* B, const double* b, double* x, double tol, int maxit, int block_size,
                   void* stream, gko_solve_info* infos);

/* Run the batched-CG autotuner: times every candidate launch on this batch
 * (the block sizes and layouts of gko_cg_batched: 64 .. 1024 with the
 * vectors in shared memory, the split layouts GKO_BATCH_SHARED_P / _PQ |
 * 32 .. 256, and, when no system exceeds 1024 rows, -128 .. -1024 with the
 * rows' vectors in registers) and keeps the fastest for
 * block_size 0.  *best receives it. */
int gko_batch_autotune(gko_batch* B, const double* b, double* x, double tol, int maxit,
                       void* stream, int* best);

/* ------------------------------------------------------------ selector */

/* The 12 matrix statistics the selector uses, computed on the device from
 * the CSR arrays: log10 n, log10 max(nnz,1), mean/std/max/min row length,
 * max/mean, fraction of empty rows, max|i-j|/n, mean|i-j|/n, fraction of
 * rows storing their diagonal, SELL-P(32) slots/nnz.  out: 12 host doubles.
 * Synchronises the stream. */
int gko_features(const gko_matrix* A, double* out, void* stream);

/* MLP 12 -> 64 -> 64 -> n_out (ReLU), FP32, parameters packed in one
 * device array in the order W1[64x12], b1[64], W2[64x64], b2[64],
 * W3[n_out x 64], b3[n_out] (row-major, output-major).
 * gko_mlp_param_count gives the packed length. */
int64_t gko_mlp_param_count(int n_out);

/* Forward pass for a batch: X[batch x 12] -> out[batch x n_out] (device,
 * FP32, row-major). */
int gko_mlp_forward(const float* params, int n_out, const float* X, int batch, float* out,
                    void* stream);

/* Loss and gradient of the masked mean squared error
 * sum M (out - Y)^2 / sum M over a batch (X[batch x 12], Y and M
 * [batch x n_out], device FP32).  grad receives d loss / d params (packed
 * like params); loss (device, 1 float) may be NULL. */
int gko_mlp_grad(const float* params, int n_out, const float* X, const float* Y, const float* M,
                 int batch, float* grad, float* loss, void* stream);

/* One Adam step on the packed parameters: m, v are the moment arrays
 * (same length, zero at t = 1), t is the 1-based step number. */
int gko_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t count, int t,
                 float lr, float beta1, float beta2, float eps, void* stream);

/* Exhaustive autotuning, the selector's fallback and the judge of its
 * regret (Sec. 6.1 observes that no SpMV kernel wins on every matrix).  The
 * candidates, in this order, are the kernels the selector chooses among:
 *   0 CSR row blocks (GKO_CFG_CSR_ROWBLOCK), 1 CSR equal-nnz split,
 *   2 CSR 4 lanes per row, 3 CSR 32 lanes per row, 4 COO, 5 ELL, 6 SELL-P,
 *   7 hybrid, 8 CSR binned by row length, 9 CSR one lane per row.
 * gko_autotune_format times every candidate the handle can run (its format
 * materialised and its configuration applicable): one warm-up and five timed
 * products each (CUDA events on stream, alpha = 1, beta = 0, on staging
 * vectors the handle owns), and returns the one with the smallest median in
 * *fmt, *config.  times_us (host, GKO_N_CANDIDATES doubles, may be NULL)
 * receives each candidate's median in microseconds, NaN where it does not
 * apply.  With no selector loaded the choice becomes the handle's
 * GKO_FMT_AUTO choice.  Synchronises the stream. */
#define GKO_N_CANDIDATES 10
int gko_autotune_format(gko_matrix* A, int* fmt, int* config, double* times_us, void* stream);

/* Install a trained selector used by GKO_FMT_AUTO: packed FP32 params
 * (host), feature normalisation mean[12], scale[12] (host doubles), and
 * the n_out (format, config) pairs the outputs stand for (host ints,
 * fmts[i], cfgs[i]).  The prediction is argmin of the outputs. */
int gko_selector_load(const float* params_host, int n_out, const double* feat_mean,
                      const double* feat_scale, const int* fmts, const int* cfgs);

/* Remove the installed selector: GKO_FMT_AUTO falls back to exhaustive
 * autotuning. */
int gko_selector_clear(void);

/* The selector's choice for A (features computed on the device, cached in
 * the handle).  Synchronises the stream. */
int gko_select_format(gko_matrix* A, int* fmt, int* config, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GKO_GB300_H */
