// Load-balanced SpMV by an equal split of the stored entries (CSR and COO).
//
// The paper's Sec. 6.1 bounds SpMV by the bytes of the value and index
// streams; on GB300 FP64 arithmetic is just as tight (one FP64 FMA per
// 12 bytes of CSR is ~97 % of the FP64 pipe at full HBM bandwidth), so
// this kernel is built to issue close to one FP64 instruction per stored
// entry whatever the row lengths are:
//
//  * the stored entries are cut into tiles of TILE = 256 * P consecutive
//    entries; a persistent grid (2 CTAs of 256 threads per SM) walks the
//    tiles round robin with two shared-memory stages: while one tile is
//    summed, the next one's values, column indices and row pointers (COO:
//    row indices) stream in through 1-D bulk copies (TMA) completing on an
//    mbarrier;
//  * thread g owns entries [g*P, g*P+P) (P odd, so shared-memory reads of
//    consecutive threads fall in distinct banks) and sums them row by row
//    with one FMA per entry; all per-entry index arithmetic is 32-bit and
//    local to the tile;
//  * a row is finalised by the thread holding its last entry (rows whose
//    end index lies in the thread's range (s, e]); contributions of earlier
//    threads are added from their outgoing partials (segmented reduction
//    by key, in a fixed order: deterministic, no floating-point atomics);
//  * a row crossing tile boundaries is finished by a tiny fix-up kernel from
//    per-tile carries (the only scratch memory the kernel uses).
//
// V is the stored value type (double, float or bf16), T the arithmetic and
// vector type (double, or float with FP32 accumulation).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace gko {

constexpr int kSegThreads = 256;
constexpr int kSegCtasPerSm = 2;

// Per-tile carries of rows that cross tile boundaries.
template <typename T>
struct SegScratchT {
    T* tail_val;        // sum of the open row's entries in this tile
    int32_t* tail_row;  // row open at the tile's end, -1 if none
    int32_t* tail_pass; // 1: the row covers the whole tile and began before it
    T* head_val;        // partial of the row this tile finalises that began before it
    int32_t* head_row;  // that row, -1 if none
};
using SegScratch = SegScratchT<double>;

template <int P>
struct SegShape {
    static constexpr int kTile = kSegThreads * P;  // a multiple of 8 entries for the P used here
    static constexpr int kBuf = kTile + 8;         // bulk copies move whole 16-byte groups
    static constexpr int kRowStage = 2048;         // CSR row_ptr entries staged per tile
};

// one pipeline stage: values | column indices | (COO rows or CSR row_ptr)
template <int P, typename V, bool kCoo>
struct SegStage {
    static constexpr size_t kVal = SegShape<P>::kBuf * sizeof(V);
    static constexpr size_t kCol = SegShape<P>::kBuf * sizeof(int32_t);
    static constexpr size_t kAux = (kCoo ? SegShape<P>::kBuf : SegShape<P>::kRowStage) * sizeof(int32_t);
    static constexpr size_t kBytes = kVal + kCol + kAux;
    static_assert(kVal % 16 == 0 && kCol % 16 == 0 && kAux % 16 == 0, "16-byte aligned stage parts");
};

template <int P, typename V, typename T, bool kCoo>
constexpr size_t seg_smem_bytes()
{
    return 2 * SegStage<P, V, kCoo>::kBytes + kSegThreads * (sizeof(T) + sizeof(int32_t)) +
           8 * (sizeof(T) + sizeof(int32_t)) + 16;
}

template <typename V>
__device__ __forceinline__ float to_float(V v);
template <>
__device__ __forceinline__ float to_float<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_float<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename V, typename T>
__device__ __forceinline__ T to_t(V v)
{
    if constexpr (sizeof(T) == 8)
        return static_cast<T>(v);
    else
        return to_float<V>(v);
}

// Sum of s_part over the run of threads h <= start with s_prow[h] == r
// (walking down), jumping over whole warps whose 32 lanes all carry row r.
// *reached is set when the run extends to thread 0.
template <typename T>
__device__ __forceinline__ T seg_walk(int start, int r, const T* s_part, const int32_t* s_prow, const T* s_wsum,
                                      const int32_t* s_wrow, bool* reached)
{
    T sum = T(0);
    int h = start;
    while (h >= 0 && s_prow[h] == r) {
        if ((h & 31) == 31 && s_wrow[h >> 5] == r) {
            sum = sum + s_wsum[h >> 5];
            h -= 32;
        } else {
            sum = sum + s_part[h];
            h -= 1;
        }
    }
    *reached = h < 0;
    return sum;
}

template <bool kAlpha, bool kBeta, typename T>
__device__ __forceinline__ void seg_store(T* y, int64_t r, T v, T alpha, T beta)
{
    T out = kAlpha ? alpha * v : v;
    if (kBeta) out = fma(beta, y[r], out);
    y[r] = out;
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Metadata of a staged tile, written by the issuing thread.
struct SegTileInfo {
    int32_t t0;
    int32_t r_lo;     // CSR: row holding entry t0;  COO: row of entry t0
    int32_t a_lo;     // CSR: first staged row_ptr index (multiple of 4)
    int32_t staged;   // CSR: row_ptr segment staged in shared memory
    int32_t began;    // COO: the tile's first row began before the tile
    int32_t next_r;   // COO: row of entry t1 (n_rows at the end)
};

// Per-thread state after phase 1 of a tile.
template <typename T>
struct SegThreadOut {
    int fin_row;   // row finalised here that began before the thread (-1: none)
    T fin_val;
    int open_row;  // row still open at the thread's end (-1: none)
    T open_val;
};

// Phase 1 of one tile for one thread: sum its entries row by row, store
// rows that start and end in its range, report the deferred and open rows.
// ls/le: the thread's entries, local to the tile; RP: CSR row pointers as
// a pointer whose index is the global row (shared or global memory).
template <int P, typename V, typename T, bool kAlpha, bool kBeta, bool kCoo, bool kSkipEmpty, typename RP>
__device__ __forceinline__ SegThreadOut<T> seg_thread(int ls, int le, int t0, int cnt, int n_rows, const V* s_val,
                                                      const int32_t* s_col, const int32_t* s_aux, RP rp,
                                                      int first_row, bool first_carried, int next_r_tile,
                                                      int my_row, const T* __restrict__ x, T* __restrict__ y,
                                                      T alpha, T beta)
{
    SegThreadOut<T> o{-1, T(0), -1, T(0)};
    const int rem = le - ls;  // entries of this thread (<= 0: none)
    T vv[P], xv[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const bool ok = j < rem;
        const int c = ok ? s_col[ls + j] : 0;
        vv[j] = ok ? to_t<V, T>(s_val[ls + j]) : T(0);
        xv[j] = ldg(x + c);
    }
    // NOTE: lanes without entries must not return before the warp vote below
    // (__all_sync over the full warp would wait for them forever).
    const bool has = rem > 0;

    int row = 0, endr = 0;  // current row; its end relative to ls (CSR)
    bool ob = false;        // current row began before the thread's range
    if (has) {
        if (kCoo) {
            row = s_aux[ls];
            ob = (ls == 0) ? first_carried : (s_aux[ls - 1] == row);
        } else {
            row = my_row;
            endr = rp[row + 1] - t0 - ls;
            ob = rp[row] - t0 < ls;
        }
        // rows before the first stored entry are empty (end position 0)
        if (!kSkipEmpty && t0 + ls == 0)
            for (int r = 0; r < row; ++r) seg_store<kAlpha, kBeta>(y, r, T(0), alpha, beta);
    }

    // ---- fast path: at most three row ends in the range, no empty row among
    // them.  Ends e0 < e1 < e2 (relative to ls, in (0, rem] when inside the
    // range) are known up front, each entry costs one FMA plus selects, and
    // the finished rows are stored after the loop: no divergent branches.
    int e0 = INT32_MAX, e1 = INT32_MAX, e2 = INT32_MAX;
    int ra = row + 1, rb = row + 2, rc = row + 3;  // rows after the 1st, 2nd, 3rd end
    bool fast = true;
    if (!has) {
        // nothing to sum; still takes part in the vote
    } else if (kCoo) {
        int cur = row, n_chg = 0;
        bool gap = false;
        e0 = e1 = e2 = INT32_MAX;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            if (j < rem) {
                const int nr = (ls + j + 1 < cnt) ? s_aux[ls + j + 1] : next_r_tile;
                const bool c = nr != cur;
                gap |= nr > cur + 1;  // rows without entries in between (or after the last row)
                e0 = (c && n_chg == 0) ? j + 1 : e0;
                e1 = (c && n_chg == 1) ? j + 1 : e1;
                e2 = (c && n_chg == 2) ? j + 1 : e2;
                ra = (c && n_chg == 0) ? nr : ra;
                rb = (c && n_chg == 1) ? nr : rb;
                rc = (c && n_chg == 2) ? nr : rc;
                n_chg += c;
                cur = nr;
            }
        }
        // rows without entries need explicit zero stores unless skipped
        fast = (kSkipEmpty || !gap) && n_chg <= 3;
    } else {
        // The end of row + k is read only when row + k - 1 ends inside the
        // range: then row + k + 1 <= R(t1) + 1 lies in the staged segment.
        auto end_at = [&](int k) { return row + k < n_rows ? rp[row + k + 1] - t0 - ls : INT32_MAX; };
        e0 = endr;
        e1 = e0 <= rem ? end_at(1) : INT32_MAX;
        e2 = e1 <= rem ? end_at(2) : INT32_MAX;
        const int e3 = e2 <= rem ? end_at(3) : INT32_MAX;
        fast = (e0 > rem || e1 > e0) && (e1 > rem || e2 > e1) && (e2 > rem || e3 > e2) && e3 > rem;
    }
    const bool warp_fast = __all_sync(0xffffffffu, fast);  // every lane of the warp reaches this
    if (!has) return o;
    if (warp_fast) {
        T v0 = T(0), v1 = T(0), v2 = T(0), acc = T(0);
#pragma unroll
        for (int j = 0; j < P; ++j) {
            if (j < rem) {
                acc = fma(vv[j], xv[j], acc);
                const bool h0 = j + 1 == e0, h1 = j + 1 == e1, h2 = j + 1 == e2;
                v0 = h0 ? acc : v0;
                v1 = h1 ? acc : v1;
                v2 = h2 ? acc : v2;
                acc = (h0 || h1 || h2) ? T(0) : acc;
            }
        }
        const int n_end = (e0 <= rem) + (e1 <= rem) + (e2 <= rem);
        if (n_end > 0) {
            if (ob) {
                o.fin_row = row;
                o.fin_val = v0;
            } else {
                seg_store<kAlpha, kBeta>(y, row, v0, alpha, beta);
            }
        }
        if (n_end > 1) seg_store<kAlpha, kBeta>(y, ra, v1, alpha, beta);
        if (n_end > 2) seg_store<kAlpha, kBeta>(y, rb, v2, alpha, beta);
        const int last_end = n_end == 0 ? 0 : (n_end == 1 ? e0 : (n_end == 2 ? e1 : e2));
        if (last_end < rem) {  // entries after the last end belong to an open row
            o.open_row = n_end == 0 ? row : (n_end == 1 ? ra : (n_end == 2 ? rb : rc));
            o.open_val = acc;
        }
        return o;
    }

    // ---- general path: any number of row ends, empty rows included
    T acc = T(0);
    bool pending = false;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        if (j < rem) {
            acc = fma(vv[j], xv[j], acc);
            pending = true;
            int nr = 0;
            bool ends;
            if (kCoo) {
                nr = (ls + j + 1 < cnt) ? s_aux[ls + j + 1] : next_r_tile;
                ends = nr != row;
            } else {
                ends = (j + 1 == endr);
            }
            if (ends) {
                if (ob) {
                    o.fin_row = row;
                    o.fin_val = acc;
                } else {
                    seg_store<kAlpha, kBeta>(y, row, acc, alpha, beta);
                }
                acc = T(0);
                pending = false;
                ob = false;
                if (kCoo) {
                    if (!kSkipEmpty)
                        for (int r = row + 1; r < nr; ++r) seg_store<kAlpha, kBeta>(y, r, T(0), alpha, beta);
                    row = nr;
                } else {
                    // skip the empty rows that end at the same position
                    ++row;
                    int e = row < n_rows ? rp[row + 1] - t0 - ls : INT32_MAX;
                    while (e == j + 1) {
                        if (!kSkipEmpty) seg_store<kAlpha, kBeta>(y, row, T(0), alpha, beta);
                        ++row;
                        e = row < n_rows ? rp[row + 1] - t0 - ls : INT32_MAX;
                    }
                    endr = e;
                }
            }
        }
    }
    if (pending) {
        o.open_row = row;
        o.open_val = acc;
    }
    (void)first_row;
    return o;
}

// kCoo = false: CSR with row_ptr and the per-thread start rows thr_row
// (thr_row[g] = row holding entry g*P).  kCoo = true: COO with row[].
// kSkipEmpty: rows without entries are left untouched (used to add the COO
// part of the hybrid format onto the ELL part's result, with beta = 1).
// kExactTail (COO only): the arrays end exactly at nnz (caller-owned, not
// padded), so the last tile bulk-copies only whole 16-byte groups and the
// threads load the remaining few entries themselves.
template <int P, typename V, typename T, bool kAlpha, bool kBeta, bool kCoo, bool kSkipEmpty, bool kExactTail = false>
__global__ void __launch_bounds__(kSegThreads, kSegCtasPerSm)
    seg_spmv_kernel(int64_t n_rows64, int64_t nnz64, const int32_t* __restrict__ row_ptr,
                    const int32_t* __restrict__ rows, const int32_t* __restrict__ col,
                    const V* __restrict__ val, const int32_t* __restrict__ thr_row, const T* __restrict__ x,
                    T* __restrict__ y, T alpha, T beta, SegScratchT<T> sc, uint32_t* err)
{
    using S = SegShape<P>;
    using G = SegStage<P, V, kCoo>;
    static_assert(!kExactTail || kCoo, "exact tails are implemented for COO");
    constexpr int kAlign = 16 / sizeof(V) > 4 ? 16 / sizeof(V) : 4;  // entries per 16-byte group
    extern __shared__ __align__(16) unsigned char smem[];
    T* s_part = reinterpret_cast<T*>(smem + 2 * G::kBytes);
    int32_t* s_prow = reinterpret_cast<int32_t*>(s_part + kSegThreads);
    T* s_wsum = reinterpret_cast<T*>(s_prow + kSegThreads);
    int32_t* s_wrow = reinterpret_cast<int32_t*>(s_wsum + 8);
    __shared__ uint64_t bar[2];
    __shared__ SegTileInfo info[2];
    __shared__ int s_head_done;

    const int n_rows = static_cast<int>(n_rows64);  // sizes fit int32 (checked at creation)
    const int nnz = static_cast<int>(nnz64);
    const int tid = threadIdx.x;
    const int n_tiles = (nnz + S::kTile - 1) / S::kTile;
    const int stride = gridDim.x;

    auto stage_val = [&](int st) { return reinterpret_cast<V*>(smem + st * G::kBytes); };
    auto stage_col = [&](int st) { return reinterpret_cast<int32_t*>(smem + st * G::kBytes + G::kVal); };
    auto stage_aux = [&](int st) { return reinterpret_cast<int32_t*>(smem + st * G::kBytes + G::kVal + G::kCol); };

    // Issue the bulk copies of `tile` into stage `st` (thread 0 only).
    // CSR: a = R(t0), b = R(t1) (n_rows at the end).  COO: a = rows[t0-1]
    // (or -1), b = rows[t0], c = rows[t1] (n_rows at the end).
    auto issue = [&](int tile, int st, int32_t a, int32_t b, int32_t c) {
        const int t0 = tile * S::kTile;
        const int t1 = min(t0 + S::kTile, nnz);
        // padded arrays: round up to whole 16-byte groups; exact arrays:
        // round down (the ragged rest is loaded by the threads)
        const int cnt_al = kExactTail ? (t1 - t0) / kAlign * kAlign : (t1 - t0 + kAlign - 1) / kAlign * kAlign;
        uint32_t bytes = cnt_al * static_cast<uint32_t>(sizeof(V) + sizeof(int32_t) + (kCoo ? sizeof(int32_t) : 0));
        SegTileInfo ti;
        ti.t0 = t0;
        ti.staged = 0;
        ti.a_lo = 0;
        ti.began = 0;
        ti.next_r = c;
        int a_cnt = 0;
        if (kCoo) {
            ti.r_lo = b;
            ti.began = (t0 > 0) && (a == b);
        } else {
            ti.r_lo = a;
            const int count = min(b + 2, n_rows + 1) - a;
            ti.a_lo = a & ~3;
            a_cnt = (a + count - ti.a_lo + 3) & ~3;
            if (a_cnt <= S::kRowStage) {
                ti.staged = 1;
                bytes += a_cnt * sizeof(int32_t);
            }
        }
        info[st] = ti;
        mbar_arrive_expect_tx(&bar[st], bytes);
        if (cnt_al > 0) {  // (an exact tail of fewer than 4 entries has no whole group)
            bulk_g2s(stage_val(st), val + t0, cnt_al * sizeof(V), &bar[st]);
            bulk_g2s(stage_col(st), col + t0, cnt_al * sizeof(int32_t), &bar[st]);
            if (kCoo) bulk_g2s(stage_aux(st), rows + t0, cnt_al * sizeof(int32_t), &bar[st]);
        }
        if (!kCoo && ti.staged) bulk_g2s(stage_aux(st), row_ptr + ti.a_lo, a_cnt * sizeof(int32_t), &bar[st]);
    };
    // metadata loads needed to issue `tile` (read early, used later)
    auto meta_a = [&](int tile) -> int32_t {
        if (kCoo) return tile > 0 ? rows[tile * S::kTile - 1] : -1;
        return thr_row[tile * kSegThreads];
    };
    auto meta_b = [&](int tile) -> int32_t {
        if (kCoo) return rows[tile * S::kTile];
        return (tile + 1) * S::kTile < nnz ? thr_row[(tile + 1) * kSegThreads] : n_rows;
    };
    auto meta_c = [&](int tile) -> int32_t {
        if (!kCoo) return 0;
        return (tile + 1) * S::kTile < nnz ? rows[(tile + 1) * S::kTile] : n_rows;
    };
    // start row of this thread's entries in a tile (threads whose first
    // entry exists only: thr_row has ceil(nnz / P) entries)
    auto start_row = [&](int tile) -> int32_t {
        const int g = tile * kSegThreads + tid;
        return (!kCoo && tile < n_tiles && static_cast<int64_t>(g) * P < nnz) ? thr_row[g] : 0;
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
        s_head_done = 0;
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            const int t = blockIdx.x + k * stride;
            if (t < n_tiles) issue(t, k, meta_a(t), meta_b(t), meta_c(t));
        }
    }
    int32_t my_row = start_row(blockIdx.x);

    for (int it = 0;; ++it) {
        const int tile = blockIdx.x + it * stride;
        if (tile >= n_tiles) break;
        const int st = it & 1;
        const uint32_t parity = (it >> 1) & 1;
        bool landed = mbar_wait_bounded(&bar[st], parity, err);
        if (!landed) landed = mbar_wait_bounded(&bar[st], parity, err);  // copies still in flight: once more
        if (!__syncthreads_and(landed)) return;                           // CTA-uniform exit
        if (kExactTail) {  // entries past the last whole 16-byte group (last tile only)
            const int tx0 = info[st].t0;
            const int cx = min(tx0 + S::kTile, nnz) - tx0;
            for (int i = cx / kAlign * kAlign + tid; i < cx; i += kSegThreads) {
                stage_val(st)[i] = val[tx0 + i];
                stage_col(st)[i] = col[tx0 + i];
                stage_aux(st)[i] = rows[tx0 + i];
            }
            __syncthreads();
        }

        // prefetch what the next issue and the next tile need
        const int t_issue = tile + 2 * stride;
        int32_t pa = 0, pb = 0, pc = 0;
        if (tid == 0 && t_issue < n_tiles) {
            pa = meta_a(t_issue);
            pb = meta_b(t_issue);
            pc = meta_c(t_issue);
        }
        const int32_t next_row = start_row(tile + stride);

        const SegTileInfo ti = info[st];
        const int t0 = ti.t0;
        const int cnt = min(t0 + S::kTile, nnz) - t0;
        const int ls = tid * P;
        const int le = min(ls + P, cnt);
        const V* s_val = stage_val(st);
        const int32_t* s_col = stage_col(st);
        const int32_t* s_aux = stage_aux(st);
        const int first_row = ti.r_lo;
        bool first_carried;
        SegThreadOut<T> o;
        if (kCoo) {
            first_carried = ti.began != 0;
            o = seg_thread<P, V, T, kAlpha, kBeta, kCoo, kSkipEmpty>(ls, le, t0, cnt, n_rows, s_val, s_col, s_aux,
                                                                     s_aux, first_row, first_carried, ti.next_r,
                                                                     my_row, x, y, alpha, beta);
        } else if (ti.staged) {
            const int32_t* rps = s_aux - ti.a_lo;  // shared memory, indexed by global row
            first_carried = rps[first_row] < t0;
            o = seg_thread<P, V, T, kAlpha, kBeta, kCoo, kSkipEmpty>(ls, le, t0, cnt, n_rows, s_val, s_col, s_aux,
                                                                     rps, first_row, first_carried, 0, my_row, x, y,
                                                                     alpha, beta);
        } else {
            first_carried = row_ptr[first_row] < t0;
            o = seg_thread<P, V, T, kAlpha, kBeta, kCoo, kSkipEmpty>(ls, le, t0, cnt, n_rows, s_val, s_col, s_aux,
                                                                     row_ptr, first_row, first_carried, 0, my_row,
                                                                     x, y, alpha, beta);
        }

        // outgoing partial: the row still open at the thread's end
        s_prow[tid] = o.open_row;
        s_part[tid] = o.open_val;
        __syncthreads();

        // ------------------------------------------------------------ phase 2
        {
            const int lane = tid & 31, w = tid >> 5;
            const int32_t pr = s_prow[tid];
            const int32_t pr0 = __shfl_sync(0xffffffffu, pr, 0);
            const bool uni = __all_sync(0xffffffffu, pr == pr0 && pr0 >= 0);
            if (uni) {
                const T t = subwarp<32>::reduce_sum(s_part[tid]);
                if (lane == 0) {
                    s_wsum[w] = t;
                    s_wrow[w] = pr0;
                }
            } else if (lane == 0) {
                s_wrow[w] = -1;
            }
        }
        __syncthreads();

        // A row is carried across tiles only if it is the tile's first row and
        // that row began before the tile; a row whose run of partials merely
        // reaches thread 0 may have started inside thread 0's range.
        if (o.fin_row >= 0) {
            bool reached;
            const T carry = seg_walk<T>(tid - 1, o.fin_row, s_part, s_prow, s_wsum, s_wrow, &reached);
            const T total = carry + o.fin_val;
            if (reached && first_carried && o.fin_row == first_row) {
                sc.head_val[tile] = total;
                sc.head_row[tile] = o.fin_row;
                s_head_done = 1;
            } else {
                seg_store<kAlpha, kBeta>(y, o.fin_row, total, alpha, beta);
            }
        }
        // the tile's last active thread publishes the carry of a row open at t1
        if (tid == (cnt - 1) / P) {
            const int32_t r = s_prow[tid];
            if (r >= 0) {
                bool reached;
                const T sum = seg_walk<T>(tid, r, s_part, s_prow, s_wsum, s_wrow, &reached);
                sc.tail_val[tile] = sum;
                sc.tail_row[tile] = r;
                sc.tail_pass[tile] = (reached && first_carried && r == first_row) ? 1 : 0;
            } else {
                sc.tail_row[tile] = -1;
            }
        }
        my_row = next_row;
        __syncthreads();  // stage st and the partial arrays are free again
        if (tid == 0) {
            if (!s_head_done) sc.head_row[tile] = -1;
            s_head_done = 0;
            if (t_issue < n_tiles) {
                fence_proxy_async_smem();  // generic-proxy reads of the stage before the async refill
                issue(t_issue, st, pa, pb, pc);
            }
        }
    }
}

// Finish rows that cross tile boundaries: for each tile f that deferred a
// row r, add the carries of the preceding tiles whose open row is r.
template <bool kAlpha, bool kBeta, typename T>
__global__ void seg_fixup_kernel(int64_t n_tiles, SegScratchT<T> sc, T* __restrict__ y, T alpha, T beta)
{
    const int64_t f = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (f >= n_tiles) return;
    const int32_t r = sc.head_row[f];
    if (r < 0) return;
    T acc = T(0);
    for (int64_t t = f - 1; t >= 0 && sc.tail_row[t] == r; --t) {
        acc = acc + sc.tail_val[t];
        if (!sc.tail_pass[t]) break;
    }
    const T total = acc + sc.head_val[f];
    seg_store<kAlpha, kBeta>(y, r, total, alpha, beta);
}

inline int seg_grid_ctas()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms * kSegCtasPerSm;
}

// Host-side launcher of the load-balanced kernel + fix-up for one
// (V, T) pair.  sc must hold ceil(nnz / TILE) tiles.  Sets the dynamic
// shared-memory attribute on first use (per instantiation).
template <int P, typename V, typename T, bool kAlpha, bool kBeta, bool kCoo, bool kSkip, bool kExact = false>
inline cudaError_t seg_launch(int64_t n_rows, int64_t nnz, const int32_t* row_ptr, const int32_t* rows,
                              const int32_t* col, const V* val, const int32_t* thr_row, SegScratchT<T> sc,
                              const T* x, T* y, T alpha, T beta, uint32_t* err, cudaStream_t st)
{
    constexpr size_t smem = seg_smem_bytes<P, V, T, kCoo>();
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(seg_spmv_kernel<P, V, T, kAlpha, kBeta, kCoo, kSkip, kExact>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int64_t tiles = (nnz + SegShape<P>::kTile - 1) / SegShape<P>::kTile;
    const int64_t grid = tiles < seg_grid_ctas() ? tiles : seg_grid_ctas();
    seg_spmv_kernel<P, V, T, kAlpha, kBeta, kCoo, kSkip, kExact>
        <<<static_cast<unsigned>(grid), kSegThreads, smem, st>>>(n_rows, nnz, row_ptr, rows, col, val, thr_row, x, y,
                                                                 alpha, beta, sc, err);
    if (tiles > 1)
        seg_fixup_kernel<kAlpha, kBeta, T>
            <<<static_cast<unsigned>((tiles + 255) / 256), 256, 0, st>>>(tiles, sc, y, alpha, beta);
    return cudaGetLastError();
}

}  // namespace gko
