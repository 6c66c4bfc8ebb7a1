// Load-balanced SpMV by an equal split of the stored entries (CSR and COO).
//
// The paper's Sec. 6.1 bounds SpMV by the bytes of the value and index
// streams; on GB300 FP64 arithmetic is just as tight (one FP64 FMA per
// 12 bytes of CSR is ~97 % of the FP64 pipe at full HBM bandwidth), so
// this kernel is built to issue close to one FP64 instruction per stored
// entry whatever the row lengths are:
//
//  * the stored entries are cut into tiles of TILE = NT * P consecutive
//    entries; a persistent grid of CTAs of NT threads (512 threads per SM:
//    2 CTAs of 256 for CSR, 8 CTAs of 64 for COO) walks the tiles round
//    robin with two shared-memory stages: while one tile is
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

constexpr int kSegThreads = 256;        // threads per CTA (= per tile) unless a launch picks NT
constexpr int kSegThreadsPerSm = 512;   // resident threads per SM (registers, shared memory)
constexpr int kSegCtasPerSm = kSegThreadsPerSm / kSegThreads;

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

template <int P, int NT = kSegThreads>
struct SegShape {
    static constexpr int kTile = NT * P;  // a multiple of 8 entries for the P and NT used here
    static constexpr int kBuf = kTile + 8;         // bulk copies move whole 16-byte groups
    static constexpr int kRowStage = 2048;         // CSR row_ptr entries staged per tile
};

// one pipeline stage: values | column indices | (COO rows or CSR row_ptr)
template <int P, typename V, bool kCoo, int NT = kSegThreads>
struct SegStage {
    static constexpr size_t kVal = SegShape<P, NT>::kBuf * sizeof(V);
    static constexpr size_t kCol = SegShape<P, NT>::kBuf * sizeof(int32_t);
    static constexpr size_t kAux = (kCoo ? SegShape<P, NT>::kBuf : SegShape<P, NT>::kRowStage) * sizeof(int32_t);
    static constexpr size_t kBytes = kVal + kCol + kAux;
    static_assert(kVal % 16 == 0 && kCol % 16 == 0 && kAux % 16 == 0, "16-byte aligned stage parts");
};

template <int P, typename V, typename T, bool kCoo, int NT = kSegThreads>
constexpr size_t seg_smem_bytes()
{
    return 2 * SegStage<P, V, kCoo, NT>::kBytes + NT * (sizeof(T) + sizeof(int32_t)) +
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

// y[r] = alpha v + beta y[r].  kRed (accumulate mode of the hybrid format's
// COO part, beta = 1): y[r] += alpha v as a fire-and-forget reduction in L2,
// so no load of y stalls the thread; every row gets exactly one such add per
// launch (rows crossing tiles only from the fix-up), so the result does not
// depend on the order of the adds.
template <bool kAlpha, bool kBeta, bool kRed = false, typename T>
__device__ __forceinline__ void seg_store(T* y, int64_t r, T v, T alpha, T beta)
{
    if constexpr (kRed) {
        atomicAdd(y + r, kAlpha ? alpha * v : v);
    } else {
        T out = kAlpha ? alpha * v : v;
        if (kBeta) out = fma(beta, y[r], out);
        y[r] = out;
    }
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

// Phase 1 of one tile for one thread, COO.  The thread's entries
// [ls, ls + rem) are loaded with their rows; a bit mask marks the entries
// after which a row ends (the row of the next entry differs; rows are
// sorted), so the row structure costs one compare per entry.  Each entry
// then costs one FMA into a running sum that is reset at each end; the
// first finished row goes to fin when it began before the thread.  Three
// paths, chosen per warp: at most three ends (the sums at the ends kept in
// registers, stored after the loop); any number of ends with no row
// without entries in between (the sums parked in the thread's own stage
// slots, stored after the loop); the general path (rows without entries
// get their zero stores).  kFull: every thread of the tile holds P entries
// (all tiles but the last), so no per-entry bounds predicates are needed.
template <int P, typename V, typename T, bool kAlpha, bool kBeta, bool kSkipEmpty, bool kFull, bool kGatherL2>
__device__ __forceinline__ SegThreadOut<T> seg_thread_coo(int ls, int rem, int t0, int cnt, const V* s_val,
                                                          const int32_t* s_col, const int32_t* s_row,
                                                          bool first_carried, int next_r_tile,
                                                          const T* __restrict__ x, T* __restrict__ y, T alpha, T beta)
{
    SegThreadOut<T> o{-1, T(0), -1, T(0)};
    T vv[P], xv[P];
    int rr[P];
    // the gathers of x are issued first, as volatile loads, so that they are
    // all in flight before the row logic and are not moved to their uses
    // behind the warp vote (random columns miss in L1 and L2)
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const bool ok = kFull || j < rem;
        const int c = ok ? s_col[ls + j] : 0;
        vv[j] = ok ? to_t<V, T>(s_val[ls + j]) : T(0);
        xv[j] = ldg_early<T, kGatherL2>(x + c);
    }
#pragma unroll
    for (int j = 0; j < P; ++j) rr[j] = (kFull || j < rem) ? s_row[ls + j] : 0;
    // NOTE: lanes without entries must not return before the warp vote below.
    const bool has = rem > 0;
    const int n_mine = kFull ? P : max(0, min(rem, P));
    const int after = ls + n_mine;  // position after the thread's last entry
    const int r_next = has ? (after < cnt ? s_row[after] : next_r_tile) : 0;
    const int r_first = rr[0];
    const bool ob = has && ((ls == 0) ? first_carried : (s_row[ls - 1] == r_first));
    uint32_t mask = 0;  // bit j: a row ends after entry j
#pragma unroll
    for (int j = 0; j < P; ++j) {
        if (kFull || j < n_mine) {
            const int nx = (j + 1 < P && (kFull || j + 1 < n_mine)) ? rr[j + 1] : r_next;
            mask |= static_cast<uint32_t>(nx != rr[j]) << j;
        }
    }
    const int n_end = __popc(mask);
    // rows are sorted: a row without entries lies between the thread's first
    // row and the next one exactly when they are further apart than the
    // number of row changes
    const bool gap = has && (r_next - r_first > n_end);
    if (has && !kSkipEmpty && t0 + ls == 0)  // rows before the first stored entry
        for (int r = 0; r < r_first; ++r) seg_store<kAlpha, kBeta>(y, r, T(0), alpha, beta);
    const bool fast = n_end <= 3 && (kSkipEmpty || !gap);
    const bool warp_fast = __all_sync(0xffffffffu, fast);  // every lane of the warp reaches this
    const bool warp_flat = !warp_fast && __all_sync(0xffffffffu, kSkipEmpty || !gap);
    if (!has) return o;
    if (warp_fast) {
        // at most three ends: the sums at the ends are captured in registers
        // and stored after the loop
        const int e0 = __ffs(mask);  // 1 + position of the first end (0: none)
        const uint32_t m1 = mask & (mask - 1u);
        const int e1 = __ffs(m1);
        const int e2 = __ffs(m1 & (m1 - 1u));
        T acc = T(0), v0 = T(0), v1 = T(0), v2 = T(0);
#pragma unroll
        for (int j = 0; j < P; ++j) {
            if (kFull || j < n_mine) {
                acc = fma(vv[j], xv[j], acc);
                v0 = (j + 1 == e0) ? acc : v0;
                v1 = (j + 1 == e1) ? acc : v1;
                v2 = (j + 1 == e2) ? acc : v2;
                acc = ((mask >> j) & 1u) ? T(0) : acc;
            }
        }
        if (n_end > 0) {
            if (ob) {
                o.fin_row = r_first;
                o.fin_val = v0;
            } else {
                seg_store<kAlpha, kBeta, kSkipEmpty>(y, r_first, v0, alpha, beta);
            }
        }
        if (n_end > 1) seg_store<kAlpha, kBeta, kSkipEmpty>(y, s_row[ls + e0], v1, alpha, beta);
        if (n_end > 2) seg_store<kAlpha, kBeta, kSkipEmpty>(y, s_row[ls + e1], v2, alpha, beta);
        if (!((mask >> (n_mine - 1)) & 1u)) {  // the last entry's row is still open
            o.open_row = s_row[ls + n_mine - 1];
            o.open_val = acc;
        }
        return o;
    }
    if (warp_flat) {
        // any number of ends (rows without entries are skipped or absent):
        // the finished rows go to this thread's own slots of the stage (its
        // values and columns are in registers already) and are written out
        // after the FMA loop, loads of y first when beta != 0
        V* sv = const_cast<V*>(s_val) + ls;
        int32_t* sr = const_cast<int32_t*>(s_col) + ls;
        const int e0 = __ffs(mask);
        T acc = T(0), f0 = T(0);
        int k = 0;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            if (kFull || j < n_mine) {
                acc = fma(vv[j], xv[j], acc);
                const bool end = (mask >> j) & 1u;
                const bool first = j + 1 == e0;
                const bool put = end && !(first && ob);
                if (put) {
                    sv[k] = static_cast<V>(acc);
                    sr[k] = rr[j];
                }
                k += put ? 1 : 0;
                f0 = first ? acc : f0;
                acc = end ? T(0) : acc;
            }
        }
        if (ob && n_end > 0) {
            o.fin_row = r_first;
            o.fin_val = f0;
        }
        if (!((mask >> (n_mine - 1)) & 1u)) {
            o.open_row = s_row[ls + n_mine - 1];
            o.open_val = acc;
        }
        if (kSkipEmpty) {  // accumulate mode: reductions, no loads of y
#pragma unroll
            for (int q = 0; q < P; ++q)
                if (q < k) seg_store<kAlpha, kBeta, true>(y, sr[q], to_t<V, T>(sv[q]), alpha, beta);
        } else if (kBeta) {
            T yo[P];
#pragma unroll
            for (int q = 0; q < P; ++q) yo[q] = q < k ? y[sr[q]] : T(0);
#pragma unroll
            for (int q = 0; q < P; ++q)
                if (q < k) {
                    const T vq = kAlpha ? alpha * to_t<V, T>(sv[q]) : to_t<V, T>(sv[q]);
                    y[sr[q]] = fma(beta, yo[q], vq);
                }
        } else {
#pragma unroll
            for (int q = 0; q < P; ++q)
                if (q < k) seg_store<kAlpha, kBeta>(y, sr[q], to_t<V, T>(sv[q]), alpha, beta);
        }
        return o;
    }

    // ---- general path: any number of row ends, empty rows included
    T acc = T(0);
    bool pending = false, obb = ob;
    int row = r_first;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        if (kFull || j < n_mine) {
            acc = fma(vv[j], xv[j], acc);
            pending = true;
            const int nr = (j + 1 < P && (kFull || j + 1 < n_mine)) ? rr[j + 1] : r_next;
            if (nr != row) {
                if (obb) {
                    o.fin_row = row;
                    o.fin_val = acc;
                } else {
                    seg_store<kAlpha, kBeta, kSkipEmpty>(y, row, acc, alpha, beta);
                }
                acc = T(0);
                pending = false;
                obb = false;
                if (!kSkipEmpty)
                    for (int r = row + 1; r < nr; ++r) seg_store<kAlpha, kBeta>(y, r, T(0), alpha, beta);
                row = nr;
            }
        }
    }
    if (pending) {
        o.open_row = row;
        o.open_val = acc;
    }
    return o;
}

// kCoo = false: CSR with row_ptr and the per-thread start rows thr_row
// (thr_row[g] = row holding entry g*P).  kCoo = true: COO with row[].
// kSkipEmpty: accumulate mode, y[r] += alpha (A x)_r by L2 reductions for
// the rows with entries, the others left untouched (adds the COO part of the
// hybrid format onto the ELL part's result; COO only, beta = 1).
// kExactTail (COO only): the arrays end exactly at nnz (caller-owned, not
// padded), so the last tile bulk-copies only whole 16-byte groups and the
// threads load the remaining few entries themselves.
// NT: threads per CTA and per tile (a multiple of 32, at most 256).
// kGatherL2 (COO): gathers of x cached in L2 only (columns scattered at
// random: L1 would not reuse them and its lines are better left to the
// gathers in flight).
template <int P, typename V, typename T, bool kAlpha, bool kBeta, bool kCoo, bool kSkipEmpty, bool kExactTail = false,
          int NT = kSegThreads, bool kGatherL2 = false>
__global__ void __launch_bounds__(NT, kSegThreadsPerSm / NT)
    seg_spmv_kernel(int64_t n_rows64, int64_t n_cols64, int64_t nnz64, const int32_t* __restrict__ row_ptr,
                    const int32_t* __restrict__ rows, const int32_t* __restrict__ col,
                    const V* __restrict__ val, const int32_t* __restrict__ thr_row, const T* __restrict__ x,
                    T* __restrict__ y, T alpha, T beta, SegScratchT<T> sc, uint32_t* err, uint32_t polls)
{
    using S = SegShape<P, NT>;
    using G = SegStage<P, V, kCoo, NT>;
    static_assert(!kExactTail || kCoo, "exact tails are implemented for COO");
    static_assert(NT % 32 == 0 && NT <= 256, "whole warps, at most 8 (s_wsum)");
    constexpr int kAlign = 16 / sizeof(V) > 4 ? 16 / sizeof(V) : 4;  // entries per 16-byte group
    extern __shared__ __align__(16) unsigned char smem[];
    T* s_part = reinterpret_cast<T*>(smem + 2 * G::kBytes);
    int32_t* s_prow = reinterpret_cast<int32_t*>(s_part + NT);
    T* s_wsum = reinterpret_cast<T*>(s_prow + NT);
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
        return thr_row[tile * NT];
    };
    auto meta_b = [&](int tile) -> int32_t {
        if (kCoo) return rows[tile * S::kTile];
        return (tile + 1) * S::kTile < nnz ? thr_row[(tile + 1) * NT] : n_rows;
    };
    auto meta_c = [&](int tile) -> int32_t {
        if (!kCoo) return 0;
        const int32_t r = (tile + 1) * S::kTile < nnz ? rows[(tile + 1) * S::kTile] : n_rows;
#ifdef GKO_CHECK_BOUNDS
        return min(max(r, 0), n_rows);  // bounds rows of empty-row stores at n_rows
#else
        return r;
#endif
    };
    // start row of this thread's entries in a tile (threads whose first
    // entry exists only: thr_row has ceil(nnz / P) entries)
    auto start_row = [&](int tile) -> int32_t {
        const int g = tile * NT + tid;
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
        const bool landed = mbar_wait_bounded(&bar[st], parity, err, polls);
        if (!__syncthreads_and(landed)) {  // CTA-uniform exit (y is left undefined)
            // first wait for the copies this CTA still has in flight (this
            // stage and the next tile's, default limit), so that no bulk copy
            // writes its shared memory after it has exited
            if (tid == 0) {
                mbar_wait_bounded(&bar[st], parity, err);
                if (tile + stride < n_tiles) mbar_wait_bounded(&bar[st ^ 1], ((it + 1) >> 1) & 1, err);
            }
            // the tiles left undone carry nothing: the fix-up then reads only
            // carries written in this launch
            for (int t = tile + tid * stride; t < n_tiles; t += NT * stride) {
                sc.head_row[t] = -1;
                sc.tail_row[t] = -1;
            }
            __syncthreads();
            return;
        }
        if (kExactTail) {  // entries past the last whole 16-byte group (last tile only)
            const int tx0 = info[st].t0;
            const int cx = min(tx0 + S::kTile, nnz) - tx0;
            for (int i = cx / kAlign * kAlign + tid; i < cx; i += NT) {
                stage_val(st)[i] = val[tx0 + i];
                stage_col(st)[i] = col[tx0 + i];
                stage_aux(st)[i] = rows[tx0 + i];
            }
            __syncthreads();
        }
#ifdef GKO_CHECK_BOUNDS
        // checked build: indices the caller did not validate (the allocation-
        // free COO entry) are checked in shared memory before use; an entry
        // with a column or row out of range gets column 0 (row n_rows - 1)
        // and value 0 and kErrBadIndex is raised: no load or store leaves
        // the arrays (a bad column then adds nothing; a bad row may leave y
        // wrong, which the error bit reports)
        if constexpr (kCoo && sizeof(V) == 8) {
            const int cx = min(info[st].t0 + S::kTile, nnz) - info[st].t0;
            int32_t* sc_col = stage_col(st);
            int32_t* sc_row = stage_aux(st);
            V* sc_val = stage_val(st);
            for (int i = tid; i < cx; i += NT) {
                const bool bad_c = static_cast<uint32_t>(sc_col[i]) >= static_cast<uint32_t>(n_cols64);
                const bool bad_r = static_cast<uint32_t>(sc_row[i]) >= static_cast<uint32_t>(n_rows);
                if (bad_c || bad_r) {
                    raise_error(err, kErrBadIndex);
                    sc_col[i] = 0;
                    sc_val[i] = V(0);
                    if (bad_r) sc_row[i] = n_rows - 1;
                }
            }
            __syncthreads();
        }
#endif

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
        if constexpr (kCoo) {
            first_carried = ti.began != 0;
            if (cnt == S::kTile)  // tile-uniform: every thread holds P entries
                o = seg_thread_coo<P, V, T, kAlpha, kBeta, kSkipEmpty, true, kGatherL2>(ls, le - ls, t0, cnt, s_val, s_col,
                                                                            s_aux, first_carried, ti.next_r, x, y,
                                                                            alpha, beta);
            else
                o = seg_thread_coo<P, V, T, kAlpha, kBeta, kSkipEmpty, false, kGatherL2>(ls, le - ls, t0, cnt, s_val, s_col,
                                                                             s_aux, first_carried, ti.next_r, x, y,
                                                                             alpha, beta);
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
                seg_store<kAlpha, kBeta, kCoo && kSkipEmpty>(y, o.fin_row, total, alpha, beta);
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
template <bool kAlpha, bool kBeta, typename T, bool kRed = false>
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
    seg_store<kAlpha, kBeta, kRed>(y, r, total, alpha, beta);
}

// 2 CTAs per SM (the row-block CSR kernel's grid uses the same count)
inline int seg_grid_ctas() { return device_sm_count() * kSegCtasPerSm; }

// Host-side launcher of the load-balanced kernel + fix-up for one
// (V, T) pair.  sc must hold ceil(nnz / (NT * P)) tiles.  Raises the dynamic
// shared-memory limit once per instantiation and device.
template <int P, typename V, typename T, bool kAlpha, bool kBeta, bool kCoo, bool kSkip, bool kExact = false,
          int NT = kSegThreads, bool kGatherL2 = false>
inline cudaError_t seg_launch(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* row_ptr, const int32_t* rows,
                              const int32_t* col, const V* val, const int32_t* thr_row, SegScratchT<T> sc,
                              const T* x, T* y, T alpha, T beta, uint32_t* err, cudaStream_t st)
{
    constexpr size_t smem = seg_smem_bytes<P, V, T, kCoo, NT>();
    const cudaError_t e = smem_limit_once(
        reinterpret_cast<const void*>(seg_spmv_kernel<P, V, T, kAlpha, kBeta, kCoo, kSkip, kExact, NT, kGatherL2>),
        static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int64_t tiles = (nnz + SegShape<P, NT>::kTile - 1) / SegShape<P, NT>::kTile;
    const int64_t ctas = static_cast<int64_t>(device_sm_count()) * (kSegThreadsPerSm / NT);
    const int64_t grid = tiles < ctas ? tiles : ctas;
    seg_spmv_kernel<P, V, T, kAlpha, kBeta, kCoo, kSkip, kExact, NT, kGatherL2>
        <<<static_cast<unsigned>(grid), NT, smem, st>>>(n_rows, n_cols, nnz, row_ptr, rows, col, val, thr_row, x, y,
                                                        alpha, beta, sc, err, first_wait_polls());
    if (tiles > 1)
        seg_fixup_kernel<kAlpha, kBeta, T, kCoo && kSkip>
            <<<static_cast<unsigned>((tiles + 255) / 256), 256, 0, st>>>(tiles, sc, y, alpha, beta);
    return cudaGetLastError();
}

}  // namespace gko
