// Device-side building blocks shared by every kernel of the library:
// error plumbing, the subwarp (cooperative-group) primitives of the paper's
// Sec. 4 ("Cooperative groups"), the xor-butterfly reduction of Listing 2,
// and thin inline-PTX wrappers for mbarrier + 1-D bulk (TMA) copies.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gko_gb300.h"

namespace gko {

constexpr int kWarp = 32;

// ---------------------------------------------------------------- errors

// Bits of the device error word every handle owns.  Kernels OR bits into
// it instead of trapping; the host reads it with gko_matrix_errors().
enum : uint32_t {
    kErrTimeout = 1u << 0,    // a bounded wait on an mbarrier ran out
    kErrBadIndex = 1u << 1,   // a column/row index outside the matrix (checked builds)
    kErrOverflow = 1u << 2,   // an int32 size computed on the device overflowed
};

__device__ __forceinline__ void raise_error(uint32_t* err, uint32_t bit)
{
    if (err) atomicOr(err, bit);
}

// ------------------------------------------------------ subwarp primitives
//
// Subwarps are groups of Size contiguous lanes (Size a power of two <= 32).
// With tid the thread index inside the block (paper, Sec. 4):
//   Rank       = tid % Size
//   LaneOffset = floor((tid % warpsize) / Size) * Size
//   Mask       = (~0 >> (warpsize - Size)) << LaneOffset
//   ballot(p)  = (warp_ballot(p) & Mask) >> LaneOffset
//   any(p)     = (warp_ballot(p) & Mask) != 0
//   all(p)     = (warp_ballot(p) & Mask) == Mask
// On sm_103a the native *_sync intrinsics take the subwarp mask directly.
template <int Size>
struct subwarp {
    static_assert(Size >= 1 && Size <= 32 && (Size & (Size - 1)) == 0, "power of two");
    __device__ __forceinline__ static int rank() { return threadIdx.x % Size; }
    __device__ __forceinline__ static int lane_offset() { return (threadIdx.x % kWarp) / Size * Size; }
    __device__ __forceinline__ static uint32_t mask()
    {
        return (0xffffffffu >> (kWarp - Size)) << lane_offset();
    }
    __device__ __forceinline__ static uint32_t ballot(bool p)
    {
        return (__ballot_sync(0xffffffffu, p) & mask()) >> lane_offset();
    }
    __device__ __forceinline__ static bool any(bool p) { return (__ballot_sync(0xffffffffu, p) & mask()) != 0; }
    __device__ __forceinline__ static bool all(bool p)
    {
        return (__ballot_sync(0xffffffffu, p) & mask()) == mask();
    }
    template <typename T>
    __device__ __forceinline__ static T shfl_xor(T v, int lane_mask)
    {
        return __shfl_xor_sync(0xffffffffu, v, lane_mask, Size);
    }
    // Butterfly all-reduce over the subwarp (paper, Listing 2): after
    // log2(Size) xor-shuffle steps every lane holds the subwarp's sum.
    template <typename T>
    __device__ __forceinline__ static T reduce_sum(T v)
    {
#pragma unroll
        for (int m = 1; m < Size; m <<= 1) v = v + shfl_xor(v, m);
        return v;
    }
};

__device__ __forceinline__ int popcnt(uint32_t m) { return __popc(m); }
__device__ __forceinline__ int popcnt(uint64_t m) { return __popcll(m); }

// -------------------------------------------------- mbarrier + bulk copies

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after max_spins polls, flags kErrTimeout and
// returns false.  Every poll of try_wait may suspend the thread for a
// hardware-chosen time, so the bound is a few seconds at most.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t* err,
                                                  uint32_t max_spins = (1u << 22))
{
    for (uint32_t i = 0; i < max_spins; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    raise_error(err, kErrTimeout);
    return false;
}

// 1-D bulk copy global -> shared completing on an mbarrier (TMA engine).
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// L2 policy for data read exactly once (a matrix streamed by one SpMV):
// its lines are the first to be evicted, so vectors that are read again
// (the gathered x, a solver's work vectors) stay in L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// bulk_g2s with an L2 cache policy for the source lines.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// Read-only, L1-allocating load for gathered vector entries.
template <typename T>
__device__ __forceinline__ T ldg(const T* p)
{
    return __ldg(p);
}

// ldg as a volatile load: issued where it stands in the source (the
// compiler neither removes it nor moves it into the branches that use it).
// kL2: cached in L2 only (ld.global.cg), for gathers at random columns that
// L1 would not reuse.
template <typename T, bool kL2 = false>
__device__ __forceinline__ T ldg_early(const T* p)
{
    if constexpr (sizeof(T) == 8) {
        double v;
        if constexpr (kL2)
            asm volatile("ld.global.cg.f64 %0, [%1];" : "=d"(v) : "l"(p));
        else
            asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
        return static_cast<T>(v);
    } else {
        float v;
        if constexpr (kL2)
            asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(p));
        else
            asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
        return static_cast<T>(v);
    }
}

// ----------------------------------------------------------- host helpers

inline int ceil_div(int64_t a, int64_t b) { return static_cast<int>((a + b - 1) / b); }

// SM count of the current device, looked up once per device (thread-safe).
int device_sm_count();

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device.  cudaFuncSetAttribute acts on the current device only, so
// the library remembers the limit per (kernel, device) and calls it again
// for each new device or larger size (thread-safe).
cudaError_t smem_limit_once(const void* kernel, int bytes);

// Poll limit of the first bounded wait for a bulk copy in the staged
// kernels (default 2^22 polls; gko_set_wait_limit changes it, for tests of
// the timeout path).  Read by the launchers and passed to the kernels.
uint32_t first_wait_polls();

}  // namespace gko
