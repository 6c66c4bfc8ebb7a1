// Hardware ceilings the sparse kernels are judged against, measured on the
// running GPU the way the paper's Sec. 6 characterises each platform before
// its SpMV and solver results (a stream benchmark for bandwidth, mixbench
// for arithmetic): here the FP64 FMA rate, which co-binds FP64 SpMV on this
// part (one FMA per 12 or 16 bytes of matrix), and the rate of random 8-byte
// gathers, which bounds unstructured matrices (one gather of x per entry).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace gko {

constexpr int kProbeThreads = 256;
constexpr int kFmaChains = 8;    // independent FMA chains per thread
constexpr int kFmaIters = 4096;  // FMAs per chain

// Every thread runs kFmaChains independent chains a = a * m + c (m just
// below 1, so the values stay bounded); the sum is stored so that nothing
// is optimised away.
template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(T* out, T m, T c)
{
    T a[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = static_cast<T>(threadIdx.x + k);
    for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
        for (int k = 0; k < kFmaChains; ++k) a[k] = fma(a[k], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) s += a[k];
    out[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

// Random gathers: thread i reads x[h(i, k)] for k < per_thread, with h a
// SplitMix64-style counter hash (no index array is read), m a power of two.
__global__ void __launch_bounds__(kProbeThreads)
    gather_probe_kernel(const double* __restrict__ x, uint64_t mask, int per_thread, double* out)
{
    const uint64_t i = blockIdx.x * static_cast<uint64_t>(kProbeThreads) + threadIdx.x;
    double s = 0.0;
    for (int k = 0; k < per_thread; k += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            uint64_t z = (i * 0x9E3779B97F4A7C15ull) ^ static_cast<uint64_t>(k + u) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 31)) * 0x94D049BB133111EBull;
            z ^= z >> 29;
            v[u] = __ldg(x + (z & mask));
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
    }
    out[i] = s;
}

template <typename F>
static int time_ms(cudaStream_t st, F launch, float* ms)
{
    cudaEvent_t e0, e1;
    GKO_CUDA(cudaEventCreate(&e0));
    GKO_CUDA(cudaEventCreate(&e1));
    launch();  // warm-up
    float best = 0.0f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep == 0 || t < best) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    GKO_CUDA(cudaGetLastError());
    *ms = best;
    return GKO_OK;
}

}  // namespace gko

using namespace gko;

extern "C" int gko_measure_ceilings(double* fp64_tfma, double* fp32_tfma, double* gathers_g, int64_t gather_span,
                                    void* stream)
{
    if (!fp64_tfma || !fp32_tfma || !gathers_g) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    if (gather_span < 1024 || (gather_span & (gather_span - 1)))
        return fail(GKO_ERR_INVALID_ARG, "gather_span must be a power of two >= 1024");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = device_sm_count() * 8;
    const int64_t threads = static_cast<int64_t>(blocks) * kProbeThreads;
    constexpr int kGathers = 256;  // per thread
    double* buf = nullptr;
    const int64_t need = std::max<int64_t>(gather_span, threads);
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&buf), (need + threads) * sizeof(double), st));
    double* out = buf + need;
    int s = GKO_OK;
    float ms = 0.0f;
    const double fmas = static_cast<double>(threads) * kFmaChains * kFmaIters;
    if (s == GKO_OK)
        s = time_ms(st, [&] { fma_probe_kernel<double><<<blocks, kProbeThreads, 0, st>>>(out, 0.999999, 1e-6); },
                    &ms);
    if (s == GKO_OK) *fp64_tfma = fmas / (ms * 1e-3) / 1e12;
    if (s == GKO_OK)
        s = time_ms(st,
                    [&] {
                        fma_probe_kernel<float><<<blocks, kProbeThreads, 0, st>>>(reinterpret_cast<float*>(out),
                                                                                 0.999f, 1e-3f);
                    },
                    &ms);
    if (s == GKO_OK) *fp32_tfma = fmas / (ms * 1e-3) / 1e12;
    if (s == GKO_OK) {
        cudaError_t e = cudaMemsetAsync(buf, 0, gather_span * sizeof(double), st);
        if (e != cudaSuccess) s = cuda_fail(e, "gather probe input");
    }
    if (s == GKO_OK)
        s = time_ms(st,
                    [&] {
                        gather_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(
                            buf, static_cast<uint64_t>(gather_span - 1), kGathers, out);
                    },
                    &ms);
    if (s == GKO_OK) *gathers_g = static_cast<double>(threads) * kGathers / (ms * 1e-3) / 1e9;
    cudaFreeAsync(buf, st);
    if (s == GKO_OK) GKO_CUDA(cudaStreamSynchronize(st));
    return s;
}
