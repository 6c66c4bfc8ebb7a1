// Device-side pieces shared by the Krylov solvers: the device-resident
// solver scalars, block and grid-wide sums (one grid reduction per dot: block
// partials + a last-block ticket, summed in block order so results do not
// depend on scheduling) and the stop of a graph's conditional WHILE loop.
#pragma once

#include <algorithm>
#include <vector>

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gko_gb300.h"

namespace gko {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 152 * 4;

// Device-resident solver scalars.
struct SolverState {
    double rho;       // r.r of the current residual
    double rho0;      // r.r at the start (inner solves stop relative to it)
    double pq;        // p.q
    double alpha, beta;
    double stop_ref;  // ||b|| (outer CG) or sqrt(rho0) (inner CG)
    double tol;
    double dot_out;   // result of a plain dot
    int32_t iter, maxit, done, status, conv, rel_inner;
    int32_t skip_test;  // single-reduction CG: skip the next stop test once
    int32_t step_ok;    // CG: this step's alpha was formed (x += alpha p is still due)
    uint32_t ticket;
};

__device__ __forceinline__ double block_sum(double v, double* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = lane < static_cast<int>(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// Grid-wide sum: partials by block, last block reduces them in index order
// and runs epi(total) on thread 0.
template <typename Epi>
__device__ __forceinline__ void grid_sum(double v, double* part, uint32_t* ticket, Epi epi)
{
    __shared__ double sh[32];
    __shared__ bool last;
    const double b = block_sum(v, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc = 0.0;
    for (int i = threadIdx.x; i < static_cast<int>(gridDim.x); i += blockDim.x) acc += __ldcg(part + i);
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        *ticket = 0;
        epi(tot);
    }
}

// Two sums at once (part holds 2 * gridDim.x doubles).
template <typename Epi>
__device__ __forceinline__ void grid_sum2(double v0, double v1, double* part, uint32_t* ticket, Epi epi)
{
    __shared__ double sh[32];
    __shared__ bool last;
    const double b0 = block_sum(v0, sh);
    const double b1 = block_sum(v1, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = b0;
        part[2 * blockIdx.x + 1] = b1;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a0 = 0.0, a1 = 0.0;
    for (int i = threadIdx.x; i < static_cast<int>(gridDim.x); i += blockDim.x) {
        a0 += __ldcg(part + 2 * i);
        a1 += __ldcg(part + 2 * i + 1);
    }
    const double t0 = block_sum(a0, sh);
    const double t1 = block_sum(a1, sh);
    if (threadIdx.x == 0) {
        *ticket = 0;
        epi(t0, t1);
    }
}

__device__ __forceinline__ void stop_loop(SolverState* s, cudaGraphConditionalHandle h)
{
    s->done = 1;
    if (h) cudaGraphSetConditional(h, 0);
}

// Scalar step of the single-reduction CG of Chronopoulos and Gear (1989):
// with gamma = r.r and delta = (A r).r of the current residual,
//   beta  = gamma / gamma_old                      (0 at the first step)
//   alpha = gamma / (delta - beta * gamma / alpha_old)   (gamma / delta at the first step)
// which equal the Hestenes-Stiefel beta and alpha = gamma / (p.Ap) in exact
// arithmetic.  Stops (loop condition cleared) on convergence of the
// recursive residual sqrt(gamma) <= tol * stop_ref, at maxit, or on a NaN
// or a non-positive denominator (breakdown; a timed-out bulk copy shows up
// as NaN with the handle's timeout bit set).
__device__ __forceinline__ void cg1_scalars(SolverState* s, double gamma, double delta, const uint32_t* err,
                                            cudaGraphConditionalHandle h)
{
    if (s->done) {  // stopped before this launch (the host re-arms done = 0)
        stop_loop(s, h);
        return;
    }
    if (!(gamma == gamma) || !(delta == delta)) {
        // a block whose bulk copies never landed contributes NaN and sets
        // the timeout bit of the handle's error word
        const bool timed_out = err && (*reinterpret_cast<const volatile uint32_t*>(err) & 1u);
        s->status = timed_out ? GKO_ERR_TIMEOUT : GKO_ERR_BREAKDOWN;
        stop_loop(s, h);
        return;
    }
    if (s->iter == 0 && s->rel_inner) s->stop_ref = sqrt(gamma);
    if (s->skip_test) {
        s->skip_test = 0;
    } else if (sqrt(gamma) <= s->tol * s->stop_ref) {
        s->conv = 1;
        s->status = GKO_OK;
        stop_loop(s, h);
        return;
    }
    if (s->iter >= s->maxit) {
        s->status = GKO_ERR_NOT_CONVERGED;
        stop_loop(s, h);
        return;
    }
    const double beta = s->iter == 0 ? 0.0 : gamma / s->rho;
    const double denom = s->iter == 0 ? delta : delta - beta * gamma / s->alpha;
    if (!(denom > 0.0)) {
        s->status = GKO_ERR_BREAKDOWN;
        stop_loop(s, h);
        return;
    }
    s->beta = beta;
    s->alpha = gamma / denom;
    s->rho = gamma;
    s->iter += 1;
}

// The grid reduction of a single-reduction CG step, done by the product
// kernel itself: every thread passes its partial (r.r, (A r).r).
struct Cg1Reduce {
    SolverState* s;
    double* part;  // 2 * gridDim.x doubles
    const uint32_t* err;
    cudaGraphConditionalHandle h;
};

// ----------------------------------------------------------- workspace

struct Workspace {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit Workspace(cudaStream_t s) : st(s) {}
    template <typename T>
    int get(T** p, int64_t count)
    {
        *p = nullptr;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(p), std::max<int64_t>(count, 1) * sizeof(T), st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (solver workspace)");
        ptrs.push_back(*p);
        return GKO_OK;
    }
    ~Workspace()
    {
        for (void* q : ptrs) cudaFreeAsync(q, st);
    }
};

struct GraphHolder {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~GraphHolder()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (g) cudaGraphDestroy(g);
    }
};

// Build a graph whose single node is WHILE(cond){ body(handle, cap) }.
// The body is captured on a private non-blocking stream `cap` (capture is
// not allowed on the legacy default stream the caller may be using); the
// instantiated graph is then launched on the caller's stream.
template <typename Body>
inline int build_while_graph(GraphHolder* gh, Body body)
{
    GKO_CUDA(cudaGraphCreate(&gh->g, 0));
    cudaGraphConditionalHandle handle;
    GKO_CUDA(cudaGraphConditionalHandleCreate(&handle, gh->g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams params = {};
    params.type = cudaGraphNodeTypeConditional;
    params.conditional.handle = handle;
    params.conditional.type = cudaGraphCondTypeWhile;
    params.conditional.size = 1;
    cudaGraphNode_t node;
    GKO_CUDA(cudaGraphAddNode(&node, gh->g, nullptr, nullptr, 0, &params));
    cudaGraph_t bodyg = params.conditional.phGraph_out[0];
    cudaStream_t cap;
    GKO_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCaptureToGraph(cap, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    int s = GKO_OK;
    if (e == cudaSuccess) {
        s = body(handle, cap);
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(cap, &captured);
    }
    cudaStreamDestroy(cap);
    if (s != GKO_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "capturing the CG body");
    GKO_CUDA(cudaGraphInstantiate(&gh->exec, gh->g, 0));
    return GKO_OK;
}

}  // namespace gko
