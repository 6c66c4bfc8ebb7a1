// Learned format selector: matrix statistics, a small MLP (12 -> 64 -> 64
// -> n_out, ReLU, FP32) trained on the GPU, and the choice it makes for
// GKO_FMT_AUTO.  The paper's Sec. 6.1 observes that no SpMV kernel wins on
// every matrix; the selector predicts the fastest (format, kernel) class
// from the statistics instead of timing every candidate.
//
// All reductions (over rows for the statistics, over samples for the
// gradients) run in a fixed order or in exact integer arithmetic, so every
// call is deterministic.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace gko {

// ------------------------------------------------------------ statistics

struct FeatStats {
    unsigned long long sum_l2;    // sum of squared row lengths
    unsigned long long sum_dist;  // sum of |i - j| over entries
    unsigned long long slots32;   // SELL-P(32, f=1) slots
    unsigned long long empty, diag;
    int max_len, min_len, max_dist, pad;
};

__global__ void feat_kernel(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            FeatStats* fs)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    int L = 0, dmax = 0, has_diag = 0;
    unsigned long long dsum = 0;
    const bool ok = r < n;
    if (ok) {
        const int32_t a = row_ptr[r], b = row_ptr[r + 1];
        L = b - a;
        for (int32_t k = a; k < b; ++k) {
            const int64_t d = col[k] - r;
            const int ad = static_cast<int>(d < 0 ? -d : d);
            dmax = max(dmax, ad);
            dsum += static_cast<unsigned long long>(ad);
            has_diag |= (col[k] == r);
        }
    }
    // slices of 32 rows are warps (blockDim is a multiple of 32, rows start at 0)
    int smax = L;
    for (int o = 16; o; o >>= 1) smax = max(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    if (ok) {
        atomicAdd(&fs->sum_l2, static_cast<unsigned long long>(L) * static_cast<unsigned long long>(L));
        if (dsum) atomicAdd(&fs->sum_dist, dsum);
        if (L == 0) atomicAdd(&fs->empty, 1ull);
        if (has_diag) atomicAdd(&fs->diag, 1ull);
        atomicMax(&fs->max_len, L);
        atomicMin(&fs->min_len, L);
        atomicMax(&fs->max_dist, dmax);
        if ((threadIdx.x & 31) == 0) atomicAdd(&fs->slots32, 32ull * static_cast<unsigned long long>(smax));
    }
}

__global__ void feat_final_kernel(int64_t n, int64_t nnz, const FeatStats* fs, double* f)
{
    if (threadIdx.x || blockIdx.x) return;
    const double dn = static_cast<double>(n);
    const double mean = static_cast<double>(nnz) / dn;
    double var = static_cast<double>(fs->sum_l2) / dn - mean * mean;
    var = var > 0.0 ? var : 0.0;
    f[0] = log10(dn);
    f[1] = log10(static_cast<double>(nnz > 0 ? nnz : 1));
    f[2] = mean;
    f[3] = sqrt(var);
    f[4] = fs->max_len;
    f[5] = fs->min_len;
    f[6] = mean > 0.0 ? fs->max_len / mean : 0.0;
    f[7] = static_cast<double>(fs->empty) / dn;
    f[8] = fs->max_dist / dn;
    f[9] = nnz > 0 ? static_cast<double>(fs->sum_dist) / static_cast<double>(nnz) / dn : 0.0;
    f[10] = static_cast<double>(fs->diag) / dn;
    f[11] = nnz > 0 ? static_cast<double>(fs->slots32) / static_cast<double>(nnz) : 0.0;
}

int features_compute(const gko_matrix* A, double* out, cudaStream_t st)
{
    FeatStats* fs = nullptr;
    double* f = nullptr;
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&fs), sizeof(FeatStats), st));
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&f), 12 * sizeof(double), st));
    FeatStats init = {};
    init.min_len = INT32_MAX;
    GKO_CUDA(cudaMemcpyAsync(fs, &init, sizeof(init), cudaMemcpyHostToDevice, st));
    feat_kernel<<<ceil_div(A->n_rows, 256), 256, 0, st>>>(A->n_rows, A->csr.row_ptr, A->csr.col, fs);
    feat_final_kernel<<<1, 32, 0, st>>>(A->n_rows, A->nnz, fs, f);
    GKO_CUDA(cudaMemcpyAsync(out, f, 12 * sizeof(double), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaFreeAsync(fs, st));
    GKO_CUDA(cudaFreeAsync(f, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

// ------------------------------------------------------------------- MLP

constexpr int kIn = 12, kHid = 64, kMaxOut = 64;

struct MlpView {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};

__host__ __device__ inline int64_t mlp_count(int n_out)
{
    return static_cast<int64_t>(kHid) * kIn + kHid + kHid * kHid + kHid + static_cast<int64_t>(n_out) * kHid + n_out;
}

__device__ __forceinline__ MlpView mlp_view(const float* p, int n_out)
{
    MlpView v;
    v.W1 = p;
    v.b1 = v.W1 + kHid * kIn;
    v.W2 = v.b1 + kHid;
    v.b2 = v.W2 + kHid * kHid;
    v.W3 = v.b2 + kHid;
    v.b3 = v.W3 + n_out * kHid;
    return v;
}

// One block of 64 threads per sample (grid-stride over samples): forward
// pass; optionally keeps z1, z2 (pre-activations) and h1, h2 for backward.
__global__ void __launch_bounds__(kHid)
    mlp_forward_kernel(const float* __restrict__ params, int n_out, const float* __restrict__ X, int batch,
                       float* __restrict__ out, float* __restrict__ z1s, float* __restrict__ h1s,
                       float* __restrict__ z2s, float* __restrict__ h2s)
{
    __shared__ float xs[kIn], h1[kHid], h2[kHid];
    const MlpView P = mlp_view(params, n_out);
    const int j = threadIdx.x;
    for (int s = blockIdx.x; s < batch; s += gridDim.x) {
        if (j < kIn) xs[j] = X[static_cast<int64_t>(s) * kIn + j];
        __syncthreads();
        float z = P.b1[j];
        for (int k = 0; k < kIn; ++k) z = fmaf(P.W1[j * kIn + k], xs[k], z);
        const float a1 = fmaxf(z, 0.0f);
        h1[j] = a1;
        if (z1s) {
            z1s[static_cast<int64_t>(s) * kHid + j] = z;
            h1s[static_cast<int64_t>(s) * kHid + j] = a1;
        }
        __syncthreads();
        float z2 = P.b2[j];
        for (int k = 0; k < kHid; ++k) z2 = fmaf(P.W2[j * kHid + k], h1[k], z2);
        const float a2 = fmaxf(z2, 0.0f);
        h2[j] = a2;
        if (z2s) {
            z2s[static_cast<int64_t>(s) * kHid + j] = z2;
            h2s[static_cast<int64_t>(s) * kHid + j] = a2;
        }
        __syncthreads();
        if (j < n_out) {
            float o = P.b3[j];
            for (int k = 0; k < kHid; ++k) o = fmaf(P.W3[j * kHid + k], h2[k], o);
            out[static_cast<int64_t>(s) * n_out + j] = o;
        }
        __syncthreads();
    }
}

// dout = 2 M (out - Y) / sum(M) and the loss; one block, fixed order
__global__ void mlp_dout_kernel(int n, const float* __restrict__ out, const float* __restrict__ Y,
                                const float* __restrict__ M, float* __restrict__ dout, float* loss)
{
    __shared__ double sh_m[256], sh_l[256];
    double m = 0.0, l = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = static_cast<double>(out[i]) - static_cast<double>(Y[i]);
        m += M[i];
        l += M[i] * d * d;
    }
    sh_m[threadIdx.x] = m;
    sh_l[threadIdx.x] = l;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) {
            sh_m[threadIdx.x] += sh_m[threadIdx.x + o];
            sh_l[threadIdx.x] += sh_l[threadIdx.x + o];
        }
        __syncthreads();
    }
    const double denom = sh_m[0] > 0.0 ? sh_m[0] : 1.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        dout[i] = static_cast<float>(2.0 * M[i] * (static_cast<double>(out[i]) - Y[i]) / denom);
    if (threadIdx.x == 0 && loss) *loss = static_cast<float>(sh_l[0] / denom);
}

// dh = (dnext @ W) * (z > 0) for one layer: dz[s, k] = (sum_j dnext[s, j] W[j, k]) * (z[s, k] > 0)
__global__ void mlp_back_act_kernel(int batch, int n_next, const float* __restrict__ dnext,
                                    const float* __restrict__ W, const float* __restrict__ z, float* __restrict__ dz)
{
    const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (t >= static_cast<int64_t>(batch) * kHid) return;
    const int64_t s = t / kHid;
    const int k = static_cast<int>(t % kHid);
    float acc = 0.0f;
    for (int j = 0; j < n_next; ++j) acc = fmaf(dnext[s * n_next + j], W[j * kHid + k], acc);
    dz[t] = z[t] > 0.0f ? acc : 0.0f;
}

// weight gradient dW[j, k] = sum_s d[s, j] a[s, k] (and db[j] = sum_s d[s, j]),
// one thread per weight, samples summed in order
__global__ void mlp_wgrad_kernel(int batch, int n_out, int n_in, const float* __restrict__ d,
                                 const float* __restrict__ a, float* __restrict__ dW, float* __restrict__ db)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nw = n_out * n_in;
    if (t < nw) {
        const int j = t / n_in, k = t % n_in;
        float acc = 0.0f;
        for (int s = 0; s < batch; ++s)
            acc = fmaf(d[static_cast<int64_t>(s) * n_out + j], a[static_cast<int64_t>(s) * n_in + k], acc);
        dW[t] = acc;
    } else if (t < nw + n_out) {
        const int j = t - nw;
        float acc = 0.0f;
        for (int s = 0; s < batch; ++s) acc += d[static_cast<int64_t>(s) * n_out + j];
        db[j] = acc;
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ------------------------------------------------------- installed model

struct Selector {
    bool loaded = false;
    int n_out = 0;
    std::vector<float> params;
    double mean[12], scale[12];
    std::vector<int> fmts, cfgs;
    float* d_params = nullptr;
    int device = -1;
};
static Selector g_sel;
static std::mutex g_sel_mu;
static uint64_t g_sel_gen = 0;  // bumped by every load/clear; 0 until the first load

uint64_t selector_generation()
{
    std::lock_guard<std::mutex> lk(g_sel_mu);
    return g_sel.loaded ? g_sel_gen : 0;
}

}  // namespace gko

using namespace gko;

extern "C" {

int64_t gko_mlp_param_count(int n_out) { return (n_out < 1 || n_out > kMaxOut) ? -1 : mlp_count(n_out); }

int gko_mlp_forward(const float* params, int n_out, const float* X, int batch, float* out, void* stream)
{
    if (!params || !X || !out) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    if (n_out < 1 || n_out > kMaxOut || batch < 0) return fail(GKO_ERR_INVALID_ARG, "bad n_out or batch");
    if (batch == 0) return GKO_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mlp_forward_kernel<<<std::min(batch, 152 * 16), kHid, 0, st>>>(params, n_out, X, batch, out, nullptr, nullptr,
                                                                   nullptr, nullptr);
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

int gko_mlp_grad(const float* params, int n_out, const float* X, const float* Y, const float* M, int batch,
                 float* grad, float* loss, void* stream)
{
    if (!params || !X || !Y || !M || !grad) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    if (n_out < 1 || n_out > kMaxOut || batch < 1) return fail(GKO_ERR_INVALID_ARG, "bad n_out or batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t B = batch;
    float* buf = nullptr;
    const int64_t need = B * (4 * kHid + 2 * n_out + 2 * kHid);
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&buf), need * sizeof(float), st));
    float *z1 = buf, *h1 = z1 + B * kHid, *z2 = h1 + B * kHid, *h2 = z2 + B * kHid;
    float *out = h2 + B * kHid, *dout = out + B * n_out, *dz2 = dout + B * n_out, *dz1 = dz2 + B * kHid;
    mlp_forward_kernel<<<std::min(batch, 152 * 16), kHid, 0, st>>>(params, n_out, X, batch, out, z1, h1, z2, h2);
    mlp_dout_kernel<<<1, 256, 0, st>>>(batch * n_out, out, Y, M, dout, loss);
    // parameter offsets (same packing as mlp_view)
    const int64_t oW1 = 0, ob1 = oW1 + kHid * kIn, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid, oW3 = ob2 + kHid,
                  ob3 = oW3 + static_cast<int64_t>(n_out) * kHid;
    const int tb = 256;
    const int g_act = ceil_div(B * kHid, tb);
    mlp_back_act_kernel<<<g_act, tb, 0, st>>>(batch, n_out, dout, params + oW3, z2, dz2);
    mlp_back_act_kernel<<<g_act, tb, 0, st>>>(batch, kHid, dz2, params + oW2, z1, dz1);
    mlp_wgrad_kernel<<<ceil_div(n_out * kHid + n_out, tb), tb, 0, st>>>(batch, n_out, kHid, dout, h2, grad + oW3,
                                                                        grad + ob3);
    mlp_wgrad_kernel<<<ceil_div(kHid * kHid + kHid, tb), tb, 0, st>>>(batch, kHid, kHid, dz2, h1, grad + oW2,
                                                                      grad + ob2);
    mlp_wgrad_kernel<<<ceil_div(kHid * kIn + kHid, tb), tb, 0, st>>>(batch, kHid, kIn, dz1, X, grad + oW1,
                                                                     grad + ob1);
    GKO_CUDA(cudaFreeAsync(buf, st));
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

int gko_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t count, int t, float lr, float beta1,
                 float beta2, float eps, void* stream)
{
    if (!params || !grad || !m || !v || count < 0 || t < 1) return fail(GKO_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float c1 = 1.0f - powf(beta1, static_cast<float>(t));
    const float c2 = 1.0f - powf(beta2, static_cast<float>(t));
    if (count > 0)
        adam_kernel<<<std::min(ceil_div(count, 256), 152 * 4), 256, 0, st>>>(params, grad, m, v, count, lr, beta1,
                                                                           beta2, eps, c1, c2);
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

int gko_selector_load(const float* params_host, int n_out, const double* feat_mean, const double* feat_scale,
                      const int* fmts, const int* cfgs)
{
    if (!params_host || !feat_mean || !feat_scale || !fmts || !cfgs) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    if (n_out < 1 || n_out > kMaxOut) return fail(GKO_ERR_INVALID_ARG, "bad n_out");
    std::lock_guard<std::mutex> lk(g_sel_mu);
    const int64_t cnt = mlp_count(n_out);
    g_sel.params.assign(params_host, params_host + cnt);
    for (int i = 0; i < 12; ++i) {
        g_sel.mean[i] = feat_mean[i];
        g_sel.scale[i] = feat_scale[i] != 0.0 ? feat_scale[i] : 1.0;
    }
    g_sel.fmts.assign(fmts, fmts + n_out);
    g_sel.cfgs.assign(cfgs, cfgs + n_out);
    g_sel.n_out = n_out;
    if (g_sel.d_params) cudaFree(g_sel.d_params);
    g_sel.d_params = nullptr;
    GKO_TRY(dev_alloc(&g_sel.d_params, cnt));
    GKO_CUDA(cudaMemcpy(g_sel.d_params, g_sel.params.data(), cnt * sizeof(float), cudaMemcpyHostToDevice));
    GKO_CUDA(cudaGetDevice(&g_sel.device));
    g_sel.loaded = true;
    ++g_sel_gen;
    return GKO_OK;
}

int gko_selector_clear(void)
{
    std::lock_guard<std::mutex> lk(g_sel_mu);
    if (g_sel.d_params) cudaFree(g_sel.d_params);
    g_sel.d_params = nullptr;
    g_sel.loaded = false;
    ++g_sel_gen;
    return GKO_OK;
}

int gko_select_format(gko_matrix* A, int* fmt, int* config, void* stream)
{
    if (!A || !fmt || !config) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(g_sel_mu);
    *fmt = GKO_FMT_CSR;
    *config = GKO_CFG_DEFAULT;
    if (!g_sel.loaded || A->n_rows == 0) return GKO_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!A->feats_valid) {
        GKO_TRY(features_compute(A, A->feats, st));
        A->feats_valid = true;
    }
    float xin[12];
    for (int i = 0; i < 12; ++i) xin[i] = static_cast<float>((A->feats[i] - g_sel.mean[i]) / g_sel.scale[i]);
    float* d = nullptr;
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d), (12 + kMaxOut) * sizeof(float), st));
    GKO_CUDA(cudaMemcpyAsync(d, xin, sizeof(xin), cudaMemcpyHostToDevice, st));
    mlp_forward_kernel<<<1, kHid, 0, st>>>(g_sel.d_params, g_sel.n_out, d, 1, d + 12, nullptr, nullptr, nullptr,
                                          nullptr);
    float out[kMaxOut];
    GKO_CUDA(cudaMemcpyAsync(out, d + 12, g_sel.n_out * sizeof(float), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaFreeAsync(d, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    // argmin over the candidates this handle can run: its format is
    // materialised and the kernel configuration applies to the matrix
    int best = -1;
    for (int i = 0; i < g_sel.n_out; ++i) {
        const int f = g_sel.fmts[i], c = g_sel.cfgs[i];
        if (f < 0 || f > GKO_FMT_HYBRID || !A->has[f]) continue;
        if ((c == GKO_CFG_CSR_ROWBLOCK || c == GKO_CFG_CSR_BANDED) && rowblock_rows(A) == 0) continue;
        if (c == GKO_CFG_CSR_BANDED && (A->csr.band < 0 || A->csr.band > 1024)) continue;
        if (best < 0 || out[i] < out[best]) best = i;
    }
    if (best >= 0) {
        *fmt = g_sel.fmts[best];
        *config = g_sel.cfgs[best];
    }
    return GKO_OK;
}

}  // extern "C"
