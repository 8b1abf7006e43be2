// Proposal network of the importance-sampled level-l estimate: a small MLP
// (ReLU hidden layers, linear scalar output) whose weights are used in bf16
// with fp32 accumulation, trained on the GPU by the kernels below (forward,
// backward, Adam on fp32 master weights, mean-squared-error loss).
//
// Parameters, flattened in this order: for each layer l, W_l (out x in,
// row-major) then b_l (out).  The bf16 copy of every W_l is what the forward
// and backward passes read; gradients flow to the fp32 masters.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "nqs_internal.h"

namespace nqs {

namespace {

constexpr int kTile = 32;

// C[M x N] = op(A)[M x K] * op(B)[K x N] (+ bias[N]) (+ ReLU), fp32 accumulation.
//   A: fp32, row-major; transA -> A stored [K x M]
//   B: bf16 (weights) or fp32, row-major; transB -> B stored [N x K]
//   accumulate: C += result (weight gradients)
template <typename TB, bool TA_T, bool TB_T>
__global__ void gemm_kernel(int M, int N, int K, const float* __restrict__ A, const TB* __restrict__ B,
                            float* __restrict__ C, const float* __restrict__ bias, int relu, int accumulate) {
    __shared__ float As[kTile][kTile + 1];
    __shared__ float Bs[kTile][kTile + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8 threads, each 4 rows
    const int row0 = blockIdx.y * kTile, col = blockIdx.x * kTile + tx;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += kTile) {
        for (int r = ty; r < kTile; r += 8) {
            const int m = row0 + r, k = k0 + tx;
            float a = 0.f;
            if (m < M && k < K) a = TA_T ? A[(size_t)k * M + m] : A[(size_t)m * K + k];
            As[r][tx] = a;
            const int kk = k0 + r, n = blockIdx.x * kTile + tx;
            float b = 0.f;
            if (kk < K && n < N) {
                if constexpr (TB_T) b = (float)B[(size_t)n * K + kk];
                else b = (float)B[(size_t)kk * N + n];
            }
            Bs[r][tx] = b;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kTile; ++k) {
            const float b = Bs[k][tx];
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i] = fmaf(As[ty + 8 * i][k], b, acc[i]);
        }
        __syncthreads();
    }
    if (col >= N) return;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = row0 + ty + 8 * i;
        if (m >= M) continue;
        float v = acc[i];
        if (bias) v += bias[col];
        if (relu) v = fmaxf(v, 0.f);
        float* dst = C + (size_t)m * N + col;
        *dst = accumulate ? *dst + v : v;
    }
}

template <typename TB, bool TA_T, bool TB_T>
void gemm(int M, int N, int K, const float* A, const TB* B, float* C, const float* bias, bool relu, bool accumulate,
          cudaStream_t st) {
    dim3 block(kTile, 8), grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
    gemm_kernel<TB, TA_T, TB_T><<<grid, block, 0, st>>>(M, N, K, A, B, C, bias, relu ? 1 : 0, accumulate ? 1 : 0);
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) wb[i] = __float2bfloat16(w[i]);
}

// dZ = dY * (Y > 0) in place (Y is the post-ReLU activation)
__global__ void relu_back_kernel(float* __restrict__ d, const float* __restrict__ y, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (y[i] <= 0.f) d[i] = 0.f;
}

// column sums (bias gradients): db[n] += sum_m dY[m][n]
__global__ void colsum_kernel(const float* __restrict__ d, float* __restrict__ db, int M, int N) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += d[(size_t)m * N + n];
    db[n] += s;
}

// MSE: loss partials and dY = 2 (pred - y) / B
__global__ void mse_kernel(const float* __restrict__ pred, const float* __restrict__ y, float* __restrict__ d, int B,
                           double* __restrict__ loss) {
    __shared__ double part[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        const float e = pred[i] - y[i];
        d[i] = 2.f * e / (float)B;
        s += (double)e * e;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0] / B;
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// rows of (X, y) picked by a counter-based generator (SplitMix64 of seed + step*B + i)
__device__ __forceinline__ unsigned long long splitmix(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void gather_batch_kernel(const float* __restrict__ X, const float* __restrict__ y, int n, int in,
                                    float* __restrict__ Xb, float* __restrict__ yb, int B, unsigned long long seed,
                                    long long step) {
    const int i = blockIdx.x;
    if (i >= B) return;
    const unsigned long long r = splitmix(seed + (unsigned long long)step * B + i);
    const int src = (int)(r % (unsigned long long)n);
    for (int k = threadIdx.x; k < in; k += blockDim.x) Xb[(size_t)i * in + k] = X[(size_t)src * in + k];
    if (threadIdx.x == 0) yb[i] = y[src];
}

}  // namespace

struct Mlp {
    std::vector<int> dims;        // in, hidden..., 1
    size_t n_params = 0;
    std::vector<size_t> w_off, b_off;
    float* w = nullptr;           // fp32 masters
    __nv_bfloat16* wb = nullptr;  // bf16 copies of the weight matrices (same offsets as w)
    float* g = nullptr;           // gradients
    float* m = nullptr;
    float* v = nullptr;           // Adam moments
    long long adam_t = 0;
    // activations for a batch
    int cap_B = 0;
    std::vector<float*> acts;     // acts[0] = input copy, acts[l] = output of layer l
    std::vector<float*> dacts;
    double* loss_dev = nullptr;
    float* Xb = nullptr;
    float* yb = nullptr;
    std::vector<void*> blocks;
    std::vector<size_t> block_bytes;
};

namespace {

void* mlp_alloc(Mlp& M, size_t bytes) {
    void* p = dev_alloc(bytes, nullptr);
    if (p) {
        M.blocks.push_back(p);
        M.block_bytes.push_back(bytes);
    }
    return p;
}

int ensure_batch(Mlp& M, int B) {
    if (B <= M.cap_B) return NQS_OK;
    // activation buffers are re-allocated for the larger batch
    for (size_t i = 0; i < M.acts.size(); ++i) {
        dev_free(M.acts[i], 0, nullptr);
        dev_free(M.dacts[i], 0, nullptr);
    }
    dev_free(M.Xb, 0, nullptr);
    dev_free(M.yb, 0, nullptr);
    const int L = (int)M.dims.size();
    M.acts.assign(L, nullptr);
    M.dacts.assign(L, nullptr);
    for (int l = 0; l < L; ++l) {
        M.acts[l] = (float*)dev_alloc((size_t)B * M.dims[l] * sizeof(float), nullptr);
        M.dacts[l] = (float*)dev_alloc((size_t)B * M.dims[l] * sizeof(float), nullptr);
        if (!M.acts[l] || !M.dacts[l]) return NQS_ERR_NOMEM;
    }
    M.Xb = (float*)dev_alloc((size_t)B * M.dims[0] * sizeof(float), nullptr);
    M.yb = (float*)dev_alloc((size_t)B * sizeof(float), nullptr);
    if (!M.Xb || !M.yb) return NQS_ERR_NOMEM;
    M.cap_B = B;
    return NQS_OK;
}

int forward(Mlp& M, const float* X, int B, cudaStream_t st) {
    const int L = (int)M.dims.size() - 1;
    const float* in = X;
    for (int l = 0; l < L; ++l) {
        const int K = M.dims[l], N = M.dims[l + 1];
        gemm<__nv_bfloat16, false, true>(B, N, K, in, M.wb + M.w_off[l], M.acts[l + 1], M.w + M.b_off[l], l + 1 < L,
                                         false, st);
        in = M.acts[l + 1];
    }
    return cudaGetLastError() == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
}

// gradients of the mean-squared error of the batch (X, y) into M.g
int backward(Mlp& M, const float* X, const float* y, int B, cudaStream_t st) {
    const int L = (int)M.dims.size() - 1;
    cudaMemsetAsync(M.g, 0, M.n_params * sizeof(float), st);
    mse_kernel<<<1, 256, 0, st>>>(M.acts[L], y, M.dacts[L], B, M.loss_dev);
    for (int l = L - 1; l >= 0; --l) {
        const int K = M.dims[l], N = M.dims[l + 1];
        float* dY = M.dacts[l + 1];
        if (l + 1 < L) relu_back_kernel<<<256, 256, 0, st>>>(dY, M.acts[l + 1], B * N);
        const float* Xin = (l == 0) ? X : M.acts[l];
        // dW[N x K] = dY^T [N x B] * X [B x K]
        gemm<float, true, false>(N, K, B, dY, Xin, M.g + M.w_off[l], nullptr, false, true, st);
        colsum_kernel<<<(N + 255) / 256, 256, 0, st>>>(dY, M.g + M.b_off[l], B, N);
        // dX[B x K] = dY [B x N] * W [N x K]
        if (l > 0) gemm<__nv_bfloat16, false, false>(B, K, N, dY, M.wb + M.w_off[l], M.dacts[l], nullptr, false, false, st);
    }
    return cudaGetLastError() == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
}

void refresh_bf16(Mlp& M, cudaStream_t st) {
    to_bf16_kernel<<<256, 256, 0, st>>>(M.w, M.wb, (int)M.n_params);
}

}  // namespace

void mlp_destroy(Mlp* M) {
    if (!M) return;
    cudaDeviceSynchronize();
    for (size_t i = 0; i < M->blocks.size(); ++i) dev_free(M->blocks[i], M->block_bytes[i], nullptr);
    for (size_t i = 0; i < M->acts.size(); ++i) {
        dev_free(M->acts[i], 0, nullptr);
        dev_free(M->dacts[i], 0, nullptr);
    }
    dev_free(M->Xb, 0, nullptr);
    dev_free(M->yb, 0, nullptr);
    delete M;
}

int mlp_create(int n_in, int hidden, int layers, unsigned long long seed, Mlp** out) {
    if (n_in < 1 || n_in > 4096 || hidden < 1 || hidden > 4096 || layers < 1 || layers > 8) return NQS_ERR_ARG;
    Mlp* M = new Mlp();
    M->dims.push_back(n_in);
    for (int l = 0; l < layers; ++l) M->dims.push_back(hidden);
    M->dims.push_back(1);
    size_t off = 0;
    for (size_t l = 0; l + 1 < M->dims.size(); ++l) {
        M->w_off.push_back(off);
        off += (size_t)M->dims[l] * M->dims[l + 1];
        M->b_off.push_back(off);
        off += M->dims[l + 1];
    }
    M->n_params = off;
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, from SplitMix64
    std::vector<float> h(off, 0.f);
    unsigned long long state = seed;
    auto next = [&]() {
        state += 0x9E3779B97F4A7C15ull;
        unsigned long long z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    for (size_t l = 0; l + 1 < M->dims.size(); ++l) {
        const double a = 1.0 / std::sqrt((double)M->dims[l]);
        for (size_t i = 0; i < (size_t)M->dims[l] * M->dims[l + 1]; ++i) {
            const double u = (next() >> 11) * (1.0 / 9007199254740992.0);
            h[M->w_off[l] + i] = (float)((2.0 * u - 1.0) * a);
        }
    }
    M->w = (float*)mlp_alloc(*M, off * sizeof(float));
    M->wb = (__nv_bfloat16*)mlp_alloc(*M, off * sizeof(__nv_bfloat16));
    M->g = (float*)mlp_alloc(*M, off * sizeof(float));
    M->m = (float*)mlp_alloc(*M, off * sizeof(float));
    M->v = (float*)mlp_alloc(*M, off * sizeof(float));
    M->loss_dev = (double*)mlp_alloc(*M, sizeof(double));
    if (!M->w || !M->wb || !M->g || !M->m || !M->v || !M->loss_dev) {
        mlp_destroy(M);
        return NQS_ERR_NOMEM;
    }
    if (cudaMemcpy(M->w, h.data(), off * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(M->m, 0, off * sizeof(float)) != cudaSuccess ||
        cudaMemset(M->v, 0, off * sizeof(float)) != cudaSuccess) {
        mlp_destroy(M);
        return NQS_ERR_CUDA;
    }
    refresh_bf16(*M, nullptr);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        mlp_destroy(M);
        return NQS_ERR_CUDA;
    }
    *out = M;
    return NQS_OK;
}

size_t mlp_n_params(const Mlp* M) { return M->n_params; }
int mlp_n_in(const Mlp* M) { return M->dims[0]; }

int mlp_get_params(Mlp* M, float* host, size_t cap) {
    if (cap < M->n_params) return NQS_ERR_ARG;
    return cudaMemcpy(host, M->w, M->n_params * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? NQS_OK
                                                                                                   : NQS_ERR_CUDA;
}

int mlp_set_params(Mlp* M, const float* host, size_t count) {
    if (count != M->n_params) return NQS_ERR_ARG;
    if (cudaMemcpy(M->w, host, count * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return NQS_ERR_CUDA;
    refresh_bf16(*M, nullptr);
    return cudaDeviceSynchronize() == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
}

int mlp_forward(Mlp* M, const float* X, int B, float* y, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_batch(*M, B);
    if (rc) return rc;
    rc = forward(*M, X, B, st);
    if (rc) return rc;
    return cudaMemcpyAsync(y, M->acts.back(), (size_t)B * sizeof(float), cudaMemcpyDefault, st) == cudaSuccess
               ? NQS_OK
               : NQS_ERR_CUDA;
}

int mlp_loss_grad(Mlp* M, const float* X, const float* y, int B, double* loss, float* grad_host, size_t cap,
                  void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (cap < M->n_params) return NQS_ERR_ARG;
    int rc = ensure_batch(*M, B);
    if (rc) return rc;
    rc = forward(*M, X, B, st);
    if (rc) return rc;
    rc = backward(*M, X, y, B, st);
    if (rc) return rc;
    if (cudaMemcpyAsync(loss, M->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return NQS_ERR_CUDA;
    if (cudaMemcpyAsync(grad_host, M->g, M->n_params * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return NQS_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
}

int mlp_train(Mlp* M, const float* X, const float* y, int n, int batch, int steps, float lr, unsigned long long seed,
              double* final_loss, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (n < 1 || batch < 1 || steps < 0) return NQS_ERR_ARG;
    int rc = ensure_batch(*M, batch);
    if (rc) return rc;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int s = 0; s < steps; ++s) {
        gather_batch_kernel<<<batch, 64, 0, st>>>(X, y, n, M->dims[0], M->Xb, M->yb, batch, seed, M->adam_t);
        rc = forward(*M, M->Xb, batch, st);
        if (rc) return rc;
        rc = backward(*M, M->Xb, M->yb, batch, st);
        if (rc) return rc;
        ++M->adam_t;
        const float c1 = 1.f - std::pow(b1, (float)M->adam_t), c2 = 1.f - std::pow(b2, (float)M->adam_t);
        adam_kernel<<<256, 256, 0, st>>>(M->w, M->g, M->m, M->v, (int)M->n_params, lr, b1, b2, eps, c1, c2);
        refresh_bf16(*M, st);
    }
    if (final_loss) {
        if (cudaMemcpyAsync(final_loss, M->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return NQS_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return NQS_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
}

}  // namespace nqs
