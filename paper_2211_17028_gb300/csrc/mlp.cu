// Proposal network of the importance-sampled level-l estimate: a small MLP
// (ReLU hidden layers, linear scalar output) whose weights are used in bf16
// with fp32 accumulation, trained on the GPU by the kernels below (forward,
// backward, Adam on fp32 master weights, mean-squared-error loss).  The
// matrix products run on the bf16 tensor cores (warp-level mma.sync).
//
// Parameters, flattened in this order: for each layer l, W_l (out x in,
// row-major) then b_l (out).  The bf16 copy of every W_l is what the forward
// and backward passes read; gradients flow to the fp32 masters.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include "nqs_internal.h"

namespace nqs {

namespace {

// C[M x N] = op(A)[M x K] * op(B)[K x N] (+ bias[N]) (+ ReLU), on the bf16
// tensor cores (mma.sync m16n8k16, fp32 accumulation).
//   A: fp32, row-major; transA -> A stored [K x M]
//   B: bf16 (weights) or fp32, row-major; transB -> B stored [N x K]
//   accumulate: C += result (weight gradients)
// Both MMA operands are bf16, so an fp32 operand x enters as two bf16 parts,
// x_hi = bf16(x) and x_lo = bf16(x - x_hi) (x = x_hi + x_lo to about 2^-16 of
// |x|): C = A_hi B + A_lo B for bf16 weights, A_hi B_hi + A_lo B_hi + A_hi B_lo
// when both are fp32 (the lo * lo product is below fp32 resolution).
// Block tile 64 x 64, k-step 16, 4 warps of 32 x 32 (2 x 4 MMAs of 16 x 8).
constexpr int kBM = 64, kBN = 64, kBK = 16, kPad = 8;

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <typename TB, bool TA_T, bool TB_T>
__global__ void __launch_bounds__(128) gemm_kernel(int M, int N, int K, const float* __restrict__ A,
                                                   const TB* __restrict__ B, float* __restrict__ C,
                                                   const float* __restrict__ bias, int relu, int accumulate,
                                                   int kchunk, float* __restrict__ part) {
    constexpr bool kSplitB = !std::is_same<TB, __nv_bfloat16>::value;
    // tiles: A as [m][k], B as [n][k] (k contiguous: one 32-bit word holds the k, k+1 pair)
    __shared__ __nv_bfloat16 Ah[kBM][kBK + kPad], Al[kBM][kBK + kPad];
    __shared__ __nv_bfloat16 Bh[kBN][kBK + kPad], Bl[kBN][kBK + kPad];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;   // warp's 32 x 32 sub-tile
    const int g = lane >> 2, t = lane & 3;                    // fragment row group, thread in group
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    // split K: block z covers [z * kchunk, (z + 1) * kchunk) and writes its
    // partial product to part[z] (summed in a fixed order by splitk_sum_kernel)
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    for (int k0 = kb; k0 < ke; k0 += kBK) {
        for (int e = tid; e < kBM * kBK; e += blockDim.x) {
            const int r = e / kBK, k = e % kBK, m = m0 + r, kk = k0 + k;
            float a = 0.f;
            if (m < M && kk < ke) a = TA_T ? A[(size_t)kk * M + m] : A[(size_t)m * K + kk];
            const __nv_bfloat16 hi = __float2bfloat16(a);
            Ah[r][k] = hi;
            Al[r][k] = __float2bfloat16(a - __bfloat162float(hi));
        }
        for (int e = tid; e < kBN * kBK; e += blockDim.x) {
            const int c = e / kBK, k = e % kBK, n = n0 + c, kk = k0 + k;
            float b = 0.f;
            if (n < N && kk < ke) {
                if constexpr (TB_T) b = (float)B[(size_t)n * K + kk];
                else b = (float)B[(size_t)kk * N + n];
            }
            const __nv_bfloat16 hi = __float2bfloat16(b);
            Bh[c][k] = hi;
            if constexpr (kSplitB) Bl[c][k] = __float2bfloat16(b - __bfloat162float(hi));
        }
        __syncthreads();
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = wm + 16 * i + g;
            ah[i][0] = pack_bf16(Ah[r][2 * t], Ah[r][2 * t + 1]);
            ah[i][1] = pack_bf16(Ah[r + 8][2 * t], Ah[r + 8][2 * t + 1]);
            ah[i][2] = pack_bf16(Ah[r][2 * t + 8], Ah[r][2 * t + 9]);
            ah[i][3] = pack_bf16(Ah[r + 8][2 * t + 8], Ah[r + 8][2 * t + 9]);
            al[i][0] = pack_bf16(Al[r][2 * t], Al[r][2 * t + 1]);
            al[i][1] = pack_bf16(Al[r + 8][2 * t], Al[r + 8][2 * t + 1]);
            al[i][2] = pack_bf16(Al[r][2 * t + 8], Al[r][2 * t + 9]);
            al[i][3] = pack_bf16(Al[r + 8][2 * t + 8], Al[r + 8][2 * t + 9]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = wn + 8 * j + g;
            const uint32_t bh[2] = {pack_bf16(Bh[c][2 * t], Bh[c][2 * t + 1]),
                                    pack_bf16(Bh[c][2 * t + 8], Bh[c][2 * t + 9])};
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                mma_bf16(acc[i][j], ah[i], bh);
                mma_bf16(acc[i][j], al[i], bh);
            }
            if constexpr (kSplitB) {
                const uint32_t bl[2] = {pack_bf16(Bl[c][2 * t], Bl[c][2 * t + 1]),
                                        pack_bf16(Bl[c][2 * t + 8], Bl[c][2 * t + 9])};
#pragma unroll
                for (int i = 0; i < 2; ++i) mma_bf16(acc[i][j], ah[i], bl);
            }
        }
        __syncthreads();
    }
    // accumulator element e of the 16 x 8 tile: row g (+8 for e >= 2), column 2t + (e & 1)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm + 16 * i + g + (e >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * t + (e & 1);
                if (m >= M || n >= N) continue;
                float v = acc[i][j][e];
                if (part) {
                    part[((size_t)blockIdx.z * M + m) * N + n] = v;
                    continue;
                }
                if (bias) v += bias[n];
                if (relu) v = fmaxf(v, 0.f);
                float* dst = C + (size_t)m * N + n;
                *dst = accumulate ? *dst + v : v;
            }
}

// C (+)= sum over z of part[z] (fixed order), for split-K products
__global__ void splitk_sum_kernel(const float* __restrict__ part, int splits, size_t mn, float* __restrict__ C,
                                  int accumulate) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < mn; i += (size_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int z = 0; z < splits; ++z) v += part[(size_t)z * mn + i];
        C[i] = accumulate ? C[i] + v : v;
    }
}

// ksplit > 1 (no bias or ReLU): K is cut into ksplit chunks computed by
// separate blocks into `part` (ksplit * M * N floats) and summed afterwards
template <typename TB, bool TA_T, bool TB_T>
void gemm(int M, int N, int K, const float* A, const TB* B, float* C, const float* bias, bool relu, bool accumulate,
          cudaStream_t st, int ksplit = 1, float* part = nullptr) {
    if (ksplit < 1 || !part || bias || relu) ksplit = 1;
    int kchunk = (K + ksplit - 1) / ksplit;
    kchunk = (kchunk + kBK - 1) / kBK * kBK;
    ksplit = (K + kchunk - 1) / kchunk;
    dim3 block(128), grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, ksplit);
    gemm_kernel<TB, TA_T, TB_T><<<grid, block, 0, st>>>(M, N, K, A, B, C, bias, relu ? 1 : 0, accumulate ? 1 : 0,
                                                         kchunk, ksplit > 1 ? part : nullptr);
    if (ksplit > 1) {
        const size_t mn = (size_t)M * N;
        const int blocks = (int)std::min<size_t>(1024, (mn + 255) / 256);
        splitk_sum_kernel<<<blocks, 256, 0, st>>>(part, ksplit, mn, C, accumulate ? 1 : 0);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) wb[i] = __float2bfloat16(w[i]);
}

// dZ = dY * (Y > 0) in place (Y is the post-ReLU activation)
__global__ void relu_back_kernel(float* __restrict__ d, const float* __restrict__ y, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (y[i] <= 0.f) d[i] = 0.f;
}

// column sums (bias gradients): db[n] += sum_m dY[m][n]; a block of 32 x 8
// threads covers 32 columns, each thread a strided eighth of the rows, then
// the eight partial sums are added in a fixed order
__global__ void colsum_kernel(const float* __restrict__ d, float* __restrict__ db, int M, int N) {
    __shared__ float part[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + tx;
    float s = 0.f;
    if (n < N)
        for (int m = ty; m < M; m += 8) s += d[(size_t)m * N + n];
    part[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && n < N) {
        float t = 0.f;
        for (int r = 0; r < 8; ++r) t += part[r][tx];
        db[n] += t;
    }
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
    int ksplit = 1;               // K splits of the weight-gradient products
    float* part = nullptr;        // their partial products
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
    // weight-gradient products: about 256 blocks of 64 x 64 outputs in all
    size_t wmax = 0, tiles = 1;
    for (size_t l = 0; l + 1 < M.dims.size(); ++l) {
        wmax = std::max(wmax, (size_t)M.dims[l] * M.dims[l + 1]);
        tiles = std::max(tiles, (size_t)((M.dims[l] + 63) / 64) * ((M.dims[l + 1] + 63) / 64));
    }
    M.ksplit = (int)std::max<size_t>(1, std::min<size_t>((size_t)(B + kBK - 1) / kBK, 256 / tiles));
    dev_free(M.part, 0, nullptr);
    M.part = M.ksplit > 1 ? (float*)dev_alloc((size_t)M.ksplit * wmax * sizeof(float), nullptr) : nullptr;
    if (M.ksplit > 1 && !M.part) return NQS_ERR_NOMEM;
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
        // (the batch is the long dimension: split it so the product fills the GPU)
        gemm<float, true, false>(N, K, B, dY, Xin, M.g + M.w_off[l], nullptr, false, true, st, M.ksplit, M.part);
        colsum_kernel<<<(N + 31) / 32, 256, 0, st>>>(dY, M.g + M.b_off[l], B, N);
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
    dev_free(M->part, 0, nullptr);
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
