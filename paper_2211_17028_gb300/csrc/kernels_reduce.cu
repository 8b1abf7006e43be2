// Reductions and bookkeeping kernels: the standalone reduced-matrix kernel,
// the fixed-order finishers that turn per-block partial sums into term
// values, the Neumaier-compensated per-level sums, and the basis-state fill.
#include "sweep_types.h"
#include "nqs_internal.h"

namespace nqs {

// Standalone reduced-matrix kernel (nqs_reduced_matrix and the N = 0 path):
// grid-stride over amplitude pairs of qubit q.
__global__ void __launch_bounds__(kThreads) reduce2x2_kernel(const float2* __restrict__ phi,
                                                             const float2* __restrict__ chi, int n, int q,
                                                             double* __restrict__ partials) {
    __shared__ double acc[kWarps][8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < kWarps * 8) (&acc[0][0])[tid] = 0.0;
    __syncthreads();
    const long long npairs = 1ll << (n - 1);
    const long long bit = 1ll << q;
    const long long stride = (long long)gridDim.x * kThreads;
    long long p = (long long)blockIdx.x * kThreads + tid;
    while (__any_sync(0xffffffffu, p < npairs)) {
        float r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int it = 0; it < 16 && p < npairs; ++it, p += stride) {
            long long lo = p & (bit - 1);
            long long i0 = ((p - lo) << 1) | lo, i1 = i0 | bit;
            float2 f0 = __ldcs(phi + i0), f1 = __ldcs(phi + i1);
            float2 x0 = __ldcs(chi + i0), x1 = __ldcs(chi + i1);
            r[0] += f0.x * x0.x + f0.y * x0.y;  r[1] += f0.x * x0.y - f0.y * x0.x;
            r[2] += f0.x * x1.x + f0.y * x1.y;  r[3] += f0.x * x1.y - f0.y * x1.x;
            r[4] += f1.x * x0.x + f1.y * x0.y;  r[5] += f1.x * x0.y - f1.y * x0.x;
            r[6] += f1.x * x1.x + f1.y * x1.y;  r[7] += f1.x * x1.y - f1.y * x1.x;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float v = r[e];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) acc[warp][e] += (double)v;
        }
    }
    __syncthreads();
    if (tid < 8) {
        double v = 0.0;
        for (int w = 0; w < kWarps; ++w) v += acc[w][tid];
        partials[(size_t)blockIdx.x * 8 + tid] = v;
    }
}

// Sum per-block partials of one reduction slot in a fixed order: thread t
// takes blocks t, t+256, ...; then a fixed tree.
__device__ void sum_partials(const double* part, int grid, double* R, double* scratch) {
    const int tid = threadIdx.x;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = tid; b < grid; b += kThreads)
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] += part[(size_t)b * 8 + e];
#pragma unroll
    for (int e = 0; e < 8; ++e) scratch[e * kThreads + tid] = v[e];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (tid < w)
#pragma unroll
            for (int e = 0; e < 8; ++e) scratch[e * kThreads + tid] += scratch[e * kThreads + tid + w];
        __syncthreads();
    }
    if (tid < 8) R[tid] = scratch[tid * kThreads];
    __syncthreads();
}

// One block per reduction slot (event, state): R from the partials, then
// X = |sum_ab K[a][b] R[a][b]|^2 for each factor of the slot.
__device__ __forceinline__ void finish_slot(const double* __restrict__ partials, int grid, int slot,
                                            const FinishDesc* __restrict__ desc, const double* __restrict__ kmats,
                                            double* __restrict__ term_vals) {
    __shared__ double scratch[8 * kThreads];
    __shared__ double R[8];
    sum_partials(partials + (size_t)slot * grid * 8, grid, R, scratch);
    if (threadIdx.x < 4) {
        FinishDesc d = desc[slot * 4 + threadIdx.x];
        if (d.rank >= 0) {
            const double* K = kmats + d.kmat;
            double re = 0, im = 0;
            for (int e = 0; e < 4; ++e) {
                double kr = K[2 * e], ki = K[2 * e + 1], rr = R[2 * e], ri = R[2 * e + 1];
                re += kr * rr - ki * ri;
                im += kr * ri + ki * rr;
            }
            term_vals[d.rank] = re * re + im * im;
        }
    }
}

__global__ void __launch_bounds__(kThreads) finish_kernel(const double* __restrict__ partials, int grid,
                                                          const FinishDesc* __restrict__ desc,
                                                          const double* __restrict__ kmats,
                                                          double* __restrict__ term_vals) {
    finish_slot(partials, grid, blockIdx.x, desc, kmats, term_vals);
}

// finishers of many circuits: unit u owns blocks [blk_begin[u], blk_begin[u+1])
__global__ void __launch_bounds__(kThreads) finish_kernel_batched(const FinishUnit* __restrict__ units,
                                                                  const int* __restrict__ blk_begin, int n_units) {
    int lo = 0, hi = n_units;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (blk_begin[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid;
    }
    const FinishUnit u = units[lo];
    finish_slot(u.partials, u.grid, (int)blockIdx.x - blk_begin[lo], u.desc, u.kmats, u.vals);
}

// One block: fixed-order sum of per-block partials into 8 doubles.
__global__ void __launch_bounds__(kThreads) partials_sum_kernel(const double* __restrict__ part, int grid,
                                                                double* __restrict__ R) {
    __shared__ double scratch[8 * kThreads];
    __shared__ double r[8];
    sum_partials(part, grid, r, scratch);
    if (threadIdx.x < 8) R[threadIdx.x] = r[threadIdx.x];
}

// Neumaier-compensated per-level sums in canonical order, one block.
__device__ __forceinline__ void level_sum_body(const double* __restrict__ vals,
                                                             const long long* __restrict__ level_off, int level,
                                                             nqs_result* __restrict__ res, double bound,
                                                             long long n_terms, const int* __restrict__ err,
                                               nqs_result* __restrict__ copy) {
    __shared__ double s_sum[kThreads], s_comp[kThreads];
    __shared__ double T[NQS_MAX_LEVEL + 1];
    const int tid = threadIdx.x;
    for (int u = 0; u <= level; ++u) {
        long long lo = level_off[u], hi = level_off[u + 1];
        long long len = hi - lo;
        long long chunk = (len + kThreads - 1) / kThreads;
        long long a = lo + chunk * tid, b = min(hi, a + chunk);
        double sum = 0.0, comp = 0.0;
        for (long long i = a; i < b; ++i) {
            double x = vals[i];
            double t = sum + x;
            if (fabs(sum) >= fabs(x)) comp += (sum - t) + x;
            else comp += (x - t) + sum;
            sum = t;
        }
        s_sum[tid] = sum;
        s_comp[tid] = comp;
        __syncthreads();
        if (tid == 0) {
            double S = 0.0, C = 0.0;
            for (int i = 0; i < kThreads; ++i) {
                double x = s_sum[i];
                double t = S + x;
                if (fabs(S) >= fabs(x)) C += (S - t) + x;
                else C += (x - t) + S;
                S = t;
                C += s_comp[i];
            }
            T[u] = S + C;
        }
        __syncthreads();
    }
    if (tid == 0) {
        double S = 0.0, C = 0.0;
        for (int u = 0; u <= NQS_MAX_LEVEL; ++u) {
            double x = (u <= level) ? T[u] : 0.0;
            res->T[u] = x;
            double t = S + x;
            if (fabs(S) >= fabs(x)) C += (S - t) + x;
            else C += (x - t) + S;
            S = t;
        }
        res->F = S + C;
        res->imag_residual = 0.0;
        res->n_terms = (uint64_t)n_terms;
        res->bound = bound;
        res->level = level;
        res->status = (err && *err) ? *err : NQS_OK;
        if (copy) *copy = *res;
    }
}

__global__ void __launch_bounds__(kThreads) level_sum_kernel(const double* __restrict__ vals,
                                                             const long long* __restrict__ level_off, int level,
                                                             nqs_result* __restrict__ res, double bound,
                                                             long long n_terms, const int* __restrict__ err) {
    level_sum_body(vals, level_off, level, res, bound, n_terms, err, nullptr);
}

// per-level sums of many circuits, one block each; results also gathered into one array
__global__ void __launch_bounds__(kThreads) level_sum_kernel_batched(const SumUnit* __restrict__ units) {
    const SumUnit u = units[blockIdx.x];
    level_sum_body(u.vals, u.level_off, u.level, u.res, u.bound, u.n_terms, u.err, u.copy);
}

// basis-state fills of many circuits: blockIdx.y selects the unit
__global__ void basis_fill_kernel_batched(const FillUnit* __restrict__ units) {
    const FillUnit u = units[blockIdx.y];
    long long stride = (long long)gridDim.x * blockDim.x;
    float4* o4 = reinterpret_cast<float4*>(u.dst);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (u.dim >> 1); i += stride) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((unsigned long long)(2 * i) == u.bits) v.x = 1.f;
        if ((unsigned long long)(2 * i + 1) == u.bits) v.z = 1.f;
        o4[i] = v;
    }
}

__global__ void basis_fill_kernel(float2* out, long long dim, unsigned long long bits) {
    long long stride = (long long)gridDim.x * blockDim.x;
    float4* o4 = reinterpret_cast<float4*>(out);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (dim >> 1); i += stride) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((unsigned long long)(2 * i) == bits) v.x = 1.f;
        if ((unsigned long long)(2 * i + 1) == bits) v.z = 1.f;
        o4[i] = v;
    }
}


cudaError_t launch_reduce2x2(const float2* phi, const float2* chi, int n, int q, double* partials, int grid,
                             cudaStream_t st) {
    reduce2x2_kernel<<<grid, kThreads, 0, st>>>(phi, chi, n, q, partials);
    return cudaGetLastError();
}

cudaError_t launch_finish(const double* partials, int grid, const FinishDesc* desc, const double* kmats,
                          double* vals, int n_red, cudaStream_t st) {
    finish_kernel<<<n_red, kThreads, 0, st>>>(partials, grid, desc, kmats, vals);
    return cudaGetLastError();
}

// v <- v / ||v||, the norm from the per-block partials of reduce2x2_kernel(v,
// v, qubit 0): ||v||^2 = Re R00 + Re R11, summed in a fixed order by every
// block.  The noiseless circuit keeps the norm of a basis state, 1; complex64
// gates lose a little of it, and v enters F twice.
__global__ void __launch_bounds__(kThreads) normalize_kernel(float2* __restrict__ v, long long dim,
                                                             const double* __restrict__ part, int grid) {
    __shared__ float scale;
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int g = 0; g < grid; ++g) a += part[(size_t)g * 8] + part[(size_t)g * 8 + 6];
        scale = a > 0.0 ? (float)(1.0 / sqrt(a)) : 1.0f;
    }
    __syncthreads();
    const float f = scale;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride) {
        const float2 x = v[i];
        v[i] = make_float2(x.x * f, x.y * f);
    }
}

cudaError_t launch_normalize(float2* v, long long dim, const double* partials, int red_grid, int grid,
                             cudaStream_t st) {
    normalize_kernel<<<grid, kThreads, 0, st>>>(v, dim, partials, red_grid);
    return cudaGetLastError();
}

// out = x + c y for basis or dense x, y (the superposed states of the
// polarization identity); a basis state is |bits> (kind 0), dense ones are
// read from device memory (kind 1)
__global__ void __launch_bounds__(kThreads) combine_kernel(float2* __restrict__ out, long long dim, int xk,
                                                           unsigned long long xb, const float2* __restrict__ xd,
                                                           int yk, unsigned long long yb,
                                                           const float2* __restrict__ yd, float cre, float cim) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride) {
        const float2 a = xk ? xd[i] : make_float2((unsigned long long)i == xb ? 1.f : 0.f, 0.f);
        const float2 b = yk ? yd[i] : make_float2((unsigned long long)i == yb ? 1.f : 0.f, 0.f);
        out[i] = make_float2(a.x + cre * b.x - cim * b.y, a.y + cre * b.y + cim * b.x);
    }
}

cudaError_t launch_combine(float2* out, long long dim, int xk, unsigned long long xb, const float2* xd, int yk,
                           unsigned long long yb, const float2* yd, float cre, float cim, int grid, cudaStream_t st) {
    combine_kernel<<<grid, kThreads, 0, st>>>(out, dim, xk, xb, xd, yk, yb, yd, cre, cim);
    return cudaGetLastError();
}

cudaError_t launch_partials_sum(const double* part, int grid, double* R, cudaStream_t st) {
    partials_sum_kernel<<<1, kThreads, 0, st>>>(part, grid, R);
    return cudaGetLastError();
}

cudaError_t launch_level_sum(const double* vals, const long long* level_off, int level, nqs_result* res,
                             double bound, long long n_terms, const int* err, cudaStream_t st) {
    level_sum_kernel<<<1, kThreads, 0, st>>>(vals, level_off, level, res, bound, n_terms, err);
    return cudaGetLastError();
}

cudaError_t launch_basis_fill(float2* out, long long dim, unsigned long long bits, int grid, cudaStream_t st) {
    basis_fill_kernel<<<grid, kThreads, 0, st>>>(out, dim, bits);
    return cudaGetLastError();
}

cudaError_t launch_finish_batched(const FinishUnit* units, const int* blk_begin, int n_units, int total_blocks,
                                  cudaStream_t st) {
    finish_kernel_batched<<<total_blocks, kThreads, 0, st>>>(units, blk_begin, n_units);
    return cudaGetLastError();
}

cudaError_t launch_level_sum_batched(const SumUnit* units, int n_units, cudaStream_t st) {
    level_sum_kernel_batched<<<n_units, kThreads, 0, st>>>(units);
    return cudaGetLastError();
}

cudaError_t launch_fill_batched(const FillUnit* units, int n_units, cudaStream_t st) {
    basis_fill_kernel_batched<<<dim3(64, n_units), kThreads, 0, st>>>(units);
    return cudaGetLastError();
}

}  // namespace nqs
