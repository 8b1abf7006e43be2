// Shared-memory tile pass: the whole tile of every state lives in shared
// memory and each fused operation traverses it once.  Used for circuits
// narrower than the register-resident kernel's 12-qubit tile.
#include "sweep_types.h"
#include "nqs_internal.h"

namespace nqs {

template <int S>
struct PassShared {
    unsigned long long hi_off[1 << (kMaxTileQ - 5)];
    double acc[kMaxEvents][S][kWarps][8];
};

template <int S>
__global__ void __launch_bounds__(kThreads) tile_pass_kernel(const PassArgs P) {
    extern __shared__ __align__(16) float2 tile[];   // S * 2^k
    __shared__ PassShared<S> sh;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int k = P.k, c = P.c;
    const int T = 1 << k;
    const int cmask = (1 << c) - 1;
    const int nhi = 1 << (k - c);

    for (int h = tid; h < nhi; h += kThreads) {
        unsigned long long off = 0;
        for (int j = 0; j < k - c; ++j)
            if ((h >> j) & 1) off |= 1ull << P.local[c + j];
        sh.hi_off[h] = off;
    }
    for (int i = tid; i < kMaxEvents * S * kWarps * 8; i += kThreads) (&sh.acc[0][0][0][0])[i] = 0.0;
    __syncthreads();

    for (long long t = blockIdx.x; t < P.n_tiles; t += gridDim.x) {
        unsigned long long base = 0;
        for (int j = 0; j < P.n - k; ++j)
            if ((t >> j) & 1) base |= 1ull << P.nonlocal[j];
        auto gaddr = [&](int j) -> unsigned long long { return base | sh.hi_off[j >> c] | (unsigned long long)(j & cmask); };

        // load (2 amplitudes per 16-byte vector; j even so the address is aligned)
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float4* src = reinterpret_cast<const float4*>(P.in[s]);
            for (int f = tid; f < (T >> 1); f += kThreads) {
                int j = f << 1;
                float4 v = __ldcs(src + (gaddr(j) >> 1));
                tile[s * T + j] = make_float2(v.x, v.y);
                tile[s * T + j + 1] = make_float2(v.z, v.w);
            }
        }
        __syncthreads();

        for (int o = 0; o < P.n_ops; ++o) {
            const DevOp op = P.ops[o];
            if (op.type == OP_G1) {
                const float2 m0 = P.mats[op.mat], m1 = P.mats[op.mat + 1];
                const float2 m2 = P.mats[op.mat + 2], m3 = P.mats[op.mat + 3];
                const int bit = 1 << op.a;
                for (int p = tid; p < (T >> 1); p += kThreads) {
                    int j0 = insert0(p, op.a), j1 = j0 | bit;
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        float2 x0 = tile[s * T + j0], x1 = tile[s * T + j1];
                        tile[s * T + j0] = cfma(m0, x0, cmul(m1, x1));
                        tile[s * T + j1] = cfma(m2, x0, cmul(m3, x1));
                    }
                }
            } else if (op.type == OP_G2) {
                float2 m[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) m[e] = P.mats[op.mat + e];
                const int lo = min(op.a, op.b), hi = max(op.a, op.b);
                const int ba = 1 << op.a, bb = 1 << op.b;
                for (int p = tid; p < (T >> 2); p += kThreads) {
                    int j = insert0(insert0(p, lo), hi);
                    int idx[4] = {j, j | bb, j | ba, j | ba | bb};
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        float2 x[4];
#pragma unroll
                        for (int r = 0; r < 4; ++r) x[r] = tile[s * T + idx[r]];
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            float2 y = cmul(m[4 * r], x[0]);
                            y = cfma(m[4 * r + 1], x[1], y);
                            y = cfma(m[4 * r + 2], x[2], y);
                            y = cfma(m[4 * r + 3], x[3], y);
                            tile[s * T + idx[r]] = y;
                        }
                    }
                }
            } else if (op.type == OP_D1) {
                const float2 d0 = P.mats[op.mat], d1 = P.mats[op.mat + 3];
                if (op.a >= 0) {
                    for (int j = tid; j < T; j += kThreads) {
                        float2 d = ((j >> op.a) & 1) ? d1 : d0;
#pragma unroll
                        for (int s = 0; s < S; ++s) tile[s * T + j] = cmul(d, tile[s * T + j]);
                    }
                } else {
                    float2 d = ((base >> op.qa) & 1) ? d1 : d0;
                    for (int j = tid; j < T; j += kThreads)
#pragma unroll
                        for (int s = 0; s < S; ++s) tile[s * T + j] = cmul(d, tile[s * T + j]);
                }
            } else if (op.type == OP_D2) {
                float2 d[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) d[e] = P.mats[op.mat + 5 * e];
                const int fa = (op.a < 0) ? (int)((base >> op.qa) & 1) : -1;
                const int fb = (op.b < 0) ? (int)((base >> op.qb) & 1) : -1;
                for (int j = tid; j < T; j += kThreads) {
                    int b0 = fa >= 0 ? fa : ((j >> op.a) & 1);
                    int b1 = fb >= 0 ? fb : ((j >> op.b) & 1);
                    float2 f = d[2 * b0 + b1];
#pragma unroll
                    for (int s = 0; s < S; ++s) tile[s * T + j] = cmul(f, tile[s * T + j]);
                }
            } else if (op.type == OP_SITE) {
                const int fl = op.flags & 0xff;
                const int ev = (op.flags >> 8) & 0xff;
                const int nspawn = (op.flags >> 16) & 0xff;
                const int bit = 1 << op.a;
                const float2 k0 = P.mats[op.mat], k1 = P.mats[op.mat + 1];
                const float2 k2 = P.mats[op.mat + 2], k3 = P.mats[op.mat + 3];
                const float2* phi = (fl & FL_REDUCE) ? P.ckpt[op.site] : nullptr;
                float2* save = (fl & FL_SAVE) ? P.ckpt[op.site] : (fl & FL_SAVE_FWD) ? P.ckpt_fwd[op.site] : nullptr;
                float r[S][8];
#pragma unroll
                for (int s = 0; s < S; ++s)
#pragma unroll
                    for (int e = 0; e < 8; ++e) r[s][e] = 0.f;
                for (int p = tid; p < (T >> 1); p += kThreads) {
                    int j0 = insert0(p, op.a), j1 = j0 | bit;
                    unsigned long long g0 = gaddr(j0), g1 = gaddr(j1);
                    float2 f0, f1;
                    if (fl & FL_REDUCE) {
                        f0 = __ldcs(phi + g0);
                        f1 = __ldcs(phi + g1);
                    }
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        float2 x0 = tile[s * T + j0], x1 = tile[s * T + j1];
                        // phi_s excludes the site's own factor: save before applying K_0^dagger
                        if ((fl & (FL_SAVE | FL_SAVE_FWD)) && s == 0) {
                            __stcs(save + g0, x0);
                            __stcs(save + g1, x1);
                        }
                        if (fl & FL_REDUCE) {
                            // R[a][b] += conj(phi_a) * x_b
                            r[s][0] += f0.x * x0.x + f0.y * x0.y;  r[s][1] += f0.x * x0.y - f0.y * x0.x;
                            r[s][2] += f0.x * x1.x + f0.y * x1.y;  r[s][3] += f0.x * x1.y - f0.y * x1.x;
                            r[s][4] += f1.x * x0.x + f1.y * x0.y;  r[s][5] += f1.x * x0.y - f1.y * x0.x;
                            r[s][6] += f1.x * x1.x + f1.y * x1.y;  r[s][7] += f1.x * x1.y - f1.y * x1.x;
                        }
                        if (fl & FL_SPAWN) {
                            for (int i = 0; i < nspawn; ++i) {
                                const float2* K = P.mats + op.mat + 4 * (i + 1);
                                float2* dst = P.spawn[s * 3 + i];
                                __stcs(dst + g0, cfma(K[0], x0, cmul(K[1], x1)));
                                __stcs(dst + g1, cfma(K[2], x0, cmul(K[3], x1)));
                            }
                        }
                        if (fl & FL_APPLY) {
                            float2 y0, y1;
                            if (fl & FL_KDIAG) {
                                y0 = cmul(k0, x0);
                                y1 = cmul(k3, x1);
                            } else {
                                y0 = cfma(k0, x0, cmul(k1, x1));
                                y1 = cfma(k2, x0, cmul(k3, x1));
                            }
                            tile[s * T + j0] = y0;
                            tile[s * T + j1] = y1;
                        }
                    }
                }
                if (fl & FL_REDUCE) {
#pragma unroll
                    for (int s = 0; s < S; ++s) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            float v = r[s][e];
#pragma unroll
                            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                            if (lane == 0) sh.acc[ev][s][warp][e] += (double)v;
                        }
                    }
                }
            }
            __syncthreads();
        }

#pragma unroll
        for (int s = 0; s < S; ++s) {
            float4* dst = reinterpret_cast<float4*>(P.out[s]);
            for (int f = tid; f < (T >> 1); f += kThreads) {
                int j = f << 1;
                float2 a = tile[s * T + j], b = tile[s * T + j + 1];
                __stcs(dst + (gaddr(j) >> 1), make_float4(a.x, a.y, b.x, b.y));
            }
        }
        __syncthreads();
    }

    for (int i = tid; i < P.n_events * S * 8; i += kThreads) {
        int e = i & 7, s = (i >> 3) % S, ev = (i >> 3) / S;
        double v = 0.0;
        for (int w = 0; w < kWarps; ++w) v += sh.acc[ev][s][w][e];
        P.partials[((size_t)(ev * S + s) * gridDim.x + blockIdx.x) * 8 + e] = v;
    }
}


namespace {
template <int S>
void set_attr() {
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(tile_pass_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             S * (1 << kMaxTileQ) * (int)sizeof(float2));
        done = true;
    }
}
}  // namespace

int tile_pass_blocks_per_sm(int S, size_t smem) {
    int nb = 0;
    if (S == 1) {
        set_attr<1>();
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tile_pass_kernel<1>, kThreads, smem);
    } else if (S == 2) {
        set_attr<2>();
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tile_pass_kernel<2>, kThreads, smem);
    } else {
        set_attr<3>();
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tile_pass_kernel<3>, kThreads, smem);
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_tile_pass(int S, int grid, size_t smem, const PassArgs& P, cudaStream_t st) {
    if (S == 1) tile_pass_kernel<1><<<grid, kThreads, smem, st>>>(P);
    else if (S == 2) tile_pass_kernel<2><<<grid, kThreads, smem, st>>>(P);
    else tile_pass_kernel<3><<<grid, kThreads, smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace nqs
