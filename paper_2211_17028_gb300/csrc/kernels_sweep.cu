// Register-resident tile sweep for sm_103a (tile = 12 qubits = 4096 amplitudes
// per state, 256 threads, 16 amplitudes per thread per state).
//
// The next tile of every state is prefetched with TMA bulk copies
// (cp.async.bulk, 256-byte runs of the 5 contiguous low qubits) into a
// shared-memory staging buffer, completion tracked by an mbarrier, while the
// current tile is processed in registers.  The pass's fused operations are
// grouped into phases; in a phase four of the tile's qubits are "register
// qubits" (the 16 amplitudes a thread holds differ only in them), so every
// dense one- or two-qubit operation of the phase is applied without touching
// shared memory.  Between phases the tile is re-laid out through a second,
// XOR-swizzled shared-memory buffer.  Diagonal operations on any qubit --
// including qubits outside the tile -- are folded into a per-thread factor
// table (one complex factor per register qubit value plus a scalar) and
// applied once, before the next dense operation.  Site operations (checkpoint
// save, reduction against phi_site, spawning K_i x, applying K_0) act on a
// register qubit and read / write HBM directly.
#include "sweep_types.h"
#include "nqs_internal.h"

namespace nqs {

namespace {

constexpr int kT = 1 << kMaxTileQ;   // amplitudes per state tile
constexpr int kChunk = 32;           // contiguous amplitudes per TMA copy (5 low qubits)
constexpr int kChunks = kT / kChunk;
constexpr int kSpinLimit = 1 << 24;  // bounded mbarrier wait (~1-2 s with the back-off)

__device__ __forceinline__ int swz(int j) { return j ^ ((j >> 5) & 31) ^ ((j >> 10) & 3); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (int i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 32) __nanosleep(64);
    }
    return false;
}

// ---- dense operations on register qubits -----------------------------------
template <int I, int S>
__device__ __forceinline__ void g1_reg(float2 (&x)[S][kRegElems], float2 m0, float2 m1, float2 m2, float2 m3) {
#pragma unroll
    for (int r = 0; r < kRegElems; ++r) {
        if (r & (1 << I)) continue;
        const int r1 = r | (1 << I);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            float2 a = x[s][r], b = x[s][r1];
            x[s][r] = cfma(m0, a, cmul(m1, b));
            x[s][r1] = cfma(m2, a, cmul(m3, b));
        }
    }
}

template <int S>
__device__ __forceinline__ void g1_dispatch(int i, float2 (&x)[S][kRegElems], const float2* m) {
    const float2 m0 = m[0], m1 = m[1], m2 = m[2], m3 = m[3];
    switch (i) {
        case 0: g1_reg<0>(x, m0, m1, m2, m3); break;
        case 1: g1_reg<1>(x, m0, m1, m2, m3); break;
        case 2: g1_reg<2>(x, m0, m1, m2, m3); break;
        default: g1_reg<3>(x, m0, m1, m2, m3); break;
    }
}

// 4x4 matrix indexed 2*b(first) + b(second); first on register bit I0
template <int I0, int I1, int S>
__device__ __forceinline__ void g2_reg(float2 (&x)[S][kRegElems], const float2* mg) {
    float2 m[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) m[e] = mg[e];
#pragma unroll
    for (int r = 0; r < kRegElems; ++r) {
        if (r & ((1 << I0) | (1 << I1))) continue;
        const int idx[4] = {r, r | (1 << I1), r | (1 << I0), r | (1 << I0) | (1 << I1)};
#pragma unroll
        for (int s = 0; s < S; ++s) {
            float2 v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = x[s][idx[q]];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 y = cmul(m[4 * q], v[0]);
                y = cfma(m[4 * q + 1], v[1], y);
                y = cfma(m[4 * q + 2], v[2], y);
                y = cfma(m[4 * q + 3], v[3], y);
                x[s][idx[q]] = y;
            }
        }
    }
}

template <int S>
__device__ __forceinline__ void g2_dispatch(int i0, int i1, float2 (&x)[S][kRegElems], const float2* m) {
    switch (i0 * 4 + i1) {
        case 1: g2_reg<0, 1>(x, m); break;
        case 2: g2_reg<0, 2>(x, m); break;
        case 3: g2_reg<0, 3>(x, m); break;
        case 4: g2_reg<1, 0>(x, m); break;
        case 6: g2_reg<1, 2>(x, m); break;
        case 7: g2_reg<1, 3>(x, m); break;
        case 8: g2_reg<2, 0>(x, m); break;
        case 9: g2_reg<2, 1>(x, m); break;
        case 11: g2_reg<2, 3>(x, m); break;
        case 12: g2_reg<3, 0>(x, m); break;
        case 13: g2_reg<3, 1>(x, m); break;
        case 14: g2_reg<3, 2>(x, m); break;
        default: break;
    }
}

// ---- pending diagonal factor ------------------------------------------------
struct Diag {
    float2 sc;
    float2 h[kRegBits][2];
    int mask;
    bool pend;
};

__device__ __forceinline__ void diag_reset(Diag& d) {
    d.sc = make_float2(1.f, 0.f);
#pragma unroll
    for (int i = 0; i < kRegBits; ++i) d.h[i][0] = d.h[i][1] = make_float2(1.f, 0.f);
    d.mask = 0;
    d.pend = false;
}

__device__ __forceinline__ void diag_mul_reg(Diag& d, int i, float2 f0, float2 f1) {
    switch (i) {
        case 0: d.h[0][0] = cmul(d.h[0][0], f0); d.h[0][1] = cmul(d.h[0][1], f1); break;
        case 1: d.h[1][0] = cmul(d.h[1][0], f0); d.h[1][1] = cmul(d.h[1][1], f1); break;
        case 2: d.h[2][0] = cmul(d.h[2][0], f0); d.h[2][1] = cmul(d.h[2][1], f1); break;
        default: d.h[3][0] = cmul(d.h[3][0], f0); d.h[3][1] = cmul(d.h[3][1], f1); break;
    }
    d.mask |= 1 << i;
    d.pend = true;
}

template <int S>
__device__ __forceinline__ void diag_flush(Diag& d, float2 (&x)[S][kRegElems]) {
    if (!d.pend) return;
#pragma unroll
    for (int r = 0; r < kRegElems; ++r) {
        float2 f = d.sc;
#pragma unroll
        for (int i = 0; i < kRegBits; ++i)
            if (d.mask & (1 << i)) f = cmul(f, d.h[i][(r >> i) & 1]);
#pragma unroll
        for (int s = 0; s < S; ++s) x[s][r] = cmul(f, x[s][r]);
    }
    diag_reset(d);
}

// ---- layouts ----------------------------------------------------------------
struct Layout {
    int jT;                          // tile index bits owned by the thread (lanes, warps)
    int jR[kRegBits];                // tile index bit of each register qubit
    unsigned long long gT;           // the same in global index bits
    unsigned long long gR[kRegBits];
};

__device__ __forceinline__ Layout make_layout(const DevPhase& ph, const int* local, int tid) {
    Layout L;
    L.jT = 0;
    L.gT = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i)
        if ((tid >> i) & 1) {
            L.jT |= 1 << ph.L[i];
            L.gT |= 1ull << local[ph.L[i]];
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
        if ((tid >> (5 + i)) & 1) {
            L.jT |= 1 << ph.W[i];
            L.gT |= 1ull << local[ph.W[i]];
        }
#pragma unroll
    for (int i = 0; i < kRegBits; ++i) {
        L.jR[i] = 1 << ph.R[i];
        L.gR[i] = 1ull << local[ph.R[i]];
    }
    return L;
}

__device__ __forceinline__ int jr_of(const Layout& L, int r) {
    int j = 0;
#pragma unroll
    for (int i = 0; i < kRegBits; ++i)
        if (r & (1 << i)) j |= L.jR[i];
    return j;
}

__device__ __forceinline__ unsigned long long gr_of(const Layout& L, int r) {
    unsigned long long g = 0;
#pragma unroll
    for (int i = 0; i < kRegBits; ++i)
        if (r & (1 << i)) g |= L.gR[i];
    return g;
}

// bit of a qubit for this thread: location code from the phase layout
__device__ __forceinline__ int const_bit(int loc, int qubit, int tid, unsigned long long base) {
    return (loc >= LOC_THREAD) ? ((tid >> (loc - LOC_THREAD)) & 1) : (int)((base >> qubit) & 1);
}

// ---- site operation on register qubit I ---------------------------------------
template <int I, int S>
__device__ __forceinline__ void site_reg(const PassArgs& P, const DevOp& op, float2 (&x)[S][kRegElems],
                                         const Layout& L, unsigned long long base, double (*acc)[kWarps][8],
                                         int lane, int warp) {
    const int fl = op.flags & 0xff;
    const int ev = (op.flags >> 8) & 0xff;
    const int nspawn = (op.flags >> 16) & 0xff;
    const float2* km = P.mats + op.mat;
    const float2 k0 = km[0], k1 = km[1], k2 = km[2], k3 = km[3];
    const float2* phi = (fl & FL_REDUCE) ? P.ckpt[op.site] : nullptr;
    float2* save = (fl & FL_SAVE) ? P.ckpt[op.site] : nullptr;
    float rr[S][8];
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
        for (int e = 0; e < 8; ++e) rr[s][e] = 0.f;
#pragma unroll
    for (int r = 0; r < kRegElems; ++r) {
        if (r & (1 << I)) continue;
        const int r1 = r | (1 << I);
        const unsigned long long g0 = base | L.gT | gr_of(L, r);
        const unsigned long long g1 = g0 | L.gR[I];
        float2 f0 = make_float2(0.f, 0.f), f1 = f0;
        if (fl & FL_REDUCE) {
            f0 = __ldcs(phi + g0);
            f1 = __ldcs(phi + g1);
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float2 a = x[s][r], b = x[s][r1];
            if ((fl & FL_SAVE) && s == 0) {
                __stcs(save + g0, a);
                __stcs(save + g1, b);
            }
            if (fl & FL_REDUCE) {
                rr[s][0] += f0.x * a.x + f0.y * a.y;  rr[s][1] += f0.x * a.y - f0.y * a.x;
                rr[s][2] += f0.x * b.x + f0.y * b.y;  rr[s][3] += f0.x * b.y - f0.y * b.x;
                rr[s][4] += f1.x * a.x + f1.y * a.y;  rr[s][5] += f1.x * a.y - f1.y * a.x;
                rr[s][6] += f1.x * b.x + f1.y * b.y;  rr[s][7] += f1.x * b.y - f1.y * b.x;
            }
            if (fl & FL_SPAWN) {
                for (int i = 0; i < nspawn; ++i) {
                    const float2* K = km + 4 * (i + 1);
                    float2* dst = P.spawn[s * 3 + i];
                    __stcs(dst + g0, cfma(K[0], a, cmul(K[1], b)));
                    __stcs(dst + g1, cfma(K[2], a, cmul(K[3], b)));
                }
            }
            if (fl & FL_APPLY) {
                if (fl & FL_KDIAG) {
                    x[s][r] = cmul(k0, a);
                    x[s][r1] = cmul(k3, b);
                } else {
                    x[s][r] = cfma(k0, a, cmul(k1, b));
                    x[s][r1] = cfma(k2, a, cmul(k3, b));
                }
            }
        }
    }
    if (fl & FL_REDUCE) {
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                float v = rr[s][e];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == 0) acc[ev * S + s][warp][e] += (double)v;
            }
    }
}

template <int S>
__device__ __forceinline__ void site_dispatch(int i, const PassArgs& P, const DevOp& op, float2 (&x)[S][kRegElems],
                                              const Layout& L, unsigned long long base, double (*acc)[kWarps][8],
                                              int lane, int warp) {
    switch (i) {
        case 0: site_reg<0>(P, op, x, L, base, acc, lane, warp); break;
        case 1: site_reg<1>(P, op, x, L, base, acc, lane, warp); break;
        case 2: site_reg<2>(P, op, x, L, base, acc, lane, warp); break;
        default: site_reg<3>(P, op, x, L, base, acc, lane, warp); break;
    }
}

template <int S>
__global__ void __launch_bounds__(kThreads, 1) sweep_kernel(const PassArgs P) {
    extern __shared__ __align__(128) unsigned char dyn[];
    float2* pf = reinterpret_cast<float2*>(dyn);                          // [S][kT], TMA destination
    float* tr = reinterpret_cast<float*>(dyn + (size_t)S * kT * sizeof(float2));   // [S][2][kT], swizzled
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned long long hi_off[kChunks];
    __shared__ double acc[kMaxEvents * S][kWarps][8];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int h = tid; h < kChunks; h += kThreads) {
        unsigned long long off = 0;
        for (int j = 0; j < kMaxTileQ - 5; ++j)
            if ((h >> j) & 1) off |= 1ull << P.local[5 + j];
        hi_off[h] = off;
    }
    for (int i = tid; i < kMaxEvents * S * kWarps * 8; i += kThreads) (&acc[0][0][0])[i] = 0.0;
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto tile_base = [&](long long t) {
        unsigned long long b = 0;
        for (int j = 0; j < P.n - kMaxTileQ; ++j)
            if ((t >> j) & 1) b |= 1ull << P.nonlocal[j];
        return b;
    };
    auto prefetch = [&](long long t) {   // called by warp 0
        const unsigned long long b = tile_base(t);
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_expect_tx(&bar, (uint32_t)(S * kT * sizeof(float2)));
        }
        __syncwarp();
        for (int q = lane; q < S * kChunks; q += 32) {
            const int s = q / kChunks, h = q % kChunks;
            bulk_copy_g2s(pf + s * kT + h * kChunk, P.in[s] + (b | hi_off[h]), kChunk * sizeof(float2), &bar);
        }
    };

    long long t = blockIdx.x;
    if (t < P.n_tiles && warp == 0) prefetch(t);
    uint32_t parity = 0;
    bool failed = false;
    float2 x[S][kRegElems];
    Diag dg;
    diag_reset(dg);

    for (; t < P.n_tiles; t += gridDim.x) {
        const unsigned long long base = tile_base(t);
        const bool ok = mbar_wait_bounded(&bar, parity);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        parity ^= 1u;

        DevPhase ph = P.phases[0];
        Layout L = make_layout(ph, P.local, tid);
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int r = 0; r < kRegElems; ++r) x[s][r] = pf[s * kT + (L.jT | jr_of(L, r))];
        __syncthreads();   // the staging buffer is free again
        if (warp == 0 && t + gridDim.x < P.n_tiles) prefetch(t + gridDim.x);

        for (int p = 0; p < P.n_phases; ++p) {
            if (p > 0) {
                // re-layout through the swizzled transpose buffer
#pragma unroll
                for (int s = 0; s < S; ++s)
#pragma unroll
                    for (int r = 0; r < kRegElems; ++r) {
                        const int j = swz(L.jT | jr_of(L, r));
                        tr[(2 * s) * kT + j] = x[s][r].x;
                        tr[(2 * s + 1) * kT + j] = x[s][r].y;
                    }
                __syncthreads();
                ph = P.phases[p];
                L = make_layout(ph, P.local, tid);
#pragma unroll
                for (int s = 0; s < S; ++s)
#pragma unroll
                    for (int r = 0; r < kRegElems; ++r) {
                        const int j = swz(L.jT | jr_of(L, r));
                        x[s][r] = make_float2(tr[(2 * s) * kT + j], tr[(2 * s + 1) * kT + j]);
                    }
                __syncthreads();
            }
            for (int o = ph.op_begin; o < ph.op_end; ++o) {
                const DevOp op = P.ops[o];
                if (op.type == OP_G1) {
                    diag_flush(dg, x);
                    g1_dispatch(op.la, x, P.mats + op.mat);
                } else if (op.type == OP_G2) {
                    diag_flush(dg, x);
                    g2_dispatch(op.la, op.lb, x, P.mats + op.mat);
                } else if (op.type == OP_D1) {
                    const float2 d0 = P.mats[op.mat], d1 = P.mats[op.mat + 3];
                    if (op.la >= 0 && op.la < kRegBits) {
                        diag_mul_reg(dg, op.la, d0, d1);
                    } else {
                        dg.sc = cmul(dg.sc, const_bit(op.la, op.qa, tid, base) ? d1 : d0);
                        dg.pend = true;
                    }
                } else if (op.type == OP_D2) {
                    float2 d[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) d[e] = P.mats[op.mat + 5 * e];
                    const bool ra = op.la >= 0 && op.la < kRegBits;
                    const bool rb = op.lb >= 0 && op.lb < kRegBits;
                    if (ra && rb) {
                        // both qubits in registers: apply now (diagonals commute)
#pragma unroll
                        for (int r = 0; r < kRegElems; ++r) {
                            const float2 f = d[2 * ((r >> op.la) & 1) + ((r >> op.lb) & 1)];
#pragma unroll
                            for (int s = 0; s < S; ++s) x[s][r] = cmul(f, x[s][r]);
                        }
                    } else if (ra) {
                        const int c = const_bit(op.lb, op.qb, tid, base);
                        diag_mul_reg(dg, op.la, d[c], d[2 + c]);
                    } else if (rb) {
                        const int c = const_bit(op.la, op.qa, tid, base);
                        diag_mul_reg(dg, op.lb, d[2 * c], d[2 * c + 1]);
                    } else {
                        const int c0 = const_bit(op.la, op.qa, tid, base);
                        const int c1 = const_bit(op.lb, op.qb, tid, base);
                        dg.sc = cmul(dg.sc, d[2 * c0 + c1]);
                        dg.pend = true;
                    }
                } else if (op.type == OP_SITE) {
                    diag_flush(dg, x);
                    site_dispatch(op.la, P, op, x, L, base, acc, lane, warp);
                }
            }
            diag_flush(dg, x);
        }

#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int r = 0; r < kRegElems; ++r) __stcs(P.out[s] + (base | L.gT | gr_of(L, r)), x[s][r]);
    }

    if (failed) {
        if (tid == 0) atomicExch(P.err, NQS_ERR_DEVICE_TIMEOUT);
        // let copies still in flight land before the block's shared memory goes away
        mbar_wait_bounded(&bar, parity);
        return;
    }
    __syncthreads();
    for (int i = tid; i < P.n_events * S * 8; i += kThreads) {
        const int e = i & 7, s = (i >> 3) % S, ev = (i >> 3) / S;
        double v = 0.0;
        for (int w = 0; w < kWarps; ++w) v += acc[ev * S + s][w][e];
        P.partials[((size_t)(ev * S + s) * gridDim.x + blockIdx.x) * 8 + e] = v;
    }
}

template <int S>
void set_attr() {
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(sweep_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_smem_bytes(S));
        done = true;
    }
}

}  // namespace

size_t sweep_smem_bytes(int S) { return (size_t)S * kT * (sizeof(float2) + 2 * sizeof(float)); }

int sweep_blocks_per_sm(int S) {
    int nb = 0;
    const size_t smem = sweep_smem_bytes(S);
    if (S == 1) {
        set_attr<1>();
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<1>, kThreads, smem);
    } else if (S == 2) {
        set_attr<2>();
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<2>, kThreads, smem);
    } else {
        set_attr<3>();
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<3>, kThreads, smem);
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_sweep(int S, int grid, const PassArgs& P, cudaStream_t st) {
    const size_t smem = sweep_smem_bytes(S);
    if (S == 1) {
        set_attr<1>();
        sweep_kernel<1><<<grid, kThreads, smem, st>>>(P);
    } else if (S == 2) {
        set_attr<2>();
        sweep_kernel<2><<<grid, kThreads, smem, st>>>(P);
    } else {
        set_attr<3>();
        sweep_kernel<3><<<grid, kThreads, smem, st>>>(P);
    }
    return cudaGetLastError();
}

}  // namespace nqs
