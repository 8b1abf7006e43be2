// Register-resident tile sweep for sm_103a: a tile is 12 qubits (4096
// amplitudes) of each of S states; each thread holds E = 2^RB amplitudes per
// state in registers (RB "register qubits"), so a block has 4096 / E threads.
//
// * Prefetch: the next tile of every state is brought into a shared-memory
//   staging buffer by TMA bulk copies (cp.async.bulk, one 256-byte run of
//   the 5 contiguous low qubits per copy) whose completion is tracked by an
//   mbarrier, while the current tile is processed in registers.  Every wait
//   on the mbarrier is bounded; a wait that gives up sets the device status
//   word, lets the copies in flight land and returns.
// * Program: the launch's phases, 16-byte operation records and matrices are
//   copied into shared memory once per block.
// * Phases: in a phase RB of the tile's qubits are register qubits, so every
//   dense one- or two-qubit operation of the phase is applied without
//   touching shared memory; between phases the tile is re-laid out through
//   a second, XOR-swizzled shared-memory buffer.
// * Diagonal operations on any qubit, inside or outside the tile, are folded
//   into a per-thread factor (a scalar plus one pair of factors per register
//   qubit) and applied once, before the next dense operation.
// * Site operations (checkpoint save, reduction against phi_site, spawning
//   K_i x, applying K_0) act on a register qubit and read / write HBM
//   directly; reductions go FP32 per thread -> FP32 warp shuffle -> FP64
//   per-warp slot, then per-block partials summed in a fixed order later.
//
// This header holds the kernel templates; each (states, register qubits)
// pair is instantiated in its own translation unit (kernels_sweep_s*.cu) so
// the pairs compile in parallel, and kernels_sweep.cu dispatches to them.
#pragma once

#include <cstdlib>

#include "sweep_types.h"
#include "nqs_internal.h"

namespace nqs {

namespace {

constexpr int kT = 1 << kMaxTileQ;   // amplitudes per state tile
constexpr int kChunk = 32;           // contiguous amplitudes per TMA copy (5 low qubits)
constexpr int kChunks = kT / kChunk;
constexpr int kSpinLimit = 1 << 19;  // bounded mbarrier wait: ~2 s with the back-off (~3.8 us per try)

// Swizzle of the re-layout buffer (8-byte complex64 words): bits 4-7 and 8-11
// of the tile index are folded into bits 0-3, so the bank pair of word j is
// the XOR of its three 4-bit groups.  Lanes 0-3 of a warp sit on tile
// positions of distinct residue mod 4 (chosen by the planner), so each
// half-warp of a 64-bit access touches 16 distinct bank pairs.  XOR-linear.
__device__ __forceinline__ int swz(int j) { return j ^ ((j >> 4) & 15) ^ ((j >> 8) & 15); }

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

// bulk prefetch of global memory into L2 (no shared-memory destination)
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
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
// Packed FP32x2 form of a complex product on interleaved (re, im) pairs:
//   m a = (m.x, m.x) * (a.x, a.y) + (-m.y, m.y) * (a.y, a.x)
// so one output of the 2x2 gate is four packed operations (multi-state passes).
template <int I, int S, int E>
__device__ __forceinline__ void g1_reg(float2 (&x)[S][E], float2 m0, float2 m1, float2 m2, float2 m3) {
    if constexpr (S == 1) {   // the 16-amplitude single-state layout has no registers to spare
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if (r & (1 << I)) continue;
            const int r1 = r | (1 << I);
            const float2 a = x[0][r], b = x[0][r1];
            x[0][r] = cfma(m0, a, cmul(m1, b));
            x[0][r1] = cfma(m2, a, cmul(m3, b));
        }
        return;
    }
    const float2 p0 = make_float2(m0.x, m0.x), q0 = make_float2(-m0.y, m0.y);
    const float2 p1 = make_float2(m1.x, m1.x), q1 = make_float2(-m1.y, m1.y);
    const float2 p2 = make_float2(m2.x, m2.x), q2 = make_float2(-m2.y, m2.y);
    const float2 p3 = make_float2(m3.x, m3.x), q3 = make_float2(-m3.y, m3.y);
#pragma unroll
    for (int r = 0; r < E; ++r) {
        if (r & (1 << I)) continue;
        const int r1 = r | (1 << I);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float2 a = x[s][r], b = x[s][r1];
            const float2 as = make_float2(a.y, a.x), bs = make_float2(b.y, b.x);
            float2 y0 = __fmul2_rn(p0, a);
            y0 = __ffma2_rn(q0, as, y0);
            y0 = __ffma2_rn(p1, b, y0);
            y0 = __ffma2_rn(q1, bs, y0);
            float2 y1 = __fmul2_rn(p2, a);
            y1 = __ffma2_rn(q2, as, y1);
            y1 = __ffma2_rn(p3, b, y1);
            y1 = __ffma2_rn(q3, bs, y1);
            x[s][r] = y0;
            x[s][r1] = y1;
        }
    }
}

template <int S, int E, int RB>
__device__ __forceinline__ void g1_dispatch(int i, float2 (&x)[S][E], const float2* m) {
    const float2 m0 = m[0], m1 = m[1], m2 = m[2], m3 = m[3];
    if (i == 0) g1_reg<0>(x, m0, m1, m2, m3);
    else if (i == 1) g1_reg<1>(x, m0, m1, m2, m3);
    else if (i == 2) g1_reg<2>(x, m0, m1, m2, m3);
    else if constexpr (RB > 3) g1_reg<3>(x, m0, m1, m2, m3);
}

// 4x4 matrix indexed 2*b(first) + b(second); first qubit on register bit I0
template <int I0, int I1, int S, int E>
__device__ __forceinline__ void g2_reg(float2 (&x)[S][E], const float2* mg) {
    float2 m[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) m[e] = mg[e];
#pragma unroll
    for (int r = 0; r < E; ++r) {
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

template <int S, int E, int RB>
__device__ __forceinline__ void g2_dispatch(int i0, int i1, float2 (&x)[S][E], const float2* m) {
    switch (i0 * 4 + i1) {
        case 1: g2_reg<0, 1>(x, m); break;
        case 2: g2_reg<0, 2>(x, m); break;
        case 4: g2_reg<1, 0>(x, m); break;
        case 6: g2_reg<1, 2>(x, m); break;
        case 8: g2_reg<2, 0>(x, m); break;
        case 9: g2_reg<2, 1>(x, m); break;
        default:
            if constexpr (RB > 3) {
                switch (i0 * 4 + i1) {
                    case 3: g2_reg<0, 3>(x, m); break;
                    case 7: g2_reg<1, 3>(x, m); break;
                    case 11: g2_reg<2, 3>(x, m); break;
                    case 12: g2_reg<3, 0>(x, m); break;
                    case 13: g2_reg<3, 1>(x, m); break;
                    case 14: g2_reg<3, 2>(x, m); break;
                    default: break;
                }
            }
            break;
    }
}

// ---- layouts ----------------------------------------------------------------
template <int RB>
struct Layout {
    int jT;                          // tile index bits owned by the thread (lanes, warps)
    int jR[RB];                      // tile index bit of each register qubit
    int sT, sR[RB];                  // swz(jT), swz(jR[i]): swz is XOR-linear in the index bits
    unsigned long long gT;           // the same in global index bits
    unsigned long long gR[RB];
};

template <int RB>
__device__ __forceinline__ void make_layout(Layout<RB>& L, const DevPhase& ph, const int* local, int tid) {
    constexpr int WB = kMaxTileQ - RB - 5;
    L.jT = 0;
    L.gT = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i)
        if ((tid >> i) & 1) {
            L.jT |= 1 << ph.L[i];
            L.gT |= 1ull << local[ph.L[i]];
        }
#pragma unroll
    for (int i = 0; i < WB; ++i)
        if ((tid >> (5 + i)) & 1) {
            L.jT |= 1 << ph.W[i];
            L.gT |= 1ull << local[ph.W[i]];
        }
#pragma unroll
    for (int i = 0; i < RB; ++i) {
        L.jR[i] = 1 << ph.R[i];
        L.gR[i] = 1ull << local[ph.R[i]];
        L.sR[i] = swz(L.jR[i]);
    }
    L.sT = swz(L.jT);
}

template <int RB>
__device__ __forceinline__ int sr_of(const Layout<RB>& L, int r) {
    int j = L.sT;
#pragma unroll
    for (int i = 0; i < RB; ++i)
        if (r & (1 << i)) j ^= L.sR[i];
    return j;
}

template <int RB>
__device__ __forceinline__ int jr_of(const Layout<RB>& L, int r) {
    int j = 0;
#pragma unroll
    for (int i = 0; i < RB; ++i)
        if (r & (1 << i)) j |= L.jR[i];
    return j;
}

template <int RB>
__device__ __forceinline__ unsigned long long gr_of(const Layout<RB>& L, int r) {
    unsigned long long g = 0;
#pragma unroll
    for (int i = 0; i < RB; ++i)
        if (r & (1 << i)) g |= L.gR[i];
    return g;
}

// bit of a qubit that is not a register qubit: a thread bit, or (code 0xff)
// a bit of the tile's base index
__device__ __forceinline__ int const_bit(int loc, int qubit, int tid, unsigned long long base) {
    return (loc != 0xff) ? ((tid >> (loc - LOC_THREAD)) & 1) : (int)((base >> qubit) & 1);
}

template <int I, int S, int E, int RB>
__device__ __forceinline__ void site_reg(const PassArgs& P, const OpRec& op, const float2* m, float2 (&x)[S][E],
                                         const Layout<RB>& L, unsigned long long base, double* acc, int lane,
                                         int warp) {
    constexpr int NW = (kT >> RB) / 32;
    const int fl = op.flags;
    const float2 k0 = m[0], k1 = m[1], k2 = m[2], k3 = m[3];
    const float2* phi = (fl & FL_REDUCE) ? P.ckpt[op.site] : nullptr;
    float2* save = (fl & FL_SAVE) ? P.ckpt[op.site] : (fl & FL_SAVE_FWD) ? P.ckpt_fwd[op.site] : nullptr;
    float rr[S][8];
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
        for (int e = 0; e < 8; ++e) rr[s][e] = 0.f;
#pragma unroll
    for (int r = 0; r < E; ++r) {
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
            if ((fl & (FL_SAVE | FL_SAVE_FWD)) && s == 0) {
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
                for (int i = 0; i < op.nspawn; ++i) {
                    const float2* K = m + 4 * (i + 1);
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
        // reduce-scatter over the warp: after halving steps 16, 8, 4 lane l
        // holds the warp sum (over lanes with equal l & 7... completed by
        // steps 2, 1) of component l & 7 in v[0]
#pragma unroll
        for (int s = 0; s < S; ++s) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = rr[s][e];
            // step 16: lanes with bit 4 set keep components 4..7, others 0..3
            {
                const bool hi = lane & 16;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float send = hi ? v[e] : v[e + 4];
                    const float keep = hi ? v[e + 4] : v[e];
                    v[e] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                }
            }
            // step 8: keep 2 of the 4
            {
                const bool hi = lane & 8;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const float send = hi ? v[e] : v[e + 2];
                    const float keep = hi ? v[e + 2] : v[e];
                    v[e] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                }
            }
            // step 4: keep 1 of the 2
            {
                const bool hi = lane & 4;
                const float send = hi ? v[0] : v[1];
                const float keep = hi ? v[1] : v[0];
                v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
            }
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
            // lane bits 4, 3, 2 select the component: ((l>>4)&1)*4 + ((l>>3)&1)*2 + ((l>>2)&1)
            if ((lane & 3) == 0) {
                const int e = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                acc[((op.ev * S + s) * NW + warp) * 8 + e] += (double)v[0];
            }
        }
    }
}

template <int S, int E, int RB>
__device__ __forceinline__ void site_dispatch(int i, const PassArgs& P, const OpRec& op, const float2* m,
                                              float2 (&x)[S][E], const Layout<RB>& L, unsigned long long base,
                                              double* acc, int lane, int warp) {
    if (i == 0) site_reg<0>(P, op, m, x, L, base, acc, lane, warp);
    else if (i == 1) site_reg<1>(P, op, m, x, L, base, acc, lane, warp);
    else if (i == 2) site_reg<2>(P, op, m, x, L, base, acc, lane, warp);
    else if constexpr (RB > 3) site_reg<3>(P, op, m, x, L, base, acc, lane, warp);
}

// The tiles of one pass, processed by block `cta` of `nctas` (tiles cta,
// cta + nctas, ...).  Shared by the single-pass kernel and the batched kernel
// that runs the passes of many circuits in one launch.
template <int S, int RB>
__device__ __forceinline__ void sweep_body(const PassArgs& P, const int cta, const int nctas) {
    constexpr int E = 1 << RB;
    constexpr int NT = kT >> RB;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(128) unsigned char dyn[];
    float2* pf = reinterpret_cast<float2*>(dyn);                                  // [S][kT] TMA staging
    float2* tr = reinterpret_cast<float2*>(dyn + (size_t)S * kT * sizeof(float2));   // [S][kT] swizzled
    uint4* prog = reinterpret_cast<uint4*>(dyn + (size_t)S * kT * 16);              // phases, ops, matrices
    double* acc = reinterpret_cast<double*>(prog + P.prog_words);                   // [ev][S][NW][8]
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned long long hi_off[kChunks];
    __shared__ const float2* red_phi[kMaxEvents];   // phi of the pass's reductions, prefetched into L2
    __shared__ int n_red;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < P.prog_words; i += NT) prog[i] = P.prog[i];
    for (int h = tid; h < kChunks; h += NT) {
        unsigned long long off = 0;
        for (int j = 0; j < kMaxTileQ - 5; ++j)
            if ((h >> j) & 1) off |= 1ull << P.local[5 + j];
        hi_off[h] = off;
    }
    for (int i = tid; i < P.n_events * S * NW * 8; i += NT) acc[i] = 0.0;
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const DevPhase* phases = reinterpret_cast<const DevPhase*>(prog);
    const OpRec* ops = reinterpret_cast<const OpRec*>(prog + P.ops_word);
    const float2* mats = reinterpret_cast<const float2*>(prog + P.mats_word);
    if (tid == 0) {
        int c = 0;
        for (int o = 0; o < P.n_ops && c < kMaxEvents; ++o)
            if (ops[o].type == OP_SITE && (ops[o].flags & FL_REDUCE)) red_phi[c++] = P.ckpt[ops[o].site];
        n_red = c;
    }
    __syncthreads();

    auto tile_base = [&](long long t) {
        unsigned long long b = 0;
        for (int j = 0; j < P.n - kMaxTileQ; ++j)
            if ((t >> j) & 1) b |= 1ull << P.nonlocal[j];
        return b;
    };
    // every thread issues its share of the copies (no warp arrives late at
    // the next barrier); the mbarrier phase cannot complete before thread 0's
    // arrive.expect_tx, whatever order the copies land in
    // the phi tiles the pass's reductions will read go to L2 at the same time
    auto prefetch = [&](unsigned long long b) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (tid == 0) mbar_arrive_expect_tx(&bar, (uint32_t)(S * kT * sizeof(float2)));
        for (int q = tid; q < S * kChunks; q += NT) {
            const int s = q / kChunks, h = q % kChunks;
            bulk_copy_g2s(pf + s * kT + h * kChunk, P.in[s] + (b | hi_off[h]), kChunk * sizeof(float2), &bar);
        }
        for (int q = tid; q < n_red * kChunks; q += NT) {
            const int e = q / kChunks, h = q % kChunks;
            bulk_prefetch_l2(red_phi[e] + (b | hi_off[h]), kChunk * sizeof(float2));
        }
    };

    long long t = cta;
    unsigned long long base_next = t < P.n_tiles ? tile_base(t) : 0ull;
    if (t < P.n_tiles) prefetch(base_next);
    uint32_t parity = 0;
    bool failed = false;
    float2 x[S][E];
    Layout<RB> L;

    for (; t < P.n_tiles; t += nctas) {
        const unsigned long long base = base_next;
        const bool ok = mbar_wait_bounded(&bar, parity);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        parity ^= 1u;
        make_layout<RB>(L, phases[0], P.local, tid);
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int r = 0; r < E; ++r) x[s][r] = pf[s * kT + (L.jT | jr_of(L, r))];
        __syncthreads();   // the staging buffer is free again
        if (t + nctas < P.n_tiles) {
            base_next = tile_base(t + nctas);
            prefetch(base_next);
        }

        // pending diagonal factor: scalar + per-register-qubit pairs
        float2 dsc = make_float2(1.f, 0.f);
        float2 dh[RB][2];
#pragma unroll
        for (int i = 0; i < RB; ++i) dh[i][0] = dh[i][1] = make_float2(1.f, 0.f);
        int dmask = 0;
        bool dpend = false;
        auto flush = [&]() {
            if (!dpend) return;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                float2 f = dsc;
#pragma unroll
                for (int i = 0; i < RB; ++i)
                    if (dmask & (1 << i)) f = cmul(f, dh[i][(r >> i) & 1]);
#pragma unroll
                for (int s = 0; s < S; ++s) x[s][r] = cmul(f, x[s][r]);
            }
            dsc = make_float2(1.f, 0.f);
#pragma unroll
            for (int i = 0; i < RB; ++i) dh[i][0] = dh[i][1] = make_float2(1.f, 0.f);
            dmask = 0;
            dpend = false;
        };
        auto dmul = [&](int i, float2 f0, float2 f1) {
#pragma unroll
            for (int k = 0; k < RB; ++k)
                if (k == i) {
                    dh[k][0] = cmul(dh[k][0], f0);
                    dh[k][1] = cmul(dh[k][1], f1);
                }
            dmask |= 1 << i;
            dpend = true;
        };

        for (int p = 0; p < P.n_phases; ++p) {
            if (p > 0) {
                flush();
#pragma unroll
                for (int s = 0; s < S; ++s)
#pragma unroll
                    for (int r = 0; r < E; ++r) {
                        const int j = sr_of(L, r);
                        tr[s * kT + j] = x[s][r];
                    }
                __syncthreads();
                make_layout<RB>(L, phases[p], P.local, tid);
#pragma unroll
                for (int s = 0; s < S; ++s)
#pragma unroll
                    for (int r = 0; r < E; ++r) {
                        const int j = sr_of(L, r);
                        x[s][r] = tr[s * kT + j];
                    }
                __syncthreads();
            }
            const int ob = phases[p].op_begin, oe = phases[p].op_end;
            for (int o = ob; o < oe; ++o) {
                const OpRec op = ops[o];
                const float2* m = mats + op.mat;
                if (op.type == OP_G1) {
                    // the pending factor on this register qubit is absorbed into the
                    // matrix columns; the rest of the pending diagonal commutes
                    float2 mm[4] = {m[0], m[1], m[2], m[3]};
                    if (dpend) {   // the pending scalar multiplies every amplitude the gate touches
#pragma unroll
                        for (int e = 0; e < 4; ++e) mm[e] = cmul(mm[e], dsc);
                        dsc = make_float2(1.f, 0.f);
                        dpend = dmask != 0;
                    }
                    if (dmask & (1 << op.la)) {
#pragma unroll
                        for (int k = 0; k < RB; ++k)
                            if (k == op.la) {
                                mm[0] = cmul(mm[0], dh[k][0]);
                                mm[2] = cmul(mm[2], dh[k][0]);
                                mm[1] = cmul(mm[1], dh[k][1]);
                                mm[3] = cmul(mm[3], dh[k][1]);
                                dh[k][0] = dh[k][1] = make_float2(1.f, 0.f);
                            }
                        dmask &= ~(1 << op.la);
                        dpend = dmask != 0;
                    }
                    g1_dispatch<S, E, RB>(op.la, x, mm);
                } else if (op.type == OP_D1) {
                    if (op.la < RB) {
                        dmul(op.la, m[0], m[3]);
                    } else {
                        dsc = cmul(dsc, const_bit(op.la, op.qa, tid, base) ? m[3] : m[0]);
                        dpend = true;
                    }
                } else if (op.type == OP_D2) {
                    const bool ra = op.la < RB, rb = op.lb < RB;
                    if (ra && rb) {
#pragma unroll
                        for (int r = 0; r < E; ++r) {
                            const float2 f = m[5 * (2 * ((r >> op.la) & 1) + ((r >> op.lb) & 1))];
#pragma unroll
                            for (int s = 0; s < S; ++s) x[s][r] = cmul(f, x[s][r]);
                        }
                    } else if (ra) {
                        const int c = const_bit(op.lb, op.qb, tid, base);
                        dmul(op.la, m[5 * c], m[5 * (2 + c)]);
                    } else if (rb) {
                        const int c = const_bit(op.la, op.qa, tid, base);
                        dmul(op.lb, m[5 * (2 * c)], m[5 * (2 * c + 1)]);
                    } else {
                        const int c0 = const_bit(op.la, op.qa, tid, base);
                        const int c1 = const_bit(op.lb, op.qb, tid, base);
                        dsc = cmul(dsc, m[5 * (2 * c0 + c1)]);
                        dpend = true;
                    }
                } else if (op.type == OP_G2) {
                    float2 mm[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) mm[e] = m[e];
                    if (dpend) {
#pragma unroll
                        for (int e = 0; e < 16; ++e) mm[e] = cmul(mm[e], dsc);
                        dsc = make_float2(1.f, 0.f);
                        dpend = dmask != 0;
                    }
                    const int both = (1 << op.la) | (1 << op.lb);
                    if (dmask & both) {
                        float2 fa[2] = {make_float2(1.f, 0.f), make_float2(1.f, 0.f)};
                        float2 fb[2] = {fa[0], fa[1]};
#pragma unroll
                        for (int k = 0; k < RB; ++k) {
                            if (k == op.la) {
                                fa[0] = dh[k][0];
                                fa[1] = dh[k][1];
                                dh[k][0] = dh[k][1] = make_float2(1.f, 0.f);
                            }
                            if (k == op.lb) {
                                fb[0] = dh[k][0];
                                fb[1] = dh[k][1];
                                dh[k][0] = dh[k][1] = make_float2(1.f, 0.f);
                            }
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float2 f = cmul(fa[c >> 1], fb[c & 1]);
#pragma unroll
                            for (int q = 0; q < 4; ++q) mm[4 * q + c] = cmul(mm[4 * q + c], f);
                        }
                        dmask &= ~both;
                        dpend = dmask != 0;
                    }
                    g2_dispatch<S, E, RB>(op.la, op.lb, x, mm);
                } else if (op.type == OP_SITE) {
                    flush();
                    site_dispatch<S, E, RB>(op.la, P, op, m, x, L, base, acc, lane, warp);
                }
            }
            flush();
        }

        const unsigned long long gb = base | L.gT;
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int r = 0; r < E; ++r) __stcs(P.out[s] + (gb | gr_of(L, r)), x[s][r]);
    }

    if (failed) {
        if (tid == 0) atomicExch(P.err, NQS_ERR_DEVICE_TIMEOUT);
        mbar_wait_bounded(&bar, parity);   // let copies still in flight land
        return;
    }
    __syncthreads();
    for (int i = tid; i < P.n_events * S * 8; i += NT) {
        const int e = i & 7, s = (i >> 3) % S, ev = (i >> 3) / S;
        double v = 0.0;
        for (int w = 0; w < NW; ++w) v += acc[((ev * S + s) * NW + w) * 8 + e];
        P.partials[((size_t)(ev * S + s) * nctas + cta) * 8 + e] = v;
    }
}

template <int S, int RB>
__global__ void __launch_bounds__(kT >> RB, (S == 1 ? 2 : 1)) sweep_kernel(const PassArgs P) {
    sweep_body<S, RB>(P, blockIdx.x, gridDim.x);
}

// Passes of many circuits in one launch: unit u owns blocks
// [cta_begin[u], cta_begin[u+1]); its arguments are staged in shared memory.
template <int S, int RB>
__global__ void __launch_bounds__(kT >> RB, (S == 1 ? 2 : 1))
    sweep_kernel_batched(const PassArgs* __restrict__ units, const int* __restrict__ cta_begin, int n_units) {
    __shared__ __align__(16) PassArgs sP;
    int lo = 0, hi = n_units;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (cta_begin[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid;
    }
    const int* src = reinterpret_cast<const int*>(units + lo);
    int* dst = reinterpret_cast<int*>(&sP);
    for (int i = threadIdx.x; i < (int)(sizeof(PassArgs) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    sweep_body<S, RB>(sP, (int)blockIdx.x - cta_begin[lo], cta_begin[lo + 1] - cta_begin[lo]);
}

template <int S, int RB>
size_t smem_for(int prog_words, int n_events) {
    constexpr int NW = (kT >> RB) / 32;
    return (size_t)S * kT * 16 + (size_t)prog_words * 16 + (size_t)n_events * S * NW * 8 * sizeof(double);
}

template <int S, int RB>
cudaError_t launch_t(int grid, const PassArgs& P, cudaStream_t st) {
    const size_t smem = smem_for<S, RB>(P.prog_words, P.n_events);
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<S, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sweep_kernel<S, RB><<<grid, kT >> RB, smem, st>>>(P);
    return cudaGetLastError();
}


template <int S, int RB>
cudaError_t launch_batched_t(const PassArgs* units, const int* cta_begin, int n_units, int total_ctas, size_t smem,
                             cudaStream_t st) {
    cudaError_t e =
        cudaFuncSetAttribute(sweep_kernel_batched<S, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sweep_kernel_batched<S, RB><<<total_ctas, kT >> RB, smem, st>>>(units, cta_begin, n_units);
    return cudaGetLastError();
}

template <int S, int RB>
int occupancy_t(size_t smem) {
    int nb = 0;
    cudaFuncSetAttribute(sweep_kernel<S, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<S, RB>, kT >> RB, smem);
    return nb > 0 ? nb : 1;
}

}  // namespace

// per-pair entry points (defined by NQS_SWEEP_PAIR in kernels_sweep_s*.cu)
#define NQS_SWEEP_PAIR_DECL(S, RB)                                                                         \
    cudaError_t sweep_launch_##S##_##RB(int grid, const PassArgs& P, cudaStream_t st);                     \
    cudaError_t sweep_launch_batched_##S##_##RB(const PassArgs* units, const int* cta_begin, int n_units, \
                                                int total_ctas, size_t smem, cudaStream_t st);            \
    int sweep_occupancy_##S##_##RB(size_t smem);
NQS_SWEEP_PAIR_DECL(1, 4)
NQS_SWEEP_PAIR_DECL(2, 3)
NQS_SWEEP_PAIR_DECL(2, 4)
NQS_SWEEP_PAIR_DECL(3, 3)
NQS_SWEEP_PAIR_DECL(3, 4)

#define NQS_SWEEP_PAIR(S, RB)                                                                              \
    cudaError_t sweep_launch_##S##_##RB(int grid, const PassArgs& P, cudaStream_t st) {                    \
        return launch_t<S, RB>(grid, P, st);                                                               \
    }                                                                                                      \
    cudaError_t sweep_launch_batched_##S##_##RB(const PassArgs* units, const int* cta_begin, int n_units, \
                                                int total_ctas, size_t smem, cudaStream_t st) {           \
        return launch_batched_t<S, RB>(units, cta_begin, n_units, total_ctas, smem, st);                  \
    }                                                                                                      \
    int sweep_occupancy_##S##_##RB(size_t smem) { return occupancy_t<S, RB>(smem); }

}  // namespace nqs
