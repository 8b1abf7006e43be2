// Pass-specialised sweep kernels, generated from a launch's program and
// compiled at run time with NVRTC for sm_103a.
//
// The register-resident sweep kernel (kernels_sweep.cu) interprets a
// per-launch program: for every operation it loads a record, dispatches on
// its type and register qubit, loads the matrix from shared memory and works
// out layouts and addresses at run time.  Here the same program becomes
// straight-line code: operations, register positions, tile layouts, global
// offsets and matrix entries are compile-time constants, zero matrix entries
// drop out, pending diagonal factors that are known when the code is
// generated (one-qubit diagonals, diagonals between register qubits,
// diagonal K_0) are multiplied together on the host, and only factors that
// depend on the thread or the tile stay run-time values.  Amplitudes whose
// addresses are adjacent (the site's qubit or a register qubit being qubit 0)
// move as 16-byte vectors.  The semantics are those of the interpreted
// kernel: same tile (12 qubits; 13 with 512-thread blocks as an option), same
// TMA bulk prefetch with bounded mbarrier waits, same phases and XOR-swizzled
// re-layouts, same site actions and the same per-block FP64 partials, so the
// finishers and term sums are shared.  The organisation differs: each kernel
// holds one state of 16 amplitudes per thread, and a pass over the three (or
// nine) states of a branch group sweeps a tile's states one after another
// (twice the resident warps of holding them together; the tile's phi values
// come from DRAM once and from L2 for the later states, under L2 eviction
// policies), consecutive re-layouts alternate between two buffers, and site
// reductions accumulate with split real/imaginary partners.
//
// Kernels are cached by their source text for the life of the process;
// the distinct kernels of a schedule are compiled in parallel.  When NVRTC
// cannot be loaded the engine keeps the interpreted kernel (still on the GPU)
// and reports it through nqs_info.jit_state == -1 (jit_launches == 0).
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "fp32_round.h"
#include "jit.h"

namespace nqs {

namespace {

using cd = std::complex<double>;

// ------------------------------------------------------------------ device prelude
const char* kPrelude = R"PRELUDE(
typedef unsigned long long u64;
typedef unsigned int u32;
struct JitArgs {
    const float2* in[3];
    float2* out[3];
    float2* const* ckpt;
    float2* const* ckpt_fwd;
    float2* spawn[9];
    double* partials;
    int* err;
    long long n_tiles;
};
#define SPIN_LIMIT (1 << 19)
static __device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }
static __device__ __forceinline__ void mbar_init(u64* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
static __device__ __forceinline__ void mbar_arrive_expect_tx(u64* bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
static __device__ __forceinline__ void bulk_g2s(void* dst, const void* src, u32 bytes, u64* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
static __device__ __forceinline__ void bulk_l2(const void* src, u32 bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// L2 eviction policies and the copies / loads that carry them
static __device__ __forceinline__ u64 pol_first() {
    u64 p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
static __device__ __forceinline__ u64 pol_last() {
    u64 p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
static __device__ __forceinline__ void bulk_g2s_h(void* dst, const void* src, u32 bytes, u64* bar, u64 pol) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol) : "memory");
}
static __device__ __forceinline__ void bulk_l2_h(const void* src, u32 bytes, u64 pol) {
    asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(src), "r"(bytes), "l"(pol) : "memory");
}
static __device__ __forceinline__ float4 ld4_h(const float2* p, u64 pol) {
    float4 v;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
    return v;
}
static __device__ __forceinline__ float2 ld2_h(const float2* p, u64 pol) {
    float2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
static __device__ __forceinline__ bool mbar_try(u64* bar, u32 parity) {
    u32 ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
static __device__ __noinline__ bool mbar_wait(u64* bar, u32 parity) {
    for (int i = 0; i < SPIN_LIMIT; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (i > 32) __nanosleep(64);
    }
    return false;
}
static __device__ __forceinline__ float2 sw(float2 a) { return make_float2(a.y, a.x); }
// c * a for a run-time c (packed FP32x2)
static __device__ __forceinline__ float2 mulR(float2 c, float2 a) {
    float2 y = __fmul2_rn(make_float2(c.x, c.x), a);
    return __ffma2_rn(make_float2(-c.y, c.y), sw(a), y);
}
static __device__ __forceinline__ float2 fmaR(float2 c, float2 a, float2 acc) {
    acc = __ffma2_rn(make_float2(c.x, c.x), a, acc);
    return __ffma2_rn(make_float2(-c.y, c.y), sw(a), acc);
}
// (cr + i ci) * a for literal constants: the tests fold when the code is compiled
static __device__ __forceinline__ float2 mulK(float cr, float ci, float2 a) {
    if (ci == 0.f) {
        if (cr == 1.f) return a;
        if (cr == 0.f) return make_float2(0.f, 0.f);
        return __fmul2_rn(make_float2(cr, cr), a);
    }
    if (cr == 0.f) return __fmul2_rn(make_float2(-ci, ci), sw(a));
    float2 y = __fmul2_rn(make_float2(cr, cr), a);
    return __ffma2_rn(make_float2(-ci, ci), sw(a), y);
}
static __device__ __forceinline__ float2 fmaK(float cr, float ci, float2 a, float2 acc) {
    if (cr != 0.f) acc = __ffma2_rn(make_float2(cr, cr), a, acc);
    if (ci != 0.f) acc = __ffma2_rn(make_float2(-ci, ci), sw(a), acc);
    return acc;
}
// acc += conj(f) * a
static __device__ __forceinline__ float2 cjfma(float2 f, float2 a, float2 acc) {
    acc = __ffma2_rn(make_float2(f.x, f.x), a, acc);
    return __ffma2_rn(make_float2(f.y, -f.y), sw(a), acc);
}
// conj(f) * a accumulated as A += f.x * a, B += f.y * a (no swapped or negated
// operands); conj(f) a = (A.x + B.y, A.y - B.x)
static __device__ __forceinline__ void cjacc(float2 f, float2 a, float2& A, float2& B) {
    A = __ffma2_rn(make_float2(f.x, f.x), a, A);
    B = __ffma2_rn(make_float2(f.y, f.y), a, B);
}
static __device__ __forceinline__ float2 cjfin(float2 A, float2 B) { return make_float2(A.x + B.y, A.y - B.x); }
static __device__ __forceinline__ float2 sel(int c, float2 a, float2 b) { return c ? b : a; }
// reduce-scatter of 8 floats over a warp; lane l ends with the warp sum of
// component ((l>>4)&1)*4 + ((l>>3)&1)*2 + ((l>>2)&1) in the return value
static __device__ __forceinline__ float warp_rs8(const float (&w)[8], int lane) {
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = w[e];
    {
        const bool hi = lane & 16;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float send = hi ? v[e] : v[e + 4];
            const float keep = hi ? v[e + 4] : v[e];
            v[e] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
    }
    {
        const bool hi = lane & 8;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float send = hi ? v[e] : v[e + 2];
            const float keep = hi ? v[e + 2] : v[e];
            v[e] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
    }
    {
        const bool hi = lane & 4;
        const float send = hi ? v[0] : v[1];
        const float keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    return v[0];
}
)PRELUDE";

// ------------------------------------------------------------------ code generation
}  // namespace

// resident blocks per SM of the kernels that hold one state in registers
int jit_blocks_per_sm() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("NQS_JIT_MINB");
        v = (e && (e[0] == '2' || e[0] == '3')) ? e[0] - '0' : 2;
    }
    return v;
}

namespace {

bool flush_rt_enabled() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("NQS_JIT_FLUSH");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

std::string flit(float v) {
    char buf[64];
    if (v == 0.f) return std::signbit(v) ? "-0.0f" : "0.0f";
    std::snprintf(buf, sizeof buf, "%af", (double)v);
    return buf;
}

struct Cf {   // complex constant rounded to float
    float re, im;
};
Cf to_cf(cd c) {
    const float2 f = round_c64(c);   // unit-modulus constants stay as close to the unit circle as FP32 allows
    return Cf{f.x, f.y};
}
bool is_one(cd c) {
    const Cf f = to_cf(c);
    return f.re == 1.f && f.im == 0.f;
}
bool is_zero(cd c) {
    const Cf f = to_cf(c);
    return f.re == 0.f && f.im == 0.f;
}
std::string kargs(cd c) {
    const Cf f = to_cf(c);
    return flit(f.re) + ", " + flit(f.im);
}

struct Gen {
    const JitPass& J;
    std::ostringstream o;
    int S, RB, E, NT, NW, WB;
    int K = 12, KT = 4096, CH = 128;   // tile qubits, amplitudes per tile, 256-byte chunks per tile
    // SEQ: the S states of a multi-state pass are swept one after another
    // through the same code (one state in registers, runtime state index st);
    // SS is the number of states, S the states held in registers
    bool SEQ = false;
    int SS = 1;
    bool PP = false;   // two re-layout buffers (one-state kernels)
    // layout of the current phase
    int R[4] = {}, Lp[5] = {}, Wp[4] = {};
    int ph = 0;
    // pending diagonal factor: cs * dsc(if rs) * prod_i cp[i][b_i] * dh_i[b_i](if rp[i]) * T[r]
    cd cs = 1.0;
    bool rs = false;
    cd cp[4][2];
    bool rp[4] = {};
    std::vector<cd> T;
    int tmp = 0;
    std::set<int> early_phi;   // reductions of the current phase whose phi is loaded at the phase start

    // reductions per phase whose phi values may be held in registers from the
    // phase start: only kernels holding several states in registers default to
    // it (measured no gain for the one-state kernels)
    int early_phi_budget() const {
        if (const char* e = std::getenv("NQS_JIT_EARLY_PHI")) return std::atoi(e);
        return (RB >= 4 && S > 1) ? 2 : 0;
    }

    explicit Gen(const JitPass& j) : J(j) {
        SS = J.S;
        SEQ = J.seq && J.S > 1;
        S = SEQ ? 1 : J.S;
        RB = J.RB;
        E = 1 << RB;
        K = J.k;
        KT = 1 << K;
        CH = 1 << (K - 5);
        NT = KT >> RB;
        NW = NT / 32;
        WB = K - RB - 5;
        T.assign(E, 1.0);
        reset_pending();
    }

    void reset_pending() {
        cs = 1.0;
        rs = false;
        rs_new.clear();
        for (auto& v : rp_new) v.clear();
        for (int i = 0; i < 4; ++i) {
            cp[i][0] = cp[i][1] = 1.0;
            rp[i] = false;
        }
        std::fill(T.begin(), T.end(), cd(1.0));
    }

    std::string name(const char* p) { return std::string(p) + std::to_string(tmp++); }

    bool has_spawn() const {
        for (const OpRec& op : J.ops)
            if (op.type == 5 && (op.flags & 2)) return true;
        return false;
    }

    void set_phase(int p) {
        ph = p;
        const DevPhase& d = J.phases[p];
        for (int i = 0; i < RB; ++i) R[i] = d.R[i];
        for (int i = 0; i < 5; ++i) Lp[i] = d.L[i];
        for (int i = 0; i < WB; ++i) Wp[i] = d.W[i];
    }
    // tile index / swizzled index / global offset of register amplitude r in phase p
    int jr(const DevPhase& d, int r) const {
        int j = 0;
        for (int i = 0; i < RB; ++i)
            if (r >> i & 1) j |= 1 << d.R[i];
        return j;
    }
    static int swz(int j) { return j ^ ((j >> 4) & 15) ^ ((j >> 8) & 15) ^ ((j >> 12) & 15); }
    unsigned long long gr(int r) const {
        unsigned long long g = 0;
        for (int i = 0; i < RB; ++i)
            if (r >> i & 1) g |= 1ull << J.local[R[i]];
        return g;
    }
    // per-thread tile index of phase p (lane and warp bits)
    std::string jt_expr(const DevPhase& d) const {
        std::ostringstream s;
        s << "(0";
        for (int i = 0; i < 5; ++i) s << " | (((tid >> " << i << ") & 1) << " << (int)d.L[i] << ")";
        for (int i = 0; i < WB; ++i) s << " | (((tid >> " << 5 + i << ") & 1) << " << (int)d.W[i] << ")";
        s << ")";
        return s.str();
    }
    std::string gt_expr(const DevPhase& d) const {
        std::ostringstream s;
        s << "(0ull";
        for (int i = 0; i < 5; ++i) s << " | ((u64)((tid >> " << i << ") & 1) << " << J.local[d.L[i]] << ")";
        for (int i = 0; i < WB; ++i)
            s << " | ((u64)((tid >> " << 5 + i << ") & 1) << " << J.local[d.W[i]] << ")";
        s << ")";
        return s.str();
    }
    // run-time value of a qubit that is not a register qubit: a thread bit or a tile-base bit
    std::string bit_expr(int loc, int qubit) const {
        if (loc != 0xff) return "((tid >> " + std::to_string(loc - 8) + ") & 1)";
        return "(int)((b >> " + std::to_string(qubit) + ") & 1ull)";
    }
    cd mat(int off) const { return cd(J.mats[off].x, J.mats[off].y); }

    // register bit of qubit 0 in this phase (adjacent amplitudes), -1 if none
    int bit_of_q0() const {
        for (int i = 0; i < RB; ++i)
            if (J.local[R[i]] == 0) return i;
        return -1;
    }

    // loads/stores of E amplitudes at global offsets gr(r) from `ptr` + gb;
    // pairs (r, r | 1 << v) with v the register bit of qubit 0 move as float4
    void emit_gather(const std::string& dst, const std::string& ptr, bool stream) {
        const int v = bit_of_q0();
        const bool hinted = (J.hint & 2) && !stream;   // phi loads with the L2 policy polphi
        for (int r = 0; r < E; ++r) {
            if (v >= 0 && (r >> v & 1)) continue;
            const std::string off = std::to_string(gr(r)) + "ull";
            if (hinted) {
                if (v >= 0) {
                    const int r1 = r | 1 << v;
                    o << "    { const float4 q = ld4_h(" << ptr << " + " << off << ", polphi); " << dst << "[" << r
                      << "] = make_float2(q.x, q.y); " << dst << "[" << r1 << "] = make_float2(q.z, q.w); }\n";
                } else {
                    o << "    " << dst << "[" << r << "] = ld2_h(" << ptr << " + " << off << ", polphi);\n";
                }
                continue;
            }
            if (v >= 0) {
                const int r1 = r | 1 << v;
                o << "    { const float4 q = " << (stream ? "__ldcs" : "__ldg") << "((const float4*)(" << ptr << " + "
                  << off << ")); " << dst << "[" << r << "] = make_float2(q.x, q.y); " << dst << "[" << r1
                  << "] = make_float2(q.z, q.w); }\n";
            } else {
                o << "    " << dst << "[" << r << "] = " << (stream ? "__ldcs" : "__ldg") << "(" << ptr << " + " << off
                  << ");\n";
            }
        }
    }
    // store value expressions val(r)
    template <typename F>
    void emit_scatter(const std::string& ptr, F val) {
        const int v = bit_of_q0();
        for (int r = 0; r < E; ++r) {
            if (v >= 0 && (r >> v & 1)) continue;
            const std::string off = std::to_string(gr(r)) + "ull";
            if (v >= 0) {
                const int r1 = r | 1 << v;
                o << "    { const float2 a0 = " << val(r) << ", a1 = " << val(r1) << "; __stcs((float4*)(" << ptr
                  << " + " << off << "), make_float4(a0.x, a0.y, a1.x, a1.y)); }\n";
            } else {
                o << "    __stcs(" << ptr << " + " << off << ", " << val(r) << ");\n";
            }
        }
    }

    // ---- pending diagonal ------------------------------------------------
    bool t_depends(int i) const {
        for (int r = 0; r < E; ++r)
            if (!(r >> i & 1) && to_cf(T[r]).re != to_cf(T[r | 1 << i]).re) return true;
        for (int r = 0; r < E; ++r)
            if (!(r >> i & 1) && to_cf(T[r]).im != to_cf(T[r | 1 << i]).im) return true;
        return false;
    }
    bool t_trivial() const {
        for (int r = 0; r < E; ++r)
            if (!is_one(T[r])) return false;
        return true;
    }
    void flush_t() {
        for (int r = 0; r < E; ++r) {
            if (is_one(T[r])) continue;
            for (int s = 0; s < S; ++s)
                o << "    x[" << s << "][" << r << "] = mulK(" << kargs(T[r]) << ", x[" << s << "][" << r << "]);\n";
        }
        std::fill(T.begin(), T.end(), cd(1.0));
    }
    // Apply the pending diagonal to the amplitudes.  keep_scalar: a constant
    // scalar (the same for every amplitude of every thread) stays pending --
    // it survives re-layouts and is absorbed later by a dense gate, a spawn
    // factor or the reduced matrix at no per-amplitude cost.
    void flush_all(bool keep_scalar = false) {
        const cd kept = keep_scalar ? cs : cd(1.0);
        if (keep_scalar) cs = 1.0;
        flush_now();
        cs = kept;
    }
    // consts: also apply the compile-time part (else it stays pending)
    void flush_now(bool consts = true) {
        materialize();
        // constant part per amplitude and run-time part over the run-time pairs
        std::vector<int> rbits;
        for (int i = 0; i < RB; ++i)
            if (rp[i]) rbits.push_back(i);
        const bool any_rt = rs || !rbits.empty();
        std::vector<cd> C(E, cd(1.0));
        if (consts)
            for (int r = 0; r < E; ++r) {
                cd c = cs * T[r];
                for (int i = 0; i < RB; ++i) c *= cp[i][r >> i & 1];
                C[r] = c;
            }
        if (!any_rt) {
            for (int r = 0; r < E; ++r) {
                if (is_one(C[r])) continue;
                for (int s = 0; s < S; ++s)
                    o << "    x[" << s << "][" << r << "] = mulK(" << kargs(C[r]) << ", x[" << s << "][" << r
                      << "]);\n";
            }
            reset_pending();
            return;
        }
        // products of the run-time factors over the bits in rbits
        std::map<int, std::string> prod;   // key: bits of r restricted to rbits (packed)
        std::string base = rs ? "dsc" : "";
        std::vector<std::pair<int, std::string>> cur = {{0, base}};
        for (size_t k = 0; k < rbits.size(); ++k) {
            std::vector<std::pair<int, std::string>> nx;
            for (auto& kv : cur)
                for (int b = 0; b < 2; ++b) {
                    const std::string f = "dh" + std::to_string(rbits[k]) + "_" + std::to_string(b);
                    std::string v;
                    if (kv.second.empty()) {
                        v = f;
                    } else {
                        v = name("g");
                        o << "    const float2 " << v << " = mulR(" << kv.second << ", " << f << ");\n";
                    }
                    nx.push_back({kv.first | (b << k), v});
                }
            cur.swap(nx);
        }
        for (auto& kv : cur) prod[kv.first] = kv.second;
        for (int r = 0; r < E; ++r) {
            int key = 0;
            for (size_t k = 0; k < rbits.size(); ++k) key |= ((r >> rbits[k]) & 1) << k;
            std::string g = prod[key];
            std::string f = g;
            if (!is_one(C[r])) {
                f = name("f");
                o << "    const float2 " << f << " = mulK(" << kargs(C[r]) << ", " << g << ");\n";
            }
            for (int s = 0; s < S; ++s)
                o << "    x[" << s << "][" << r << "] = mulR(" << f << ", x[" << s << "][" << r << "]);\n";
        }
        if (consts) {
            reset_pending();
        } else {
            rs = false;
            for (int i = 0; i < 4; ++i) rp[i] = false;
        }
    }
    // Before a dense gate that would take run-time diagonal factors into its
    // matrix: when two or more dense gates up to the next site would do so,
    // multiply the run-time factors into the amplitudes once instead, so the
    // gates keep constant (and often structured: real or imaginary) entries.
    void maybe_flush_rt(int oi, int end) {
        if (!(rs_pending() || rt_pending(0) || rt_pending(1) || rt_pending(2) || rt_pending(3))) return;
        int k = 0;
        bool scalar = rs_pending();
        for (int j = oi; j < end; ++j) {
            const OpRec& op = J.ops[j];
            if (op.type == 5) break;
            if (op.type == 1) {
                if (scalar || rt_pending(op.la)) ++k;
                scalar = false;
            } else if (op.type == 2) {
                if (scalar || rt_pending(op.la) || rt_pending(op.lb)) ++k;
                scalar = false;
            }
        }
        if (k >= 2) flush_now(false);
    }
    // Run-time factors are collected and multiplied as balanced product trees
    // when first needed (short dependency chains instead of one serial chain
    // through an accumulator).
    std::vector<std::string> rs_new;                       // scalar factors not yet in dsc
    std::vector<std::pair<std::string, std::string>> rp_new[4];
    std::string tree(std::vector<std::string> v) {
        while (v.size() > 1) {
            std::vector<std::string> nx;
            for (size_t k = 0; k + 1 < v.size(); k += 2) {
                const std::string t = name("t");
                o << "    const float2 " << t << " = mulR(" << v[k] << ", " << v[k + 1] << ");\n";
                nx.push_back(t);
            }
            if (v.size() & 1) nx.push_back(v.back());
            v.swap(nx);
        }
        return v.empty() ? "" : v[0];
    }
    void materialize() {
        if (!rs_new.empty()) {
            if (rs) rs_new.push_back("dsc");
            const std::string t = tree(rs_new);
            o << "    dsc = " << t << ";\n";
            rs_new.clear();
            rs = true;
        }
        for (int i = 0; i < 4; ++i) {
            if (rp_new[i].empty()) continue;
            std::vector<std::string> a, b;
            for (auto& pr : rp_new[i]) {
                a.push_back(pr.first);
                b.push_back(pr.second);
            }
            if (rp[i]) {
                a.push_back("dh" + std::to_string(i) + "_0");
                b.push_back("dh" + std::to_string(i) + "_1");
            }
            const std::string ta = tree(a), tb = tree(b);
            o << "    dh" << i << "_0 = " << ta << "; dh" << i << "_1 = " << tb << ";\n";
            rp_new[i].clear();
            rp[i] = true;
        }
    }
    bool rt_pending(int i) const { return rp[i] || !rp_new[i].empty(); }
    bool rs_pending() const { return rs || !rs_new.empty(); }
    void scalar_mul_rt(const std::string& v) { rs_new.push_back(v); }
    void pair_mul_rt(int i, const std::string& v0, const std::string& v1) { rp_new[i].push_back({v0, v1}); }
    static std::string c2(cd c) {
        const Cf f = to_cf(c);
        return "make_float2(" + flit(f.re) + ", " + flit(f.im) + ")";
    }

    // the FP32 matrix closest to unitary (when the exact one is), returned as the
    // doubles of those floats so the emitters print them unchanged
    static void round_matrix(cd* K, int dim) {
        float2 f[16];
        round_matrix_c64(K, dim, f);
        for (int e = 0; e < dim * dim; ++e) K[e] = cd(f[e].x, f[e].y);
    }

    // ---- operations ---------------------------------------------------------
    // run-time column factor rho_c of a dense gate: scalar times run-time pairs
    std::string column_rt(const std::vector<std::pair<int, int>>& bits) {
        materialize();
        std::vector<std::string> fs;
        if (rs) fs.push_back("dsc");
        for (auto& ib : bits)
            if (rp[ib.first]) fs.push_back("dh" + std::to_string(ib.first) + "_" + std::to_string(ib.second));
        if (fs.empty()) return "";
        std::string v = fs[0];
        for (size_t k = 1; k < fs.size(); ++k) {
            const std::string nv = name("rho");
            o << "    const float2 " << nv << " = mulR(" << v << ", " << fs[k] << ");\n";
            v = nv;
        }
        return v;
    }

    void op_g1(int i, cd m[4]) {
        if (t_depends(i)) flush_t();
        cd K[4];
        std::string rho[2];
        for (int c = 0; c < 2; ++c) rho[c] = column_rt({{i, c}});
        for (int rr = 0; rr < 2; ++rr)
            for (int c = 0; c < 2; ++c) K[2 * rr + c] = m[2 * rr + c] * cs * cp[i][c];
        round_matrix(K, 2);
        const bool rt = !rho[0].empty() || !rho[1].empty();
        std::string mv[4];
        if (rt) {
            for (int e = 0; e < 4; ++e) {
                const std::string& rc = rho[e & 1];
                mv[e] = name("m");
                if (rc.empty()) o << "    const float2 " << mv[e] << " = " << c2(K[e]) << ";\n";
                else o << "    const float2 " << mv[e] << " = mulK(" << kargs(K[e]) << ", " << rc << ");\n";
            }
        }
        cs = 1.0;
        rs = false;
        cp[i][0] = cp[i][1] = 1.0;
        rp[i] = false;
        for (int r = 0; r < E; ++r) {
            if (r >> i & 1) continue;
            const int r1 = r | 1 << i;
            for (int s = 0; s < S; ++s) {
                const std::string a = "x[" + std::to_string(s) + "][" + std::to_string(r) + "]";
                const std::string b = "x[" + std::to_string(s) + "][" + std::to_string(r1) + "]";
                o << "    { const float2 a = " << a << ", b = " << b << "; ";
                if (rt) {
                    o << a << " = fmaR(" << mv[1] << ", b, mulR(" << mv[0] << ", a)); " << b << " = fmaR(" << mv[3]
                      << ", b, mulR(" << mv[2] << ", a)); }\n";
                } else {
                    o << a << " = fmaK(" << kargs(K[1]) << ", b, mulK(" << kargs(K[0]) << ", a)); " << b << " = fmaK("
                      << kargs(K[3]) << ", b, mulK(" << kargs(K[2]) << ", a)); }\n";
                }
            }
        }
    }

    // 4x4 matrix indexed 2*b(first) + b(second); first on register bit i0
    void op_g2(int i0, int i1, const cd* m) {
        if (t_depends(i0) || t_depends(i1)) flush_t();
        cd K[16];
        std::string rho[4];
        for (int c = 0; c < 4; ++c) rho[c] = column_rt({{i0, c >> 1}, {i1, c & 1}});
        for (int q = 0; q < 4; ++q)
            for (int c = 0; c < 4; ++c) K[4 * q + c] = m[4 * q + c] * cs * cp[i0][c >> 1] * cp[i1][c & 1];
        round_matrix(K, 4);
        bool rt = false;
        for (int c = 0; c < 4; ++c) rt = rt || !rho[c].empty();
        std::string mv[16];
        if (rt) {
            for (int e = 0; e < 16; ++e) {
                const std::string& rc = rho[e & 3];
                mv[e] = name("m");
                if (rc.empty()) o << "    const float2 " << mv[e] << " = " << c2(K[e]) << ";\n";
                else o << "    const float2 " << mv[e] << " = mulK(" << kargs(K[e]) << ", " << rc << ");\n";
            }
        }
        cs = 1.0;
        rs = false;
        cp[i0][0] = cp[i0][1] = cp[i1][0] = cp[i1][1] = 1.0;
        rp[i0] = rp[i1] = false;
        for (int r = 0; r < E; ++r) {
            if (r & ((1 << i0) | (1 << i1))) continue;
            const int idx[4] = {r, r | 1 << i1, r | 1 << i0, r | 1 << i0 | 1 << i1};
            for (int s = 0; s < S; ++s) {
                o << "    { const float2 v0 = x[" << s << "][" << idx[0] << "], v1 = x[" << s << "][" << idx[1]
                  << "], v2 = x[" << s << "][" << idx[2] << "], v3 = x[" << s << "][" << idx[3] << "];\n";
                for (int q = 0; q < 4; ++q) {
                    o << "      x[" << s << "][" << idx[q] << "] = ";
                    if (rt) {
                        o << "fmaR(" << mv[4 * q + 3] << ", v3, fmaR(" << mv[4 * q + 2] << ", v2, fmaR(" << mv[4 * q + 1]
                          << ", v1, mulR(" << mv[4 * q] << ", v0))));\n";
                    } else {
                        o << "fmaK(" << kargs(K[4 * q + 3]) << ", v3, fmaK(" << kargs(K[4 * q + 2]) << ", v2, fmaK("
                          << kargs(K[4 * q + 1]) << ", v1, mulK(" << kargs(K[4 * q]) << ", v0))));\n";
                    }
                }
                o << "    }\n";
            }
        }
    }

    void op_d1(const OpRec& op, const cd* m) {
        if (op.la < RB) {
            cp[op.la][0] *= m[0];
            cp[op.la][1] *= m[3];
        } else {
            const std::string v = name("d");
            o << "    const float2 " << v << " = sel(" << bit_expr(op.la, op.qa) << ", " << c2(m[0]) << ", " << c2(m[3])
              << ");\n";
            scalar_mul_rt(v);
        }
    }

    void op_d2(const OpRec& op, const cd* m) {
        const bool ra = op.la < RB, rb = op.lb < RB;
        if (ra && rb) {
            for (int r = 0; r < E; ++r) T[r] *= m[5 * (2 * ((r >> op.la) & 1) + ((r >> op.lb) & 1))];
        } else if (ra || rb) {
            const int i = ra ? op.la : op.lb;
            const std::string c = ra ? bit_expr(op.lb, op.qb) : bit_expr(op.la, op.qa);
            // factors for b_i = 0, 1 given the other qubit's bit c
            cd f0c0, f1c0, f0c1, f1c1;
            if (ra) {   // index 2*b_a + c
                f0c0 = m[5 * 0]; f1c0 = m[5 * 2]; f0c1 = m[5 * 1]; f1c1 = m[5 * 3];
            } else {    // index 2*c + b_b
                f0c0 = m[5 * 0]; f1c0 = m[5 * 1]; f0c1 = m[5 * 2]; f1c1 = m[5 * 3];
            }
            const std::string cv = name("c");
            o << "    const int " << cv << " = " << c << ";\n";
            const std::string v0 = name("p"), v1 = name("p");
            o << "    const float2 " << v0 << " = sel(" << cv << ", " << c2(f0c0) << ", " << c2(f0c1) << ");\n";
            o << "    const float2 " << v1 << " = sel(" << cv << ", " << c2(f1c0) << ", " << c2(f1c1) << ");\n";
            pair_mul_rt(i, v0, v1);
        } else {
            const std::string c0 = name("c"), c1 = name("c"), v = name("d");
            o << "    const int " << c0 << " = " << bit_expr(op.la, op.qa) << ", " << c1 << " = "
              << bit_expr(op.lb, op.qb) << ";\n";
            o << "    const float2 " << v << " = " << c0 << " ? sel(" << c1 << ", " << c2(m[10]) << ", " << c2(m[15])
              << ") : sel(" << c1 << ", " << c2(m[0]) << ", " << c2(m[5]) << ");\n";
            scalar_mul_rt(v);
        }
    }

    void op_site(const OpRec& op, const cd* m, int phase_idx) {
        flush_all(true);
        const cd sc = cs;   // pending constant scalar: folded into what the site writes or reduces
        const int i = op.la;
        const int fl = op.flags;
        const DevPhase& d = J.phases[phase_idx];
        (void)d;
        const bool red = fl & 1, spawn = fl & 2, save = fl & 4, apply = fl & 8, save_fwd = fl & 16, kdiag = fl & 32;
        o << "    {\n";
        if (red || save || save_fwd || spawn) o << "    const u64 gb = b | gT" << phase_idx << ";\n";
        if (save || save_fwd) {
            const std::string p = save ? ("P.ckpt[" + std::to_string(op.site) + "]")
                                       : ("P.ckpt_fwd[" + std::to_string(op.site) + "]");
            o << "    float2* const sv = " << p << " + gb;\n";
            emit_scatter("sv", [&](int r) {
                const std::string v = "x[0][" + std::to_string(r) + "]";
                return is_one(sc) ? v : "mulK(" + kargs(sc) + ", " + v + ")";
            });
        }
        if (red) {
            if (early_phi.count(op.ev)) {
                o << "    const float2 (&ph)[" << E << "] = phe" << (int)op.ev << ";\n";
            } else {
                o << "    float2 ph[" << E << "];\n";
                o << "    const float2* const pp = phi" << (int)op.ev << " + gb;\n";
                emit_gather("ph", "pp", !SEQ && !(J.hint & 2));   // the other states re-read phi from L2
            }
            for (int s = 0; s < S; ++s) {
                o << "    { float2 R00 = make_float2(0.f, 0.f), R01 = R00, R10 = R00, R11 = R00;\n";
                if (J.rv == 2) {
                    o << "      float2 A00 = R00, B00 = R00, A01 = R00, B01 = R00, A10 = R00, B10 = R00, A11 = R00, B11 = R00;\n";
                    for (int r = 0; r < E; ++r) {
                        if (r >> i & 1) continue;
                        const int r1 = r | 1 << i;
                        const std::string f0 = "ph[" + std::to_string(r) + "]", f1 = "ph[" + std::to_string(r1) + "]";
                        const std::string x0 = "x[" + std::to_string(s) + "][" + std::to_string(r) + "]";
                        const std::string x1 = "x[" + std::to_string(s) + "][" + std::to_string(r1) + "]";
                        o << "      cjacc(" << f0 << ", " << x0 << ", A00, B00); cjacc(" << f0 << ", " << x1
                          << ", A01, B01); cjacc(" << f1 << ", " << x0 << ", A10, B10); cjacc(" << f1 << ", " << x1
                          << ", A11, B11);\n";
                    }
                    o << "      R00 = cjfin(A00, B00); R01 = cjfin(A01, B01); R10 = cjfin(A10, B10); R11 = cjfin(A11, B11);\n";
                } else {
                    for (int r = 0; r < E; ++r) {
                        if (r >> i & 1) continue;
                        const int r1 = r | 1 << i;
                        o << "      R00 = cjfma(ph[" << r << "], x[" << s << "][" << r << "], R00); R01 = cjfma(ph[" << r
                          << "], x[" << s << "][" << r1 << "], R01); R10 = cjfma(ph[" << r1 << "], x[" << s << "][" << r
                          << "], R10); R11 = cjfma(ph[" << r1 << "], x[" << s << "][" << r1 << "], R11);\n";
                    }
                }
                if (!is_one(sc))
                    o << "      R00 = mulK(" << kargs(sc) << ", R00); R01 = mulK(" << kargs(sc) << ", R01); R10 = mulK("
                      << kargs(sc) << ", R10); R11 = mulK(" << kargs(sc) << ", R11);\n";
                o << "      const float w[8] = {R00.x, R00.y, R01.x, R01.y, R10.x, R10.y, R11.x, R11.y};\n";
                o << "      const float v = warp_rs8(w, lane);\n";
                o << "      if ((lane & 3) == 0) acc[((" << (int)op.ev << " * " << SS << " + " << (SEQ ? std::string("st") : std::to_string(s)) << ") * " << NW
                  << " + warp) * 8 + ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)] += (double)v;\n";
                o << "    }\n";
            }
        }
        if (spawn) {
            const int ns = op.nspawn;
            for (int s = 0; s < S; ++s)
                for (int k = 0; k < ns; ++k) {
                    const cd K[4] = {m[4 * (k + 1)] * sc, m[4 * (k + 1) + 1] * sc, m[4 * (k + 1) + 2] * sc,
                                     m[4 * (k + 1) + 3] * sc};
                    if (SEQ)
                        o << "    { float2* const dp = spw" << k << " + gb;\n";
                    else
                        o << "    { float2* const dp = P.spawn[" << s * 3 + k << "] + gb;\n";
                    // value of amplitude r of K x: rows by the site's bit
                    emit_scatter("dp", [&](int r) {
                        const int r0 = r & ~(1 << i), r1 = r | 1 << i;
                        const bool hi = r >> i & 1;
                        const cd k0 = hi ? K[2] : K[0], k1 = hi ? K[3] : K[1];
                        return "fmaK(" + kargs(k1) + ", x[" + std::to_string(s) + "][" + std::to_string(r1) +
                               "], mulK(" + kargs(k0) + ", x[" + std::to_string(s) + "][" + std::to_string(r0) + "]))";
                    });
                    o << "    }\n";
                }
        }
        o << "    }\n";
        if (apply) {
            if (kdiag) {
                cp[i][0] *= m[0];
                cp[i][1] *= m[3];
            } else {
                cd mm[4] = {m[0], m[1], m[2], m[3]};
                op_g1(i, mm);
            }
        }
    }

    std::string generate() {
        const int n_ph = (int)J.phases.size();
        std::vector<int> red_sites(J.n_events, -1);
        for (const OpRec& op : J.ops)
            if (op.type == 5 && (op.flags & 1)) red_sites[op.ev] = op.site;
        unsigned long long nl_mask = 0;
        for (int j = 0; j < J.n - K; ++j) nl_mask |= 1ull << J.nonlocal[j];
        // one-state kernels of 12-qubit tiles: several 256-thread blocks per SM;
        // 13-qubit tiles: one 512-thread block
        const int minb = (S == 1 && K == 12) ? jit_blocks_per_sm() : 1;
        o << kPrelude;
        o << "#define KT " << KT << "\n";
        o << "extern \"C\" __global__ void __launch_bounds__(" << NT << ", " << minb
          << ") nqs_pass(const JitArgs P) {\n";
        o << "  extern __shared__ __align__(128) unsigned char dyn[];\n";
        // kernels holding one state in registers (one state, or SEQ) stage
        // their tiles through a ring of DB buffers, one mbarrier each
        const bool ONE = (S == 1);
        const int DB = ONE ? std::max(1, std::min(2, J.db)) : 1;
        PP = ONE && J.pp;
        o << "  float2* const pf = (float2*)dyn;\n";
        o << "  float2* const tr = pf + " << (ONE ? DB : S) << " * KT;\n";
        o << "  double* const acc = (double*)(tr + " << (PP ? 2 : S) << " * KT);\n";
        o << "  __shared__ __align__(8) u64 bar[" << DB << "];\n";
        o << "  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;\n";
        o << "  const int cta = blockIdx.x, nctas = gridDim.x;\n";
        o << "  (void)lane; (void)warp;\n";
        o << "  for (int i = tid; i < " << J.n_events * SS * NW * 8 << "; i += " << NT << ") acc[i] = 0.0;\n";
        o << "  if (tid == 0) { for (int i = 0; i < " << DB << "; ++i) mbar_init(&bar[i], 1); "
             "asm volatile(\"fence.mbarrier_init.release.cluster;\" ::: \"memory\"); }\n";
        o << "  __syncthreads();\n";
        for (int p = 0; p < n_ph; ++p) {
            o << "  const int jT" << p << " = " << jt_expr(J.phases[p]) << ";\n";
            o << "  const int sT" << p << " = jT" << p << " ^ ((jT" << p << " >> 4) & 15) ^ ((jT" << p
              << " >> 8) & 15) ^ ((jT" << p << " >> 12) & 15);\n";
            o << "  const u64 gT" << p << " = " << gt_expr(J.phases[p]) << ";\n";
            o << "  (void)jT" << p << "; (void)sT" << p << "; (void)gT" << p << ";\n";
        }
        for (int e = 0; e < J.n_events; ++e)
            o << "  const float2* const phi" << e << " = P.ckpt[" << std::max(0, red_sites[e]) << "];\n";
        // tile bases: deposit the tile number into the non-tile qubits
        o << "  const u64 NL = " << nl_mask << "ull;\n";
        o << "  u64 step = 0, base = 0;\n";
        o << "  { u64 m = NL; long long v = nctas, w = cta; while (m) { const u64 low = m & (~m + 1ull); "
             "if (v & 1) step |= low; if (w & 1) base |= low; v >>= 1; w >>= 1; m ^= low; } }\n";
        // chunk offsets: bits 5..11 of the tile index on qubits local[5..11]
        o << "  auto hi_off = [&](int h) -> u64 { return 0ull";
        for (int j = 0; j < K - 5; ++j) o << " | ((u64)((h >> " << j << ") & 1) << " << J.local[5 + j] << ")";
        o << "; };\n";
        if (J.hint) {
            o << "  const u64 pol_ef = pol_first(), pol_el = pol_last();\n";
            o << "  const u64 polst = pol_ef;\n  const u64 polpf = " << (SS > 1 ? "pol_el" : "pol_ef") << ";\n";
            o << "  (void)polst; (void)polpf;\n";
        }
        // state selection by the runtime index st (SEQ)
        auto pick = [&](const std::string& arr, int stride, int k) {
            std::string e = arr + "[" + std::to_string((SS - 1) * stride + k) + "]";
            for (int q = SS - 2; q >= 0; --q)
                e = "(st == " + std::to_string(q) + " ? " + arr + "[" + std::to_string(q * stride + k) + "] : " + e + ")";
            return e;
        };
        if (ONE) {
            o << "  auto prefetch = [&](u64 bb, int st, int buf) {\n";
            o << "    asm volatile(\"fence.proxy.async.shared::cta;\" ::: \"memory\");\n";
            o << "    if (tid == 0) mbar_arrive_expect_tx(&bar[buf], " << KT * 8 << "u);\n";
            o << "    const float2* const src = " << pick("P.in", 1, 0) << ";\n";
            o << "    float2* const dst = pf + buf * KT;\n";
            if (J.hint & 1)
                o << "    for (int h = tid; h < " << CH << "; h += " << NT << ") bulk_g2s_h(dst + h * 32, src + (bb | hi_off(h)), 256u, &bar[buf], polst);\n";
            else
                o << "    for (int h = tid; h < " << CH << "; h += " << NT << ") bulk_g2s(dst + h * 32, src + (bb | hi_off(h)), 256u, &bar[buf]);\n";
            o << "    if (st != 0) return;\n";
        } else {
            o << "  auto prefetch = [&](u64 bb) {\n";
            o << "    asm volatile(\"fence.proxy.async.shared::cta;\" ::: \"memory\");\n";
            o << "    if (tid == 0) mbar_arrive_expect_tx(&bar[0], " << S * KT * 8 << "u);\n";
            o << "    for (int q = tid; q < " << S * CH << "; q += " << NT << ") { const int s = q >> " << K - 5
              << ", h = q & " << CH - 1 << "; "
                 "bulk_g2s(pf + s * KT + h * 32, P.in[s] + (bb | hi_off(h)), 256u, &bar[0]); }\n";
        }
        if (J.n_events > 0) {
            o << "    for (int q = tid; q < " << J.n_events * CH << "; q += " << NT << ") { const int e = q >> " << K - 5
              << ", h = q & " << CH - 1 << "; "
                 "const float2* ph = ";
            for (int e = 0; e < J.n_events; ++e) o << (e + 1 < J.n_events ? "e == " + std::to_string(e) + " ? phi" + std::to_string(e) + " : " : "phi" + std::to_string(e));
            if (J.hint & 2)
                o << "; bulk_l2_h(ph + (bb | hi_off(h)), 256u, polpf); }\n";
            else
                o << "; bulk_l2(ph + (bb | hi_off(h)), 256u); }\n";
        }
        o << "  };\n";
        o << "  long long t = cta;\n";
        if (ONE) {
            // consumer cursor (t, base, st), producer cursor (pt, pbase, pst)
            o << "  int st = 0;\n  (void)st;\n";
            o << "  long long pt = t;\n  u64 pbase = base;\n  int pst = 0;\n";
            o << "  u32 par = 0u, infl = 0u;\n  int cb = 0;\n";
            o << "  for (int i = 0; i < " << DB << "; ++i) if (pt < P.n_tiles) { prefetch(pbase, pst, i); infl |= 1u << i; "
                 "if (++pst == " << SS << ") { pst = 0; pt += nctas; pbase = ((pbase | ~NL) + step) & NL; } }\n";
            o << "  bool failed = false;\n";
        } else {
            o << "  if (t < P.n_tiles) prefetch(base);\n";
            o << "  u32 parity = 0;\n  bool failed = false;\n";
        }
        o << "  float2 x[" << S << "][" << E << "];\n";
        o << "  float2 dsc = make_float2(1.f, 0.f);\n";
        for (int i = 0; i < RB; ++i) o << "  float2 dh" << i << "_0 = dsc, dh" << i << "_1 = dsc;\n";
        o << "  (void)dsc;\n";
        for (int i = 0; i < RB; ++i) o << "  (void)dh" << i << "_0; (void)dh" << i << "_1;\n";
        if (ONE) {
            // (tile, state) pairs; with several states (SEQ) the states of a
            // tile follow one another, so the tile's phi values are read from
            // DRAM once and from L2 for the other states
            o << "  #pragma unroll 1\n";
            o << "  while (t < P.n_tiles) {\n";
            o << "    const u64 b = base;\n";
            o << "    const bool ok = mbar_wait(&bar[cb], (par >> cb) & 1u);\n";
            o << "    if (__syncthreads_or(!ok)) { failed = true; break; }\n";
            o << "    par ^= 1u << cb;\n    infl &= ~(1u << cb);\n";
            if (J.hint) o << "    const u64 polphi = st == " << SS - 1 << " ? pol_ef : pol_el;\n    (void)polphi;\n";
            set_phase(0);
            o << "    { const float2* const cur = pf + cb * KT;\n";
            for (int r = 0; r < E; ++r)
                o << "    x[0][" << r << "] = cur[" << jr(J.phases[0], r) << " + jT0];\n";
            o << "    }\n";
            o << "    __syncthreads();\n";
            o << "    if (pt < P.n_tiles) { prefetch(pbase, pst, cb); infl |= 1u << cb; "
                 "if (++pst == " << SS << ") { pst = 0; pt += nctas; pbase = ((pbase | ~NL) + step) & NL; } }\n";
        } else {
            o << "  for (; t < P.n_tiles; t += nctas) {\n";
            o << "    const u64 b = base;\n";
            o << "    const bool ok = mbar_wait(&bar[0], parity);\n";
            o << "    if (__syncthreads_or(!ok)) { failed = true; break; }\n";
            o << "    parity ^= 1u;\n";
            // every state of the tile is in registers: phi is read once per tile
            if (J.hint) o << "    const u64 polphi = pol_ef;\n    (void)polphi;\n";
            // load phase 0 from the staging buffer
            set_phase(0);
            for (int s = 0; s < S; ++s)
                for (int r = 0; r < E; ++r)
                    o << "    x[" << s << "][" << r << "] = pf[" << s * KT + jr(J.phases[0], r) << " + jT0];\n";
            o << "    __syncthreads();\n";
        }
        if (SEQ) {
            if (has_spawn())
                for (int k = 0; k < 3; ++k) o << "    float2* const spw" << k << " = " << pick("P.spawn", 3, k) << ";\n";
        } else if (!ONE) {
            o << "    if (t + nctas < P.n_tiles) { base = ((base | ~NL) + step) & NL; prefetch(base); }\n";
        }
        for (int p = 0; p < n_ph; ++p) {
            if (p > 0) {
                // re-layout through the swizzled buffer
                const DevPhase& a = J.phases[p - 1];
                const DevPhase& c = J.phases[p];
                // PP: consecutive re-layouts alternate between two buffers, so
                // the barrier of the next re-layout (or of the next tile) already
                // orders this one's reads before the buffer is written again
                const int tb = PP ? ((p - 1) & 1) * KT : 0;
                for (int s = 0; s < S; ++s)
                    for (int r = 0; r < E; ++r)
                        o << "    tr[" << tb + s * KT << " + (sT" << p - 1 << " ^ " << swz(jr(a, r)) << ")] = x[" << s
                          << "][" << r << "];\n";
                o << "    __syncthreads();\n";
                set_phase(p);
                for (int s = 0; s < S; ++s)
                    for (int r = 0; r < E; ++r)
                        o << "    x[" << s << "][" << r << "] = tr[" << tb + s * KT << " + (sT" << p << " ^ "
                          << swz(jr(c, r)) << ")];\n";
                if (!PP) o << "    __syncthreads();\n";
            }
            const DevPhase& d = J.phases[p];
            // the phi values of this phase's reductions are loaded at the start
            // of the phase (when the registers allow), so their latency overlaps
            // the phase's gates
            early_phi.clear();
            if (early_phi_budget() > 0) {
                int budget = early_phi_budget();
                for (int oi = d.op_begin; oi < d.op_end && budget > 0; ++oi) {
                    const OpRec& op = J.ops[oi];
                    if (op.type != 5 || !(op.flags & 1)) continue;
                    early_phi.insert(op.ev);
                    --budget;
                    o << "    float2 phe" << (int)op.ev << "[" << E << "];\n";
                    o << "    { const float2* const pp = phi" << (int)op.ev << " + (b | gT" << p << ");\n";
                    emit_gather("phe" + std::to_string((int)op.ev), "pp", !SEQ && !(J.hint & 2));
                    o << "    }\n";
                }
            }
            for (int oi = d.op_begin; oi < d.op_end; ++oi) {
                const OpRec& op = J.ops[oi];
                cd m[16];
                const int cnt = (op.type == 2 || op.type == 4 || (op.type == 5 && (op.flags & 2))) ? 16 : 4;
                for (int e = 0; e < cnt; ++e) m[e] = mat(op.mat + e);
                o << "    // op " << oi << " type " << (int)op.type << "\n";
                if ((op.type == 1 || op.type == 2) && flush_rt_enabled()) maybe_flush_rt(oi, d.op_end);
                switch (op.type) {
                    case 1: op_g1(op.la, m); break;
                    case 2: op_g2(op.la, op.lb, m); break;
                    case 3: op_d1(op, m); break;
                    case 4: op_d2(op, m); break;
                    case 5: op_site(op, m, p); break;
                    default: break;
                }
            }
            flush_all(p + 1 < n_ph);
        }
        // store the tile
        o << "    {\n";
        for (int s = 0; s < S; ++s) {
            if (SEQ)
                o << "    { float2* const op = " << pick("P.out", 1, 0) << " + (b | gT" << n_ph - 1 << ");\n";
            else
                o << "    { float2* const op = P.out[" << s << "] + (b | gT" << n_ph - 1 << ");\n";
            emit_scatter("op", [&](int r) { return "x[" + std::to_string(s) + "][" + std::to_string(r) + "]"; });
            o << "    }\n";
        }
        o << "    }\n";
        if (ONE) {
            o << "    if (++st == " << SS << ") { st = 0; t += nctas; base = ((base | ~NL) + step) & NL; }\n";
            o << "    cb = (cb + 1 == " << DB << ") ? 0 : cb + 1;\n";
        }
        o << "  }\n";
        o << "  if (failed) {\n";
        o << "    if (tid == 0) atomicExch(P.err, " << J.err_timeout << ");\n";
        if (ONE)   // the copies still in flight land before the block exits
            o << "    for (int i = 0; i < " << DB << "; ++i) if ((infl >> i) & 1u) mbar_wait(&bar[i], (par >> i) & 1u);\n";
        else
            o << "    mbar_wait(&bar[0], parity);\n";
        o << "    return;\n";
        o << "  }\n";
        if (J.n_events > 0) {
            o << "  __syncthreads();\n";
            o << "  for (int i = tid; i < " << J.n_events * SS * 8 << "; i += " << NT << ") {\n";
            o << "    const int e = i & 7, s = (i >> 3) % " << SS << ", ev = (i >> 3) / " << SS << ";\n";
            o << "    double v = 0.0;\n";
            o << "    for (int w = 0; w < " << NW << "; ++w) v += acc[((ev * " << SS << " + s) * " << NW << " + w) * 8 + e];\n";
            o << "    P.partials[((size_t)(ev * " << SS << " + s) * nctas + cta) * 8 + e] = v;\n";
            o << "  }\n";
        }
        o << "}\n";
        return o.str();
    }
};

// ------------------------------------------------------------------ NVRTC and loading
typedef int (*nvrtcCreateProgram_t)(void**, const char*, const char*, int, const char* const*, const char* const*);
typedef int (*nvrtcCompileProgram_t)(void*, int, const char* const*);
typedef int (*nvrtcGetSize_t)(void*, size_t*);
typedef int (*nvrtcGetData_t)(void*, char*);
typedef int (*nvrtcDestroyProgram_t)(void**);

struct Nvrtc {
    bool tried = false, ok = false;
    nvrtcCreateProgram_t create = nullptr;
    nvrtcCompileProgram_t compile = nullptr;
    nvrtcGetSize_t log_size = nullptr, cubin_size = nullptr;
    nvrtcGetData_t log = nullptr, cubin = nullptr;
    nvrtcDestroyProgram_t destroy = nullptr;
};

Nvrtc& nvrtc() {
    static Nvrtc N;
    static std::mutex mu;
    std::lock_guard<std::mutex> g(mu);
    if (N.tried) return N;
    N.tried = true;
    std::vector<std::string> cand;
    if (const char* e = std::getenv("NQS_NVRTC")) cand.push_back(e);
    cand.push_back("libnvrtc.so.13");
    cand.push_back("libnvrtc.so");
    const char* roots[] = {std::getenv("CUDA_HOME"), std::getenv("CUDA_PATH"), "/usr/local/cuda"};
    for (const char* root : roots)
        if (root) {
            cand.push_back(std::string(root) + "/lib64/libnvrtc.so.13");
            cand.push_back(std::string(root) + "/lib64/libnvrtc.so");
            cand.push_back(std::string(root) + "/targets/sbsa-linux/lib/libnvrtc.so.13");
            cand.push_back(std::string(root) + "/targets/x86_64-linux/lib/libnvrtc.so.13");
        }
    void* h = nullptr;
    for (const auto& c : cand) {
        h = dlopen(c.c_str(), RTLD_NOW | RTLD_LOCAL);
        if (h) break;
    }
    if (!h) return N;
    N.create = (nvrtcCreateProgram_t)dlsym(h, "nvrtcCreateProgram");
    N.compile = (nvrtcCompileProgram_t)dlsym(h, "nvrtcCompileProgram");
    N.log_size = (nvrtcGetSize_t)dlsym(h, "nvrtcGetProgramLogSize");
    N.log = (nvrtcGetData_t)dlsym(h, "nvrtcGetProgramLog");
    N.cubin_size = (nvrtcGetSize_t)dlsym(h, "nvrtcGetCUBINSize");
    N.cubin = (nvrtcGetData_t)dlsym(h, "nvrtcGetCUBIN");
    N.destroy = (nvrtcDestroyProgram_t)dlsym(h, "nvrtcDestroyProgram");
    N.ok = N.create && N.compile && N.log_size && N.log && N.cubin_size && N.cubin && N.destroy;
    return N;
}

struct CacheEntry {
    std::vector<char> cubin;
    std::string error;
    bool done = false;
    std::map<int, void*> kernel;   // per device: cudaKernel_t (libraries load into every context)
    cudaLibrary_t lib = nullptr;
    int smem_set = 0;
};

std::mutex g_cache_mu;
std::map<std::string, CacheEntry*>& cache() {
    static std::map<std::string, CacheEntry*> c;
    return c;
}
std::atomic<long long> g_compiles{0};

bool compile_one(const std::string& src, CacheEntry& ce) {
    Nvrtc& N = nvrtc();
    if (!N.ok) {
        ce.error = "NVRTC not available";
        return false;
    }
    void* prog = nullptr;
    if (N.create(&prog, src.c_str(), "nqs_pass.cu", 0, nullptr, nullptr) != 0) {
        ce.error = "nvrtcCreateProgram failed";
        return false;
    }
    const bool verbose = std::getenv("NQS_JIT_VERBOSE") != nullptr;
    const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", "--ptxas-options=-v"};
    const int rc = N.compile(prog, verbose ? 4 : 3, opts);
    if (verbose && rc == 0) {
        size_t n = 0;
        N.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) N.log(prog, &log[0]);
        std::fprintf(stderr, "nqs jit ptxas: %s\n", log.c_str());
    }
    if (rc != 0) {
        size_t n = 0;
        N.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) N.log(prog, &log[0]);
        ce.error = "nvrtc: " + log.substr(0, 2000);
        N.destroy(&prog);
        return false;
    }
    size_t n = 0;
    N.cubin_size(prog, &n);
    ce.cubin.resize(n);
    N.cubin(prog, ce.cubin.data());
    N.destroy(&prog);
    ++g_compiles;
    return true;
}

}  // namespace

std::string jit_source(const JitPass& p) {
    Gen g(p);
    return g.generate();
}

bool jit_available() { return nvrtc().ok; }

long long jit_compile_count() { return g_compiles.load(); }

int jit_compile(std::vector<JitPass*>& passes, std::string* error) {
    // distinct sources, compiled in parallel
    std::vector<std::pair<std::string, CacheEntry*>> todo;
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        for (JitPass* p : passes) {
            p->source = jit_source(*p);
            auto it = cache().find(p->source);
            if (it == cache().end()) {
                CacheEntry* ce = new CacheEntry();
                cache()[p->source] = ce;
                todo.push_back({p->source, ce});
            }
        }
    }
    if (!todo.empty()) {
        unsigned hw = std::thread::hardware_concurrency();
        const int nthr = (int)std::max(1u, std::min<unsigned>(hw ? hw : 4, (unsigned)todo.size()));
        std::atomic<size_t> next{0};
        std::vector<std::thread> th;
        for (int k = 0; k < nthr; ++k)
            th.emplace_back([&]() {
                for (;;) {
                    const size_t i = next++;
                    if (i >= todo.size()) break;
                    compile_one(todo[i].first, *todo[i].second);
                    todo[i].second->done = true;
                }
            });
        for (auto& t : th) t.join();
    }
    std::lock_guard<std::mutex> g(g_cache_mu);
    for (JitPass* p : passes) {
        CacheEntry* ce = cache()[p->source];
        if (ce->cubin.empty()) {
            if (error) *error = ce->error;
            return -1;
        }
    }
    return 0;
}

int jit_build(std::vector<JitPass*>& passes, std::string* error) {
    if (jit_compile(passes, error) != 0) return -1;
    std::lock_guard<std::mutex> g(g_cache_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        if (error) *error = "no CUDA device";
        return -1;
    }
    for (JitPass* p : passes) {
        CacheEntry* ce = cache()[p->source];
        if (!ce->lib) {
            if (cudaLibraryLoadData(&ce->lib, ce->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) !=
                cudaSuccess) {
                if (error) *error = "cudaLibraryLoadData failed";
                return -1;
            }
        }
        if (!ce->kernel.count(dev)) {
            cudaKernel_t k = nullptr;
            if (cudaLibraryGetKernel(&k, ce->lib, "nqs_pass") != cudaSuccess) {
                if (error) *error = "cudaLibraryGetKernel failed";
                return -1;
            }
            ce->kernel[dev] = (void*)k;
        }
        const size_t smem = p->smem_bytes();
        if (cudaFuncSetAttribute((const void*)ce->kernel[dev], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess) {
            if (error) *error = "cudaFuncSetAttribute failed";
            return -1;
        }
        p->kernel = ce->kernel[dev];
    }
    return 0;
}

size_t JitPass::smem_bytes() const {
    const int NT = (1 << k) >> RB, NW = NT / 32;
    // one state in registers: a ring of db staging tiles and one re-layout
    // tile; otherwise a staging and a re-layout tile per state
    const bool one = S == 1 || seq;
    const size_t tiles = one ? (size_t)std::max(1, std::min(2, db)) + (pp ? 2 : 1) : (size_t)2 * S;
    return tiles * ((size_t)8 << k) + (size_t)n_events * S * NW * 8 * sizeof(double);
}

cudaError_t jit_launch(const JitPass& p, int grid, const PassArgs& a, cudaStream_t st) {
    JitArgsHost j{};
    for (int s = 0; s < 3; ++s) {
        j.in[s] = a.in[s];
        j.out[s] = a.out[s];
    }
    j.ckpt = a.ckpt;
    j.ckpt_fwd = a.ckpt_fwd;
    for (int i = 0; i < 9; ++i) j.spawn[i] = a.spawn[i];
    j.partials = a.partials;
    j.err = a.err;
    j.n_tiles = a.n_tiles;
    void* args[] = {&j};
    return cudaLaunchKernel((const void*)p.kernel, dim3(grid), dim3((1 << p.k) >> p.RB), args, p.smem_bytes(), st);
}

}  // namespace nqs
