// Sweep engine: complex64 state-vector passes on sm_103a and the schedule
// that turns them into the level-l expansion of Algorithm 1 (Sec. IV).
//
// Every kept term of the expansion is X = |<v| C[K_sigma] |psi>|^2, where
// C[K_sigma] is the noiseless gate sequence with the 2x2 factor K_{sigma_s}
// inserted at each noise site s (K_0 = dominant factor).  Instead of one
// contraction per term, the engine
//   1. sweeps v backwards (adjoint operations, K_0^dagger at sites) and stores
//      phi_s = (operations after site s)^dagger |v> at every site;
//   2. sweeps psi forwards; at site s the state is chi_s and the 2x2 reduced
//      matrix R_s[a][b] = sum_rest conj(phi_s[rest,a]) chi_s[rest,b] gives
//      every level-1 amplitude <phi_s| K_i |chi_s> = sum_ab K_i[a][b] R_s[a][b]
//      (and, with K_0, the level-0 amplitude);
//   3. for level >= 2 spawns w_i = K_i chi_s at each site and re-sweeps the
//      three branch states from there, reducing against phi_t at every later
//      site t, recursing depth first up to the level.
// A pass holds 2^k amplitudes of each state in shared memory (the tile's
// qubits are the low c qubits plus those the pass acts on), applies a run of
// fused operations and writes the tile back; site operations inside a pass
// read phi_t straight from HBM, write checkpoints and spawned states, and
// accumulate reductions in FP32 per thread, FP32 per warp (shuffle), then FP64
// per warp slot in shared memory; per-block partials are summed in a fixed
// order by a finisher, so results are bit-reproducible.  Terms are summed
// per level with Neumaier compensation in canonical order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

#include "engine_internal.h"

namespace nqs {


int cuda_err(cudaError_t e) { return e == cudaSuccess ? NQS_OK : NQS_ERR_CUDA; }

// NQS_JIT=0 in the environment turns the automatic choice of pass-specialised kernels off
static bool jit_env_enabled() {
    const char* e = std::getenv("NQS_JIT");
    return !(e && e[0] == '0');
}

// multi-state generated passes sweep their states one at a time (NQS_JIT_SEQ=0:
// all states in registers together)
static bool jit_seq_enabled() {
    const char* e = std::getenv("NQS_JIT_SEQ");
    return !(e && e[0] == '0');
}

// two re-layout buffers in the generated one-state kernels (NQS_JIT_PP=0: one)
static bool jit_pingpong() {
    const char* e = std::getenv("NQS_JIT_PP");
    return !(e && e[0] == '0');
}

// L2 eviction policies of the generated kernels (NQS_JIT_HINT bits, default 3:
// state tiles evict-first, phi kept in L2 until the last state of a tile read it)
static int jit_hint() {
    const char* e = std::getenv("NQS_JIT_HINT");
    return e ? (std::atoi(e) & 3) : 3;
}

// site reduction form of the generated kernels (NQS_JIT_RV=1: conjugate
// multiply-add per product; default 2: split accumulators, no swapped operands)
static int jit_reduction_form() {
    const char* e = std::getenv("NQS_JIT_RV");
    return (e && e[0] == '1') ? 1 : 2;
}

// 13-qubit tiles for the generated kernels (NQS_JIT_WIDE=1)
static bool jit_wide_enabled() {
    const char* e = std::getenv("NQS_JIT_WIDE");
    return e && e[0] == '1';
}

// the handle's plan re-cut into passes of 13-qubit tiles, with the handle's
// segmentation options (the operation order is the same for every tile width)
static void make_wide_plan(const Handle& h, Plan& w) {
    w = h.plan;
    w.k = std::min(h.plan.n, kWideTileQ);
    const int sites = h.opt_max_sites > 0 ? h.opt_max_sites : 4;
    const int ops = h.opt_max_ops > 0 ? h.opt_max_ops : 96;
    w.free_passes = segment(w, false, sites, ops);
    w.sitecut_passes = segment(w, true, sites, ops);
}

// staging buffers of the generated kernels that hold one state in registers
static int jit_staging_buffers() {
    const char* e = std::getenv("NQS_JIT_DB");
    return (e && e[0] == '2') ? 2 : 1;
}



// Program of one register-resident launch, appended to `prog` (16-byte
// words): the phases, one 16-byte record per operation, then the matrices.
// The operations (execution order) are grouped into phases: a phase gathers
// consecutive operations whose dense qubits fit in the RB register qubits;
// diagonal operations never constrain it.  Each phase pads its register set
// with the highest free tile positions, gives lane bits 0-3 to the lowest
// free position of each residue class mod 4 (the bank-pair bits of the
// swizzled 64-bit re-layout buffer), lane bit 4 to the lowest free position
// left and the warp bits to the rest.  Returns the offsets
// (in words) of the operations and matrices and the phase count.


ProgInfo build_program(const std::vector<DevOp>& dops, int off, int n, int RB, const Tables& tab,
                       std::vector<uint4>& prog, int k) {
    const int WB = k - RB - 5;
    std::vector<std::pair<int, int>> ranges;
    std::vector<std::vector<int>> regs;
    std::vector<int> cur;
    int begin = 0;
    for (int o = 0; o < n; ++o) {
        const DevOp& d = dops[off + o];
        std::vector<int> need;
        if (d.type == OP_G1 || d.type == OP_SITE) need.push_back(d.a);
        else if (d.type == OP_G2) {
            need.push_back(d.a);
            need.push_back(d.b);
        }
        std::vector<int> u = cur;
        for (int q : need)
            if (std::find(u.begin(), u.end(), q) == u.end()) u.push_back(q);
        if ((int)u.size() > RB) {
            ranges.push_back({begin, o});
            regs.push_back(cur);
            cur = need;
            begin = o;
        } else {
            cur = u;
        }
    }
    ranges.push_back({begin, n});
    regs.push_back(cur);

    std::vector<DevPhase> phases;
    std::vector<OpRec> recs(n);
    std::vector<float2> mats;
    for (size_t p = 0; p < ranges.size(); ++p) {
        std::vector<int> R = regs[p];
        std::vector<char> used(k, 0);
        for (int q : R) used[q] = 1;
        for (int q = k - 1; q >= 0 && (int)R.size() < RB; --q)
            if (!used[q]) {
                R.push_back(q);
                used[q] = 1;
            }
        std::sort(R.begin(), R.end());
        // lanes 0-3 (a half-warp) on free positions of distinct residue mod 4
        // (conflict-free 64-bit re-layouts, see the kernel's swizzle), lowest
        // first; lane 4 on the lowest free position left
        std::vector<int> lanes;
        bool res_used[4] = {false, false, false, false};
        for (int q = 0; q < k && (int)lanes.size() < 4; ++q)
            if (!used[q] && !res_used[q % 4]) {
                lanes.push_back(q);
                res_used[q % 4] = true;
            }
        for (int q : lanes) used[q] = 1;
        for (int q = 0; q < k && (int)lanes.size() < 5; ++q)
            if (!used[q]) {
                lanes.push_back(q);
                used[q] = 1;
            }
        std::sort(lanes.begin(), lanes.begin() + std::min<size_t>(4, lanes.size()));
        std::vector<int> warps;
        for (int q = 0; q < k; ++q)
            if (!used[q]) warps.push_back(q);
        DevPhase ph{};
        int loc[kTileSlots];
        for (int i = 0; i < RB; ++i) {
            ph.R[i] = (signed char)R[i];
            loc[R[i]] = i;
        }
        for (int i = 0; i < 5; ++i) {
            ph.L[i] = (signed char)lanes[i];
            loc[lanes[i]] = LOC_THREAD + i;
        }
        for (int i = 0; i < WB; ++i) {
            ph.W[i] = (signed char)warps[i];
            loc[warps[i]] = LOC_THREAD + 5 + i;
        }
        ph.op_begin = ranges[p].first;
        ph.op_end = ranges[p].second;
        phases.push_back(ph);
        for (int o = ph.op_begin; o < ph.op_end; ++o) {
            const DevOp& d = dops[off + o];
            OpRec& r = recs[o];
            r = OpRec{};
            r.type = (unsigned char)d.type;
            r.la = (unsigned char)(d.a >= 0 ? loc[d.a] : 0xff);
            r.lb = (unsigned char)(d.b >= 0 ? loc[d.b] : 0xff);
            r.flags = (unsigned char)(d.flags & 0xff);
            r.qa = (unsigned char)(d.qa >= 0 ? d.qa : 0xff);
            r.qb = (unsigned char)(d.qb >= 0 ? d.qb : 0xff);
            r.ev = (unsigned char)((d.flags >> 8) & 0xff);
            r.nspawn = (unsigned char)((d.flags >> 16) & 0xff);
            r.site = (unsigned short)(d.site >= 0 ? d.site : 0);
            int cnt = (d.type == OP_G2 || d.type == OP_D2) ? 16 : 4;
            if (d.type == OP_SITE && (d.flags & FL_SPAWN)) cnt = 16;
            r.mat = (unsigned short)mats.size();
            for (int e = 0; e < cnt; ++e) mats.push_back(tab.mats[d.mat + e]);
        }
    }
    ProgInfo info;
    info.words_begin = (int)prog.size();
    info.n_phases = (int)phases.size();
    static_assert(sizeof(DevPhase) == 32 && sizeof(OpRec) == 16, "program record sizes");
    const uint4* pw = reinterpret_cast<const uint4*>(phases.data());
    prog.insert(prog.end(), pw, pw + 2 * phases.size());
    info.ops_word = (int)prog.size() - info.words_begin;
    const uint4* ow = reinterpret_cast<const uint4*>(recs.data());
    prog.insert(prog.end(), ow, ow + recs.size());
    info.mats_word = (int)prog.size() - info.words_begin;
    if (mats.size() & 1) mats.push_back(make_float2(0.f, 0.f));
    const uint4* mw = reinterpret_cast<const uint4*>(mats.data());
    prog.insert(prog.end(), mw, mw + mats.size() / 2);
    info.n_words = (int)prog.size() - info.words_begin;
    return info;
}

Run make_run(const Plan& plan, const std::vector<PassSpec>& segs, RunType rt, bool reduce, bool spawn,
             bool level0_only, const std::vector<Factors>& fac, Tables& tab, std::vector<DevOp>& dops,
             const std::vector<char>* save_only) {
    Run run;
    std::vector<int> fwd_mat(plan.ops.size(), -1), bwd_mat(plan.ops.size(), -1);
    for (size_t i = 0; i < plan.ops.size(); ++i) {
        const HostOp& o = plan.ops[i];
        int dim = (o.type == OP_G2 || o.type == OP_D2) ? 4 : 2;
        if (rt == RT_BWD) {
            bwd_mat[i] = tab.add(o.m.data(), dim * dim, true, dim);
        } else if (o.type == OP_SITE) {
            // K_0 followed by the kept non-dominant factors
            fwd_mat[i] = tab.add(o.m.data(), 4, false, 2);
            const Factors& f = fac[o.site];
            for (int j = 0; j < 3; ++j) {
                Mat2 z{};
                const Mat2& K = (j < f.m) ? f.K[f.keep[j]] : z;
                tab.add(K.data(), 4, false, 2);
            }
        } else {
            fwd_mat[i] = tab.add(o.m.data(), dim * dim, false, dim);
        }
    }
    int first_site_done = 0;
    auto build_pass = [&](const PassSpec& ps, bool reversed) {
        RunPass rp;
        rp.k = plan.k;
        rp.c = plan.c;
        std::vector<int> pos(plan.n, -1);
        for (int j = 0; j < plan.k; ++j) {
            rp.local[j] = ps.local[j];
            pos[ps.local[j]] = j;
        }
        int nl = 0;
        for (int q = 0; q < plan.n; ++q)
            if (pos[q] < 0) rp.nonlocal[nl++] = q;
        rp.op_off = (int)dops.size();
        auto emit = [&](int i) {
            const HostOp& o = plan.ops[i];
            DevOp d{};
            d.type = o.type;
            d.qa = o.q0;
            d.qb = o.q1;
            d.a = o.q0 >= 0 ? pos[o.q0] : -1;
            d.b = o.q1 >= 0 ? pos[o.q1] : -1;
            d.site = o.site;
            d.mat = (rt == RT_BWD) ? bwd_mat[i] : fwd_mat[i];
            if (o.type == OP_SITE) {
                int fl = 0;
                if (rt == RT_IDEAL) {
                    return;   // noiseless sweep: sites are absent
                } else if (rt == RT_BWD) {
                    fl = FL_APPLY | ((!save_only || (*save_only)[o.site]) ? FL_SAVE : 0);
                } else {
                    fl = FL_APPLY;
                    bool red = reduce && (!level0_only || first_site_done == 0);
                    if (red) {
                        fl |= FL_REDUCE | ((int)rp.ev_site.size() << 8);
                        rp.ev_site.push_back(o.site);
                    }
                    if (spawn && fac[o.site].m > 0) {
                        fl |= FL_SPAWN | (fac[o.site].m << 16);
                        rp.spawn_site = o.site;
                    }
                    first_site_done = 1;
                }
                if (o.diag) fl |= FL_KDIAG;
                d.flags = fl;
            }
            dops.push_back(d);
            rp.lin.push_back(i);
        };
        if (!reversed)
            for (int i = ps.op_begin; i < ps.op_end; ++i) emit(i);
        else
            for (int i = ps.op_end - 1; i >= ps.op_begin; --i) emit(i);
        rp.n_ops = (int)dops.size() - rp.op_off;
        return rp;
    };
    if (rt == RT_BWD) {
        for (int p = (int)segs.size() - 1; p >= 0; --p) run.passes.push_back(build_pass(segs[p], true));
    } else {
        for (const auto& ps : segs) run.passes.push_back(build_pass(ps, false));
    }
    return run;
}

// ------------------------------------------------------------------ schedule
namespace {

struct Builder {
    Handle& h;
    Engine& E;
    const Plan& plan;
    int level;
    TermIndex ti;
    Tables tab;
    std::vector<DevOp> dops;
    std::vector<uint4> prog;          // programs of the register-resident launches
    bool too_big = false;             // a launch would not fit in shared memory
    bool rt = false;                  // register-resident kernel (tile of exactly 12 qubits)
    bool use_jit = false;             // passes will get pass-specialised kernels
    std::vector<FinishDesc> descs;
    std::vector<Launch> L;
    size_t partial_doubles = 0;
    long long dim;
    // device buffers (resolved after allocation)
    float2* main_buf = nullptr;
    float2* work_buf = nullptr;                     // spaced checkpoints: block recomputation
    std::vector<float2*> phi;                       // checkpoint table (spaced: ring per site, then boundary per site)
    std::vector<float2*> bd;                        // spaced checkpoints: phi at the last site of each block
    std::vector<std::vector<float2*>> group_bufs;   // per depth (1..level-1)
    float2** ckpt_dev = nullptr;
    Run run_ideal, run_bwd, run_mat;   // run_mat: per-block phi recomputation (spaced checkpoints)
    std::vector<Run> run_fwd;    // per depth

    Builder(Handle& hh, Engine& ee, int lvl, const Plan& pl) : h(hh), E(ee), plan(pl), level(lvl) {
        dim = 1ll << plan.n;
        const int N = (int)hh.factors.size();
        if (N > 0) {
            first_site_pos = plan.site_pos[0];
            last_site_pos = plan.site_pos[lvl == 0 ? 0 : N - 1];
        }
    }

    // Sweeps need nothing outside [first site, last reducing site]: the
    // backward sweep stops once phi of the first site is saved, forward and
    // branch sweeps once the last site that reduces or spawns is passed.
    // Passes lying entirely outside that range are skipped.
    int first_site_pos = -1;
    int last_site_pos = 1 << 30;
    bool before_first(const RunPass& rp) const {
        if (rp.lin.empty()) return false;
        return *std::max_element(rp.lin.begin(), rp.lin.end()) < first_site_pos;
    }
    bool after_last(const RunPass& rp) const {
        if (rp.lin.empty()) return false;
        return *std::min_element(rp.lin.begin(), rp.lin.end()) > last_site_pos;
    }

    int grid_for(int S, int RB, long long tiles, int prog_words, int n_events) {
        int per_sm;
        if (rt) {
            per_sm = sweep_blocks_per_sm(S, RB, sweep_smem_bytes(S, RB, prog_words, n_events));
        } else {
            size_t smem = (size_t)S * (1 << plan.k) * sizeof(float2);
            per_sm = tile_pass_blocks_per_sm(S, smem);
        }
        long long g = (long long)per_sm * E.sm_count;
        return (int)std::max<long long>(1, std::min<long long>(g, tiles));
    }

    PassArgs pass_args(const RunPass& rp, int start, int S) {
        PassArgs a{};
        a.ops = nullptr;
        a.n_ops = rp.n_ops - start;
        a.mats = nullptr;
        a.n = plan.n;
        a.k = rp.k;
        a.c = rp.c;
        a.n_events = (int)rp.ev_site.size();
        for (int j = 0; j < kTileSlots; ++j) a.local[j] = rp.local[j];
        for (int j = 0; j < kMaxQ; ++j) a.nonlocal[j] = rp.nonlocal[j];
        a.n_tiles = 1ll << (plan.n - rp.k);
        a.ckpt = ckpt_dev;
        return a;
    }

    void add_pass(const RunPass& rp, int start, int S, const float2* const* in, float2* const* out,
                  float2* const* spawn, int n_spawn) {
        if (rp.n_ops - start <= 0 && in[0] == out[0]) return;
        Launch l;
        l.kind = L_PASS;
        l.S = S;
        l.args = pass_args(rp, start, S);
        l.op_index = rp.op_off + start;
        l.rt = rt;
        if (rt) {
            // pass-specialised multi-state passes hold 16 amplitudes per state and
            // thread (more work per instruction stream, registers for early phi loads)
            l.rb = plan.k == kWideTileQ ? 4
                   : (S > 1 && h.opt_rb_multi) ? h.opt_rb_multi : (S > 1 && use_jit) ? 4 : sweep_reg_bits(S);
            ProgInfo pi = build_program(dops, rp.op_off + start, rp.n_ops - start, l.rb, tab, prog, plan.k);
            l.prog_index = pi.words_begin;
            l.args.prog_words = pi.n_words;
            l.args.ops_word = pi.ops_word;
            l.args.mats_word = pi.mats_word;
            l.args.n_phases = pi.n_phases;
            // static shared memory of the kernel stays below 4 KiB (13-qubit tiles:
            // staging and two re-layout tiles of 64 KiB and the reduction slots)
            if (plan.k == kWideTileQ) {
                if ((size_t)3 * (8 << kWideTileQ) + (size_t)l.args.n_events * S * 16 * 64 + 4096 > E.smem_optin)
                    too_big = true;
            } else if (sweep_smem_bytes(S, l.rb, pi.n_words, l.args.n_events) + 4096 > E.smem_optin) {
                too_big = true;
            }
        }
        for (int s = 0; s < S; ++s) {
            l.args.in[s] = in[s];
            l.args.out[s] = out[s];
        }
        for (int i = 0; i < n_spawn; ++i) l.args.spawn[i] = spawn[i];
        l.seq = rt && use_jit && S > 1 && (jit_seq_enabled() || plan.k == kWideTileQ);
        // state-sequential generated passes: two 256-thread blocks per SM (13-qubit
        // tiles: one 512-thread block)
        const long long per_sm = plan.k == kWideTileQ ? 1 : jit_blocks_per_sm();
        l.grid = (l.seq || (rt && use_jit && S == 1))
                     ? (int)std::max<long long>(1, std::min<long long>(per_sm * E.sm_count, l.args.n_tiles))
                     : grid_for(S, l.rb, l.args.n_tiles, l.args.prog_words, l.args.n_events);
        l.smem = (size_t)S * (1 << plan.k) * sizeof(float2);
        partial_doubles = std::max(partial_doubles, (size_t)std::max(1, l.args.n_events) * S * l.grid * 8);
        // algorithmic bytes: state load + store, phi reads, checkpoint and spawn writes
        double b = 16.0 * dim * S;
        int n_red = 0, n_save = 0, n_sp = 0;
        for (int o = start; o < rp.n_ops; ++o) {
            const DevOp& d = dops[rp.op_off + o];
            if (d.type >= OP_G1 && d.type <= OP_SITE) ++l.op_counts[d.type - OP_G1];
            if (d.type != OP_SITE) continue;
            if (d.flags & FL_REDUCE) ++n_red;
            if (d.flags & FL_SAVE) ++n_save;
            if (d.flags & FL_SPAWN) n_sp += (d.flags >> 16) & 0xff;
        }
        b += 8.0 * dim * (n_red + n_save + (double)n_sp * S);
        l.bytes = b;
        l.op_counts[5] = n_red;
        l.op_counts[6] = n_sp * S;
        l.op_counts[7] = n_save;
        L.push_back(l);
    }

    // finisher for the last pass launch: slot (event e, state s) -> term ranks
    template <typename RankFn>
    void add_finish(const RunPass& rp, int start, int S, RankFn rank_of) {
        const Launch& pl = L.back();
        int n_ev = (int)rp.ev_site.size();
        if (n_ev == 0) return;
        // events executed in this launch
        std::vector<char> executed(n_ev, 0);
        for (int o = start; o < rp.n_ops; ++o) {
            const DevOp& d = dops[rp.op_off + o];
            if (d.type == OP_SITE && (d.flags & FL_REDUCE)) executed[(d.flags >> 8) & 0xff] = 1;
        }
        Launch f;
        f.kind = L_FINISH;
        f.n_red = n_ev * S;
        f.fin_grid = pl.grid;
        f.desc_off = descs.size();
        for (int e = 0; e < n_ev; ++e)
            for (int s = 0; s < S; ++s)
                for (int i = 0; i < 4; ++i) {
                    FinishDesc d{-1, 0, 0};
                    if (executed[e]) rank_of(rp.ev_site[e], s, i, d);
                    descs.push_back(d);
                }
        L.push_back(f);
    }

    int kmat_off(int site, int factor) { return site * 32 + factor * 8; }

    // Group of S sibling states spawned at site `s_last` (state s carries the
    // s-th kept factor there); `prefix` holds the earlier insertions.  The
    // group sweeps from the operation after the site to the end of the
    // circuit, reducing against phi_t at every later site t; when the level
    // allows, it spawns children at each site into the next depth's buffers
    // (3 per state) and recurses depth first.
    void dfs_group(int depth, const std::vector<std::pair<int, int>>& prefix, int s_last, int S,
                   const std::vector<float2*>& bufs) {
        const Run& run = run_fwd[depth];
        int pos = plan.site_pos[s_last];
        int pi = -1, start = 0;
        for (size_t p = 0; p < run.passes.size() && pi < 0; ++p) {
            const RunPass& rp = run.passes[p];
            for (int o = 0; o < rp.n_ops; ++o)
                if (rp.lin[o] > pos) {
                    pi = (int)p;
                    start = o;
                    break;
                }
        }
        if (pi < 0) {
            // nothing after the site: the branch states are final, nothing to reduce
            return;
        }
        const bool can_spawn = depth + 1 < (int)group_bufs.size();
        for (size_t p = pi; p < run.passes.size(); ++p) {
            const RunPass& rp = run.passes[p];
            if (after_last(rp)) break;
            int st = (p == (size_t)pi) ? start : 0;
            bool spawns = can_spawn && rp.spawn_site >= 0 && rp.lin.size() > 0;
            // a spawn before `st` (partial first pass) does not execute
            if (spawns) {
                int sp_pos = plan.site_pos[rp.spawn_site];
                if (sp_pos <= pos) spawns = false;
            }
            std::vector<float2*> child;
            if (spawns)
                for (int i = 0; i < S * 3; ++i) child.push_back(group_bufs[depth + 1][i]);
            add_pass(rp, st, S, (const float2* const*)bufs.data(), bufs.data(),
                     child.empty() ? nullptr : child.data(), (int)child.size());
            add_finish(rp, st, S, [&](int t, int s, int i, FinishDesc& d) {
                const Factors& ft = h.factors[t];
                if (i == 0 || i > ft.m || depth + 1 > level) return;
                std::vector<std::pair<int, int>> terms = prefix;
                terms.push_back({s_last, s});
                terms.push_back({t, i - 1});
                std::sort(terms.begin(), terms.end());
                int sites[NQS_MAX_LEVEL + 1], fp[NQS_MAX_LEVEL + 1];
                for (size_t j = 0; j < terms.size(); ++j) {
                    sites[j] = terms[j].first;
                    fp[j] = terms[j].second;
                }
                d.rank = (long long)ti.rank((int)terms.size(), sites, fp);
                d.kmat = kmat_off(t, ft.keep[i - 1]);
            });
            if (spawns) {
                int t = rp.spawn_site;
                for (int s = 0; s < S; ++s) {
                    std::vector<std::pair<int, int>> pre = prefix;
                    pre.push_back({s_last, s});
                    std::vector<float2*> cb(group_bufs[depth + 1].begin() + 3 * s,
                                            group_bufs[depth + 1].begin() + 3 * s + 3);
                    dfs_group(depth + 1, pre, t, h.factors[t].m, cb);
                }
            }
        }
    }

    // ---- spaced checkpoints --------------------------------------------
    // Block c holds the operations after the last site of block c-1 up to
    // the last site of block c; the operations after the last site form
    // block nb, which no forward sweep needs.
    int block_of_op(int op, int k) const {
        const int N = (int)h.factors.size();
        const int nb = (N + k - 1) / k;
        for (int c = 0; c < nb; ++c)
            if (op <= plan.site_pos[std::min(N, (c + 1) * k) - 1]) return c;
        return nb;
    }

    std::vector<int> blocks_of(const Run& run, int k) const {
        const int N = (int)h.factors.size();
        std::vector<int> b(run.passes.size());
        for (size_t p = 0; p < run.passes.size(); ++p)
            b[p] = run.passes[p].lin.empty() ? (N + k - 1) / k : block_of_op(run.passes[p].lin[0], k);
        return b;
    }

    // The group of states spawned at site s sweeps through block c, reducing
    // against the block's recomputed phi (level 2).
    void group_block(int s, int c, int k, const std::vector<int>& blk) {
        const Run& run = run_fwd[1];
        const int pos = plan.site_pos[s];
        const int S = h.factors[s].m;
        if (S == 0) return;
        float2* bufs[3] = {group_bufs[1][3 * (s % k)], group_bufs[1][3 * (s % k) + 1], group_bufs[1][3 * (s % k) + 2]};
        for (size_t p = 0; p < run.passes.size(); ++p) {
            if (blk[p] != c) continue;
            const RunPass& rp = run.passes[p];
            int st = 0;
            while (st < rp.n_ops && rp.lin[st] <= pos) ++st;
            if (st >= rp.n_ops) continue;
            add_pass(rp, st, S, (const float2* const*)bufs, bufs, nullptr, 0);
            add_finish(rp, st, S, [&](int t, int si, int i, FinishDesc& d) {
                const Factors& ft = h.factors[t];
                if (i == 0 || i > ft.m) return;
                int sites[2] = {s, t}, fp[2] = {si, i - 1};
                d.rank = (long long)ti.rank(2, sites, fp);
                d.kmat = kmat_off(t, ft.keep[i - 1]);
            });
        }
    }

    // Forward part of a spaced schedule.  For every block b: recompute the
    // block's phi from its boundary, sweep the main state through the block
    // (level-0/1 reductions, spawning three states per site), then sweep the
    // block's spawned groups through every later block, recomputing each
    // block's phi once for all of them.
    template <typename RankFn, typename OwnFn>
    void spaced_forward(int k, const float2* ext, RankFn main_rank, OwnFn owns_group) {
        const int N = (int)h.factors.size();
        const int nb = (N + k - 1) / k;
        const Run& fwd0 = run_fwd[0];
        const bool groups = level >= 2;
        const std::vector<int> b0 = blocks_of(fwd0, k), bm = blocks_of(run_mat, k);
        const std::vector<int> b1 = groups ? blocks_of(run_fwd[1], k) : std::vector<int>();
        int ring_block = -1;
        auto materialize = [&](int c) {
            if (ring_block == c) return;
            bool first_in = true;
            for (size_t p = 0; p < run_mat.passes.size(); ++p) {
                if (bm[p] != c || before_first(run_mat.passes[p])) continue;
                const float2* in[1] = {first_in ? bd[c] : work_buf};
                float2* out[1] = {work_buf};
                add_pass(run_mat.passes[p], 0, 1, in, out, nullptr, 0);
                first_in = false;
            }
            ring_block = c;
        };
        bool first = true;
        for (int b = 0; b < nb; ++b) {
            materialize(b);
            for (size_t p = 0; p < fwd0.passes.size(); ++p) {
                if (b0[p] != b) continue;
                const RunPass& rp = fwd0.passes[p];
                const float2* in[1] = {(first && ext) ? ext : main_buf};
                float2* out[1] = {main_buf};
                first = false;
                float2* sp[3];
                int n_sp = 0;
                if (groups && rp.spawn_site >= 0)
                    for (int i = 0; i < 3; ++i) sp[n_sp++] = group_bufs[1][3 * (rp.spawn_site % k) + i];
                add_pass(rp, 0, 1, in, out, n_sp ? sp : nullptr, n_sp);
                add_finish(rp, 0, 1, main_rank);
            }
            if (!groups) continue;
            const int s_lo = b * k, s_hi = std::min(N, (b + 1) * k);
            for (int c = b; c < nb; ++c) {
                materialize(c);
                for (int s = s_lo; s < s_hi; ++s)
                    if (owns_group(s)) group_block(s, c, k, b1);
            }
        }
    }
};

}  // namespace

int engine_init(Engine& E) {
    if (E.device >= 0) return NQS_OK;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return NQS_ERR_CUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return NQS_ERR_CUDA;
    E.device = dev;
    E.sm_count = prop.multiProcessorCount;
    E.smem_optin = prop.sharedMemPerBlockOptin;
    return NQS_OK;
}

void engine_release(Engine& E, void* stream) {
    if (E.buf) dev_free(E.buf, E.buf_bytes, stream);
    if (E.aux) dev_free(E.aux, E.aux_bytes, stream);
    E.buf = E.aux = nullptr;
    E.buf_bytes = E.aux_bytes = 0;
    E.level = -1;
    E.launches.clear();
    E.jit.clear();
    E.jit_launches = 0;
    E.jit_state = 0;
}

// States held by a schedule that keeps phi every `k` sites: the block
// boundaries, the ring of one block, main, the recomputation buffer and, at
// level 2, three spawned states per site of a block.
static size_t spaced_states(int N, int level, int k) {
    return (size_t)((N + k - 1) / k) + (size_t)k + 2 + (level >= 2 ? 3 * (size_t)k : 0);
}

// The block size with the fewest states.
static int best_spacing(int N, int level) {
    int best = 1;
    size_t fewest = spaced_states(N, level, 1);
    for (int k = 2; k < N; ++k) {
        const size_t st = spaced_states(N, level, k);
        if (st < fewest) {
            fewest = st;
            best = k;
        }
    }
    return best;
}

// Build (or reuse) the schedule for this level and state kinds.
int build_schedule(Handle& h, Engine& E, const nqs_state* psi, const nqs_state* v, int level, void* stream,
                   bool allow_jit) {
    const int N = (int)h.factors.size();
    // automatic: circuits of 26 qubits or more, where one call's sweeps outlast
    // the compilation of its distinct passes
    const bool want_jit =
        allow_jit && (h.opt_jit == 1 || (h.opt_jit == 0 && h.plan.n >= 26 && jit_env_enabled()));
    if (E.level == level && E.psi_kind == psi->kind && E.v_kind == v->kind && E.psi_bits == psi->bits &&
        E.v_bits == v->bits && E.psi_dev == psi->dev && E.v_dev == v->dev && !(want_jit && E.jit_state == 0))
        return NQS_OK;
    engine_release(E, stream);
    ++E.gen;

    // generated kernels may sweep 13-qubit tiles (fewer passes); if their
    // kernels cannot be built the schedule is rebuilt for 12-qubit tiles
    E.wide = want_jit && !E.wide_failed && h.plan.k == kMaxTileQ && h.plan.n > kWideTileQ && jit_wide_enabled() &&
             jit_available();
    if (E.wide) make_wide_plan(h, E.wide_plan);
    const Plan& plan = E.wide ? E.wide_plan : h.plan;
    Builder B(h, E, level, plan);
    std::vector<int> m(N);
    for (int s = 0; s < N; ++s) m[s] = h.factors[s].m;
    B.ti.build(m, level);

    B.rt = plan.k == kMaxTileQ || E.wide;
    B.use_jit = want_jit && B.rt && jit_available();
    if (want_jit && B.rt && !B.use_jit) E.jit_state = -1;   // NVRTC missing: the interpreting kernel runs
    // finisher factor table (complex128)
    B.tab.kmats.assign((size_t)std::max(N, 1) * 32, 0.0);
    for (int s = 0; s < N; ++s)
        for (int i = 0; i < 4; ++i)
            for (int e = 0; e < 4; ++e) {
                B.tab.kmats[s * 32 + i * 8 + 2 * e] = h.factors[s].K[i][e].real();
                B.tab.kmats[s * 32 + i * 8 + 2 * e + 1] = h.factors[s].K[i][e].imag();
            }
    if (N == 0) {   // identity "factor" for the plain inner product
        B.tab.kmats[0] = 1.0;
        B.tab.kmats[6] = 1.0;
    }

    // state buffers.  Every site keeps its phi when the states fit (or the
    // option asks for it): phi slots, main, group buffers (3 at depth 1, 9
    // deeper).  Otherwise (levels <= 2) phi is kept only at the last site of
    // each block of `spacing` sites and a block's phi are recomputed into a
    // ring of `spacing` slots whenever a sweep enters the block.
    const size_t sbytes = (size_t)B.dim * sizeof(float2);
    int n_phi = std::max(N, 1);
    int n_group = 0;
    for (int d = 1; d < level; ++d) n_group += (d == 1) ? 3 : 9;
    int spacing = 0;
    if (h.opt_spacing > 0 && h.opt_spacing < N) {
        if (level > 2) return NQS_ERR_UNSUPPORTED;
        spacing = h.opt_spacing;
    }
    size_t n_states = (size_t)n_phi + 1 + n_group;
    if (spacing == 0) {
        E.buf_bytes = n_states * sbytes;
        E.buf = dev_alloc(E.buf_bytes, stream);
        if (!E.buf) {
            E.buf_bytes = 0;
            if (h.opt_spacing != 0 || level > 2 || N < 2) return NQS_ERR_NOMEM;
            spacing = best_spacing(N, level);
        }
    }
    if (spacing > 0) {
        n_states = spaced_states(N, level, spacing);
        E.buf_bytes = n_states * sbytes;
        E.buf = dev_alloc(E.buf_bytes, stream);
        if (!E.buf) {
            E.buf_bytes = 0;
            return NQS_ERR_NOMEM;
        }
    }
    E.spacing = spacing;
    E.n_states = n_states;
    float2* base = (float2*)E.buf;
    B.group_bufs.assign(std::max(1, level), {});
    if (spacing == 0) {
        for (int s = 0; s < n_phi; ++s) B.phi.push_back(base + (size_t)s * B.dim);
        B.main_buf = base + (size_t)n_phi * B.dim;
        size_t next = (size_t)n_phi + 1;
        for (int d = 1; d < level; ++d) {
            int cnt = (d == 1) ? 3 : 9;
            for (int i = 0; i < cnt; ++i) B.group_bufs[d].push_back(base + (next++) * B.dim);
        }
    } else {
        const int nb = (N + spacing - 1) / spacing;
        size_t next = 0;
        std::vector<float2*> ring, bd;
        for (int b = 0; b < nb; ++b) bd.push_back(base + (next++) * B.dim);
        for (int j = 0; j < spacing; ++j) ring.push_back(base + (next++) * B.dim);
        B.main_buf = base + (next++) * B.dim;
        B.work_buf = base + (next++) * B.dim;
        if (level >= 2)
            for (int i = 0; i < 3 * spacing; ++i) B.group_bufs[1].push_back(base + (next++) * B.dim);
        for (int s = 0; s < N; ++s) B.phi.push_back(ring[s % spacing]);
        for (int s = 0; s < N; ++s) B.phi.push_back(bd[s / spacing]);
        B.bd = bd;
    }

    // runs: the register-resident kernel needs a tile of exactly 12 qubits
    bool need_ideal = v->kind == NQS_STATE_IDEAL;
    if (need_ideal) B.run_ideal = make_run(plan, plan.free_passes, RT_IDEAL, false, false, false, h.factors, B.tab, B.dops);
    std::vector<char> block_last;
    std::vector<PassSpec> spaced_free;
    if (spacing == 0) {
        if (N > 0) B.run_bwd = make_run(plan, plan.free_passes, RT_BWD, false, false, false, h.factors, B.tab, B.dops);
        // forward runs per depth d: reduce if d+1 <= level (or level 0 at depth 0), spawn if d+2 <= level
        int depths = std::max(1, level);
        for (int d = 0; d < depths; ++d) {
            bool spawn = d + 2 <= level;
            bool reduce = (level == 0) ? (d == 0) : (d + 1 <= level);
            B.run_fwd.push_back(make_run(plan, spawn ? plan.sitecut_passes : plan.free_passes, RT_FWD,
                                         reduce && N > 0, spawn, level == 0, h.factors, B.tab, B.dops));
        }
    } else {
        block_last.assign(N, 0);
        for (int s = 0; s < N; ++s) block_last[s] = ((s + 1) % spacing == 0) || s == N - 1;
        spaced_free = segment(plan, false, h.opt_max_sites > 0 ? h.opt_max_sites : 4,
                              h.opt_max_ops > 0 ? h.opt_max_ops : 96, &block_last);
        // backward: boundary phi only, and the per-block recomputation (every site)
        B.run_bwd = make_run(plan, spaced_free, RT_BWD, false, false, false, h.factors, B.tab, B.dops, &block_last);
        B.run_mat = make_run(plan, spaced_free, RT_BWD, false, false, false, h.factors, B.tab, B.dops);
        const bool spawn = level >= 2;
        B.run_fwd.push_back(make_run(plan, spawn ? plan.sitecut_passes : spaced_free, RT_FWD, true, spawn,
                                     level == 0, h.factors, B.tab, B.dops));
        if (level >= 2)
            B.run_fwd.push_back(make_run(plan, spaced_free, RT_FWD, true, false, false, h.factors, B.tab, B.dops));
    }

    // --- schedule (device pointers to aux tables are patched after layout) ---
    B.ckpt_dev = nullptr;
    float2* mainb = B.main_buf;
    const float2* in1[3];
    float2* out1[3];

    auto init_state = [&](const nqs_state* st, float2* dst, bool& external, const float2*& ext) {
        external = false;
        if (st->kind == NQS_STATE_BASIS) {
            Launch l;
            l.kind = L_FILL;
            l.dst = dst;
            l.bits = st->bits;
            B.L.push_back(l);
        } else {
            external = true;
            ext = (const float2*)st->dev;
        }
    };

    // 1. v (into main), optionally the ideal sweep, then the backward sweep
    {
        bool ext = false;
        const float2* ext_ptr = nullptr;
        if (v->kind == NQS_STATE_IDEAL) {
            bool pe = false;
            const float2* pp = nullptr;
            init_state(psi, mainb, pe, pp);
            for (size_t p = 0; p < B.run_ideal.passes.size(); ++p) {
                in1[0] = (p == 0 && pe) ? pp : mainb;
                out1[0] = mainb;
                B.add_pass(B.run_ideal.passes[p], 0, 1, in1, out1, nullptr, 0);
            }
            if (B.run_ideal.passes.empty() && pe) {
                Launch l;
                l.kind = L_COPY;
                l.dst = mainb;
                l.src = pp;
                B.L.push_back(l);
            }
            if (psi->kind == NQS_STATE_BASIS && !B.run_ideal.passes.empty()) {
                // U|psi> has the norm of the basis state, 1: restore it (the
                // complex64 gates lose a little; v enters every term twice)
                Launch r;
                r.kind = L_REDUCE2;
                r.src = mainb;
                r.dst = mainb;
                r.bits = 0;
                r.grid = std::max(1, std::min<int>(E.sm_count * 4, (int)std::max<long long>(1, B.dim / (2 * kThreads * 16))));
                B.partial_doubles = std::max(B.partial_doubles, (size_t)r.grid * 8);
                B.L.push_back(r);
                Launch nl;
                nl.kind = L_NORMALIZE;
                nl.dst = mainb;
                nl.fin_grid = r.grid;
                B.L.push_back(nl);
            }
        } else {
            init_state(v, mainb, ext, ext_ptr);
        }
        if (N > 0) {
            for (size_t p = 0; p < B.run_bwd.passes.size(); ++p) {
                if (p > 0 && B.before_first(B.run_bwd.passes[p])) break;
                in1[0] = (p == 0 && ext) ? ext_ptr : mainb;
                out1[0] = mainb;
                B.add_pass(B.run_bwd.passes[p], 0, 1, in1, out1, nullptr, 0);
                if (spacing > 0) B.L.back().bd_table = true;
            }
        } else {
            // N = 0: keep v in the single phi slot for the final inner product
            Launch l;
            l.kind = L_COPY;
            l.dst = B.phi[0];
            l.src = ext ? ext_ptr : mainb;
            B.L.push_back(l);
        }
    }
    // finisher ranks of the main forward sweep: level 0 at the first site, level 1 everywhere
    bool first_red = true;
    // sharding of one call's terms: levels 0 and 1 belong to shard 0, a branch
    // group (and every deeper term below it) to shard (first site mod count)
    const int shard_count = std::max(1, h.opt_shard_count), shard_rank = h.opt_shard_rank;
    auto owns_group = [&](int s) { return s % shard_count == shard_rank; };
    auto main_rank = [&](int t, int s, int i, FinishDesc& d) {
        (void)s;
        if (shard_rank != 0) return;
        const Factors& ft = h.factors[t];
        if (i == 0) {
            if (first_red) {
                d.rank = 0;
                d.kmat = B.kmat_off(t, 0);
                first_red = false;
            }
            return;
        }
        if (level < 1 || i > ft.m) return;
        int site = t, fp = i - 1;
        d.rank = (long long)B.ti.rank(1, &site, &fp);
        d.kmat = B.kmat_off(t, ft.keep[i - 1]);
    };
    // 2. forward sweep from psi, level 0 / 1 reductions, spawns
    if (spacing == 0) {
        bool ext = false;
        const float2* ext_ptr = nullptr;
        init_state(psi, mainb, ext, ext_ptr);
        const Run& run = B.run_fwd[0];
        for (size_t p = 0; p < run.passes.size(); ++p) {
            const RunPass& rp = run.passes[p];
            if (N > 0 && p > 0 && B.after_last(rp)) break;
            in1[0] = (p == 0 && ext) ? ext_ptr : mainb;
            out1[0] = mainb;
            std::vector<float2*> sp;
            if (level >= 2 && rp.spawn_site >= 0)
                for (int i = 0; i < 3; ++i) sp.push_back(B.group_bufs[1][i]);
            B.add_pass(rp, 0, 1, in1, out1, sp.empty() ? nullptr : sp.data(), (int)sp.size());
            B.add_finish(rp, 0, 1, main_rank);
            if (level >= 2 && rp.spawn_site >= 0 && owns_group(rp.spawn_site)) {
                int s = rp.spawn_site;
                B.dfs_group(1, {}, s, h.factors[s].m, B.group_bufs[1]);
            }
        }
        if (N == 0) {
            Launch l;
            l.kind = L_REDUCE2;
            l.src = B.phi[0];
            l.dst = mainb;
            l.grid = std::max(1, std::min<int>(E.sm_count * 4, (int)std::max<long long>(1, B.dim / (2 * kThreads * 16))));
            B.partial_doubles = std::max(B.partial_doubles, (size_t)l.grid * 8);
            B.L.push_back(l);
            Launch f;
            f.kind = L_FINISH;
            f.n_red = 1;
            f.fin_grid = l.grid;
            f.desc_off = B.descs.size();
            B.descs.push_back({0, 0, 0});
            for (int i = 1; i < 4; ++i) B.descs.push_back({-1, 0, 0});
            B.L.push_back(f);
        }
    } else {
        bool ext = false;
        const float2* ext_ptr = nullptr;
        init_state(psi, mainb, ext, ext_ptr);
        B.spaced_forward(spacing, ext ? ext_ptr : nullptr, main_rank, owns_group);
    }
    {
        Launch l;
        l.kind = L_SUM;
        B.L.push_back(l);
    }
    if (B.too_big) {
        engine_release(E, stream);
        return NQS_ERR_UNSUPPORTED;
    }
    // pass-specialised kernels for the register-resident passes
    if (B.use_jit) {
        std::vector<JitPass*> todo;
        std::vector<Launch*> owner;
        for (auto& l : B.L) {
            if (l.kind != L_PASS || !l.rt) continue;
            std::unique_ptr<JitPass> jp(new JitPass());
            jp->S = l.S;
            jp->k = plan.k;
            jp->seq = l.seq;
            jp->db = jit_staging_buffers();
            jp->pp = jit_pingpong();
            jp->hint = jit_hint();
            jp->rv = jit_reduction_form();
            jp->RB = l.rb;
            jp->n = plan.n;
            for (int j = 0; j < kTileSlots; ++j) jp->local[j] = l.args.local[j];
            for (int j = 0; j < kMaxQ; ++j) jp->nonlocal[j] = l.args.nonlocal[j];
            jp->n_events = l.args.n_events;
            const uint4* w = B.prog.data() + l.prog_index;
            const DevPhase* phs = reinterpret_cast<const DevPhase*>(w);
            jp->phases.assign(phs, phs + l.args.n_phases);
            const OpRec* ops = reinterpret_cast<const OpRec*>(w + l.args.ops_word);
            jp->ops.assign(ops, ops + (l.args.mats_word - l.args.ops_word));
            const float2* mts = reinterpret_cast<const float2*>(w + l.args.mats_word);
            jp->mats.assign(mts, mts + 2 * (l.args.prog_words - l.args.mats_word));
            todo.push_back(jp.get());
            owner.push_back(&l);
            E.jit.push_back(std::move(jp));
        }
        std::string err;
        if (!todo.empty() && jit_build(todo, &err) == 0) {
            for (size_t i = 0; i < todo.size(); ++i) owner[i]->jit = todo[i];
            E.jit_launches = (int)todo.size();
            E.jit_state = 1;
        } else {
            E.jit.clear();
            E.jit_state = todo.empty() ? 0 : -1;
            if (!todo.empty() && std::getenv("NQS_JIT_VERBOSE")) std::fprintf(stderr, "nqs jit: %s\n", err.c_str());
            if (E.wide) {   // the interpreting kernel needs 12-qubit tiles
                E.wide_failed = true;
                engine_release(E, stream);
                return build_schedule(h, E, psi, v, level, stream, allow_jit);
            }
        }
    }

    // --- aux allocation: ops, mats, ckpt table, kmats, descs, partials, term values, level offsets, result
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off_ops = 0;
    size_t off_mats = align(off_ops + B.dops.size() * sizeof(DevOp) + 1);
    size_t off_ckpt = align(off_mats + B.tab.mats.size() * sizeof(float2) + 1);
    size_t off_phase = align(off_ckpt + B.phi.size() * sizeof(float2*));
    size_t off_err = align(off_phase + B.prog.size() * sizeof(uint4) + 1);
    size_t off_kmat = align(off_err + sizeof(int));
    size_t off_desc = align(off_kmat + B.tab.kmats.size() * sizeof(double));
    size_t off_part = align(off_desc + B.descs.size() * sizeof(FinishDesc) + 1);
    size_t off_vals = align(off_part + std::max<size_t>(B.partial_doubles, 8) * sizeof(double));
    size_t off_loff = align(off_vals + std::max<uint64_t>(B.ti.total, 1) * sizeof(double));
    size_t off_res = align(off_loff + (level + 2) * sizeof(long long));
    E.aux_bytes = align(off_res + sizeof(nqs_result));
    E.aux = dev_alloc(E.aux_bytes, stream);
    if (!E.aux) {
        E.aux_bytes = 0;
        engine_release(E, stream);
        return NQS_ERR_NOMEM;
    }
    char* ab = (char*)E.aux;
    DevOp* dops_dev = (DevOp*)(ab + off_ops);
    B.ckpt_dev = (float2**)(ab + off_ckpt);
    float2* mats_dev = (float2*)(ab + off_mats);
    float2** ckpt_dev = (float2**)(ab + off_ckpt);
    uint4* prog_dev = (uint4*)(ab + off_phase);
    E.err_dev = (int*)(ab + off_err);
    E.kmats_dev = (double*)(ab + off_kmat);
    E.desc_dev = (FinishDesc*)(ab + off_desc);
    E.partials = (double*)(ab + off_part);
    E.term_vals = (double*)(ab + off_vals);
    E.level_off_dev = (long long*)(ab + off_loff);
    E.res_dev = (nqs_result*)(ab + off_res);

    cudaStream_t st = (cudaStream_t)stream;
    std::vector<long long> loff(level + 2);
    for (int u = 0; u <= level + 1; ++u) loff[u] = (long long)B.ti.level_offset[u];
    int rc = NQS_OK;
    E.upload_bytes = 0;
    auto up = [&](void* dst, const void* src, size_t bytes) {
        if (bytes && rc == NQS_OK) rc = cuda_err(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
        E.upload_bytes += bytes;
    };
    up(dops_dev, B.dops.data(), B.dops.size() * sizeof(DevOp));
    up(mats_dev, B.tab.mats.data(), B.tab.mats.size() * sizeof(float2));
    up(ckpt_dev, B.phi.data(), B.phi.size() * sizeof(float2*));
    up(prog_dev, B.prog.data(), B.prog.size() * sizeof(uint4));
    up(E.kmats_dev, B.tab.kmats.data(), B.tab.kmats.size() * sizeof(double));
    up(E.desc_dev, B.descs.data(), B.descs.size() * sizeof(FinishDesc));
    up(E.level_off_dev, loff.data(), loff.size() * sizeof(long long));
    if (rc == NQS_OK) rc = cuda_err(cudaMemsetAsync(E.term_vals, 0, std::max<uint64_t>(B.ti.total, 1) * sizeof(double), st));
    // the uploads read pageable host memory: make sure they completed before the builder goes away
    if (rc == NQS_OK) rc = cuda_err(cudaStreamSynchronize(st));
    if (rc != NQS_OK) {
        engine_release(E, stream);
        return rc;
    }
    // rebase pass arguments onto the device tables
    for (auto& l : B.L) {
        if (l.kind != L_PASS) continue;
        l.args.ops = dops_dev + l.op_index;
        l.args.prog = l.rt ? prog_dev + l.prog_index : nullptr;
        l.args.err = E.err_dev;
        l.args.mats = mats_dev;
        l.args.ckpt = ckpt_dev + (l.bd_table ? N : 0);
        l.args.partials = E.partials;
    }
    E.launches = std::move(B.L);
    E.level = level;
    E.psi_kind = psi->kind;
    E.v_kind = v->kind;
    E.psi_bits = psi->bits;
    E.v_bits = v->bits;
    E.psi_dev = psi->dev;
    E.v_dev = v->dev;
    E.n_terms = (long long)B.ti.total;
    E.eff_level = level;
    // truncation bound: sum_{|S|>l} prod ||M-bar|| prod ||M'||
    std::vector<double> poly(1, 1.0);
    for (int s = 0; s < N; ++s) {
        std::vector<double> nx(poly.size() + 1, 0.0);
        for (size_t i = 0; i < poly.size(); ++i) {
            nx[i] += poly[i] * h.factors[s].norm_dom;
            nx[i + 1] += poly[i] * h.factors[s].norm_rest;
        }
        poly.swap(nx);
    }
    double bnd = 0;
    for (size_t i = level + 1; i < poly.size(); ++i) bnd += poly[i];
    E.bound = bnd;
    return NQS_OK;
}

int launch_pass(const Launch& l, cudaStream_t st) {
    if (l.jit) return cuda_err(jit_launch(*l.jit, l.grid, l.args, st));
    if (l.rt) return cuda_err(launch_sweep(l.S, l.rb, l.grid, l.args, st));
    return cuda_err(launch_tile_pass(l.S, l.grid, l.smem, l.args, st));
}

// One launch of a schedule on stream `st`.
int run_launch(Handle& h, Engine& E, const Launch& l, cudaStream_t st) {
    const long long dim = 1ll << h.plan.n;
    const int fill_grid = (int)std::max<long long>(1, std::min<long long>(E.sm_count * 8, dim / 512));
    switch (l.kind) {
        case L_PASS: return launch_pass(l, st);
        case L_FINISH:
            return cuda_err(
                launch_finish(E.partials, l.fin_grid, E.desc_dev + l.desc_off, E.kmats_dev, E.term_vals, l.n_red, st));
        case L_FILL: return cuda_err(launch_basis_fill(l.dst, dim, l.bits, fill_grid, st));
        case L_COPY:
            return cuda_err(cudaMemcpyAsync(l.dst, l.src, dim * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        case L_REDUCE2:   // bits holds the qubit
            return cuda_err(launch_reduce2x2(l.src, l.dst, h.plan.n, (int)l.bits, E.partials, l.grid, st));
        case L_SUM:
            return cuda_err(launch_level_sum(E.term_vals, E.level_off_dev, E.eff_level, E.res_dev, E.bound, E.n_terms,
                                             E.err_dev, st));
        case L_NORMALIZE:
            return cuda_err(launch_normalize(l.dst, dim, E.partials, l.fin_grid, fill_grid, st));
    }
    return NQS_ERR_ARG;
}

int run_schedule(Handle& h, Engine& E, cudaStream_t st) {
    int rc = cuda_err(cudaMemsetAsync(E.err_dev, 0, sizeof(int), st));
    if (rc != NQS_OK) return rc;
    for (const Launch& l : E.launches) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        int kind = (l.kind == L_PASS) ? 0 : (l.kind == L_FINISH || l.kind == L_SUM || l.kind == L_REDUCE2) ? 1 : 2;
        const bool timed = h.profiling && l.kind != L_COPY;
        if (timed) {
            if (E.ev_next >= E.ev_pool.size()) {
                cudaEvent_t a, b;
                cudaEventCreate(&a);
                cudaEventCreate(&b);
                E.ev_pool.push_back({a, b});
            }
            e0 = E.ev_pool[E.ev_next].first;
            e1 = E.ev_pool[E.ev_next].second;
            E.ev_used.push_back({kind, l.kind == L_PASS ? (l.S > 1 ? 3 : 4) : -1, l.bytes});
            ++E.ev_next;
            cudaEventRecord(e0, st);
        }
        rc = run_launch(h, E, l, st);
        if (timed) cudaEventRecord(e1, st);
        if (rc != NQS_OK) return rc;
    }
    return rc;
}

// Add the event timings of finished launches to the handle's statistics.
static void fold_timings(Handle& h, Engine& E) {
    for (size_t i = 0; i < E.ev_used.size(); ++i) {
        float ms = 0;
        cudaEventElapsedTime(&ms, E.ev_pool[i].first, E.ev_pool[i].second);
        for (int slot : {E.ev_used[i].kind, E.ev_used[i].sub}) {
            if (slot < 0) continue;
            nqs_kernel_stats& s = h.stats[slot];
            s.launches += 1;
            s.total_ms += ms;
            s.algorithmic_bytes += E.ev_used[i].bytes;
        }
    }
    E.ev_used.clear();
    E.ev_next = 0;
}

int engine_fidelity(Handle& h, const nqs_state* psi, const nqs_state* v, int level, nqs_result* out, void* stream) {
    if (!h.eng) h.eng = new Engine();
    Engine& E = *h.eng;
    int rc = engine_init(E);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = build_schedule(h, E, psi, v, level, stream);
    if (rc) return rc;
    if (h.profiling) {
        // fold finished timings of earlier calls before reusing the event pool
        cudaStreamSynchronize(E.last_stream);
        fold_timings(h, E);
    }
    rc = run_schedule(h, E, st);
    if (rc) return rc;
    E.last_stream = st;
    E.has_result = true;
    rc = cuda_err(cudaMemcpyAsync(out, E.res_dev, sizeof(nqs_result), cudaMemcpyDefault, st));
    return rc;
}

int engine_collect_stats(Handle& h) {
    if (!h.eng) return NQS_OK;
    Engine& E = *h.eng;
    if (cudaStreamSynchronize(E.last_stream) != cudaSuccess) return NQS_ERR_CUDA;
    fold_timings(h, E);
    return NQS_OK;
}

int engine_term_values(Handle& h, double* out, size_t cap, size_t* count) {
    if (!h.eng || !h.eng->has_result) return NQS_ERR_ORDER;
    Engine& E = *h.eng;
    *count = (size_t)E.n_terms;
    size_t nb = std::min<size_t>(cap, (size_t)E.n_terms) * sizeof(double);
    if (cudaStreamSynchronize(E.last_stream) != cudaSuccess) return NQS_ERR_CUDA;
    if (nb && cudaMemcpy(out, E.term_vals, nb, cudaMemcpyDeviceToHost) != cudaSuccess) return NQS_ERR_CUDA;
    return NQS_OK;
}

void engine_destroy(Handle& h) {
    if (!h.eng) return;
    Engine& E = *h.eng;
    if (E.last_stream) cudaStreamSynchronize(E.last_stream);
    engine_release(E, E.last_stream);
    for (auto& pr : E.ev_pool) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    delete h.eng;
    h.eng = nullptr;
}

uint64_t engine_upload_bytes(const Handle& h) { return h.eng ? h.eng->upload_bytes : 0; }

void engine_invalidate(Handle& h) {
    if (h.eng) h.eng->level = -1;
    engine_batch_forget(&h);
}

int engine_launch_list(const Handle& h, nqs_launch_info* out, size_t cap, size_t* count) {
    const size_t n = (h.eng && h.eng->level >= 0) ? h.eng->launches.size() : 0;
    *count = n;
    if (!out || cap < n) return NQS_OK;
    for (size_t i = 0; i < n; ++i) {
        const Launch& l = h.eng->launches[i];
        nqs_launch_info& o = out[i];
        std::memset(&o, 0, sizeof(o));
        o.kind = (int32_t)l.kind;
        if (l.kind == L_PASS) {
            o.states = l.S;
            o.reg_qubits = l.rt ? l.rb : 0;
            o.phases = l.rt ? l.args.n_phases : 0;
            o.grid = l.grid;
            for (int c = 0; c < 8; ++c) o.ops[c] = l.op_counts[c];
            o.jit = l.jit ? 1 : 0;
            o.algorithmic_bytes = l.bytes;
        }
    }
    return NQS_OK;
}

int engine_jit_compile_check(Handle& h, int states, int max_passes, int* compiled) {
    *compiled = 0;
    if (h.plan.k != kMaxTileQ || !jit_available()) return NQS_ERR_UNSUPPORTED;
    Plan wide;   // NQS_JIT_WIDE=1: the 13-qubit-tile form
    const bool use_wide = jit_wide_enabled() && h.plan.n > kWideTileQ;
    if (use_wide) make_wide_plan(h, wide);
    const Plan& plan = use_wide ? wide : h.plan;
    Tables tab;
    std::vector<DevOp> dops;
    std::vector<uint4> prog;
    // forward passes with reductions and spawns at the sites; for one state also
    // backward passes (adjoint operations, checkpoint saves)
    std::vector<Run> runs;
    runs.push_back(make_run(plan, plan.free_passes, RT_FWD, true, true, false, h.factors, tab, dops));
    if (states == 1) runs.push_back(make_run(plan, plan.free_passes, RT_BWD, false, false, false, h.factors, tab, dops));
    std::vector<std::unique_ptr<JitPass>> own;
    std::vector<JitPass*> todo;
    for (const Run& run : runs)
    for (size_t ip = 0; ip < run.passes.size() && (int)ip < max_passes; ++ip) {
        const RunPass& rp = run.passes[ip];
        const ProgInfo pi = build_program(dops, rp.op_off, rp.n_ops, 4, tab, prog, plan.k);
        std::unique_ptr<JitPass> jp(new JitPass());
        jp->S = states;
        jp->k = plan.k;
        jp->RB = 4;
        jp->n = plan.n;
        jp->seq = states > 1 && jit_seq_enabled();
        jp->db = jit_staging_buffers();
        jp->pp = jit_pingpong();
        jp->hint = jit_hint();
        jp->rv = jit_reduction_form();
        for (int j = 0; j < kTileSlots; ++j) jp->local[j] = rp.local[j];
        for (int j = 0; j < kMaxQ; ++j) jp->nonlocal[j] = rp.nonlocal[j];
        jp->n_events = (int)rp.ev_site.size();
        const uint4* w = prog.data() + pi.words_begin;
        const DevPhase* phs = reinterpret_cast<const DevPhase*>(w);
        jp->phases.assign(phs, phs + pi.n_phases);
        const OpRec* ops = reinterpret_cast<const OpRec*>(w + pi.ops_word);
        jp->ops.assign(ops, ops + (pi.mats_word - pi.ops_word));
        const float2* mts = reinterpret_cast<const float2*>(w + pi.mats_word);
        jp->mats.assign(mts, mts + 2 * (pi.n_words - pi.mats_word));
        todo.push_back(jp.get());
        own.push_back(std::move(jp));
    }
    std::string err;
    if (jit_compile(todo, &err) != 0) {
        std::fprintf(stderr, "nqs jit: %s\n", err.c_str());
        return NQS_ERR_COMPILE;
    }
    *compiled = (int)todo.size();
    return NQS_OK;
}

int engine_jit_info(const Handle& h, int* state) {
    *state = (h.eng && h.eng->level >= 0) ? h.eng->jit_state : 0;
    return (h.eng && h.eng->level >= 0) ? h.eng->jit_launches : 0;
}

int engine_spacing(const Handle& h, int* n_states) {
    *n_states = (h.eng && h.eng->level >= 0) ? (int)h.eng->n_states : 0;
    return (h.eng && h.eng->level >= 0) ? h.eng->spacing : 0;
}

uint64_t engine_launches_per_call(const Handle& h) {
    if (!h.eng) return 0;
    uint64_t n = 0;
    for (const auto& l : h.eng->launches) n += (l.kind != L_COPY) ? 1 : 0;
    return n;
}

uint64_t engine_workspace_bytes(const Handle& h) {
    return h.eng ? (uint64_t)(h.eng->buf_bytes + h.eng->aux_bytes) : 0;
}

// grid of the standalone reduction: about 16 pairs per thread per round,
// capped at 4 blocks per SM and 2048 blocks
static int reduced_matrix_grid(int n, int sms) {
    long long npairs = 1ll << (n - 1);
    long long g = (npairs + 16ll * kThreads - 1) / (16ll * kThreads);
    return (int)std::max<long long>(1, std::min<long long>(std::min<long long>((long long)sms * 4, g), 2048));
}

static size_t reduced_matrix_scratch(int grid) { return ((size_t)grid * 8 + 8) * sizeof(double); }

size_t engine_reduced_matrix_scratch_bytes(int n) {
    // upper bound over SM counts: the grid never exceeds 2048 blocks
    long long npairs = 1ll << (n - 1);
    long long g = std::min<long long>(2048, std::max<long long>(1, (npairs + 16ll * kThreads - 1) / (16ll * kThreads)));
    return reduced_matrix_scratch((int)g);
}

int engine_reduced_matrix(const void* phi, const void* chi, int n, int qubit, double* R_out, void* scratch,
                          size_t scratch_bytes, void* stream) {
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return NQS_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NQS_ERR_CUDA;
    const int grid = reduced_matrix_grid(n, sms);
    if (scratch_bytes < reduced_matrix_scratch(grid)) return NQS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double* part = (double*)scratch;
    double* R = part + (size_t)grid * 8;
    if (launch_reduce2x2((const float2*)phi, (const float2*)chi, n, qubit, part, grid, st) != cudaSuccess)
        return NQS_ERR_CUDA;
    if (launch_partials_sum(part, grid, R, st) != cudaSuccess) return NQS_ERR_CUDA;
    if (cudaMemcpyAsync(R_out, R, 8 * sizeof(double), cudaMemcpyDefault, st) != cudaSuccess) return NQS_ERR_CUDA;
    return NQS_OK;
}

}  // namespace nqs
