// Evaluation of chosen noise-site sets: for a set S = {s_1 < ... < s_k}
// (k <= 3), W(S) = sum over the kept non-dominant factors at every site of S
// of the term values X (the dominant factor everywhere else) -- the
// quantity an importance-sampled estimate of the level-k sum T_k draws.
//
// nqs_prepare_sets stores phi_s (backward sweep from v) and chi_s (forward
// sweep from psi, saved before K_0 is applied) at every site.  A set is then
// evaluated from its first site's checkpoint: w_i = K_i chi_{s_1} is spawned
// (three states), swept to s_2 (K_0 at the sites in between), spawned again
// into three groups of three, swept to s_3 and reduced against phi_{s_3};
// k = 1 reduces chi_{s_1} against phi_{s_1} directly.  Sets are taken in
// lexicographic order so that sets with a common first site share the sweep
// of w_i, and sets with a common first pair share the sweeps of the nine
// states, each of which reduces at every third site its sets need.
//
// When the 2N checkpoints do not fit in device memory (or the handle's
// checkpoint-spacing option asks for it), chi is kept only at the first site
// and phi only at the last site of each block of k sites: chi_{s_1} is
// recomputed by a forward sweep from its block's first site, and a block's
// phi by a backward sweep from its last site into a ring of k slots, once
// for every run of reductions that falls in the block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <iterator>
#include <map>
#include <vector>

#include "engine_internal.h"

namespace nqs {

struct SetsState {
    int N = 0, n = 0;
    void* buf = nullptr;
    size_t buf_bytes = 0;
    void* aux = nullptr;
    size_t aux_bytes = 0;
    void* call = nullptr;
    size_t call_bytes = 0;
    std::vector<float2*> phi, chi;    // spaced: boundaries per block (phi at block-last, chi at block-first sites)
    std::vector<float2*> ring;        // spaced: recomputed phi of one block
    int spacing = 0;                  // sites per checkpoint block (0: every site)
    float2* main = nullptr;
    float2* scratch = nullptr;
    float2* work = nullptr;           // spaced: recomputed chi
    float2* work_mat = nullptr;       // spaced: backward recomputation state
    float2** phi_bd_tab = nullptr;    // spaced: site -> phi boundary of its block
    std::vector<PassSpec> segs;       // spaced: passes cut after every block-last site
    std::vector<PassSpec> fsegs;      // passes of the set sweeps: up to 16 sites each (K_0 only at most of them)
    std::vector<DevOp> mat_ops;       // spaced: backward ops saving phi at every site, per pass of segs
    std::vector<std::pair<int, int>> mat_pass;   // (first op in mat_ops, count) per pass, reversed order
    std::vector<int> mat_seg;         // segment index of each entry of mat_pass
    std::vector<int> mat_block;       // block of each entry of mat_pass
    float2* g1[3] = {};
    float2* g2[9] = {};
    float2** phi_tab = nullptr;
    float2** chi_tab = nullptr;
    double* kmats = nullptr;
    double* partials = nullptr;
    size_t partial_doubles = 0;
    int* err = nullptr;
    Tables tab;
    std::vector<int> fwd_mat;        // forward matrix offset of every linear op
    int sm_count = 0;
    bool ready = false;
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Prog {
    std::vector<DevOp> dops;          // shared-memory tile kernel
    std::vector<uint4> prog;          // register-resident kernel
    std::vector<FinishDesc> descs;
    std::vector<Launch> L;
    size_t partial_doubles = 8;
};

// DevOps of the forward direction for linear ops [a, b) of pass `ps`, with
// site flags chosen by `flag_of(site)`.
template <typename F>
std::vector<DevOp> emit_range(const Plan& plan, const SetsState& S, const PassSpec& ps, int a, int b, F flag_of,
                              const std::vector<Factors>& fac) {
    std::vector<int> pos(plan.n, -1);
    for (int j = 0; j < plan.k; ++j) pos[ps.local[j]] = j;
    std::vector<DevOp> out;
    int events = 0;
    for (int i = a; i < b; ++i) {
        const HostOp& o = plan.ops[i];
        DevOp d{};
        d.type = o.type;
        d.qa = o.q0;
        d.qb = o.q1;
        d.a = o.q0 >= 0 ? pos[o.q0] : -1;
        d.b = o.q1 >= 0 ? pos[o.q1] : -1;
        d.site = o.site;
        d.mat = S.fwd_mat[i];
        if (o.type == OP_SITE) {
            int fl = flag_of(o.site);
            if (fl & FL_REDUCE) fl |= (events++) << 8;
            if (fl & FL_SPAWN) fl |= fac[o.site].m << 16;
            if (o.diag) fl |= FL_KDIAG;
            d.flags = fl;
        }
        out.push_back(d);
    }
    return out;
}

int pass_of(const std::vector<PassSpec>& segs, int lin) {
    for (size_t p = 0; p < segs.size(); ++p)
        if (segs[p].op_begin <= lin && lin < segs[p].op_end) return (int)p;
    return -1;
}

// one sweep launch over custom DevOps of one pass
void add_launch(Prog& G, const Plan& plan, const SetsState& S, const PassSpec& ps, int nstates,
                std::vector<DevOp> ops, const float2* const* in, float2* const* out, float2* const* spawn,
                int n_spawn) {
    Launch l;
    l.kind = L_PASS;
    l.S = nstates;
    PassArgs& a = l.args;
    a = PassArgs{};
    a.n = plan.n;
    a.k = plan.k;
    a.c = plan.c;
    int n_ev = 0;
    for (const DevOp& d : ops)
        if (d.type == OP_SITE && (d.flags & FL_REDUCE)) ++n_ev;
    a.n_events = n_ev;
    std::vector<char> is_local(plan.n, 0);
    for (int j = 0; j < plan.k; ++j) {
        a.local[j] = ps.local[j];
        is_local[ps.local[j]] = 1;
    }
    int nl = 0;
    for (int q = 0; q < plan.n; ++q)
        if (!is_local[q]) a.nonlocal[nl++] = q;
    a.n_tiles = 1ll << (plan.n - plan.k);
    for (int s = 0; s < nstates; ++s) {
        a.in[s] = in[s];
        a.out[s] = out[s];
    }
    for (int i = 0; i < n_spawn; ++i) a.spawn[i] = spawn[i];
    l.rt = plan.k == kMaxTileQ;
    int per_sm;
    if (l.rt) {
        l.rb = sweep_reg_bits(nstates);
        ProgInfo pi = build_program(ops, 0, (int)ops.size(), l.rb, S.tab, G.prog);
        l.prog_index = pi.words_begin;
        a.prog_words = pi.n_words;
        a.ops_word = pi.ops_word;
        a.mats_word = pi.mats_word;
        a.n_phases = pi.n_phases;
        per_sm = sweep_blocks_per_sm(nstates, l.rb, sweep_smem_bytes(nstates, l.rb, pi.n_words, n_ev));
    } else {
        l.op_index = (int)G.dops.size();
        G.dops.insert(G.dops.end(), ops.begin(), ops.end());
        a.n_ops = (int)ops.size();
        l.smem = (size_t)nstates * (1 << plan.k) * sizeof(float2);
        per_sm = tile_pass_blocks_per_sm(nstates, l.smem);
    }
    l.grid = (int)std::max<long long>(1, std::min<long long>((long long)per_sm * S.sm_count, a.n_tiles));
    G.partial_doubles = std::max(G.partial_doubles, (size_t)std::max(1, n_ev) * nstates * l.grid * 8);
    G.L.push_back(l);
}

// finisher for the last launch: its single reduction event, `nstates` slots;
// slot st, factor position f -> value index rank_of(st, f)
template <typename R>
void add_finish(Prog& G, int nstates, int site, const std::vector<Factors>& fac, R rank_of) {
    const Launch& pl = G.L.back();
    Launch f;
    f.kind = L_FINISH;
    f.n_red = nstates;
    f.fin_grid = pl.grid;
    f.desc_off = G.descs.size();
    const Factors& ft = fac[site];
    for (int st = 0; st < nstates; ++st)
        for (int i = 0; i < 4; ++i) {
            FinishDesc d{-1, 0, 0};
            if (i >= 1 && i <= ft.m) {
                d.rank = rank_of(st, i - 1);
                d.kmat = site * 32 + ft.keep[i - 1] * 8;
            }
            G.descs.push_back(d);
        }
    G.L.push_back(f);
}

// finisher for the last launch with several reduction events (sites in
// launch order); slot (event e, state st), factor position f -> rank_of(site, st, f)
template <typename R>
void add_finish_events(Prog& G, int nstates, const std::vector<int>& ev_sites, const std::vector<Factors>& fac,
                       R rank_of) {
    const Launch& pl = G.L.back();
    Launch f;
    f.kind = L_FINISH;
    f.n_red = (int)ev_sites.size() * nstates;
    f.fin_grid = pl.grid;
    f.desc_off = G.descs.size();
    for (int t : ev_sites) {
        const Factors& ft = fac[t];
        for (int st = 0; st < nstates; ++st)
            for (int i = 0; i < 4; ++i) {
                FinishDesc d{-1, 0, 0};
                if (i >= 1 && i <= ft.m) {
                    d.rank = rank_of(t, st, i - 1);
                    d.kmat = t * 32 + ft.keep[i - 1] * 8;
                }
                G.descs.push_back(d);
            }
    }
    G.L.push_back(f);
}

// sweep `nstates` states over the linear ops (a, b]; site t gets flag_of(t)
// (which may spawn only at b); every launch with reductions gets its finisher
template <typename FlagFn, typename RankFn>
void sweep_range(Prog& G, const Handle& h, const SetsState& S, int a, int b, FlagFn flag_of, int nstates,
                 float2* const* states, float2* const* spawn, int n_spawn, RankFn rank_of) {
    const Plan& plan = h.plan;
    for (int p = pass_of(S.fsegs, a + 1); p >= 0 && p < (int)S.fsegs.size(); ++p) {
        const PassSpec& ps = S.fsegs[p];
        const int lo = std::max(ps.op_begin, a + 1), hi = std::min(ps.op_end, b + 1);
        if (lo >= hi) break;
        const bool has_last = hi == b + 1;
        // one launch per run of at most four reductions (the kernels' reduction slots)
        for (int c0 = lo; c0 < hi;) {
            int c1 = c0, red = 0;
            while (c1 < hi) {
                const HostOp& o = plan.ops[c1];
                const bool r = o.type == OP_SITE && (flag_of(o.site) & FL_REDUCE);
                if (r && red == 4) break;
                red += r;
                ++c1;
            }
            auto ops = emit_range(plan, S, ps, c0, c1, flag_of, h.factors);
            const bool last_chunk = has_last && c1 == hi;
            add_launch(G, plan, S, ps, nstates, ops, (const float2* const*)states, states,
                       last_chunk ? spawn : nullptr, last_chunk ? n_spawn : 0);
            std::vector<int> ev;
            for (const DevOp& d : ops)
                if (d.type == OP_SITE && (d.flags & FL_REDUCE)) ev.push_back(d.site);
            if (!ev.empty()) add_finish_events(G, nstates, ev, h.factors, rank_of);
            c0 = c1;
        }
        if (has_last) break;
    }
}

int upload_and_run(Handle& h, SetsState& S, Prog& G, size_t extra_bytes, void** extra, cudaStream_t st) {
    // per-call buffer: device ops, programs, descriptors, partials, extra
    const size_t o_ops = 0;
    const size_t o_prog = align256(o_ops + G.dops.size() * sizeof(DevOp) + 1);
    const size_t o_desc = align256(o_prog + G.prog.size() * sizeof(uint4) + 1);
    const size_t o_part = align256(o_desc + G.descs.size() * sizeof(FinishDesc) + 1);
    const size_t o_extra = align256(o_part + G.partial_doubles * sizeof(double));
    const size_t need = align256(o_extra + extra_bytes + 1);
    if (need > S.call_bytes) {
        if (S.call) {
            cudaStreamSynchronize(st);
            dev_free(S.call, S.call_bytes, st);
        }
        S.call = dev_alloc(need, st);
        S.call_bytes = S.call ? need : 0;
        if (!S.call) return NQS_ERR_NOMEM;
    }
    char* base = (char*)S.call;
    int rc = NQS_OK;
    auto up = [&](size_t off, const void* src, size_t bytes) {
        if (bytes && rc == NQS_OK) rc = cuda_err(cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, st));
    };
    up(o_ops, G.dops.data(), G.dops.size() * sizeof(DevOp));
    up(o_prog, G.prog.data(), G.prog.size() * sizeof(uint4));
    up(o_desc, G.descs.data(), G.descs.size() * sizeof(FinishDesc));
    if (rc == NQS_OK && extra_bytes) rc = cuda_err(cudaMemsetAsync(base + o_extra, 0, extra_bytes, st));
    if (rc == NQS_OK) rc = cuda_err(cudaStreamSynchronize(st));   // pageable sources
    if (rc != NQS_OK) return rc;
    if (extra) *extra = base + o_extra;
    // a throwaway engine view carrying the pointers run_launch reads
    Engine E;
    E.sm_count = S.sm_count;
    E.partials = (double*)(base + o_part);
    E.desc_dev = (FinishDesc*)(base + o_desc);
    E.kmats_dev = S.kmats;
    E.err_dev = S.err;
    for (Launch& l : G.L) {
        if (l.kind == L_PASS) {
            l.args.ops = (const DevOp*)(base + o_ops) + l.op_index;
            l.args.prog = l.rt ? (const uint4*)(base + o_prog) + l.prog_index : nullptr;
            l.args.ckpt = l.bd_table ? S.phi_bd_tab : S.phi_tab;
            l.args.ckpt_fwd = S.chi_tab;
            l.args.partials = E.partials;
            l.args.err = S.err;
        }
    }
    E.term_vals = extra ? (double*)*extra : nullptr;
    for (const Launch& l : G.L) {
        rc = run_launch(h, E, l, st);
        if (rc != NQS_OK) break;
    }
    E.launches.clear();
    return rc;
}

}  // namespace

void sets_destroy(Handle& h) {
    if (!h.sets) return;
    SetsState& S = *h.sets;
    cudaDeviceSynchronize();
    if (S.buf) dev_free(S.buf, S.buf_bytes, nullptr);
    if (S.aux) dev_free(S.aux, S.aux_bytes, nullptr);
    if (S.call) dev_free(S.call, S.call_bytes, nullptr);
    delete h.sets;
    h.sets = nullptr;
}

int engine_prepare_sets(Handle& h, const nqs_state* psi, const nqs_state* v, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const Plan& plan = h.plan;
    const int N = (int)h.factors.size();
    if (N < 1) return NQS_ERR_ARG;
    sets_destroy(h);
    h.sets = new SetsState();
    SetsState& S = *h.sets;
    S.N = N;
    S.n = plan.n;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return NQS_ERR_CUDA;
    cudaDeviceGetAttribute(&S.sm_count, cudaDevAttrMultiProcessorCount, dev);
    const size_t dim = (size_t)1 << plan.n;
    const size_t sbytes = dim * sizeof(float2);
    // every site, else blocks of k sites: boundaries 2 ceil(N/k), ring k, five work states, 12 group states
    auto spaced_states = [&](int k) { return 2 * (size_t)((N + k - 1) / k) + (size_t)k + 5 + 12; };
    int k = (h.opt_spacing > 0 && h.opt_spacing < N) ? h.opt_spacing : 0;
    if (k == 0) {
        S.buf_bytes = (2 * (size_t)N + 2 + 3 + 9) * sbytes;
        S.buf = dev_alloc(S.buf_bytes, stream);
        if (!S.buf && h.opt_spacing == 0 && N > 1) {
            k = 1;
            for (int c = 2; c < N; ++c)
                if (spaced_states(c) < spaced_states(k)) k = c;
        }
    }
    if (k > 0) {
        S.buf_bytes = spaced_states(k) * sbytes;
        S.buf = dev_alloc(S.buf_bytes, stream);
    }
    if (!S.buf) {
        S.buf_bytes = 0;
        sets_destroy(h);
        return NQS_ERR_NOMEM;
    }
    S.spacing = k;
    float2* b = (float2*)S.buf;
    size_t next = 0;
    const int nslots = k ? (N + k - 1) / k : N;
    for (int s = 0; s < nslots; ++s) S.phi.push_back(b + (next++) * dim);
    for (int s = 0; s < nslots; ++s) S.chi.push_back(b + (next++) * dim);
    for (int j = 0; j < k; ++j) S.ring.push_back(b + (next++) * dim);
    S.main = b + (next++) * dim;
    S.scratch = b + (next++) * dim;
    if (k) {
        S.work = b + (next++) * dim;
        S.work_mat = b + (next++) * dim;
        next++;   // spare (keeps the count of spaced_states)
    }
    for (int i = 0; i < 3; ++i) S.g1[i] = b + (next++) * dim;
    for (int i = 0; i < 9; ++i) S.g2[i] = b + (next++) * dim;

    // matrices: forward factors for every op (and adjoints for the backward runs)
    std::vector<char> block_last, block_first;
    if (k) {
        block_last.assign(N, 0);
        block_first.assign(N, 0);
        for (int s = 0; s < N; ++s) {
            block_last[s] = ((s + 1) % k == 0) || s == N - 1;
            block_first[s] = s % k == 0;
        }
        S.segs = segment(plan, false, h.opt_max_sites > 0 ? h.opt_max_sites : 4,
                         h.opt_max_ops > 0 ? h.opt_max_ops : 96, &block_last);
    }
    S.fsegs = segment(plan, false, 16, h.opt_max_ops > 0 ? h.opt_max_ops : 96);
    const std::vector<PassSpec>& bsegs = k ? S.segs : plan.free_passes;
    std::vector<DevOp> run_ops;
    Run run_bwd = make_run(plan, bsegs, RT_BWD, false, false, false, h.factors, S.tab, run_ops,
                           k ? &block_last : nullptr);
    Run run_fwd = make_run(plan, plan.free_passes, RT_FWD, false, false, false, h.factors, S.tab, run_ops);
    S.fwd_mat.assign(plan.ops.size(), -1);
    for (const RunPass& rp : run_fwd.passes)
        for (int o = 0; o < rp.n_ops; ++o) S.fwd_mat[rp.lin[o]] = run_ops[rp.op_off + o].mat;
    Run run_ideal;
    if (v->kind == NQS_STATE_IDEAL) run_ideal = make_run(plan, plan.free_passes, RT_IDEAL, false, false, false, h.factors,
                                                         S.tab, run_ops);
    if (k) {
        // per-block recomputation of phi (saves at every site), kept for evaluation calls
        Run run_mat = make_run(plan, S.segs, RT_BWD, false, false, false, h.factors, S.tab, S.mat_ops);
        const int nb = (N + k - 1) / k;
        for (size_t p = 0; p < run_mat.passes.size(); ++p) {
            const RunPass& rp = run_mat.passes[p];
            int blk = nb;
            if (!rp.lin.empty())
                for (int c = 0; c < nb; ++c)
                    if (rp.lin[0] <= plan.site_pos[std::min(N, (c + 1) * k) - 1]) {
                        blk = c;
                        break;
                    }
            S.mat_pass.push_back({rp.op_off, rp.n_ops});
            S.mat_seg.push_back((int)(run_mat.passes.size() - 1 - p));
            S.mat_block.push_back(blk);
        }
    }

    // aux: checkpoint tables, factor table (complex128), status word, matrix table
    const size_t o_phi = 0, o_chi = align256(N * sizeof(float2*));
    const size_t o_kmat = align256(o_chi + N * sizeof(float2*));
    const size_t o_err = align256(o_kmat + (size_t)N * 32 * sizeof(double));
    const size_t o_mats = align256(o_err + sizeof(int));
    const size_t o_bd = align256(o_mats + S.tab.mats.size() * sizeof(float2) + 1);
    S.aux_bytes = align256(o_bd + N * sizeof(float2*));
    S.aux = dev_alloc(S.aux_bytes, stream);
    if (!S.aux) {
        S.aux_bytes = 0;
        sets_destroy(h);
        return NQS_ERR_NOMEM;
    }
    char* ab = (char*)S.aux;
    S.phi_tab = (float2**)(ab + o_phi);
    S.chi_tab = (float2**)(ab + o_chi);
    S.kmats = (double*)(ab + o_kmat);
    S.err = (int*)(ab + o_err);
    S.phi_bd_tab = (float2**)(ab + o_bd);
    float2* mats_dev = (float2*)(ab + o_mats);
    std::vector<double> kh((size_t)N * 32);
    for (int s = 0; s < N; ++s)
        for (int i = 0; i < 4; ++i)
            for (int e = 0; e < 4; ++e) {
                kh[s * 32 + i * 8 + 2 * e] = h.factors[s].K[i][e].real();
                kh[s * 32 + i * 8 + 2 * e + 1] = h.factors[s].K[i][e].imag();
            }
    std::vector<float2*> phi_t(N), chi_t(N), bd_t(N);
    for (int s = 0; s < N; ++s) {
        phi_t[s] = k ? S.ring[s % k] : S.phi[s];
        chi_t[s] = k ? S.chi[s / k] : S.chi[s];
        bd_t[s] = k ? S.phi[s / k] : S.phi[s];
    }
    int rc = NQS_OK;
    auto up = [&](void* dst, const void* src, size_t bytes) {
        if (bytes && rc == NQS_OK) rc = cuda_err(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    };
    up(S.phi_tab, phi_t.data(), N * sizeof(float2*));
    up(S.chi_tab, chi_t.data(), N * sizeof(float2*));
    up(S.phi_bd_tab, bd_t.data(), N * sizeof(float2*));
    up(S.kmats, kh.data(), kh.size() * sizeof(double));
    up(mats_dev, S.tab.mats.data(), S.tab.mats.size() * sizeof(float2));
    if (rc == NQS_OK) rc = cuda_err(cudaMemsetAsync(S.err, 0, sizeof(int), st));
    if (rc == NQS_OK) rc = cuda_err(cudaStreamSynchronize(st));
    if (rc != NQS_OK) {
        sets_destroy(h);
        return rc;
    }

    // checkpoint sweeps: (ideal v) -> backward saving phi -> forward saving chi
    Prog G;
    const float2* in1[1];
    float2* out1[1];
    auto run_passes = [&](const Run& run, const std::vector<PassSpec>& segs, const float2* first_in, bool bwd,
                          bool save_fwd) {
        for (size_t p = 0; p < run.passes.size(); ++p) {
            const RunPass& rp = run.passes[p];
            // the backward sweep is done once phi of the first site is saved, the
            // forward one once chi of the last site is
            if (p > 0 && !rp.lin.empty()) {
                if (bwd && *std::max_element(rp.lin.begin(), rp.lin.end()) < plan.site_pos[0]) break;
                if (save_fwd && *std::min_element(rp.lin.begin(), rp.lin.end()) > plan.site_pos[N - 1]) break;
            }
            std::vector<DevOp> ops(run_ops.begin() + rp.op_off, run_ops.begin() + rp.op_off + rp.n_ops);
            for (DevOp& d : ops)
                if (d.type == OP_SITE && save_fwd)
                    d.flags = FL_APPLY | ((!k || block_first[d.site]) ? FL_SAVE_FWD : 0) | (d.flags & FL_KDIAG);
            in1[0] = (p == 0 && first_in) ? first_in : S.main;
            out1[0] = S.main;
            const PassSpec& ps = segs[bwd ? run.passes.size() - 1 - p : p];
            add_launch(G, plan, S, ps, 1, ops, in1, out1, nullptr, 0);
            if (bwd) G.L.back().bd_table = true;
        }
    };
    auto fill = [&](const nqs_state* st8, const float2*& ext) {
        ext = nullptr;
        if (st8->kind == NQS_STATE_BASIS) {
            Launch l;
            l.kind = L_FILL;
            l.dst = S.main;
            l.bits = st8->bits;
            G.L.push_back(l);
        } else {
            ext = (const float2*)st8->dev;
        }
    };
    const float2* ext = nullptr;
    if (v->kind == NQS_STATE_IDEAL) {
        fill(psi, ext);
        run_passes(run_ideal, plan.free_passes, ext, false, false);
        ext = nullptr;
    } else {
        fill(v, ext);
    }
    run_passes(run_bwd, bsegs, ext, true, false);
    fill(psi, ext);
    run_passes(run_fwd, plan.free_passes, ext, false, true);
    // the matrices of the device table: programs index their own copies, the
    // shared-memory tile kernel reads the table
    for (Launch& l : G.L)
        if (l.kind == L_PASS) l.args.mats = mats_dev;
    rc = upload_and_run(h, S, G, 0, nullptr, st);
    if (rc == NQS_OK) rc = cuda_err(cudaStreamSynchronize(st));
    if (rc != NQS_OK) {
        sets_destroy(h);
        return rc;
    }
    S.ready = true;
    return NQS_OK;
}

int engine_eval_sets(Handle& h, int k, const int* sets, size_t m, double* W_out, void* stream) {
    if (!h.sets || !h.sets->ready) return NQS_ERR_ORDER;
    SetsState& S = *h.sets;
    const Plan& plan = h.plan;
    cudaStream_t st = (cudaStream_t)stream;
    if (k < 1 || k > 3 || m == 0) return NQS_ERR_ARG;
    for (size_t j = 0; j < m; ++j)
        for (int r = 0; r < k; ++r) {
            const int s = sets[j * k + r];
            if (s < 0 || s >= S.N || (r > 0 && s <= sets[j * k + r - 1])) return NQS_ERR_ARG;
        }
    Prog G;
    const float2* mats_dev = nullptr;
    {
        // the matrix table sits at the end of aux (see engine_prepare_sets)
        const size_t o_chi = align256(S.N * sizeof(float2*));
        const size_t o_kmat = align256(o_chi + S.N * sizeof(float2*));
        const size_t o_err = align256(o_kmat + (size_t)S.N * 32 * sizeof(double));
        mats_dev = (const float2*)((char*)S.aux + align256(o_err + sizeof(int)));
    }
    std::vector<size_t> order(m);
    for (size_t j = 0; j < m; ++j) order[j] = j;
    std::sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        return std::lexicographical_compare(sets + x * k, sets + x * k + k, sets + y * k, sets + y * k + k);
    });
    auto at = [&](size_t r, int c) { return sets[order[r] * k + c]; };
    const int K = S.spacing;
    // spaced checkpoints: phi of block c into the ring (once per run of reductions in it)
    int ring_block = -1;
    auto materialize = [&](int c) {
        if (!K || ring_block == c) return;
        bool first_in = true;
        for (size_t p = 0; p < S.mat_pass.size(); ++p) {
            if (S.mat_block[p] != c) continue;
            std::vector<DevOp> ops(S.mat_ops.begin() + S.mat_pass[p].first,
                                   S.mat_ops.begin() + S.mat_pass[p].first + S.mat_pass[p].second);
            const float2* in[1] = {first_in ? S.phi[c] : S.work_mat};
            float2* out[1] = {S.work_mat};
            add_launch(G, plan, S, S.segs[S.mat_seg[p]], 1, ops, in, out, nullptr, 0);
            first_in = false;
        }
        ring_block = c;
    };
    auto phi_of = [&](int t) { return K ? S.ring[t % K] : S.phi[t]; };
    // chi_{s1}: stored, or swept forward from the first site of its block
    auto chi_of = [&](int s1) -> const float2* {
        if (!K) return S.chi[s1];
        const int first = (s1 / K) * K;
        if (s1 == first) return S.chi[s1 / K];
        Launch c;
        c.kind = L_COPY;
        c.dst = S.work;
        c.src = S.chi[s1 / K];
        G.L.push_back(c);
        float2* w[1] = {S.work};
        sweep_range(G, h, S, plan.site_pos[first] - 1, plan.site_pos[s1] - 1, [](int) { return FL_APPLY; }, 1, w,
                    nullptr, 0, [](int, int, int) { return -1ll; });
        return S.work;
    };
    // sweep `states` from linear op `from` through the reduction sites of
    // `slots` (site -> value slot base), one checkpoint block at a time
    auto reduce_through = [&](int from, const std::map<int, long long>& slots, int nst, float2* const* states,
                              int mult) {
        int pos = from;
        for (auto it = slots.begin(); it != slots.end();) {
            const int blk = K ? it->first / K : 0;
            auto end = it;
            while (end != slots.end() && (!K || end->first / K == blk)) ++end;
            materialize(blk);
            const int last = std::prev(end)->first;
            sweep_range(G, h, S, pos, plan.site_pos[last],
                        [&](int t) { return FL_APPLY | (slots.count(t) ? FL_REDUCE : 0); }, nst, states, nullptr, 0,
                        [&](int t, int st, int f) { return slots.at(t) + st * mult + f; });
            pos = plan.site_pos[last];
            it = end;
        }
    };
    for (size_t i = 0; i < m;) {
        const int s1 = at(i, 0);
        size_t i1 = i;
        while (i1 < m && at(i1, 0) == s1) ++i1;
        if (k == 1) {
            const float2* chi = chi_of(s1);
            materialize(K ? s1 / K : 0);
            for (size_t r = i; r < i1; ++r) {
                const long long base = (long long)order[r] * 27;
                Launch l;
                l.kind = L_REDUCE2;
                l.src = phi_of(s1);
                l.dst = const_cast<float2*>(chi);   // read only
                l.bits = (unsigned long long)h.circ.noises[s1].qubit;
                const long long npairs = 1ll << (plan.n - 1);
                l.grid = (int)std::max<long long>(
                    1, std::min<long long>((long long)S.sm_count * 4, (npairs + 16ll * kThreads - 1) / (16ll * kThreads)));
                G.partial_doubles = std::max(G.partial_doubles, (size_t)l.grid * 8);
                G.L.push_back(l);
                add_finish(G, 1, s1, h.factors, [&](int, int f) { return base + f; });
            }
            i = i1;
            continue;
        }
        // spawn K_i chi_{s1} into the first group (shared by every set starting at s1)
        const int p1 = plan.site_pos[s1];
        const int m1 = h.factors[s1].m;
        const PassSpec& ps1 = S.fsegs[pass_of(S.fsegs, p1)];
        {
            auto ops = emit_range(plan, S, ps1, p1, p1 + 1, [&](int) { return FL_SPAWN; }, h.factors);
            const float2* in[1] = {chi_of(s1)};
            float2* out[1] = {S.scratch};
            add_launch(G, plan, S, ps1, 1, ops, in, out, S.g1, 3);
        }
        if (k == 2) {
            std::map<int, long long> base2;   // second site -> value slots of its set
            for (size_t r = i; r < i1; ++r) base2[at(r, 1)] = (long long)order[r] * 27;
            reduce_through(p1, base2, m1, S.g1, 3);
            i = i1;
            continue;
        }
        int pos = p1;
        for (size_t r = i; r < i1;) {
            const int s2 = at(r, 1), p2 = plan.site_pos[s2];
            size_t r2 = r;
            while (r2 < i1 && at(r2, 1) == s2) ++r2;
            // carry the first group to s2 (K_0 there), spawning the nine states
            sweep_range(G, h, S, pos, p2, [&](int t) { return FL_APPLY | (t == s2 ? FL_SPAWN : 0); }, m1, S.g1, S.g2, 9,
                        [](int, int, int) { return -1ll; });
            pos = p2;
            std::map<int, long long> base3;   // third site -> value slots of its set
            for (size_t q = r; q < r2; ++q) base3[at(q, 2)] = (long long)order[q] * 27;
            const int m2 = h.factors[s2].m;
            if (!K) {
                for (int g = 0; g < m1; ++g) {
                    std::map<int, long long> bg = base3;
                    for (auto& e : bg) e.second += g * 9;
                    reduce_through(p2, bg, m2, S.g2 + 3 * g, 3);
                }
            } else {
                // one block at a time for all three groups, so each block's phi is recomputed once
                int gpos[3] = {p2, p2, p2};
                for (auto it = base3.begin(); it != base3.end();) {
                    const int blk = it->first / K;
                    auto end = it;
                    while (end != base3.end() && end->first / K == blk) ++end;
                    std::map<int, long long> part(it, end);
                    for (int g = 0; g < m1; ++g) {
                        std::map<int, long long> bg = part;
                        for (auto& e : bg) e.second += g * 9;
                        reduce_through(gpos[g], bg, m2, S.g2 + 3 * g, 3);
                        gpos[g] = plan.site_pos[std::prev(end)->first];
                    }
                    it = end;
                }
            }
            r = r2;
        }
        i = i1;
    }
    for (Launch& l : G.L)
        if (l.kind == L_PASS) l.args.mats = mats_dev;
    void* vals = nullptr;
    int rc = upload_and_run(h, S, G, m * 27 * sizeof(double), &vals, st);   // value slots start at zero
    if (rc != NQS_OK) return rc;
    std::vector<double> hv(m * 27);
    rc = cuda_err(cudaMemcpyAsync(hv.data(), vals, m * 27 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (rc == NQS_OK) rc = cuda_err(cudaStreamSynchronize(st));
    if (rc != NQS_OK) return rc;
    int err = 0;
    cudaMemcpy(&err, S.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) return NQS_ERR_DEVICE_TIMEOUT;
    for (size_t j = 0; j < m; ++j) {
        double w = 0.0;
        for (int t = 0; t < 27; ++t) w += hv[j * 27 + t];
        W_out[j] = w;
    }
    return NQS_OK;
}

}  // namespace nqs
