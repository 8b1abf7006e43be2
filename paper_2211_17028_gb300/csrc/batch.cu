// Batched evaluation of many circuits (nqs_batch_fidelity).
//
// Every circuit keeps its own schedule (engine.cu).  The batch runs in
// rounds: round r executes the r-th launch of every circuit that has one.
// Launches of one round belong to different circuits and never depend on one
// another, so each launch kind of a round becomes a single multi-circuit
// launch (sweep passes grouped by state count, finishers, fills, level sums)
// with no grid-wide waiting.  Small circuits, whose single-circuit passes
// would occupy a handful of SMs, then share the GPU.  Circuits are packed
// into waves whose state buffers fit in the free device memory; when the
// whole batch fits in one wave, its launch sequence is captured once as a
// CUDA graph and replayed on later calls with the same inputs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "engine_internal.h"

namespace nqs {

namespace {

int cuda_ok(cudaError_t e) { return e == cudaSuccess ? NQS_OK : NQS_ERR_CUDA; }

// One launch of the batched sequence.
struct Group {
    enum Kind { SWEEP, FINISH, FILL, SUM, SINGLE, MEMSET } kind;
    int S = 1, RB = 4;
    size_t units = 0;      // byte offset of the unit array in the device blob
    size_t begins = 0;     // byte offset of the block-begin array
    int n_units = 0, total = 0;
    size_t smem = 0;
    int h = -1;            // SINGLE / MEMSET: which circuit
    int li = -1;           // SINGLE: which launch
};

struct BatchPlan {
    std::vector<Handle*> hs;
    std::vector<int> levels;
    std::vector<nqs_state> psis, vs;
    std::vector<Engine*> engines;   // identity of the schedules the plan was built from
    std::vector<uint64_t> gens;     // their generation counters
    void* dev = nullptr;
    size_t dev_bytes = 0;
    nqs_result* results = nullptr;
    std::vector<Group> seq;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t captured_on = nullptr;
};

std::mutex g_batch_mutex;
BatchPlan* g_cached = nullptr;

bool same_state(const nqs_state& a, const nqs_state& b) {
    return a.kind == b.kind && a.bits == b.bits && a.dev == b.dev;
}

void free_plan(BatchPlan* p, void* stream) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->dev) dev_free(p->dev, p->dev_bytes, stream);
    delete p;
}

size_t state_bytes_needed(const Handle& h, int level) {
    const int N = (int)h.factors.size();
    const int lvl = std::min(level, N);
    int n_group = 0;
    for (int d = 1; d < lvl; ++d) n_group += (d == 1) ? 3 : 9;
    return ((size_t)std::max(N, 1) + 1 + n_group) * ((size_t)8 << h.plan.n);
}

// Build the round-grouped launch sequence of the circuits [first, last) and
// upload their unit arrays.
int build_plan(BatchPlan& P, int first, int last, void* stream) {
    struct Blob {
        std::vector<char> b;
        size_t put(const void* p, size_t n) {
            size_t off = (b.size() + 255) & ~(size_t)255;
            b.resize(off + n);
            std::memcpy(b.data() + off, p, n);
            return off;
        }
    } blob;
    P.seq.clear();
    // memsets of the status words first
    for (int k = first; k < last; ++k) {
        Group g;
        g.kind = Group::MEMSET;
        g.h = k;
        P.seq.push_back(g);
    }
    size_t rounds = 0;
    for (int k = first; k < last; ++k) rounds = std::max(rounds, P.engines[k]->launches.size());
    for (size_t r = 0; r < rounds; ++r) {
        std::vector<PassArgs> sweep_units[4][5];     // [S][RB]
        std::vector<int> sweep_ctas[4][5];
        std::vector<FinishUnit> fin;
        std::vector<int> fin_blocks;
        std::vector<FillUnit> fills;
        std::vector<SumUnit> sums;
        for (int k = first; k < last; ++k) {
            Engine& E = *P.engines[k];
            if (r >= E.launches.size()) continue;
            const Launch& l = E.launches[r];
            const Handle& h = *P.hs[k];
            if (l.kind == L_PASS && l.rt) {
                sweep_units[l.S][l.rb].push_back(l.args);
                sweep_ctas[l.S][l.rb].push_back(l.grid);
            } else if (l.kind == L_FINISH) {
                FinishUnit u{};
                u.partials = E.partials;
                u.desc = E.desc_dev + l.desc_off;
                u.kmats = E.kmats_dev;
                u.vals = E.term_vals;
                u.grid = l.fin_grid;
                fin.push_back(u);
                fin_blocks.push_back(l.n_red);
            } else if (l.kind == L_FILL) {
                FillUnit u{};
                u.dst = l.dst;
                u.dim = 1ll << h.plan.n;
                u.bits = l.bits;
                fills.push_back(u);
            } else if (l.kind == L_SUM) {
                SumUnit u{};
                u.vals = E.term_vals;
                u.level_off = E.level_off_dev;
                u.res = E.res_dev;
                u.copy = P.results + k;
                u.err = E.err_dev;
                u.bound = E.bound;
                u.n_terms = E.n_terms;
                u.level = E.eff_level;
                sums.push_back(u);
            } else {
                Group g;
                g.kind = Group::SINGLE;
                g.h = k;
                g.li = (int)r;
                P.seq.push_back(g);
            }
        }
        for (int S = 1; S <= 3; ++S)
            for (int RB = 3; RB <= 4; ++RB) {
                auto& units = sweep_units[S][RB];
                if (units.empty()) continue;
                std::vector<int> begins(units.size() + 1, 0);
                int max_words = 0, max_ev = 0;
                for (size_t u = 0; u < units.size(); ++u) {
                    begins[u + 1] = begins[u] + sweep_ctas[S][RB][u];
                    max_words = std::max(max_words, units[u].prog_words);
                    max_ev = std::max(max_ev, units[u].n_events);
                }
                Group g;
                g.kind = Group::SWEEP;
                g.S = S;
                g.RB = RB;
                g.units = blob.put(units.data(), units.size() * sizeof(PassArgs));
                g.begins = blob.put(begins.data(), begins.size() * sizeof(int));
                g.n_units = (int)units.size();
                g.total = begins.back();
                g.smem = sweep_smem_bytes(S, RB, max_words, max_ev);
                P.seq.push_back(g);
            }
        if (!fin.empty()) {
            std::vector<int> begins(fin.size() + 1, 0);
            for (size_t u = 0; u < fin.size(); ++u) begins[u + 1] = begins[u] + fin_blocks[u];
            Group g;
            g.kind = Group::FINISH;
            g.units = blob.put(fin.data(), fin.size() * sizeof(FinishUnit));
            g.begins = blob.put(begins.data(), begins.size() * sizeof(int));
            g.n_units = (int)fin.size();
            g.total = begins.back();
            P.seq.push_back(g);
        }
        if (!fills.empty()) {
            Group g;
            g.kind = Group::FILL;
            g.units = blob.put(fills.data(), fills.size() * sizeof(FillUnit));
            g.n_units = (int)fills.size();
            P.seq.push_back(g);
        }
        if (!sums.empty()) {
            Group g;
            g.kind = Group::SUM;
            g.units = blob.put(sums.data(), sums.size() * sizeof(SumUnit));
            g.n_units = (int)sums.size();
            P.seq.push_back(g);
        }
    }
    // device copy of the unit arrays (the result array sits in front of it)
    const size_t res_bytes = ((P.hs.size() * sizeof(nqs_result)) + 255) & ~(size_t)255;
    const size_t need = res_bytes + blob.b.size() + 256;
    if (need > P.dev_bytes) {
        if (P.dev) dev_free(P.dev, P.dev_bytes, stream);
        P.dev = dev_alloc(need, stream);
        P.dev_bytes = P.dev ? need : 0;
        if (!P.dev) return NQS_ERR_NOMEM;
        // the result pointers baked into the SUM units must follow the new buffer
        return -1;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cuda_ok(cudaMemcpyAsync((char*)P.dev + res_bytes, blob.b.data(), blob.b.size(),
                                     cudaMemcpyHostToDevice, st));
    if (rc == NQS_OK) rc = cuda_ok(cudaStreamSynchronize(st));   // the blob is pageable host memory
    for (auto& g : P.seq) {
        g.units += res_bytes;
        g.begins += res_bytes;
    }
    return rc;
}

int run_plan(BatchPlan& P, cudaStream_t st) {
    char* base = (char*)P.dev;
    for (const Group& g : P.seq) {
        int rc = NQS_OK;
        switch (g.kind) {
            case Group::MEMSET:
                rc = cuda_ok(cudaMemsetAsync(P.engines[g.h]->err_dev, 0, sizeof(int), st));
                break;
            case Group::SWEEP:
                rc = cuda_ok(launch_sweep_batched(g.S, g.RB, (const PassArgs*)(base + g.units),
                                                  (const int*)(base + g.begins), g.n_units, g.total, g.smem, st));
                break;
            case Group::FINISH:
                rc = cuda_ok(launch_finish_batched((const FinishUnit*)(base + g.units), (const int*)(base + g.begins),
                                                   g.n_units, g.total, st));
                break;
            case Group::FILL:
                rc = cuda_ok(launch_fill_batched((const FillUnit*)(base + g.units), g.n_units, st));
                break;
            case Group::SUM:
                rc = cuda_ok(launch_level_sum_batched((const SumUnit*)(base + g.units), g.n_units, st));
                break;
            case Group::SINGLE:
                rc = run_launch(*P.hs[g.h], *P.engines[g.h], P.engines[g.h]->launches[g.li], st);
                break;
        }
        if (rc != NQS_OK) return rc;
    }
    return NQS_OK;
}

}  // namespace

int engine_batch_fidelity(Handle** hs, size_t count, const nqs_state* psis, const nqs_state* vs, const int* levels,
                          nqs_result* outs, void* stream) {
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    cudaStream_t st = (cudaStream_t)stream;
    // reuse the cached plan when the batch is the same and no schedule changed
    bool reuse = g_cached && g_cached->hs.size() == count;
    for (size_t k = 0; reuse && k < count; ++k)
        reuse = g_cached->hs[k] == hs[k] && g_cached->levels[k] == levels[k] && same_state(g_cached->psis[k], psis[k]) &&
                same_state(g_cached->vs[k], vs[k]) && hs[k]->eng == g_cached->engines[k] &&
                hs[k]->eng->gen == g_cached->gens[k];
    if (reuse && g_cached->exec) {
        if (cudaGraphLaunch(g_cached->exec, st) != cudaSuccess) return NQS_ERR_CUDA;
        for (size_t k = 0; k < count; ++k) {
            hs[k]->eng->last_stream = st;
            hs[k]->eng->has_result = true;
        }
        return cuda_ok(cudaMemcpyAsync(outs, g_cached->results, count * sizeof(nqs_result), cudaMemcpyDefault, st));
    }
    free_plan(g_cached, stream);
    g_cached = nullptr;

    BatchPlan* P = new BatchPlan();
    P->hs.assign(hs, hs + count);
    P->levels.assign(levels, levels + count);
    P->psis.assign(psis, psis + count);
    P->vs.assign(vs, vs + count);
    P->engines.assign(count, nullptr);
    P->gens.assign(count, 0);

    // waves of circuits whose state buffers fit in the free device memory
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        free_plan(P, stream);
        return NQS_ERR_CUDA;
    }
    size_t held = 0;
    for (size_t k = 0; k < count; ++k) held += engine_workspace_bytes(*hs[k]);
    const size_t budget = (size_t)(0.9 * (double)(free_b + held));
    std::vector<std::pair<int, int>> waves;
    {
        size_t acc = 0;
        int first = 0;
        for (size_t k = 0; k < count; ++k) {
            const size_t need = state_bytes_needed(*hs[k], levels[k]) + (64u << 20);
            if (acc > 0 && acc + need > budget) {
                waves.push_back({first, (int)k});
                first = (int)k;
                acc = 0;
            }
            acc += need;
        }
        waves.push_back({first, (int)count});
    }
    const bool single_wave = waves.size() == 1;

    int rc = NQS_OK;
    for (const auto& w : waves) {
        for (int k = w.first; k < w.second && rc == NQS_OK; ++k) {
            Handle& h = *hs[k];
            if (!h.eng) h.eng = new Engine();
            rc = engine_init(*h.eng);
            if (rc == NQS_OK) rc = build_schedule(h, *h.eng, &psis[k], &vs[k], std::min(levels[k], (int)h.factors.size()),
                                                  stream, false);
            P->engines[k] = h.eng;
            P->gens[k] = h.eng->gen;
        }
        if (rc != NQS_OK) break;
        // results array and unit arrays (build_plan asks once for a larger buffer)
        if (!P->dev) {
            const size_t res_bytes = ((count * sizeof(nqs_result)) + 255) & ~(size_t)255;
            P->dev = dev_alloc(res_bytes + (1u << 20), stream);
            P->dev_bytes = P->dev ? res_bytes + (1u << 20) : 0;
            if (!P->dev) {
                rc = NQS_ERR_NOMEM;
                break;
            }
        }
        P->results = (nqs_result*)P->dev;
        rc = build_plan(*P, w.first, w.second, stream);
        if (rc == -1) {
            P->results = (nqs_result*)P->dev;
            rc = build_plan(*P, w.first, w.second, stream);
        }
        if (rc != NQS_OK) break;
        if (single_wave) {
            cudaGraph_t graph = nullptr;
            bool captured = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) == cudaSuccess;
            P->captured_on = st;
            if (captured) {
                int rc2 = run_plan(*P, st);
                cudaError_t ce = cudaStreamEndCapture(st, &graph);
                if (rc2 == NQS_OK && ce == cudaSuccess && graph &&
                    cudaGraphInstantiate(&P->exec, graph, 0) == cudaSuccess) {
                    rc = cuda_ok(cudaGraphLaunch(P->exec, st));
                } else {
                    cudaGetLastError();
                    P->exec = nullptr;
                    rc = run_plan(*P, st);
                }
                if (graph) cudaGraphDestroy(graph);
            } else {
                cudaGetLastError();
                rc = run_plan(*P, st);
            }
        } else {
            rc = run_plan(*P, st);
        }
        if (rc != NQS_OK) break;
        rc = cuda_ok(cudaMemcpyAsync(outs + w.first, P->results + w.first, (w.second - w.first) * sizeof(nqs_result),
                                     cudaMemcpyDefault, st));
        for (int k = w.first; k < w.second; ++k) {
            hs[k]->eng->last_stream = st;
            hs[k]->eng->has_result = true;
        }
        if (!single_wave) {
            // make room for the next wave
            if (cudaStreamSynchronize(st) != cudaSuccess) rc = NQS_ERR_CUDA;
            for (int k = w.first; k < w.second; ++k) engine_release(*hs[k]->eng, stream);
        }
        if (rc != NQS_OK) break;
    }
    if (rc == NQS_OK && single_wave) {
        g_cached = P;
    } else {
        if (rc == NQS_OK) cudaStreamSynchronize(st);
        free_plan(P, stream);
    }
    return rc;
}

void engine_batch_forget(Handle* h) {
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    if (!g_cached) return;
    for (Handle* x : g_cached->hs)
        if (x == h) {
            if (g_cached->captured_on) cudaStreamSynchronize(g_cached->captured_on);
            free_plan(g_cached, nullptr);
            g_cached = nullptr;
            return;
        }
}

}  // namespace nqs
