// C ABI of libnqs (include/nqs.h): argument validation, handle lifetime, the
// device allocator hook, and the host-only inspection entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "nqs_internal.h"

namespace nqs {

namespace {
nqs_alloc_fn g_alloc = nullptr;
nqs_free_fn g_free = nullptr;
void* g_ctx = nullptr;
constexpr int kTileQubits = 12;
}  // namespace

void* dev_alloc(size_t bytes, void* stream) {
    if (bytes == 0) bytes = 256;
    if (g_alloc) return g_alloc(bytes, stream, g_ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void* p, size_t bytes, void* stream) {
    if (!p) return;
    if (g_free) {
        g_free(p, bytes, stream, g_ctx);
        return;
    }
    cudaFree(p);
}

int engine_collect_stats(Handle& h);

}  // namespace nqs

using namespace nqs;

extern "C" {

int nqs_set_allocator(nqs_alloc_fn alloc, nqs_free_fn release, void* ctx) {
    if ((alloc == nullptr) != (release == nullptr)) return NQS_ERR_ARG;
    g_alloc = alloc;
    g_free = release;
    g_ctx = ctx;
    return NQS_OK;
}

int nqs_load_circuit(const char* ir_text, nqs_handle* out) {
    if (!ir_text || !out) return NQS_ERR_ARG;
    Handle* h = new (std::nothrow) Handle();
    if (!h) return NQS_ERR_NOMEM;
    std::string err;
    int rc = parse_circuit(ir_text, h->circ, err);
    if (rc != NQS_OK) {
        delete h;
        return rc;
    }
    *out = reinterpret_cast<nqs_handle>(h);
    return NQS_OK;
}

int nqs_prepare_noise(nqs_handle hh, const nqs_noise* sites, size_t n_sites, uint32_t flags) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return NQS_ERR_ARG;
    if ((sites == nullptr) != (n_sites == 0)) return NQS_ERR_ARG;
    if (flags & ~(uint32_t)NQS_PREP_PRUNE_ZERO_RANK) return NQS_ERR_ARG;
    std::vector<NoiseSite> ns;
    if (sites) {
        if (n_sites > 4096) return NQS_ERR_UNSUPPORTED;
        int prev = -2;
        for (size_t i = 0; i < n_sites; ++i) {
            const nqs_noise& s = sites[i];
            if (s.qubit >= (uint32_t)h->circ.n || s.n_kraus < 1 || s.n_kraus > 16 || !s.kraus) return NQS_ERR_ARG;
            if (s.after_gate < -1 || s.after_gate >= (int)h->circ.gates.size() || s.after_gate < prev)
                return NQS_ERR_ARG;
            prev = s.after_gate;
            NoiseSite t;
            t.after_gate = s.after_gate;
            t.qubit = (int)s.qubit;
            for (uint32_t k = 0; k < s.n_kraus; ++k) {
                Mat2 m;
                for (int e = 0; e < 4; ++e) m[e] = cd(s.kraus[8 * k + 2 * e], s.kraus[8 * k + 2 * e + 1]);
                t.kraus.push_back(m);
            }
            ns.push_back(t);
        }
    } else {
        ns = h->circ.noises;
    }
    bool general = false;
    for (const auto& s : ns) general = general || s.general();
    if (general) {
        // two-qubit or superoperator noises: every site goes through the general path
        std::vector<GFactors> gf(ns.size());
        for (size_t i = 0; i < ns.size(); ++i) {
            int rc = factor_general(ns[i], gf[i]);
            if (rc != NQS_OK) return rc;
        }
        engine_batch_forget(h);
        engine_destroy(*h);
        sets_destroy(*h);
        general_destroy(*h);
        h->circ.noises = ns;
        h->factors.clear();
        h->gfac = gf;
        h->general = true;
        h->plan = Plan{};
        h->prepared = true;
        return NQS_OK;
    }
    std::vector<Factors> fac(ns.size());
    for (size_t i = 0; i < ns.size(); ++i) {
        int rc = factor_noise(ns[i], (flags & NQS_PREP_PRUNE_ZERO_RANK) != 0, fac[i]);
        if (rc != NQS_OK) return rc;
    }
    engine_batch_forget(h);
    engine_destroy(*h);
    sets_destroy(*h);
    general_destroy(*h);
    h->general = false;
    h->gfac.clear();
    h->circ.noises = ns;
    h->factors = fac;
    build_plan(h->circ, h->factors, kTileQubits, h->plan);
    h->prepared = true;
    return NQS_OK;
}

static int check_state(const Handle& h, const nqs_state* s, bool allow_ideal) {
    if (!s) return NQS_ERR_ARG;
    if (s->kind == NQS_STATE_BASIS) {
        if (h.circ.n < 64 && (s->bits >> h.circ.n) != 0) return NQS_ERR_ARG;
        return NQS_OK;
    }
    if (s->kind == NQS_STATE_DENSE) {
        if (!s->dev || ((uintptr_t)s->dev & 15u)) return NQS_ERR_ARG;
        return NQS_OK;
    }
    if (s->kind == NQS_STATE_IDEAL && allow_ideal) return NQS_OK;
    return NQS_ERR_ARG;
}

int nqs_fidelity(nqs_handle hh, const nqs_state* psi, const nqs_state* v, int level, nqs_result* out,
                 void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !out || level < 0) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    int rc = check_state(*h, psi, false);
    if (rc) return rc;
    rc = check_state(*h, v, true);
    if (rc) return rc;
    if (h->general) {
        const int lvl = std::min(level, (int)h->gfac.size());
        if (lvl > NQS_MAX_LEVEL) return NQS_ERR_ARG;
        return general_fidelity(*h, psi, v, lvl, out, stream);
    }
    int lvl = std::min(level, (int)h->factors.size());
    if (lvl > NQS_MAX_LEVEL) return NQS_ERR_ARG;
    if (h->opt_shard_rank >= std::max(1, h->opt_shard_count)) return NQS_ERR_ARG;
    return engine_fidelity(*h, psi, v, lvl, out, stream);
}

int nqs_batch_fidelity(const nqs_handle* hs, size_t count, const nqs_state* psis, const nqs_state* vs,
                       const int* levels, nqs_result* outs, void* stream) {
    if (count == 0) return NQS_OK;
    if (!hs || !psis || !vs || !levels || !outs) return NQS_ERR_ARG;
    std::vector<Handle*> H(count);
    for (size_t i = 0; i < count; ++i) {
        Handle* h = reinterpret_cast<Handle*>(hs[i]);
        if (!h || levels[i] < 0) return NQS_ERR_ARG;
        if (!h->prepared) return NQS_ERR_ORDER;
        if (h->general) return NQS_ERR_UNSUPPORTED;   // one-qubit channels only
        int rc = check_state(*h, &psis[i], false);
        if (rc) return rc;
        rc = check_state(*h, &vs[i], true);
        if (rc) return rc;
        if (std::min(levels[i], (int)h->factors.size()) > NQS_MAX_LEVEL) return NQS_ERR_ARG;
        for (size_t j = 0; j < i; ++j)
            if (H[j] == h) return NQS_ERR_ARG;   // each handle once per batch
        H[i] = h;
    }
    return engine_batch_fidelity(H.data(), count, psis, vs, levels, outs, stream);
}

int nqs_enumerate_terms(nqs_handle hh, int level, uint64_t* rec, size_t cap, size_t* count) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (h && h->general) return NQS_ERR_UNSUPPORTED;   // one-qubit channels only
    if (!h || !count || level < 0 || (cap && !rec)) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    const int N = (int)h->factors.size();
    int lvl = std::min(level, N);
    if (lvl > 4 || N > 4096) return NQS_ERR_UNSUPPORTED;
    size_t written = 0, total = 0;
    auto emit = [&](uint64_t r) {
        if (written < cap) rec[written++] = r;
        ++total;
    };
    for (int u = 0; u <= lvl; ++u) {
        std::vector<int> comb(u);
        for (int j = 0; j < u; ++j) comb[j] = j;
        while (true) {
            // factor tuples over each chosen site's kept factors, lexicographic
            std::vector<int> fp(u, 0);
            bool any = true;
            for (int j = 0; j < u; ++j)
                if (h->factors[comb[j]].m == 0) any = false;
            while (any) {
                uint64_t r = (uint64_t)u;
                for (int j = 0; j < u; ++j) {
                    uint64_t field = (uint64_t)comb[j] | ((uint64_t)h->factors[comb[j]].keep[fp[j]] << 12);
                    r |= field << (4 + 14 * j);
                }
                emit(r);
                int j = u - 1;
                while (j >= 0 && fp[j] + 1 >= h->factors[comb[j]].m) fp[j--] = 0;
                if (j < 0) break;
                ++fp[j];
            }
            if (u == 0) break;
            int j = u - 1;
            while (j >= 0 && comb[j] == N - u + j) --j;
            if (j < 0) break;
            ++comb[j];
            for (int t = j + 1; t < u; ++t) comb[t] = comb[t - 1] + 1;
        }
    }
    *count = total;
    return NQS_OK;
}

int nqs_noise_factors(nqs_handle hh, uint32_t site, double* d4, double* K) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (h && h->general) return NQS_ERR_UNSUPPORTED;   // one-qubit channels only
    if (!h || !d4 || !K) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    if (site >= h->factors.size()) return NQS_ERR_ARG;
    const Factors& f = h->factors[site];
    for (int i = 0; i < 4; ++i) {
        d4[i] = f.d[i];
        for (int e = 0; e < 4; ++e) {
            K[8 * i + 2 * e] = f.K[i][e].real();
            K[8 * i + 2 * e + 1] = f.K[i][e].imag();
        }
    }
    return NQS_OK;
}

int nqs_general_factors(nqs_handle hh, uint32_t site, int32_t* m, int32_t* dim, int32_t* same, double* sv, double* KA,
                        double* KB) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !m || !dim || !same) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    if (!h->general) return NQS_ERR_UNSUPPORTED;
    if (site >= h->gfac.size()) return NQS_ERR_ARG;
    const GFactors& f = h->gfac[site];
    *m = f.m;
    *dim = f.nq == 1 ? 2 : 4;
    *same = f.same ? 1 : 0;
    if (sv)
        for (int i = 0; i < f.m; ++i) sv[i] = f.d[i];
    for (size_t e = 0; e < f.KA.size(); ++e) {
        if (KA) {
            KA[2 * e] = f.KA[e].real();
            KA[2 * e + 1] = f.KA[e].imag();
        }
        if (KB) {
            KB[2 * e] = f.KB[e].real();
            KB[2 * e + 1] = f.KB[e].imag();
        }
    }
    return NQS_OK;
}

int nqs_shard_mask(nqs_handle hh, int level, int rank, int count, uint8_t* mask, size_t cap, size_t* n) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !n || level < 0 || count < 1 || rank < 0 || rank >= count || (cap && !mask)) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    if (h->general) return NQS_ERR_UNSUPPORTED;
    const int N = (int)h->factors.size();
    const int lvl = std::min(level, N);
    std::vector<int> m(N);
    for (int s = 0; s < N; ++s) m[s] = h->factors[s].m;
    TermIndex ti;
    ti.build(m, lvl);
    *n = (size_t)ti.total;
    if (!mask || cap < ti.total) return NQS_OK;
    for (int u = 0; u <= lvl; ++u) {
        const uint64_t lo = ti.level_offset[u], hi = ti.level_offset[u + 1];
        if (u <= 1) {
            std::memset(mask + lo, rank == 0 ? 1 : 0, hi - lo);
            continue;
        }
        // level u: site tuples in lexicographic order; the first site decides
        uint64_t at = lo;
        for (int s = 0; s < N && at < hi; ++s) {
            const uint64_t cnt = (uint64_t)m[s] * ti.E[u - 1][s + 1];   // tuples starting at s
            std::memset(mask + at, (s % count == rank) ? 1 : 0, cnt);
            at += cnt;
        }
    }
    return NQS_OK;
}

int nqs_term_values(nqs_handle hh, double* out, size_t cap, size_t* count) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !count || (cap && !out)) return NQS_ERR_ARG;
    if (h->general) return general_term_values(*h, out, cap, count);
    return engine_term_values(*h, out, cap, count);
}

int nqs_plan_check(nqs_handle hh, double* max_abs_err) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !max_abs_err) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    if (h->general) return NQS_ERR_UNSUPPORTED;
    const Plan& p = h->plan;
    *max_abs_err = p.n <= 10 ? plan_product_error(h->circ, h->factors, p) : 0.0;
    // the sweeps take the noise sites in their order: site_pos must increase
    for (size_t s = 1; s < p.site_pos.size(); ++s)
        if (p.site_pos[s] <= p.site_pos[s - 1]) *max_abs_err = HUGE_VAL;
    // pass structure of both segmentations
    const int max_sites = h->opt_max_sites > 0 ? h->opt_max_sites : 4;
    const int max_ops = h->opt_max_ops > 0 ? h->opt_max_ops : 96;
    for (const std::vector<PassSpec>* segs : {&p.free_passes, &p.sitecut_passes}) {
        int at = 0;
        for (const PassSpec& ps : *segs) {
            bool ok = ps.op_begin == at && ps.op_end > ps.op_begin && ps.op_end - ps.op_begin <= max_ops &&
                      (int)ps.local.size() == p.k;
            std::vector<char> in(p.n, 0);
            for (size_t j = 0; j < ps.local.size() && ok; ++j) {
                const int q = ps.local[j];
                ok = q >= 0 && q < p.n && !in[q] && (j == 0 || q > ps.local[j - 1]);
                if (ok) in[q] = 1;
            }
            for (int q = 0; q < p.c && ok; ++q) ok = in[q];
            int sites = 0;
            for (int i = ps.op_begin; i < ps.op_end && ok; ++i) {
                const HostOp& o = p.ops[i];
                if (o.type == OP_SITE) ++sites;
                if (o.type == OP_G1 || o.type == OP_SITE) ok = in[o.q0];
                if (o.type == OP_G2) ok = in[o.q0] && in[o.q1];
            }
            if (!ok || sites > max_sites) *max_abs_err = HUGE_VAL;
            at = ps.op_end;
        }
        if (at != (int)p.ops.size()) *max_abs_err = HUGE_VAL;
    }
    return NQS_OK;
}

int nqs_jit_compile_check(nqs_handle hh, int states, int max_passes, int* compiled) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !compiled || (states != 1 && states != 3) || max_passes < 1) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    if (h->general) return NQS_ERR_UNSUPPORTED;
    return engine_jit_compile_check(*h, states, max_passes, compiled);
}

int nqs_truncation_bound(nqs_handle hh, int level, double* out) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !out || level < 0) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    std::vector<double> poly(1, 1.0);
    std::vector<std::pair<double, double>> norms;
    for (const auto& f : h->factors) norms.push_back({f.norm_dom, f.norm_rest});
    for (const auto& f : h->gfac) norms.push_back({f.norm_dom, f.norm_rest});
    for (const auto& nr : norms) {
        std::vector<double> nx(poly.size() + 1, 0.0);
        for (size_t i = 0; i < poly.size(); ++i) {
            nx[i] += poly[i] * nr.first;
            nx[i + 1] += poly[i] * nr.second;
        }
        poly.swap(nx);
    }
    double b = 0.0;
    for (size_t i = (size_t)level + 1; i < poly.size(); ++i) b += poly[i];
    *out = b;
    return NQS_OK;
}

int nqs_fidelity_adaptive(nqs_handle hh, const nqs_state* psi, const nqs_state* v, double tol, int max_level,
                          uint32_t criteria, nqs_result* out, void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !out || !(tol >= 0.0) || max_level < 0) return NQS_ERR_ARG;
    if (!(criteria & (NQS_ADAPT_BOUND | NQS_ADAPT_OBSERVED)) || (criteria & ~3u)) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    const int N = (int)(h->general ? h->gfac.size() : h->factors.size());
    int top = std::min(std::min(max_level, N), NQS_MAX_LEVEL);
    if (criteria & NQS_ADAPT_BOUND) {
        // smallest level whose truncation bound is within tol
        int l = 0;
        double b = 0.0;
        for (; l < top; ++l) {
            if (nqs_truncation_bound(hh, l, &b) != NQS_OK) return NQS_ERR_ARG;
            if (b <= tol) break;
        }
        top = l;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int start = (criteria & NQS_ADAPT_OBSERVED) ? std::min(1, top) : top;
    for (int l = start; l <= top; ++l) {
        int rc = nqs_fidelity(hh, psi, v, l, out, stream);
        if (rc != NQS_OK) return rc;
        if (cudaStreamSynchronize(st) != cudaSuccess) return NQS_ERR_CUDA;
        if (out->status != NQS_OK) return NQS_OK;   // the device error is in out->status
        if ((criteria & NQS_ADAPT_OBSERVED) && std::fabs(out->T[l]) <= tol) break;
    }
    return NQS_OK;
}

int nqs_offdiagonal(nqs_handle hh, const nqs_state* psi, const nqs_state* x, const nqs_state* y, int level,
                    double* out, nqs_result* parts, void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !out || level < 0) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    int rc = check_state(*h, psi, false);
    if (rc) return rc;
    if (check_state(*h, x, false) || check_state(*h, y, false)) return NQS_ERR_ARG;
    const int lvl = std::min(level, (int)(h->general ? h->gfac.size() : h->factors.size()));
    if (lvl > NQS_MAX_LEVEL) return NQS_ERR_ARG;
    const long long dim = 1ll << h->circ.n;
    const size_t bytes = (size_t)dim * 8;
    cudaStream_t st = (cudaStream_t)stream;
    float2* v = (float2*)dev_alloc(bytes, stream);
    if (!v) return NQS_ERR_NOMEM;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::max<long long>(1, std::min<long long>((long long)sms * 8, dim / 256));
    // f(v) = <v|rho_l|v> for v = x + i^k y, k = 0..3;  <x|rho_l|y> = 1/4 sum_k i^(-k) f(x + i^k y)
    const float cr[4] = {1.f, 0.f, -1.f, 0.f}, ci[4] = {0.f, 1.f, 0.f, -1.f};
    double re = 0.0, im = 0.0;
    for (int k = 0; k < 4 && rc == NQS_OK; ++k) {
        if (launch_combine(v, dim, x->kind == NQS_STATE_DENSE, x->bits, (const float2*)x->dev,
                           y->kind == NQS_STATE_DENSE, y->bits, (const float2*)y->dev, cr[k], ci[k], grid,
                           st) != cudaSuccess) {
            rc = NQS_ERR_CUDA;
            break;
        }
        nqs_state vs{};
        vs.kind = NQS_STATE_DENSE;
        vs.dev = v;
        nqs_result r{};
        rc = h->general ? general_fidelity(*h, psi, &vs, lvl, &r, stream) : engine_fidelity(*h, psi, &vs, lvl, &r, stream);
        if (rc == NQS_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = NQS_ERR_CUDA;
        if (rc != NQS_OK) break;
        if (parts) parts[k] = r;
        if (r.status != NQS_OK) rc = r.status;
        // i^(-k) f_k
        const double f = r.F;
        if (k == 0) re += f;
        else if (k == 1) im -= f;
        else if (k == 2) re -= f;
        else im += f;
    }
    cudaStreamSynchronize(st);
    dev_free(v, bytes, stream);
    if (rc != NQS_OK) return rc;
    out[0] = 0.25 * re;
    out[1] = 0.25 * im;
    return NQS_OK;
}

int nqs_get_info(nqs_handle hh, nqs_info* out) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !out) return NQS_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    out->n_qubits = h->circ.n;
    out->n_gates = (int32_t)h->circ.gates.size();
    out->n_sites = (int32_t)h->circ.noises.size();
    if (h->prepared) {
        out->n_ops = (int32_t)h->plan.ops.size();
        out->n_passes = (int32_t)h->plan.free_passes.size();
        out->tile_qubits = h->plan.k;
    }
    out->workspace_bytes = engine_workspace_bytes(*h);
    out->upload_bytes = engine_upload_bytes(*h);
    out->launches_per_call = engine_launches_per_call(*h);
    int n_states = 0;
    out->ckpt_spacing = engine_spacing(*h, &n_states);
    out->n_states = n_states;
    int js = 0;
    out->jit_launches = engine_jit_info(*h, &js);
    out->jit_state = js;
    return NQS_OK;
}

namespace {

void resegment(Handle& h) {
    const int sites = h.opt_max_sites > 0 ? h.opt_max_sites : 4;
    const int ops = h.opt_max_ops > 0 ? h.opt_max_ops : 96;
    // the reordering's passes keep any bounds at least as loose as their own
    if (!h.plan.grouped_passes.empty() && sites >= 4 && ops >= 96)
        h.plan.free_passes = h.plan.grouped_passes;
    else
        h.plan.free_passes = segment(h.plan, false, sites, ops);
    h.plan.sitecut_passes = segment(h.plan, true, sites, ops);
}

}  // namespace

int nqs_schedule_launches(nqs_handle hh, nqs_launch_info* out, size_t cap, size_t* count) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !count) return NQS_ERR_ARG;
    return engine_launch_list(*h, out, cap, count);
}

int nqs_set_option(nqs_handle hh, int option, int64_t value) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || value < 0) return NQS_ERR_ARG;
    switch (option) {
        case NQS_OPT_CKPT_SPACING:
            if (value > (1 << 20)) return NQS_ERR_ARG;
            h->opt_spacing = (int)value;
            break;
        case NQS_OPT_SWEEP_RB:
            if (value != 0 && value != 3 && value != 4) return NQS_ERR_ARG;
            h->opt_rb_multi = (int)value;
            break;
        case NQS_OPT_JIT:
            if (value > 2) return NQS_ERR_ARG;
            h->opt_jit = (int)value;
            break;
        case NQS_OPT_SHARD_RANK:
            if (value > 65535) return NQS_ERR_ARG;
            h->opt_shard_rank = (int)value;
            break;
        case NQS_OPT_SHARD_COUNT:
            if (value > 65536) return NQS_ERR_ARG;
            h->opt_shard_count = (int)value;
            break;
        case NQS_OPT_MAX_OPS:
        case NQS_OPT_MAX_SITES: {
            if (!h->prepared) return NQS_ERR_ORDER;
            const bool ops = option == NQS_OPT_MAX_OPS;
            if (value != 0 && (ops ? (value < 8 || value > 160) : (value < 1 || value > 8))) return NQS_ERR_ARG;
            (ops ? h->opt_max_ops : h->opt_max_sites) = (int)value;
            resegment(*h);
            break;
        }
        default:
            return NQS_ERR_ARG;
    }
    engine_invalidate(*h);
    return NQS_OK;
}

int nqs_get_option(nqs_handle hh, int option, int64_t* value) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !value) return NQS_ERR_ARG;
    switch (option) {
        case NQS_OPT_CKPT_SPACING: *value = h->opt_spacing; break;
        case NQS_OPT_SWEEP_RB: *value = h->opt_rb_multi; break;
        case NQS_OPT_JIT: *value = h->opt_jit; break;
        case NQS_OPT_SHARD_RANK: *value = h->opt_shard_rank; break;
        case NQS_OPT_SHARD_COUNT: *value = h->opt_shard_count; break;
        case NQS_OPT_MAX_OPS: *value = h->opt_max_ops; break;
        case NQS_OPT_MAX_SITES: *value = h->opt_max_sites; break;
        default: return NQS_ERR_ARG;
    }
    return NQS_OK;
}

int nqs_autotune(nqs_handle hh, const nqs_state* psi, const nqs_state* v, int level, int trials, nqs_result* out,
                 void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (h && h->general) return NQS_ERR_UNSUPPORTED;   // one-qubit channels only
    if (!h || trials < 1 || level < 0) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return NQS_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return NQS_ERR_CUDA;
    }
    nqs_result res{};
    // register qubits matter only where multi-state passes run (level >= 2)
    const int rbs[2] = {3, 4};
    const int n_rb = level >= 2 ? 2 : 1;
    const int opss[3] = {64, 96, 128};
    float best_ms = -1.f;
    int best_rb = 0, best_ops = 0, rc = NQS_OK;
    for (int a = 0; a < n_rb && rc == NQS_OK; ++a)
        for (int b = 0; b < 3 && rc == NQS_OK; ++b) {
            const int rb = n_rb > 1 ? rbs[a] : 0;
            if ((rc = nqs_set_option(hh, NQS_OPT_SWEEP_RB, rb)) != NQS_OK) break;
            if ((rc = nqs_set_option(hh, NQS_OPT_MAX_OPS, opss[b])) != NQS_OK) break;
            int r = nqs_fidelity(hh, psi, v, level, &res, stream);   // builds the schedule
            if (r == NQS_ERR_UNSUPPORTED) continue;                   // program does not fit: skip
            if (r != NQS_OK) {
                rc = r;
                break;
            }
            if (cudaEventRecord(e0, st) != cudaSuccess) rc = NQS_ERR_CUDA;
            for (int t = 0; t < trials && rc == NQS_OK; ++t) rc = nqs_fidelity(hh, psi, v, level, &res, stream);
            if (rc == NQS_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = NQS_ERR_CUDA;
            if (rc == NQS_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = NQS_ERR_CUDA;
            float ms = 0.f;
            if (rc == NQS_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = NQS_ERR_CUDA;
            if (rc == NQS_OK && (best_ms < 0.f || ms < best_ms)) {
                best_ms = ms;
                best_rb = rb;
                best_ops = opss[b];
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != NQS_OK) return rc;
    if (best_ms < 0.f) return NQS_ERR_UNSUPPORTED;
    nqs_set_option(hh, NQS_OPT_SWEEP_RB, best_rb);
    nqs_set_option(hh, NQS_OPT_MAX_OPS, best_ops);
    if (out) *out = res;
    return NQS_OK;
}

int nqs_set_profiling(nqs_handle hh, int on) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return NQS_ERR_ARG;
    if (h->profiling) {
        int rc = engine_collect_stats(*h);
        if (rc) return rc;
    }
    h->profiling = on != 0;
    if (on)
        for (auto& s : h->stats) s = nqs_kernel_stats{};
    return NQS_OK;
}

int nqs_get_kernel_stats(nqs_handle hh, int kind, nqs_kernel_stats* out) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !out || kind < 0 || kind > 4) return NQS_ERR_ARG;
    if (h->profiling) {
        int rc = engine_collect_stats(*h);
        if (rc) return rc;
    }
    *out = h->stats[kind];
    return NQS_OK;
}

int nqs_reduced_matrix(const void* phi, const void* chi, int n, int qubit, double* R_out, void* scratch,
                       size_t scratch_bytes, void* stream) {
    if (!phi || !chi || !R_out || !scratch || n < 1 || n > 34 || qubit < 0 || qubit >= n) return NQS_ERR_ARG;
    if (((uintptr_t)phi & 15u) || ((uintptr_t)chi & 15u) || ((uintptr_t)scratch & 7u)) return NQS_ERR_ARG;
    return engine_reduced_matrix(phi, chi, n, qubit, R_out, scratch, scratch_bytes, stream);
}

size_t nqs_reduced_matrix_scratch_bytes(int n) {
    if (n < 1 || n > 34) return 0;
    return engine_reduced_matrix_scratch_bytes(n);
}

int nqs_prepare_sets(nqs_handle hh, const nqs_state* psi, const nqs_state* v, void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (h && h->general) return NQS_ERR_UNSUPPORTED;   // one-qubit channels only
    if (!h) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    int rc = check_state(*h, psi, false);
    if (rc) return rc;
    rc = check_state(*h, v, true);
    if (rc) return rc;
    return engine_prepare_sets(*h, psi, v, stream);
}

int nqs_eval_sets(nqs_handle hh, int k, const int32_t* sets, size_t m, double* W_out, void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (h && h->general) return NQS_ERR_UNSUPPORTED;   // one-qubit channels only
    if (!h || !sets || !W_out || k < 1 || k > 3) return NQS_ERR_ARG;
    if (m == 0) return NQS_OK;
    return engine_eval_sets(*h, k, sets, m, W_out, stream);
}

int nqs_mlp_create(int n_in, int hidden, int hidden_layers, uint64_t seed, nqs_mlp* out) {
    if (!out) return NQS_ERR_ARG;
    Mlp* m = nullptr;
    int rc = mlp_create(n_in, hidden, hidden_layers, seed, &m);
    if (rc == NQS_OK) *out = reinterpret_cast<nqs_mlp>(m);
    return rc;
}

size_t nqs_mlp_param_count(nqs_mlp m) { return m ? mlp_n_params(reinterpret_cast<Mlp*>(m)) : 0; }

int nqs_mlp_get_params(nqs_mlp m, float* host, size_t cap) {
    if (!m || !host) return NQS_ERR_ARG;
    return mlp_get_params(reinterpret_cast<Mlp*>(m), host, cap);
}

int nqs_mlp_set_params(nqs_mlp m, const float* host, size_t count) {
    if (!m || !host) return NQS_ERR_ARG;
    return mlp_set_params(reinterpret_cast<Mlp*>(m), host, count);
}

int nqs_mlp_forward(nqs_mlp m, const float* X, int batch, float* y, void* stream) {
    if (!m || !X || !y || batch < 1) return NQS_ERR_ARG;
    return mlp_forward(reinterpret_cast<Mlp*>(m), X, batch, y, stream);
}

int nqs_mlp_loss_grad(nqs_mlp m, const float* X, const float* y, int batch, double* loss, float* grad_host, size_t cap,
                      void* stream) {
    if (!m || !X || !y || !loss || !grad_host || batch < 1) return NQS_ERR_ARG;
    return mlp_loss_grad(reinterpret_cast<Mlp*>(m), X, y, batch, loss, grad_host, cap, stream);
}

int nqs_mlp_train(nqs_mlp m, const float* X, const float* y, int n, int batch, int steps, float lr, uint64_t seed,
                  double* final_loss, void* stream) {
    if (!m || !X || !y || !(lr > 0.f)) return NQS_ERR_ARG;
    return mlp_train(reinterpret_cast<Mlp*>(m), X, y, n, batch, steps, lr, seed, final_loss, stream);
}

void nqs_mlp_destroy(nqs_mlp m) { mlp_destroy(reinterpret_cast<Mlp*>(m)); }

int nqs_site_features(nqs_handle hh, const double* W1, float* out) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (h && h->general) return NQS_ERR_UNSUPPORTED;   // one-qubit channels only
    if (!h || !W1 || !out) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    return site_features(*h, W1, out);
}

int nqs_pair_training_data(nqs_handle hh, const float* feats, const double* W2, float* X, float* y, size_t cap,
                           size_t* count) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (h && h->general) return NQS_ERR_UNSUPPORTED;   // one-qubit channels only
    if (!h || !feats || !W2 || !count || (cap && (!X || !y))) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    return pair_training_data(*h, feats, W2, X, y, cap, count);
}

int nqs_is_estimate(nqs_handle hh, nqs_mlp mlp, int level, uint64_t samples, double alpha, uint64_t seed,
                    const float* feats, const double* W1, nqs_is_result* out, void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (h && h->general) return NQS_ERR_UNSUPPORTED;   // one-qubit channels only
    if (!h || !out || (mlp && (!feats || !W1)) || (!W1)) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    return is_estimate(*h, reinterpret_cast<Mlp*>(mlp), level, samples, alpha, seed, feats, W1, out, stream);
}

int nqs_is_proposal(nqs_handle hh, nqs_mlp mlp, int level, double alpha, const float* feats, const double* W1,
                    double* q_out, size_t cap, size_t* count, void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (h && h->general) return NQS_ERR_UNSUPPORTED;   // one-qubit channels only
    if (!h || !count || !W1 || (mlp && !feats)) return NQS_ERR_ARG;
    if (!h->prepared) return NQS_ERR_ORDER;
    return is_proposal_values(*h, reinterpret_cast<Mlp*>(mlp), level, alpha, feats, W1, q_out, cap, count, stream);
}

void nqs_destroy(nqs_handle hh) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return;
    engine_batch_forget(h);
    engine_destroy(*h);
    sets_destroy(*h);
    general_destroy(*h);
    delete h;
}

const char* nqs_strerror(int code) {
    switch (code) {
        case NQS_OK: return "ok";
        case NQS_ERR_ARG: return "invalid argument";
        case NQS_ERR_PARSE: return "malformed circuit text";
        case NQS_ERR_NOT_CPTP: return "noise channel is not trace preserving (||sum E^dag E - I|| > 1e-10)";
        case NQS_ERR_NOT_DOMINANT: return "noise channel has no unique dominant singular value";
        case NQS_ERR_NOMEM: return "device allocation failed";
        case NQS_ERR_CUDA: return "CUDA runtime error";
        case NQS_ERR_ORDER: return "call order violated (prepare the noise first)";
        case NQS_ERR_DEVICE_TIMEOUT: return "a bounded device-side wait gave up";
        case NQS_ERR_UNSUPPORTED: return "request outside the supported range";
        case NQS_ERR_TOO_LARGE: return "request exceeds the fixed scratch capacity of the allocation-free entry point";
        case NQS_ERR_COMPILE: return "a generated kernel did not compile";
        default: return "unknown status";
    }
}

int nqs_selftest_bounded_wait(int* status_out, void* stream) {
    if (!status_out) return NQS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int* dev = (int*)dev_alloc(sizeof(int), stream);
    if (!dev) return NQS_ERR_NOMEM;
    int rc = cudaMemsetAsync(dev, 0xff, sizeof(int), st) == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
    if (rc == NQS_OK) rc = selftest_bounded_wait(dev, stream);
    if (rc == NQS_OK && cudaMemcpyAsync(status_out, dev, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = NQS_ERR_CUDA;
    if (rc == NQS_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = NQS_ERR_CUDA;
    dev_free(dev, sizeof(int), stream);
    return rc;
}

const char* nqs_version(void) { return "nqs 0.1 (sm_103a)"; }

}  // extern "C"
