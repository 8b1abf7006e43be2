// Sweep planner: one linear operation order shared by every sweep, then
// segmentation of that order into tile passes.
//
// Every noise site becomes an OP_SITE carrying its dominant factor K_0
// (Sec. IV: M' = U_0 (x) V_0); the non-dominant factors enter only through
// the site's reductions and spawns.  Gates are fused while reading the
// circuit: an operation is multiplied into the last operation touching its
// qubits when that operation acts on a superset of them, is not a site, and
// is not diagonal unless the new one is too (diagonal operations never need
// their qubits inside the tile, so they are kept diagonal; CNOT-RZ-CNOT
// collapses into one diagonal two-qubit phase).  Moving a gate past
// operations on other qubits, including sites, is exact: the forward,
// backward and branch sweeps all use this one order, so every checkpoint
// <phi_s| and |chi_s> is cut at the same place.
//
// A pass keeps 2^k amplitudes in shared memory: the lowest c qubits (for
// contiguous 256-byte runs in HBM) plus the qubits of the operations it
// applies.  Diagonal operations on qubits outside the tile read the qubit's
// value from the tile's base index.
#include <algorithm>
#include <cstdlib>
#include <cmath>

#include "nqs_internal.h"

namespace nqs {

namespace {

bool is_diag2(const std::array<cd, 16>& m) {
    double mx = std::max(std::abs(m[0]), std::abs(m[3]));
    double off = std::max(std::abs(m[1]), std::abs(m[2]));
    return off <= 1e-14 * mx || (off == 0.0);
}

bool is_diag4(const std::array<cd, 16>& m) {
    double mx = 0, off = 0;
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double a = std::abs(m[4 * r + c]);
            if (r == c) mx = std::max(mx, a);
            else off = std::max(off, a);
        }
    return off <= 1e-14 * mx || off == 0.0;
}

// a 1q matrix on position `pos` (0 = first/more significant qubit) of a pair
std::array<cd, 16> expand_1q(const std::array<cd, 16>& m2, int pos) {
    std::array<cd, 16> out{};
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            int r0 = r >> 1, r1 = r & 1, c0 = c >> 1, c1 = c & 1;
            if (pos == 0) out[4 * r + c] = (r1 == c1) ? m2[2 * r0 + c0] : cd(0);
            else out[4 * r + c] = (r0 == c0) ? m2[2 * r1 + c1] : cd(0);
        }
    return out;
}

std::array<cd, 16> swap_pair(const std::array<cd, 16>& m) {
    // reorder a 4x4 from (q0, q1) to (q1, q0) indexing
    auto sw = [](int i) { return ((i & 1) << 1) | (i >> 1); };
    std::array<cd, 16> out{};
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) out[4 * sw(r) + sw(c)] = m[4 * r + c];
    return out;
}

std::array<cd, 16> matmul(const std::array<cd, 16>& a, const std::array<cd, 16>& b, int d) {
    std::array<cd, 16> out{};
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
            cd s = 0;
            for (int k = 0; k < d; ++k) s += a[d * r + k] * b[d * k + c];
            out[d * r + c] = s;
        }
    return out;
}

bool op_is_diag(const HostOp& o) { return o.type == OP_D1 || o.type == OP_D2; }

// One pass of the reordering over the remaining operations `rest` with the
// tile qubits fixed to `tile`: every operation is taken (in order) when its
// dense qubits are in the tile and it commutes with every operation skipped
// before it in this pass -- two operations commute when they share no qubit or
// are both diagonal; a noise site commutes with nothing on its qubit (the
// branch states it spawns and the reduction it makes see the state at its
// place) and sites keep their relative order.  Returns the count taken.
int take_pass(const Plan& p, const std::vector<int>& rest, const std::vector<char>& tile, int max_sites, int max_ops,
              std::vector<int>* taken, std::vector<int>* kept) {
    std::vector<char> blk_diag(p.n, 0), blk_any(p.n, 0);
    bool site_skipped = false;
    int sites = 0, cnt = 0;
    for (int idx : rest) {
        const HostOp& o = p.ops[idx];
        const int qs[2] = {o.q0, o.q1};
        const int nq = o.q1 >= 0 ? 2 : 1;
        const bool d = op_is_diag(o), site = o.type == OP_SITE;
        bool ok = !(site && site_skipped) && cnt < max_ops && !(site && sites >= max_sites);
        for (int j = 0; j < nq && ok; ++j)
            if (blk_any[qs[j]] || (!d && blk_diag[qs[j]]) || (!d && !tile[qs[j]])) ok = false;
        if (ok) {
            sites += site;
            ++cnt;
            if (taken) taken->push_back(idx);
        } else {
            for (int j = 0; j < nq; ++j) (d ? blk_diag : blk_any)[qs[j]] = 1;
            site_skipped = site_skipped || site;
            if (kept) kept->push_back(idx);
        }
    }
    return cnt;
}

// Reorders the operations so that in-order segmentation needs fewer passes.
// Pass by pass: the tile holds the always-local low qubits and the dense
// qubits of the first remaining operation, and is filled up to k qubits one
// qubit at a time, each time with the qubit that lets the pass take the most
// operations (take_pass); the pass then takes what it can.  The reordered
// product of operations equals the original one (nqs_plan_check).  `passes`
// receives the passes so formed (tile qubits ascending, padded to k with the
// lowest unused qubits).
void lookahead_order(Plan& p, int max_sites, int max_ops, std::vector<PassSpec>& passes) {
    passes.clear();
    const int nops = (int)p.ops.size();
    std::vector<int> rest(nops), order;
    for (int i = 0; i < nops; ++i) rest[i] = i;
    order.reserve(nops);
    while (!rest.empty()) {
        std::vector<char> tile(p.n, 0);
        int count = 0;
        auto add = [&](int q) {
            if (q >= 0 && !tile[q]) {
                tile[q] = 1;
                ++count;
            }
        };
        for (int q = 0; q < p.c; ++q) add(q);
        const HostOp& first = p.ops[rest[0]];
        if (!op_is_diag(first)) {
            add(first.q0);
            add(first.q1);
        }
        // candidates: dense qubits of the operations near the front
        std::vector<char> cand(p.n, 0);
        for (size_t i = 0; i < rest.size() && i < 512; ++i) {
            const HostOp& o = p.ops[rest[i]];
            if (op_is_diag(o)) continue;
            cand[o.q0] = 1;
            if (o.q1 >= 0) cand[o.q1] = 1;
        }
        while (count < p.k) {
            int best = -1, best_v = -1;
            for (int q = 0; q < p.n; ++q) {
                if (tile[q] || !cand[q]) continue;
                tile[q] = 1;
                const int v = take_pass(p, rest, tile, max_sites, max_ops, nullptr, nullptr);
                tile[q] = 0;
                if (v > best_v) {
                    best_v = v;
                    best = q;
                }
            }
            if (best < 0) break;
            add(best);
        }
        std::vector<int> keep;
        PassSpec ps;
        ps.op_begin = (int)order.size();
        take_pass(p, rest, tile, max_sites, max_ops, &order, &keep);
        ps.op_end = (int)order.size();
        for (int q = 0; q < p.n && count < p.k; ++q) add(q);
        for (int q = 0; q < p.n; ++q)
            if (tile[q]) ps.local.push_back(q);
        passes.push_back(ps);
        rest.swap(keep);
    }
    std::vector<HostOp> ops;
    ops.reserve(nops);
    for (int idx : order) ops.push_back(p.ops[idx]);
    p.ops.swap(ops);
    for (int i = 0; i < nops; ++i)
        if (p.ops[i].type == OP_SITE) p.site_pos[p.ops[i].site] = i;
}

}  // namespace

void build_plan(const Circuit& c, const std::vector<Factors>& f, int tile_qubits, Plan& p) {
    p = Plan{};
    p.n = c.n;
    p.k = std::min(c.n, tile_qubits);
    p.c = std::min(c.n, 5);
    std::vector<int> last(c.n, -1);

    auto append = [&](HostOp op) {
        int qa = op.q0, qb = op.q1;
        if (op.type != OP_SITE) {
            int cand = last[qa];
            bool ok = cand >= 0 && (qb < 0 || last[qb] == cand);
            if (ok) {
                HostOp& t = p.ops[cand];
                bool t_two = (t.type == OP_G2 || t.type == OP_D2);
                bool t_one = (t.type == OP_G1 || t.type == OP_D1);
                bool covers = (qb < 0) ? ((t_one && t.q0 == qa) || (t_two && (t.q0 == qa || t.q1 == qa)))
                                       : (t_two && ((t.q0 == qa && t.q1 == qb) || (t.q0 == qb && t.q1 == qa)));
                bool diag_ok = !op_is_diag(t) || op_is_diag(op);
                if (t.type != OP_SITE && covers && diag_ok) {
                    bool new_two = (op.type == OP_G2 || op.type == OP_D2);
                    if (t_one) {
                        t.m = matmul(op.m, t.m, 2);
                    } else {
                        std::array<cd, 16> m4;
                        if (!new_two) m4 = expand_1q(op.m, qa == t.q0 ? 0 : 1);
                        else m4 = (op.q0 == t.q0) ? op.m : swap_pair(op.m);
                        t.m = matmul(m4, t.m, 4);
                    }
                    bool d = t_one ? is_diag2(t.m) : is_diag4(t.m);
                    if (t_one) t.type = d ? OP_D1 : OP_G1;
                    else t.type = d ? OP_D2 : OP_G2;
                    return;
                }
            }
        }
        p.ops.push_back(op);
        int idx = (int)p.ops.size() - 1;
        last[qa] = idx;
        if (qb >= 0) last[qb] = idx;
    };

    auto gate_op = [&](const Gate& g) {
        HostOp o;
        o.q0 = g.q0;
        if (gate_is_two_qubit(g.kind)) {
            o.q1 = g.q1;
            Mat4 m = gate_matrix_2q(g);
            std::copy(m.begin(), m.end(), o.m.begin());
            o.type = is_diag4(o.m) ? OP_D2 : OP_G2;
        } else {
            Mat2 m = gate_matrix_1q(g);
            for (int e = 0; e < 4; ++e) o.m[e] = m[e];
            o.type = is_diag2(o.m) ? OP_D1 : OP_G1;
        }
        return o;
    };
    auto site_op = [&](int s) {
        HostOp o;
        o.type = OP_SITE;
        o.q0 = c.noises[s].qubit;
        o.site = s;
        for (int e = 0; e < 4; ++e) o.m[e] = f[s].K[0][e];
        o.diag = is_diag2(o.m);
        if (o.diag) o.m[1] = o.m[2] = cd(0);
        return o;
    };

    p.site_pos.assign(c.noises.size(), -1);
    size_t ns = 0;
    auto flush_sites = [&](int g) {
        while (ns < c.noises.size() && c.noises[ns].after_gate == g) {
            append(site_op((int)ns));
            p.site_pos[ns] = (int)p.ops.size() - 1;
            ++ns;
        }
    };
    flush_sites(-1);
    for (size_t g = 0; g < c.gates.size(); ++g) {
        append(gate_op(c.gates[g]));
        flush_sites((int)g);
    }
    // A dense two-qubit operation that is diagonal up to a Hadamard on one of
    // its qubits (a CNOT left alone, e.g. when a noise site sits inside a
    // CNOT-RZ-CNOT) is rewritten as H, diagonal, H on that qubit and the
    // order is fused again: the diagonal part needs no register qubits and
    // the Hadamards join neighbouring one-qubit operations where they can.
    {
        const double r2 = std::sqrt(0.5);
        std::array<cd, 16> h{};
        h[0] = h[1] = h[2] = cd(r2);
        h[3] = cd(-r2);
        std::vector<HostOp> old_ops;
        old_ops.swap(p.ops);
        bool changed = false;
        std::vector<HostOp> expanded;
        for (const HostOp& o : old_ops) {
            if (o.type == OP_G2) {
                bool done = false;
                for (int pos = 1; pos >= 0 && !done; --pos) {
                    const std::array<cd, 16> h4 = expand_1q(h, pos);
                    const std::array<cd, 16> m = matmul(h4, matmul(o.m, h4, 4), 4);
                    if (!is_diag4(m)) continue;
                    HostOp hg;
                    hg.type = OP_G1;
                    hg.q0 = pos == 0 ? o.q0 : o.q1;
                    hg.m = h;
                    HostOp d = o;
                    d.type = OP_D2;
                    d.m = m;
                    expanded.push_back(hg);
                    expanded.push_back(d);
                    expanded.push_back(hg);
                    done = changed = true;
                }
                if (done) continue;
            }
            expanded.push_back(o);
        }
        if (!changed) {
            p.ops.swap(old_ops);
        } else {
            std::fill(last.begin(), last.end(), -1);
            for (const HostOp& o : expanded) {
                append(o);
                if (o.type == OP_SITE) p.site_pos[o.site] = (int)p.ops.size() - 1;
            }
        }
    }
    // exact zeros for the off-diagonals of diagonal operations
    for (auto& o : p.ops) {
        if (o.type == OP_D1) o.m[1] = o.m[2] = cd(0);
        if (o.type == OP_D2)
            for (int r = 0; r < 4; ++r)
                for (int cc = 0; cc < 4; ++cc)
                    if (r != cc) o.m[4 * r + cc] = cd(0);
    }
    // bounded passes: at most 4 reductions and 96 operations each, so a pass's
    // program and reduction slots fit next to the tiles in shared memory
    {
        const char* e = std::getenv("NQS_PLAN_REORDER");   // 0: keep the circuit order
        if (!(e && e[0] == '0')) {
            lookahead_order(p, 4, 96, p.grouped_passes);
            p.free_passes = p.grouped_passes;
        } else {
            p.free_passes = segment(p, false, 4, 96);
        }
    }
    p.sitecut_passes = segment(p, true, 4, 96);
}

std::vector<PassSpec> segment(const Plan& p, bool cut_after_sites, int max_sites_per_pass, int max_ops_per_pass,
                              const std::vector<char>* cut_after) {
    std::vector<PassSpec> out;
    const int nops = (int)p.ops.size();
    auto needs = [&](const HostOp& o, int q[2]) {
        int cnt = 0;
        if (o.type == OP_G1 || o.type == OP_SITE) q[cnt++] = o.q0;
        if (o.type == OP_G2) {
            q[cnt++] = o.q0;
            q[cnt++] = o.q1;
        }
        return cnt;
    };
    int i = 0;
    if (nops == 0) {
        PassSpec ps;
        for (int q = 0; q < p.k; ++q) ps.local.push_back(q);
        ps.op_begin = ps.op_end = 0;
        out.push_back(ps);
        return out;
    }
    while (i < nops) {
        std::vector<char> in(p.n, 0);
        int count = 0;
        for (int q = 0; q < p.c; ++q) {
            in[q] = 1;
            ++count;
        }
        PassSpec ps;
        ps.op_begin = i;
        int sites = 0;
        while (i < nops) {
            int q[2];
            int cnt = needs(p.ops[i], q);
            int extra = 0;
            for (int j = 0; j < cnt; ++j) extra += in[q[j]] ? 0 : 1;
            if (cnt == 2 && q[0] == q[1]) extra = in[q[0]] ? 0 : 1;
            if (count + extra > p.k || i - ps.op_begin >= max_ops_per_pass) break;
            for (int j = 0; j < cnt; ++j)
                if (!in[q[j]]) {
                    in[q[j]] = 1;
                    ++count;
                }
            bool site = p.ops[i].type == OP_SITE;
            ++i;
            if (site) {
                ++sites;
                const bool cut = cut_after && (*cut_after)[p.ops[i - 1].site];
                if (cut_after_sites || cut || sites >= max_sites_per_pass) break;
            }
        }
        ps.op_end = i;
        // pad the tile to exactly k qubits with the lowest unused ones
        for (int q = 0; q < p.n && count < p.k; ++q)
            if (!in[q]) {
                in[q] = 1;
                ++count;
            }
        for (int q = 0; q < p.n; ++q)
            if (in[q]) ps.local.push_back(q);
        out.push_back(ps);
    }
    return out;
}

// Largest entry difference between the operator of the plan's operation order
// and that of the circuit with K_0 at every noise site (both applied to every
// basis state, FP64): fusion, the Hadamard rewrite and the reordering must
// leave the product unchanged.
double plan_product_error(const Circuit& c, const std::vector<Factors>& f, const Plan& p) {
    const int n = c.n;
    const size_t D = (size_t)1 << n;
    auto apply1 = [&](std::vector<cd>& v, int q, const cd* m) {
        const size_t b = (size_t)1 << q;
        for (size_t i = 0; i < D; ++i)
            if (!(i & b)) {
                const cd x0 = v[i], x1 = v[i | b];
                v[i] = m[0] * x0 + m[1] * x1;
                v[i | b] = m[2] * x0 + m[3] * x1;
            }
    };
    auto apply2 = [&](std::vector<cd>& v, int q0, int q1, const cd* m) {   // row 2*b(q0) + b(q1)
        const size_t b0 = (size_t)1 << q0, b1 = (size_t)1 << q1;
        for (size_t i = 0; i < D; ++i)
            if (!(i & b0) && !(i & b1)) {
                const size_t idx[4] = {i, i | b1, i | b0, i | b0 | b1};
                cd x[4], y[4];
                for (int e = 0; e < 4; ++e) x[e] = v[idx[e]];
                for (int r = 0; r < 4; ++r) {
                    y[r] = 0.0;
                    for (int e = 0; e < 4; ++e) y[r] += m[4 * r + e] * x[e];
                }
                for (int e = 0; e < 4; ++e) v[idx[e]] = y[e];
            }
    };
    double err = 0.0;
    std::vector<cd> a(D), b(D);
    for (size_t col = 0; col < D; ++col) {
        std::fill(a.begin(), a.end(), cd(0.0));
        std::fill(b.begin(), b.end(), cd(0.0));
        a[col] = b[col] = 1.0;
        size_t ns = 0;
        auto sites = [&](int g) {
            for (; ns < c.noises.size() && c.noises[ns].after_gate == g; ++ns)
                apply1(a, c.noises[ns].qubit, f[ns].K[0].data());
        };
        sites(-1);
        for (size_t g = 0; g < c.gates.size(); ++g) {
            const Gate& gt = c.gates[g];
            if (gate_is_two_qubit(gt.kind)) {
                const Mat4 m = gate_matrix_2q(gt);
                apply2(a, gt.q0, gt.q1, m.data());
            } else {
                const Mat2 m = gate_matrix_1q(gt);
                apply1(a, gt.q0, m.data());
            }
            sites((int)g);
        }
        for (const HostOp& o : p.ops) {
            if (o.type == OP_G2 || o.type == OP_D2) apply2(b, o.q0, o.q1, o.m.data());
            else apply1(b, o.q0, o.m.data());
        }
        for (size_t i = 0; i < D; ++i) err = std::max(err, std::abs(a[i] - b[i]));
    }
    return err;
}

}  // namespace nqs
