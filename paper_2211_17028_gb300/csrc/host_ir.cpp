// Circuit text reader and gate matrices (Sec. II, Table I).
//
// Single-qubit gates follow Table I; controlled gates follow the controlled-U
// construction of Sec. II with the control as the more significant index bit;
// U3 uses the OpenQASM convention (the paper does not list it).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <sstream>

#include "nqs_internal.h"

namespace nqs {

namespace {

struct GateName {
    const char* name;
    GateKind kind;
    int arity;
    int nparam;
};

const GateName kGateNames[] = {
    {"h", G_H, 1, 0},   {"x", G_X, 1, 0},   {"y", G_Y, 1, 0},  {"z", G_Z, 1, 0},
    {"t", G_T, 1, 0},   {"rx", G_RX, 1, 1}, {"ry", G_RY, 1, 1}, {"rz", G_RZ, 1, 1},
    {"u3", G_U3, 1, 3}, {"cz", G_CZ, 2, 0}, {"cx", G_CX, 2, 0},
};

bool parse_int(const std::string& s, long long& v) {
    if (s.empty()) return false;
    char* end = nullptr;
    v = std::strtoll(s.c_str(), &end, 10);
    return end && *end == '\0';
}

bool parse_double(const std::string& s, double& v) {
    if (s.empty()) return false;
    char* end = nullptr;
    v = std::strtod(s.c_str(), &end);
    return end && *end == '\0' && std::isfinite(v);
}

}  // namespace

bool gate_is_two_qubit(GateKind k) { return k == G_CZ || k == G_CX; }

int parse_circuit(const char* text, Circuit& out, std::string& err) {
    out = Circuit{};
    std::istringstream in(text);
    std::string raw;
    bool header = false;
    int line_no = 0;
    auto fail = [&](const std::string& why) {
        err = "line " + std::to_string(line_no) + ": " + why;
        return NQS_ERR_PARSE;
    };
    while (std::getline(in, raw)) {
        ++line_no;
        size_t hash = raw.find('#');
        if (hash != std::string::npos) raw.resize(hash);
        std::istringstream ls(raw);
        std::vector<std::string> tok;
        std::string t;
        while (ls >> t) tok.push_back(t);
        if (tok.empty()) continue;
        if (tok[0] == "nqs-ir") {
            if (tok.size() != 2 || tok[1] != "1") return fail("unsupported header");
            header = true;
        } else if (tok[0] == "qubits") {
            long long n;
            if (tok.size() != 2 || !parse_int(tok[1], n)) return fail("bad qubit count");
            if (n < 1 || n > 34) {
                err = "qubit count outside 1..34";
                return NQS_ERR_UNSUPPORTED;
            }
            out.n = (int)n;
        } else if (tok[0] == "gate") {
            if (!header || out.n == 0) return fail("gate before header/qubits");
            if (tok.size() < 3) return fail("short gate record");
            const GateName* gn = nullptr;
            for (const auto& g : kGateNames)
                if (tok[1] == g.name) gn = &g;
            if (!gn) return fail("unknown gate " + tok[1]);
            if ((int)tok.size() != 2 + gn->arity + gn->nparam) return fail("wrong field count");
            Gate g;
            g.kind = gn->kind;
            long long q;
            if (!parse_int(tok[2], q) || q < 0 || q >= out.n) return fail("bad qubit");
            g.q0 = (int)q;
            if (gn->arity == 2) {
                if (!parse_int(tok[3], q) || q < 0 || q >= out.n || q == g.q0) return fail("bad qubit");
                g.q1 = (int)q;
            }
            for (int i = 0; i < gn->nparam; ++i)
                if (!parse_double(tok[2 + gn->arity + i], g.p[i])) return fail("bad parameter");
            out.gates.push_back(g);
        } else if (tok[0] == "noise") {
            if (!header || out.n == 0) return fail("noise before header/qubits");
            long long ag, q, k;
            if (tok.size() < 4 || !parse_int(tok[1], ag) || !parse_int(tok[2], q) || !parse_int(tok[3], k))
                return fail("bad noise record");
            if (q < 0 || q >= out.n) return fail("bad noise qubit");
            if (k < 1 || k > 16) return fail("Kraus count outside 1..16");
            if ((long long)tok.size() != 4 + 8 * k) return fail("wrong Kraus value count");
            NoiseSite s;
            s.after_gate = (int)ag;
            s.qubit = (int)q;
            for (long long j = 0; j < k; ++j) {
                Mat2 m;
                for (int e = 0; e < 4; ++e) {
                    double re, im;
                    if (!parse_double(tok[4 + 8 * j + 2 * e], re) || !parse_double(tok[5 + 8 * j + 2 * e], im))
                        return fail("bad Kraus value");
                    m[e] = cd(re, im);
                }
                s.kraus.push_back(m);
            }
            out.noises.push_back(s);
        } else if (tok[0] == "noise2" || tok[0] == "superop" || tok[0] == "superop2") {
            // general noises: two-qubit Kraus operators (4x4, index 2*b(q0) + b(q1)),
            // or the matrix representation M of a one- / two-qubit noise
            if (!header || out.n == 0) return fail("noise before header/qubits");
            const bool two = tok[0] != "superop";
            const bool sop = tok[0] != "noise2";
            long long ag, q, q2 = -1, k = 1;
            size_t at = 2;
            if (tok.size() < 3 || !parse_int(tok[1], ag) || !parse_int(tok[at++], q)) return fail("bad noise record");
            if (two && (tok.size() <= at || !parse_int(tok[at++], q2))) return fail("bad noise record");
            if (!sop && (tok.size() <= at || !parse_int(tok[at++], k))) return fail("bad noise record");
            if (q < 0 || q >= out.n || (two && (q2 < 0 || q2 >= out.n || q2 == q))) return fail("bad noise qubit");
            if (k < 1 || k > 16) return fail("Kraus count outside 1..16");
            const int d = two ? 4 : 2;
            const size_t vals = sop ? (size_t)2 * d * d * d * d : (size_t)2 * d * d * k;
            if (tok.size() != at + vals) return fail("wrong value count");
            std::vector<cd> all(vals / 2);
            for (size_t e = 0; e < all.size(); ++e) {
                double re, im;
                if (!parse_double(tok[at + 2 * e], re) || !parse_double(tok[at + 2 * e + 1], im))
                    return fail("bad value");
                all[e] = cd(re, im);
            }
            NoiseSite s;
            s.after_gate = (int)ag;
            s.qubit = (int)q;
            s.qubit2 = two ? (int)q2 : -1;
            if (sop) {
                s.superop = all;
            } else {
                for (long long j = 0; j < k; ++j)
                    s.kraus_d.emplace_back(all.begin() + j * d * d, all.begin() + (j + 1) * d * d);
            }
            out.noises.push_back(s);
        } else {
            return fail("unknown record " + tok[0]);
        }
    }
    if (!header || out.n == 0) {
        err = "missing header or qubit count";
        return NQS_ERR_PARSE;
    }
    int prev = -2;
    for (const auto& s : out.noises) {
        if (s.after_gate < prev || s.after_gate < -1 || s.after_gate >= (int)out.gates.size()) {
            err = "noise records must be ordered by after_gate and reference existing gates";
            return NQS_ERR_PARSE;
        }
        prev = s.after_gate;
    }
    return NQS_OK;
}

Mat2 gate_matrix_1q(const Gate& g) {
    const double r2 = 1.0 / std::sqrt(2.0);
    const cd I(0, 1);
    switch (g.kind) {
        case G_H: return {cd(r2), cd(r2), cd(r2), cd(-r2)};
        case G_X: return {cd(0), cd(1), cd(1), cd(0)};
        case G_Y: return {cd(0), -I, I, cd(0)};
        case G_Z: return {cd(1), cd(0), cd(0), cd(-1)};
        case G_T: return {cd(1), cd(0), cd(0), std::polar(1.0, M_PI / 4)};
        case G_RX: {
            double c = std::cos(g.p[0] / 2), s = std::sin(g.p[0] / 2);
            return {cd(c), cd(0, -s), cd(0, -s), cd(c)};
        }
        case G_RY: {
            double c = std::cos(g.p[0] / 2), s = std::sin(g.p[0] / 2);
            return {cd(c), cd(-s), cd(s), cd(c)};
        }
        case G_RZ: return {std::polar(1.0, -g.p[0] / 2), cd(0), cd(0), std::polar(1.0, g.p[0] / 2)};
        case G_U3: {
            double c = std::cos(g.p[0] / 2), s = std::sin(g.p[0] / 2);
            return {cd(c), -std::polar(s, g.p[2]), std::polar(s, g.p[1]), std::polar(c, g.p[1] + g.p[2])};
        }
        default: break;
    }
    return {cd(1), cd(0), cd(0), cd(1)};
}

Mat4 gate_matrix_2q(const Gate& g) {
    Mat4 m{};
    for (int i = 0; i < 4; ++i) m[5 * i] = cd(1);
    if (g.kind == G_CZ) {
        m[15] = cd(-1);
    } else if (g.kind == G_CX) {
        m[10] = cd(0);
        m[15] = cd(0);
        m[11] = cd(1);
        m[14] = cd(1);
    }
    return m;
}

}  // namespace nqs
