// Factors of general noises (Sec. IV, Fig. 3) in FP64 on the host: two-qubit
// channels and noises given by their matrix representation M.
//
// M (d^2 x d^2, rows (out, out'), columns (in, in'), the original-wire index
// first in each pair) is tensor-permuted to M~ with rows (out, in) and
// columns (out', in'), and M~ = S D T^dagger by a one-sided (Hestenes)
// Jacobi SVD written here.  Permuting d_i S|i> T|i>^dagger back gives
// U_i (x) V_i with U_i = d_i reshape(S|i>) and V_i = conj(reshape(T|i>)); the
// expansion's term for an assignment sigma is the product of
// <v|C[U_sigma]|psi> and <v^*|C^*[V_sigma]|psi^*> = conj(<v|C[conj V_sigma]|psi>),
// which the general-noise path evaluates as
//   X = <v|C[KA_sigma]|psi> * conj(<v|C[KB_sigma]|psi>),
//   KA_i = sqrt(d_i) reshape(S|i>),  KB_i = sqrt(d_i) reshape(T|i>).
// For a channel M~ = sum_k vec(E_k) vec(E_k)^dagger is PSD and S = T where
// d_i > 0, so KA = KB and one network per term suffices.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "nqs_internal.h"

namespace nqs {

void svd_jacobi(const std::vector<cd>& a_in, int n, std::vector<double>& sv, std::vector<cd>& u,
                std::vector<cd>& v) {
    // columns of A (column-major work copy) rotated until mutually orthogonal
    std::vector<cd> A((size_t)n * n), V((size_t)n * n, cd(0));
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) A[(size_t)c * n + r] = a_in[(size_t)r * n + c];
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    auto col = [&](std::vector<cd>& M, int c) { return M.data() + (size_t)c * n; };
    for (int sweep = 0; sweep < 80; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                cd* ap = col(A, p);
                cd* aq = col(A, q);
                double alpha = 0.0, beta = 0.0;
                cd gamma = 0.0;
                for (int k = 0; k < n; ++k) {
                    alpha += std::norm(ap[k]);
                    beta += std::norm(aq[k]);
                    gamma += std::conj(ap[k]) * aq[k];
                }
                const double g = std::abs(gamma);
                tot += alpha * beta;
                if (g <= 1e-300 || g * g <= 1e-30 * alpha * beta) continue;
                off += g * g;
                // the 2x2 Hermitian [[alpha, gamma], [conj gamma, beta]] diagonalised by
                // W = [[c, s], [-s conj(ph), c conj(ph)]] with ph = gamma / |gamma|
                const cd ph = gamma / g;
                const double tau = (beta - alpha) / (2.0 * g);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::abs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                const cd wpp = c, wpq = s, wqp = -s * std::conj(ph), wqq = c * std::conj(ph);
                for (int k = 0; k < n; ++k) {
                    const cd x = ap[k], y = aq[k];
                    ap[k] = x * wpp + y * wqp;
                    aq[k] = x * wpq + y * wqq;
                }
                cd* vp = col(V, p);
                cd* vq = col(V, q);
                for (int k = 0; k < n; ++k) {
                    const cd x = vp[k], y = vq[k];
                    vp[k] = x * wpp + y * wqp;
                    vq[k] = x * wpq + y * wqq;
                }
            }
        if (off <= 1e-32 * std::max(tot, 1e-300)) break;
    }
    std::vector<double> s(n);
    for (int c = 0; c < n; ++c) {
        double x = 0.0;
        for (int k = 0; k < n; ++k) x += std::norm(A[(size_t)c * n + k]);
        s[c] = std::sqrt(x);
    }
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return s[x] > s[y]; });
    sv.assign(n, 0.0);
    u.assign((size_t)n * n, cd(0));
    v.assign((size_t)n * n, cd(0));
    // singular values at rounding level (below 1e-14 of the largest) are zero:
    // their left vectors are noise, and their factors carry no weight
    const double tiny = 1e-300 + (n ? s[ord[0]] : 0.0) * 1e-14;
    for (int j = 0; j < n; ++j) {
        const int c = ord[j];
        sv[j] = s[c] > tiny ? s[c] : 0.0;
        for (int k = 0; k < n; ++k) {
            v[(size_t)j * n + k] = V[(size_t)c * n + k];
            if (s[c] > tiny) u[(size_t)j * n + k] = A[(size_t)c * n + k] / s[c];
        }
    }
}

namespace {

double spectral_norm(const std::vector<cd>& a, int n) {
    std::vector<double> sv;
    std::vector<cd> u, v;
    svd_jacobi(a, n, sv, u, v);
    return n ? sv[0] : 0.0;
}

}  // namespace

int factor_general(const NoiseSite& s, GFactors& out) {
    const int d = s.dim(), D = d * d;
    std::vector<cd> M((size_t)D * D, cd(0));
    if (!s.superop.empty()) {
        if ((int)s.superop.size() != D * D) return NQS_ERR_ARG;
        M = s.superop;
    } else {
        std::vector<std::vector<cd>> ks = s.kraus_d;
        if (ks.empty())
            for (const Mat2& k : s.kraus) ks.emplace_back(k.begin(), k.end());
        if (ks.empty()) return NQS_ERR_ARG;
        // trace preservation: sum_k E_k^dagger E_k = I
        double dev = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                cd acc = 0.0;
                for (const auto& e : ks)
                    for (int r = 0; r < d; ++r) acc += std::conj(e[(size_t)r * d + i]) * e[(size_t)r * d + j];
                dev = std::max(dev, std::abs(acc - (i == j ? 1.0 : 0.0)));
            }
        if (dev > 1e-10) return NQS_ERR_NOT_CPTP;
        // M[(o, o'), (i, i')] = sum_k E[o][i] conj(E[o'][i'])
        for (const auto& e : ks)
            for (int o = 0; o < d; ++o)
                for (int op = 0; op < d; ++op)
                    for (int i = 0; i < d; ++i)
                        for (int ip = 0; ip < d; ++ip)
                            M[(size_t)(o * d + op) * D + (i * d + ip)] += e[(size_t)o * d + i] * std::conj(e[(size_t)op * d + ip]);
    }
    // tensor permutation: M~[(o, i), (o', i')] = M[(o, o'), (i, i')]
    std::vector<cd> Mt((size_t)D * D);
    for (int o = 0; o < d; ++o)
        for (int op = 0; op < d; ++op)
            for (int i = 0; i < d; ++i)
                for (int ip = 0; ip < d; ++ip)
                    Mt[(size_t)(o * d + i) * D + (op * d + ip)] = M[(size_t)(o * d + op) * D + (i * d + ip)];
    std::vector<double> sv;
    std::vector<cd> S, T;
    svd_jacobi(Mt, D, sv, S, T);
    if (!(sv[0] - sv[1] > 1e-12 * sv[0])) return NQS_ERR_NOT_DOMINANT;
    out.nq = s.qubit2 >= 0 ? 2 : 1;
    out.q0 = s.qubit;
    out.q1 = s.qubit2;
    out.m = D;
    out.d = sv;
    out.KA.assign((size_t)D * d * d, cd(0));
    out.KB.assign((size_t)D * d * d, cd(0));
    double big = 0.0, diff = 0.0;
    for (int j = 0; j < D; ++j) {
        const double w = std::sqrt(sv[j]);
        for (int e = 0; e < D; ++e) {   // reshape: entry [o][i] = vector[(o, i)] = vector[o * d + i]
            out.KA[(size_t)j * D + e] = w * S[(size_t)j * D + e];
            out.KB[(size_t)j * D + e] = w * T[(size_t)j * D + e];
            big = std::max(big, std::abs(out.KA[(size_t)j * D + e]));
            diff = std::max(diff, std::abs(out.KA[(size_t)j * D + e] - out.KB[(size_t)j * D + e]));
        }
    }
    out.same = diff <= 1e-12 * std::max(big, 1e-300);
    if (out.same) out.KB = out.KA;
    // bound norms: M' = U_0 (x) V_0, U_0 = d_0 reshape(S|0>), V_0 = conj(reshape(T|0>))
    std::vector<cd> U0((size_t)d * d), V0((size_t)d * d);
    for (int e = 0; e < d * d; ++e) {
        U0[e] = sv[0] * S[e];
        V0[e] = std::conj(T[e]);
    }
    std::vector<cd> Md((size_t)D * D), Mr((size_t)D * D);
    for (int o = 0; o < d; ++o)
        for (int op = 0; op < d; ++op)
            for (int i = 0; i < d; ++i)
                for (int ip = 0; ip < d; ++ip) {
                    const size_t at = (size_t)(o * d + op) * D + (i * d + ip);
                    Md[at] = U0[(size_t)o * d + i] * V0[(size_t)op * d + ip];
                    Mr[at] = M[at] - Md[at];
                }
    out.norm_dom = spectral_norm(Md, D);
    out.norm_rest = spectral_norm(Mr, D);
    return NQS_OK;
}

}  // namespace nqs
