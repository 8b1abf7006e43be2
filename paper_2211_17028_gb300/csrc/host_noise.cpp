// Noise factors of Sec. IV (Fig. 3), in FP64 on the host.
//
// For a channel with Kraus operators E_k the matrix representation is
// M = sum_k E_k (x) E_k^*; its tensor permutation (rows = edges 1,3,
// columns = edges 2,4) is M~ = sum_k vec(E_k) vec(E_k)^dagger with
// vec(E)[2a+b] = E[a][b].  M~ is Hermitian positive semidefinite, so its SVD
// S D T^dagger coincides with its eigendecomposition (S|i> = T|i> wherever
// d_i > 0).  Permuting d_i S|i> T|i>^dagger back gives
// U_i (x) V_i = (sqrt(d_i) A_i) (x) conj(sqrt(d_i) A_i) with A_i the 2x2
// reshape of the i-th singular vector, so each factor is carried by one 2x2
// matrix K_i = sqrt(d_i) A_i.  The eigendecomposition is a cyclic complex
// Jacobi iteration written here (no LAPACK).
#include <algorithm>
#include <cmath>

#include "nqs_internal.h"

namespace nqs {

void hermitian_jacobi4(const Mat4& a_in, double evals[4], Mat4& V) {
    cd A[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) A[i][j] = a_in[4 * i + j];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) V[4 * i + j] = cd(i == j ? 1.0 : 0.0);
    double scale = 0.0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) scale = std::max(scale, std::abs(A[i][j]));
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q) off += std::norm(A[p][q]);
        if (off <= 1e-64 * scale * scale || off == 0.0) break;
        for (int p = 0; p < 4; ++p) {
            for (int q = p + 1; q < 4; ++q) {
                double r = std::abs(A[p][q]);
                if (r <= 1e-300) continue;
                // phase making the (p,q) entry real: D = diag(1 at p, e^{-i phi} at q)
                cd ph = A[p][q] / r;   // e^{i phi}
                double app = A[p][p].real(), aqq = A[q][q].real();
                double tau = (aqq - app) / (2.0 * r);
                double t = (tau >= 0 ? 1.0 : -1.0) / (std::abs(tau) + std::sqrt(1.0 + tau * tau));
                double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                // unitary W = D R acting on columns p, q:
                //   W[p][p] = c, W[p][q] = s, W[q][p] = -s e^{-i phi}, W[q][q] = c e^{-i phi}
                cd wpp = c, wpq = s, wqp = -s * std::conj(ph), wqq = c * std::conj(ph);
                // A <- W^dag A W
                for (int k = 0; k < 4; ++k) {   // A W (columns)
                    cd akp = A[k][p], akq = A[k][q];
                    A[k][p] = akp * wpp + akq * wqp;
                    A[k][q] = akp * wpq + akq * wqq;
                }
                for (int k = 0; k < 4; ++k) {   // W^dag (rows)
                    cd apk = A[p][k], aqk = A[q][k];
                    A[p][k] = std::conj(wpp) * apk + std::conj(wqp) * aqk;
                    A[q][k] = std::conj(wpq) * apk + std::conj(wqq) * aqk;
                }
                A[p][q] = A[q][p] = cd(0);
                A[p][p] = cd(A[p][p].real());
                A[q][q] = cd(A[q][q].real());
                for (int k = 0; k < 4; ++k) {   // V <- V W
                    cd vkp = V[4 * k + p], vkq = V[4 * k + q];
                    V[4 * k + p] = vkp * wpp + vkq * wqp;
                    V[4 * k + q] = vkp * wpq + vkq * wqq;
                }
            }
        }
    }
    for (int i = 0; i < 4; ++i) evals[i] = A[i][i].real();
}

namespace {

double spectral_norm4(const Mat4& m) {
    // sqrt of the largest eigenvalue of m^dagger m
    Mat4 h{};
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cd s = 0;
            for (int k = 0; k < 4; ++k) s += std::conj(m[4 * k + i]) * m[4 * k + j];
            h[4 * i + j] = s;
        }
    double ev[4];
    Mat4 vec;
    hermitian_jacobi4(h, ev, vec);
    double mx = 0;
    for (double e : ev) mx = std::max(mx, e);
    return std::sqrt(std::max(mx, 0.0));
}

Mat4 kron_conj(const Mat2& k) {
    // K (x) conj(K): index (2a+a', 2b+b') -> K[a][b] conj(K[a'][b'])
    Mat4 out{};
    for (int a = 0; a < 2; ++a)
        for (int ap = 0; ap < 2; ++ap)
            for (int b = 0; b < 2; ++b)
                for (int bp = 0; bp < 2; ++bp)
                    out[4 * (2 * a + ap) + (2 * b + bp)] = k[2 * a + b] * std::conj(k[2 * ap + bp]);
    return out;
}

}  // namespace

int factor_noise(const NoiseSite& s, bool prune_zero_rank, Factors& f) {
    // CPTP: sum_k E_k^dagger E_k = I
    cd acc[4] = {0, 0, 0, 0};
    for (const auto& e : s.kraus)
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                for (int k = 0; k < 2; ++k) acc[2 * i + j] += std::conj(e[2 * k + i]) * e[2 * k + j];
    double dev = 0;
    for (int i = 0; i < 4; ++i) dev = std::max(dev, std::abs(acc[i] - cd((i == 0 || i == 3) ? 1.0 : 0.0)));
    if (!(dev <= 1e-10)) return NQS_ERR_NOT_CPTP;

    // M~ = sum_k vec(E_k) vec(E_k)^dagger
    Mat4 mt{};
    for (const auto& e : s.kraus)
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) mt[4 * r + c] += e[r] * std::conj(e[c]);
    double ev[4];
    Mat4 vec;
    hermitian_jacobi4(mt, ev, vec);
    int order[4] = {0, 1, 2, 3};
    std::sort(order, order + 4, [&](int a, int b) { return ev[a] > ev[b]; });
    for (int i = 0; i < 4; ++i) {
        int j = order[i];
        f.d[i] = std::max(ev[j], 0.0);
        double sq = std::sqrt(f.d[i]);
        for (int e = 0; e < 4; ++e) f.K[i][e] = sq * vec[4 * e + j];
    }
    if (!(f.d[0] - f.d[1] > 1e-12 * f.d[0])) return NQS_ERR_NOT_DOMINANT;
    f.m = 0;
    for (int i = 1; i < 4; ++i) {
        if (prune_zero_rank && f.d[i] < 1e-10 * f.d[0]) continue;
        f.keep[f.m++] = i;
    }
    for (int i = f.m; i < 3; ++i) f.keep[i] = 0;
    f.norm_dom = spectral_norm4(kron_conj(f.K[0]));
    Mat4 rest{};
    for (int i = 1; i < 4; ++i) {
        Mat4 t = kron_conj(f.K[i]);
        for (int e = 0; e < 16; ++e) rest[e] += t[e];
    }
    f.norm_rest = spectral_norm4(rest);
    {
        Mat4 m{};
        for (const auto& e : s.kraus) {
            Mat4 t = kron_conj(e);
            for (int i = 0; i < 16; ++i) m[i] += t[i];
        }
        for (int i = 0; i < 4; ++i) m[5 * i] -= cd(1);
        f.rate = spectral_norm4(m);
    }
    return NQS_OK;
}

}  // namespace nqs
