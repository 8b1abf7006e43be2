// Importance-sampled estimate of one level's sum T_k (k = 2 or 3) over site
// sets, with a proposal built from the trained network.
//
// The network scores site pairs: g(s, t) ~ log W_2(s, t), from the features
// of the two sites (position of the noise in the circuit, qubit, noise rate,
// level-1 weight W_1).  A pair is proposed with weight exp(g); a triple with
//   w(S) = exp(g(s1,s2)) W_1(s3) + exp(g(s1,s3)) W_1(s2) + exp(g(s2,s3)) W_1(s1),
// one pair interacting and the third site on its own (under independent
// noises W_3 ~ W_2 W_1 / W_0 for each split, and the sum keeps every split's
// share even when one factor vanishes).  The proposal mixes w / sum(w) with
// the uniform law (defensive weight alpha), so every set keeps probability
// >= alpha / #sets and the estimator  T_k ~ (1/m) sum_j W(S_j) / q(S_j)  is
// unbiased with finite variance.  Sets are drawn by inverse-CDF lookup of
// counter-based uniforms (SplitMix64 of seed + j) and evaluated on the GPU
// (nqs_eval_sets); repeated draws are evaluated once.  Without a network
// (mlp == NULL) q is uniform: the plain Monte-Carlo version of the method.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <vector>

#include "nqs_internal.h"

namespace nqs {

namespace {

double uniform01(unsigned long long seed, unsigned long long j) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (j + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (z >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace

int site_features(const Handle& h, const double* W1, float* out) {
    const int N = (int)h.factors.size();
    const int G = std::max(1, (int)h.circ.gates.size());
    std::vector<double> f((size_t)N * 4);
    double w1max = 0.0;
    for (int s = 0; s < N; ++s) w1max = std::max(w1max, W1[s]);
    const double w1floor = w1max > 0.0 ? 1e-12 * w1max : 1e-300;
    for (int s = 0; s < N; ++s) {
        f[s * 4 + 0] = (h.circ.noises[s].after_gate + 1.0) / G;
        f[s * 4 + 1] = (double)h.circ.noises[s].qubit / std::max(1, h.circ.n - 1);
        f[s * 4 + 2] = std::log10(std::max(h.factors[s].rate, 1e-300));
        f[s * 4 + 3] = std::log10(std::max(W1[s], w1floor));
    }
    // standardise every column over the sites
    for (int c = 0; c < 4; ++c) {
        double mu = 0, var = 0;
        for (int s = 0; s < N; ++s) mu += f[s * 4 + c];
        mu /= N;
        for (int s = 0; s < N; ++s) var += (f[s * 4 + c] - mu) * (f[s * 4 + c] - mu);
        const double sd = std::sqrt(var / N) + 1e-12;
        for (int s = 0; s < N; ++s) out[s * 4 + c] = (float)((f[s * 4 + c] - mu) / sd);
    }
    return NQS_OK;
}

int pair_training_data(const Handle& h, const float* feats, const double* W2, float* X, float* y, size_t cap,
                       size_t* count) {
    const int N = (int)h.factors.size();
    const size_t P = (size_t)N * (N - 1) / 2;
    *count = P;
    if (cap < P) return NQS_OK;
    double w2max = 0.0;
    for (int s = 0; s < N; ++s)
        for (int t = s + 1; t < N; ++t) w2max = std::max(w2max, W2[(size_t)s * N + t]);
    const double w2floor = w2max > 0.0 ? 1e-12 * w2max : 1e-300;
    size_t r = 0;
    for (int s = 0; s < N; ++s)
        for (int t = s + 1; t < N; ++t, ++r) {
            for (int c = 0; c < 4; ++c) {
                X[r * 8 + c] = feats[s * 4 + c];
                X[r * 8 + 4 + c] = feats[t * 4 + c];
            }
            y[r] = (float)std::log(std::max(W2[(size_t)s * N + t], w2floor));
        }
    return NQS_OK;
}

// The proposal q over all site sets of the level, in canonical (lexicographic)
// order, with the sets themselves; alpha becomes 1 without a network (or
// when the network's weights sum to nothing).
int is_proposal(Handle& h, Mlp* mlp, int level, double& alpha, const float* feats, const double* W1,
                std::vector<int>& sets, std::vector<double>& q, void* stream) {
    const int N = (int)h.factors.size();
    if (level < 2 || level > 3 || N < level || !(alpha >= 0.0 && alpha <= 1.0)) return NQS_ERR_ARG;
    if (!mlp) alpha = 1.0;
    if (mlp && mlp_n_in(mlp) != 8) return NQS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // pair scores from the network
    std::vector<double> g((size_t)N * N, 0.0);
    if (mlp && alpha < 1.0) {
        const size_t P = (size_t)N * (N - 1) / 2;
        std::vector<float> X(P * 8);
        size_t r = 0;
        for (int s = 0; s < N; ++s)
            for (int t = s + 1; t < N; ++t, ++r)
                for (int c = 0; c < 4; ++c) {
                    X[r * 8 + c] = feats[s * 4 + c];
                    X[r * 8 + 4 + c] = feats[t * 4 + c];
                }
        float* Xd = (float*)dev_alloc(P * 8 * sizeof(float), stream);
        float* yd = (float*)dev_alloc(P * sizeof(float), stream);
        if (!Xd || !yd) {
            dev_free(Xd, 0, stream);
            dev_free(yd, 0, stream);
            return NQS_ERR_NOMEM;
        }
        std::vector<float> ys(P);
        int rc = cudaMemcpyAsync(Xd, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, st) == cudaSuccess
                     ? NQS_OK
                     : NQS_ERR_CUDA;
        if (rc == NQS_OK) rc = mlp_forward(mlp, Xd, (int)P, yd, stream);
        if (rc == NQS_OK && cudaMemcpyAsync(ys.data(), yd, P * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = NQS_ERR_CUDA;
        if (rc == NQS_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = NQS_ERR_CUDA;
        dev_free(Xd, 0, stream);
        dev_free(yd, 0, stream);
        if (rc) return rc;
        r = 0;
        for (int s = 0; s < N; ++s)
            for (int t = s + 1; t < N; ++t, ++r) g[(size_t)s * N + t] = g[(size_t)t * N + s] = ys[r];
    }
    // proposal over all site sets, canonical (lexicographic) order
    sets.clear();
    std::vector<double> w;
    const bool learned = mlp && alpha < 1.0;
    std::vector<double> w2(g.size());
    if (learned) {
        double gmax = -1e300;
        for (int a = 0; a < N; ++a)
            for (int b = a + 1; b < N; ++b) gmax = std::max(gmax, g[(size_t)a * N + b]);
        for (size_t i = 0; i < g.size(); ++i) w2[i] = std::exp(g[i] - gmax);   // common scale drops out
    }
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b) {
            if (level == 2) {
                sets.push_back(a);
                sets.push_back(b);
                w.push_back(learned ? w2[(size_t)a * N + b] : 1.0);
                continue;
            }
            for (int c = b + 1; c < N; ++c) {
                sets.push_back(a);
                sets.push_back(b);
                sets.push_back(c);
                w.push_back(learned ? w2[(size_t)a * N + b] * std::max(W1[c], 0.0) +
                                          w2[(size_t)a * N + c] * std::max(W1[b], 0.0) +
                                          w2[(size_t)b * N + c] * std::max(W1[a], 0.0)
                                    : 1.0);
            }
        }
    const size_t n_sets = w.size();
    q.assign(n_sets, 0.0);
    {
        double z = 0.0;
        for (double x : w) z += x;
        if (!(z > 0.0) || !std::isfinite(z)) alpha = 1.0;   // nothing learned to go on
        for (size_t i = 0; i < n_sets; ++i)
            q[i] = (alpha < 1.0 ? (1.0 - alpha) * w[i] / z : 0.0) + alpha / (double)n_sets;
    }
    return NQS_OK;
}

int is_estimate(Handle& h, Mlp* mlp, int level, unsigned long long samples, double alpha, unsigned long long seed,
                const float* feats, const double* W1, nqs_is_result* out, void* stream) {
    if (samples < 2) return NQS_ERR_ARG;
    std::vector<int> sets;
    std::vector<double> q;
    int rc0 = is_proposal(h, mlp, level, alpha, feats, W1, sets, q, stream);
    if (rc0) return rc0;
    const size_t n_sets = q.size();
    std::vector<double> cdf(n_sets);
    {
        double acc = 0.0;
        for (size_t i = 0; i < n_sets; ++i) cdf[i] = (acc += q[i]);
        for (size_t i = 0; i < n_sets; ++i) cdf[i] /= acc;
    }
    // draws, evaluated once per distinct set
    std::vector<size_t> draw(samples);
    std::unordered_map<size_t, size_t> slot;
    std::vector<int> uniq;
    for (unsigned long long j = 0; j < samples; ++j) {
        const double u = uniform01(seed, j);
        size_t i = (size_t)(std::lower_bound(cdf.begin(), cdf.end(), u) - cdf.begin());
        if (i >= n_sets) i = n_sets - 1;
        draw[j] = i;
        if (slot.emplace(i, slot.size()).second)
            for (int r = 0; r < level; ++r) uniq.push_back(sets[i * level + r]);
    }
    std::vector<double> Wu(slot.size());
    int rc = engine_eval_sets(h, level, uniq.data(), slot.size(), Wu.data(), stream);
    if (rc) return rc;
    double sum = 0.0, sum2 = 0.0, sw = 0.0, sw2 = 0.0;
    for (unsigned long long j = 0; j < samples; ++j) {
        const size_t i = draw[j];
        const double x = Wu[slot[i]] / q[i];
        sum += x;
        sum2 += x * x;
        const double w = 1.0 / q[i];
        sw += w;
        sw2 += w * w;
    }
    const double m = (double)samples;
    const double est = sum / m;
    const double var = std::max(0.0, (sum2 - m * est * est) / (m - 1.0));
    out->estimate = est;
    out->stderr_ = std::sqrt(var / m);
    out->ess = sw * sw / sw2;
    out->samples = samples;
    out->distinct = slot.size();
    out->alpha = alpha;
    out->n_sets = n_sets;
    out->level = level;
    out->status = NQS_OK;
    return NQS_OK;
}

int is_proposal_values(Handle& h, Mlp* mlp, int level, double alpha, const float* feats, const double* W1,
                       double* q_out, size_t cap, size_t* count, void* stream) {
    std::vector<int> sets;
    std::vector<double> q;
    const int rc = is_proposal(h, mlp, level, alpha, feats, W1, sets, q, stream);
    if (rc) return rc;
    *count = q.size();
    if (q_out && cap >= q.size()) std::copy(q.begin(), q.end(), q_out);
    return NQS_OK;
}

}  // namespace nqs
