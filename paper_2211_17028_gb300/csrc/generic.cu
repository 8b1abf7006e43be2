// General-noise path: circuits with two-qubit noise channels or noises given
// by their matrix representation (Sec. IV's SVD in its general form, with
// d^2 factors per site and two factor sets when the tensor-permuted matrix
// is not positive semidefinite).
//
// Every kept assignment sigma is X = a_sigma * conj(b_sigma) with
// a = <v|C[KA_sigma]|psi>, b = <v|C[KB_sigma]|psi> (host_generic.cpp); b = a
// when every site has KA = KB.  Each network is evaluated for all kept
// assignments at once from checkpoints, on the device, one kernel per
// operation (complex64 states, FP64 reductions):
//   backward: phi_t = (events after site t with KX_0 at later sites)^dagger v,
//   forward:  depth-first from psi -- at site t the reduced matrix
//             R[a][b] = sum_rest conj(phi_t[rest, a]) w[rest, b] over the
//             site's qubits gives <phi_t| K_j |w> = sum_ab K_j[a][b] R[a][b]
//             for every factor j, and each non-dominant K_j w is swept on to
//             the later sites while the level allows.
// The amplitudes land at the canonical ranks of the kept-term list (level,
// site tuple, factor tuple, all lexicographic); a last kernel forms
// X = a conj(b), the per-level Neumaier sums of Re X and |sum Im X|.  This
// path is not the tuned hot path of one-qubit channels (engine.cu): it has no
// gate fusion, tiling or pass specialisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "nqs_internal.h"

namespace nqs {

struct GEngine {
    void* buf = nullptr;
    size_t buf_bytes = 0;
    void* aux = nullptr;
    size_t aux_bytes = 0;
    long long n_terms = 0;
    bool has_result = false;
    cudaStream_t last = nullptr;
    double* vals = nullptr;
};

namespace {

constexpr int kT = 256;

struct GMat {
    float2 m[16];
};

__global__ void __launch_bounds__(kT) g_apply_kernel(float2* __restrict__ s, long long count, int nq, int q0, int q1,
                                                     GMat g) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < count; p += stride) {
        if (nq == 1) {
            const long long bit = 1ll << q0;
            const long long lo = p & (bit - 1);
            const long long i0 = ((p - lo) << 1) | lo, i1 = i0 | bit;
            const float2 a = s[i0], b = s[i1];
            s[i0] = make_float2(g.m[0].x * a.x - g.m[0].y * a.y + g.m[1].x * b.x - g.m[1].y * b.y,
                                g.m[0].x * a.y + g.m[0].y * a.x + g.m[1].x * b.y + g.m[1].y * b.x);
            s[i1] = make_float2(g.m[2].x * a.x - g.m[2].y * a.y + g.m[3].x * b.x - g.m[3].y * b.y,
                                g.m[2].x * a.y + g.m[2].y * a.x + g.m[3].x * b.y + g.m[3].y * b.x);
        } else {
            const long long b0 = 1ll << q0, b1 = 1ll << q1;
            const long long lob = b0 < b1 ? b0 : b1, hib = b0 < b1 ? b1 : b0;
            long long x = p;
            long long lo = x & (lob - 1);
            x = ((x - lo) << 1) | lo;
            lo = x & (hib - 1);
            x = ((x - lo) << 1) | lo;
            const long long idx[4] = {x, x | b1, x | b0, x | b0 | b1};
            float2 in[4];
            for (int k = 0; k < 4; ++k) in[k] = s[idx[k]];
            for (int r = 0; r < 4; ++r) {
                float re = 0.f, im = 0.f;
                for (int c = 0; c < 4; ++c) {
                    const float2 m = g.m[4 * r + c];
                    re += m.x * in[c].x - m.y * in[c].y;
                    im += m.x * in[c].y + m.y * in[c].x;
                }
                s[idx[r]] = make_float2(re, im);
            }
        }
    }
}

// per-block FP64 partials of R[a][b] (d^2 complex, d = 2 or 4) in a fixed order
__global__ void __launch_bounds__(kT) g_reduce_kernel(const float2* __restrict__ phi, const float2* __restrict__ w,
                                                      long long count, int nq, int q0, int q1,
                                                      double* __restrict__ part) {
    const int d = nq == 1 ? 2 : 4;
    double acc[32];
    for (int e = 0; e < 32; ++e) acc[e] = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < count; p += stride) {
        long long idx[4];
        if (nq == 1) {
            const long long bit = 1ll << q0;
            const long long lo = p & (bit - 1);
            idx[0] = ((p - lo) << 1) | lo;
            idx[1] = idx[0] | bit;
        } else {
            const long long b0 = 1ll << q0, b1 = 1ll << q1;
            const long long lob = b0 < b1 ? b0 : b1, hib = b0 < b1 ? b1 : b0;
            long long x = p;
            long long lo = x & (lob - 1);
            x = ((x - lo) << 1) | lo;
            lo = x & (hib - 1);
            x = ((x - lo) << 1) | lo;
            idx[0] = x;
            idx[1] = x | b1;
            idx[2] = x | b0;
            idx[3] = x | b0 | b1;
        }
        for (int a = 0; a < d; ++a) {
            const float2 f = phi[idx[a]];
            for (int b = 0; b < d; ++b) {
                const float2 x = w[idx[b]];
                acc[2 * (d * a + b)] += (double)f.x * x.x + (double)f.y * x.y;
                acc[2 * (d * a + b) + 1] += (double)f.x * x.y - (double)f.y * x.x;
            }
        }
    }
    __shared__ double sm[32][kT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = 0; e < 2 * d * d; ++e) {
        double v = acc[e];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sm[e][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * d * d) {
        double v = 0.0;
        for (int k = 0; k < kT / 32; ++k) v += sm[threadIdx.x][k];
        part[(size_t)blockIdx.x * 32 + threadIdx.x] = v;
    }
}

// R from the partials (fixed order), then amps[pos[c]] = sum_ab K_{j[c]}[a][b] R[a][b]
__global__ void __launch_bounds__(kT) g_finish_kernel(const double* __restrict__ part, int grid, int dd,
                                                      const double2* __restrict__ K, const int* __restrict__ js,
                                                      const long long* __restrict__ pos, int cnt,
                                                      double2* __restrict__ amps) {
    __shared__ double R[32];
    if (threadIdx.x < 2 * dd) {
        double v = 0.0;
        for (int g = 0; g < grid; ++g) v += part[(size_t)g * 32 + threadIdx.x];
        R[threadIdx.x] = v;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < cnt; c += blockDim.x) {
        const double2* k = K + (size_t)js[c] * dd;
        double re = 0.0, im = 0.0;
        for (int e = 0; e < dd; ++e) {
            re += k[e].x * R[2 * e] - k[e].y * R[2 * e + 1];
            im += k[e].x * R[2 * e + 1] + k[e].y * R[2 * e];
        }
        amps[pos[c]] = make_double2(re, im);
    }
}

__global__ void g_fill_kernel(float2* __restrict__ s, long long dim, unsigned long long bits) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride)
        s[i] = make_float2((unsigned long long)i == bits ? 1.f : 0.f, 0.f);
}

// X = a conj(b) (b = a when b is null); per-level Neumaier sums of Re X in
// canonical order, |sum Im X|, the result record
__global__ void __launch_bounds__(kT) g_sum_kernel(const double2* __restrict__ a, const double2* __restrict__ b,
                                                   const long long* __restrict__ level_off, int level,
                                                   long long n_terms, double bound, double* __restrict__ vals,
                                                   nqs_result* __restrict__ res) {
    __shared__ double s_re[kT], s_c[kT], s_im[kT];
    __shared__ double T[NQS_MAX_LEVEL + 1];
    __shared__ double imag_tot;
    const int tid = threadIdx.x;
    if (tid == 0) imag_tot = 0.0;
    __syncthreads();
    for (int u = 0; u <= level; ++u) {
        const long long lo = level_off[u], hi = level_off[u + 1];
        const long long len = hi - lo, chunk = (len + kT - 1) / kT;
        double s = 0.0, c = 0.0, si = 0.0;
        for (long long i = lo + tid * chunk; i < lo + (tid + 1) * chunk && i < hi; ++i) {
            const double2 x = a[i];
            const double2 y = b ? b[i] : a[i];
            const double re = x.x * y.x + x.y * y.y, im = x.y * y.x - x.x * y.y;
            vals[i] = re;
            const double t = s + re;
            c += (fabs(s) >= fabs(re)) ? (s - t) + re : (re - t) + s;
            s = t;
            si += im;
        }
        s_re[tid] = s;
        s_c[tid] = c;
        s_im[tid] = si;
        __syncthreads();
        if (tid == 0) {
            double S = 0.0, C = 0.0, I = 0.0;
            for (int k = 0; k < kT; ++k) {
                const double v = s_re[k];
                const double t = S + v;
                C += (fabs(S) >= fabs(v)) ? (S - t) + v : (v - t) + S;
                S = t;
                C += s_c[k];
                I += s_im[k];
            }
            T[u] = S + C;
            imag_tot += I;
        }
        __syncthreads();
    }
    if (tid == 0) {
        nqs_result r;
        double F = 0.0, C = 0.0;
        for (int u = 0; u <= NQS_MAX_LEVEL; ++u) r.T[u] = 0.0;
        for (int u = 0; u <= level; ++u) {
            r.T[u] = T[u];
            const double t = F + T[u];
            C += (fabs(F) >= fabs(T[u])) ? (F - t) + T[u] : (T[u] - t) + F;
            F = t;
        }
        r.F = F + C;
        r.imag_residual = fabs(imag_tot);
        r.n_terms = (uint64_t)n_terms;
        r.bound = bound;
        r.level = level;
        r.status = NQS_OK;
        *res = r;
    }
}

int cu(cudaError_t e) { return e == cudaSuccess ? NQS_OK : NQS_ERR_CUDA; }

struct Run {
    Handle& h;
    cudaStream_t st;
    int n, level, grid;
    long long dim;
    const TermIndex& ti;
    std::vector<float2*> phi;      // per site
    std::vector<float2*> work;     // per depth
    double* part;                  // reduce partials (grid x 32)
    double2* kdev;                 // factor tables of this side: site s at kofs[s]
    std::vector<size_t> kofs;
    double2* amps;                 // this side's amplitudes
    std::vector<int> site_ev;      // event index of each site
    std::vector<int> ev_gate;      // event -> gate index or -1
    std::vector<int> ev_site;      // event -> site index or -1
    int last_site_ev = -1;
    bool side_b;
    int* js_dev;                   // finisher descriptor scratch (device)
    long long* pos_dev;
    int rc = NQS_OK;

    GMat gate_mat(int g, bool adjoint) {
        const Gate& gt = h.circ.gates[g];
        GMat m{};
        if (gate_is_two_qubit(gt.kind)) {
            Mat4 a = gate_matrix_2q(gt);
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c) {
                    const cd v = adjoint ? std::conj(a[4 * c + r]) : a[4 * r + c];
                    m.m[4 * r + c] = make_float2((float)v.real(), (float)v.imag());
                }
        } else {
            Mat2 a = gate_matrix_1q(gt);
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) {
                    const cd v = adjoint ? std::conj(a[2 * c + r]) : a[2 * r + c];
                    m.m[2 * r + c] = make_float2((float)v.real(), (float)v.imag());
                }
        }
        return m;
    }
    GMat factor_mat(int s, int j, bool adjoint) {
        const GFactors& f = h.gfac[s];
        const int d = f.nq == 1 ? 2 : 4;
        const std::vector<cd>& K = side_b ? f.KB : f.KA;
        GMat m{};
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c) {
                const cd v = adjoint ? std::conj(K[(size_t)j * d * d + d * c + r]) : K[(size_t)j * d * d + d * r + c];
                m.m[d * r + c] = make_float2((float)v.real(), (float)v.imag());
            }
        return m;
    }
    void apply(float2* s, int nq, int q0, int q1, const GMat& m) {
        if (rc) return;
        const long long count = dim >> nq;
        g_apply_kernel<<<grid, kT, 0, st>>>(s, count, nq, q0, q1, m);
        rc = cu(cudaGetLastError());
    }
    void apply_event(float2* s, int e, bool adjoint) {
        if (ev_gate[e] >= 0) {
            const Gate& g = h.circ.gates[ev_gate[e]];
            const bool two = gate_is_two_qubit(g.kind);
            apply(s, two ? 2 : 1, g.q0, g.q1, gate_mat(ev_gate[e], adjoint));
        } else {
            const GFactors& f = h.gfac[ev_site[e]];
            apply(s, f.nq, f.q0, f.q1, factor_mat(ev_site[e], 0, adjoint));
        }
    }
    // reduce (phi_t, w) and write amps for the listed (factor, rank) pairs
    void reduce_finish(int t, const float2* w, const std::vector<int>& js, const std::vector<long long>& pos) {
        if (rc || js.empty()) return;
        const GFactors& f = h.gfac[t];
        const long long count = dim >> f.nq;
        g_reduce_kernel<<<grid, kT, 0, st>>>(phi[t], w, count, f.nq, f.q0, f.q1, part);
        rc = cu(cudaGetLastError());
        if (rc) return;
        // the descriptor lists go through a small staging copy (stream ordered)
        rc = cu(cudaMemcpyAsync(js_dev, js.data(), js.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        if (!rc) rc = cu(cudaMemcpyAsync(pos_dev, pos.data(), pos.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
        if (rc) return;
        const int dd = f.nq == 1 ? 4 : 16;
        g_finish_kernel<<<1, kT, 0, st>>>(part, grid, dd, kdev + kofs[t], js_dev, pos_dev, (int)js.size(), amps);
        rc = cu(cudaGetLastError());
        // the host lists are reused by the next call: wait until the copies have been read
        if (!rc) rc = cu(cudaStreamSynchronize(st));
    }

    void expand(float2* w, int e0, int depth, std::vector<int>& c, std::vector<int>& fp) {
        for (int e = e0; e <= last_site_ev && !rc; ++e) {
            if (ev_gate[e] >= 0) {
                apply_event(w, e, false);
                continue;
            }
            const int t = ev_site[e];
            const GFactors& f = h.gfac[t];
            const bool last0 = depth == 0 && e == last_site_ev;
            if (depth < level || last0) {
                std::vector<int> js;
                std::vector<long long> pos;
                if (last0) {
                    js.push_back(0);
                    pos.push_back(0);
                }
                if (depth < level) {
                    c[depth] = t;
                    for (int j = 1; j < f.m; ++j) {
                        fp[depth] = j - 1;
                        js.push_back(j);
                        pos.push_back((long long)ti.rank(depth + 1, c.data(), fp.data()));
                    }
                }
                reduce_finish(t, w, js, pos);
                if (depth + 1 < level)
                    for (int j = 1; j < f.m && !rc; ++j) {
                        c[depth] = t;
                        fp[depth] = j - 1;
                        float2* w2 = work[depth + 1];
                        rc = cu(cudaMemcpyAsync(w2, w, dim * sizeof(float2), cudaMemcpyDeviceToDevice, st));
                        apply(w2, f.nq, f.q0, f.q1, factor_mat(t, j, false));
                        expand(w2, e + 1, depth + 1, c, fp);
                    }
            }
            apply_event(w, e, false);
        }
    }

    // the whole network for one factor set: backward checkpoints, forward expansion
    void network(const float2* psi0, const float2* v0) {
        const int n_ev = (int)ev_gate.size();
        float2* p = work[0];
        rc = cu(cudaMemcpyAsync(p, v0, dim * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        for (int e = n_ev - 1; e >= 0 && !rc; --e) {
            if (ev_gate[e] >= 0) {
                apply_event(p, e, true);
            } else {
                rc = cu(cudaMemcpyAsync(phi[ev_site[e]], p, dim * sizeof(float2), cudaMemcpyDeviceToDevice, st));
                apply_event(p, e, true);
            }
        }
        if (rc) return;
        rc = cu(cudaMemcpyAsync(work[0], psi0, dim * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        std::vector<int> c(level + 1), fp(level + 1);
        expand(work[0], 0, 0, c, fp);
    }
};

void release(GEngine& G, void* stream) {
    if (G.buf) dev_free(G.buf, G.buf_bytes, stream);
    if (G.aux) dev_free(G.aux, G.aux_bytes, stream);
    G.buf = G.aux = nullptr;
    G.buf_bytes = G.aux_bytes = 0;
}

}  // namespace

int general_fidelity(Handle& h, const nqs_state* psi, const nqs_state* v, int level, nqs_result* out, void* stream) {
    if (!h.geng) h.geng = new GEngine();
    GEngine& G = *h.geng;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = h.circ.n, N = (int)h.gfac.size();
    const long long dim = 1ll << n;
    level = std::min(level, N);
    std::vector<int> m(N);
    bool two_sided = false;
    for (int s = 0; s < N; ++s) {
        m[s] = h.gfac[s].m - 1;
        two_sided = two_sided || !h.gfac[s].same;
    }
    TermIndex ti;
    ti.build(m, level);
    // events in circuit order
    std::vector<int> ev_gate, ev_site, site_ev(N, -1);
    {
        size_t ns = 0;
        auto sites_after = [&](int g) {
            while (ns < h.circ.noises.size() && h.circ.noises[ns].after_gate == g) {
                site_ev[ns] = (int)ev_gate.size();
                ev_gate.push_back(-1);
                ev_site.push_back((int)ns);
                ++ns;
            }
        };
        sites_after(-1);
        for (size_t g = 0; g < h.circ.gates.size(); ++g) {
            ev_gate.push_back((int)g);
            ev_site.push_back(-1);
            sites_after((int)g);
        }
    }
    int last_site_ev = -1;
    for (int s = 0; s < N; ++s) last_site_ev = std::max(last_site_ev, site_ev[s]);
    if (N == 0) return NQS_ERR_UNSUPPORTED;   // the general path needs at least one noise
    // device memory: N phi, level + 1 work states, psi, v; aux: factors, partials, amps, values, tables
    const size_t sb = (size_t)dim * sizeof(float2);
    const size_t n_states = (size_t)N + level + 1 + 2;
    const size_t kcount = [&] {
        size_t c = 0;
        for (const auto& f : h.gfac) c += (size_t)f.m * (f.nq == 1 ? 4 : 16);
        return c;
    }();
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::max<long long>(1, std::min<long long>((long long)sms * 4, (dim / 2 + kT - 1) / kT));
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_k = 0;
    const size_t o_part = al(o_k + 2 * kcount * sizeof(double2));
    const size_t o_amps = al(o_part + (size_t)grid * 32 * sizeof(double));
    const size_t o_vals = al(o_amps + (two_sided ? 2 : 1) * (size_t)ti.total * sizeof(double2));
    const size_t o_loff = al(o_vals + (size_t)ti.total * sizeof(double));
    const size_t o_res = al(o_loff + (size_t)(level + 2) * sizeof(long long));
    const size_t o_js = al(o_res + sizeof(nqs_result));
    const size_t o_pos = al(o_js + 16 * sizeof(int));
    const size_t aux_bytes = al(o_pos + 16 * sizeof(long long));
    if (G.buf_bytes < n_states * sb || G.aux_bytes < aux_bytes) {
        release(G, stream);
        G.buf = dev_alloc(n_states * sb, stream);
        G.aux = dev_alloc(aux_bytes, stream);
        if (!G.buf || !G.aux) {
            release(G, stream);
            return NQS_ERR_NOMEM;
        }
        G.buf_bytes = n_states * sb;
        G.aux_bytes = aux_bytes;
    }
    char* ab = (char*)G.aux;
    double2* kdevA = (double2*)(ab + o_k);
    double2* kdevB = kdevA + kcount;
    double* part = (double*)(ab + o_part);
    double2* ampsA = (double2*)(ab + o_amps);
    double2* ampsB = two_sided ? ampsA + ti.total : nullptr;
    double* vals = (double*)(ab + o_vals);
    long long* loff = (long long*)(ab + o_loff);
    nqs_result* res = (nqs_result*)(ab + o_res);
    int* js_dev = (int*)(ab + o_js);
    long long* pos_dev = (long long*)(ab + o_pos);
    float2* base = (float2*)G.buf;
    float2* psi_buf = base + (size_t)(N + level + 1) * dim;
    float2* v_buf = psi_buf + dim;
    // factor tables (complex128) of both sides
    std::vector<double2> kh(2 * kcount);
    std::vector<size_t> kofs(N);
    {
        size_t at = 0;
        for (int s = 0; s < N; ++s) {
            const GFactors& f = h.gfac[s];
            kofs[s] = at;
            for (size_t e = 0; e < f.KA.size(); ++e) {
                kh[at + e] = make_double2(f.KA[e].real(), f.KA[e].imag());
                kh[kcount + at + e] = make_double2(f.KB[e].real(), f.KB[e].imag());
            }
            at += f.KA.size();
        }
    }
    std::vector<long long> lo(level + 2);
    for (int u = 0; u <= level + 1; ++u) lo[u] = (long long)ti.level_offset[u];
    int rc = cu(cudaMemcpyAsync(kdevA, kh.data(), kh.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    if (!rc) rc = cu(cudaMemcpyAsync(loff, lo.data(), lo.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
    if (!rc) rc = cu(cudaMemsetAsync(ampsA, 0, (two_sided ? 2 : 1) * (size_t)ti.total * sizeof(double2), st));
    // psi, v
    const int fill_grid = (int)std::max<long long>(1, std::min<long long>((long long)sms * 8, dim / kT));
    if (!rc) {
        if (psi->kind == NQS_STATE_BASIS) g_fill_kernel<<<fill_grid, kT, 0, st>>>(psi_buf, dim, psi->bits);
        else rc = cu(cudaMemcpyAsync(psi_buf, psi->dev, sb, cudaMemcpyDeviceToDevice, st));
        if (!rc) rc = cu(cudaGetLastError());
    }
    Run R{h, st, n, level, grid, dim, ti, {}, {}, part, kdevA, kofs, ampsA, site_ev, ev_gate, ev_site,
          last_site_ev, false, js_dev, pos_dev};
    for (int s = 0; s < N; ++s) R.phi.push_back(base + (size_t)s * dim);
    for (int d = 0; d <= level; ++d) R.work.push_back(base + (size_t)(N + d) * dim);
    R.rc = rc;
    if (!R.rc) {
        if (v->kind == NQS_STATE_BASIS) {
            g_fill_kernel<<<fill_grid, kT, 0, st>>>(v_buf, dim, v->bits);
            R.rc = cu(cudaGetLastError());
        } else if (v->kind == NQS_STATE_DENSE) {
            R.rc = cu(cudaMemcpyAsync(v_buf, v->dev, sb, cudaMemcpyDeviceToDevice, st));
        } else {   // U |psi>
            R.rc = cu(cudaMemcpyAsync(v_buf, psi_buf, sb, cudaMemcpyDeviceToDevice, st));
            for (size_t e = 0; e < ev_gate.size() && !R.rc; ++e)
                if (ev_gate[e] >= 0) R.apply_event(v_buf, (int)e, false);
        }
    }
    if (!R.rc) R.network(psi_buf, v_buf);
    if (!R.rc && two_sided) {
        R.side_b = true;
        R.kdev = kdevB;
        R.amps = ampsB;
        R.network(psi_buf, v_buf);
    }
    rc = R.rc;
    if (!rc) {
        double bound = 0.0;
        std::vector<double> poly(1, 1.0);
        for (const auto& f : h.gfac) {
            std::vector<double> nx(poly.size() + 1, 0.0);
            for (size_t i = 0; i < poly.size(); ++i) {
                nx[i] += poly[i] * f.norm_dom;
                nx[i + 1] += poly[i] * f.norm_rest;
            }
            poly.swap(nx);
        }
        for (size_t i = level + 1; i < poly.size(); ++i) bound += poly[i];
        g_sum_kernel<<<1, kT, 0, st>>>(ampsA, ampsB, loff, level, (long long)ti.total, bound, vals, res);
        rc = cu(cudaGetLastError());
    }
    if (!rc) rc = cu(cudaMemcpyAsync(out, res, sizeof(nqs_result), cudaMemcpyDefault, st));
    G.n_terms = (long long)ti.total;
    G.vals = vals;
    G.last = st;
    G.has_result = rc == NQS_OK;
    return rc;
}

int general_term_values(Handle& h, double* out, size_t cap, size_t* count) {
    if (!h.geng || !h.geng->has_result) return NQS_ERR_ORDER;
    GEngine& G = *h.geng;
    *count = (size_t)G.n_terms;
    const size_t nb = std::min<size_t>(cap, (size_t)G.n_terms) * sizeof(double);
    if (cudaStreamSynchronize(G.last) != cudaSuccess) return NQS_ERR_CUDA;
    if (nb && cudaMemcpy(out, G.vals, nb, cudaMemcpyDeviceToHost) != cudaSuccess) return NQS_ERR_CUDA;
    return NQS_OK;
}

void general_destroy(Handle& h) {
    if (!h.geng) return;
    if (h.geng->last) cudaStreamSynchronize(h.geng->last);
    release(*h.geng, h.geng->last);
    delete h.geng;
    h.geng = nullptr;
}

}  // namespace nqs
