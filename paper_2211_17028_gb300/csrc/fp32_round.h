// Rounding of unitary operations to complex64 that keeps them unitary as far
// as FP32 allows (host code).
//
// A gate's matrix rounded entry by entry to FP32 is off unitarity by up to
// about one ulp in its singular values.  The sweeps apply hundreds of gates,
// and in the circuits of interest many share their angles (a QAOA layer
// applies the same mixer rotation to every qubit and the same ZZ phase to
// every edge), so those errors add up coherently: the state's norm drifts by
// the gate count times the per-gate error, about 1e-5 over 700 gates -- as
// much as the whole parity budget.  Choosing, among the FP32 neighbours of
// the exact entries, the ones whose matrix is closest to unitary removes the
// coherent part; what remains is the random rounding of the arithmetic.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <complex>

namespace nqs {

namespace fp32r {

using cdr = std::complex<double>;

inline double unitarity_defect(const float* x, int dim) {
    // || M^dagger M - I ||_F^2 in double for M with interleaved (re, im) entries
    double acc = 0.0;
    for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) {
            cdr s = 0.0;
            for (int k = 0; k < dim; ++k) {
                const cdr a(x[2 * (dim * k + i)], -x[2 * (dim * k + i) + 1]);
                const cdr b(x[2 * (dim * k + j)], x[2 * (dim * k + j) + 1]);
                s += a * b;
            }
            if (i == j) s -= 1.0;
            acc += std::norm(s);
        }
    return acc;
}

inline double distance2(const float* x, const cdr* m, int n) {
    double acc = 0.0;
    for (int e = 0; e < n; ++e) acc += std::norm(cdr(x[2 * e], x[2 * e + 1]) - m[e]);
    return acc;
}

}  // namespace fp32r

// A complex number of modulus 1 (to 1e-9) rounded to the FP32 pair, among the
// nine neighbours of the nearest one, with modulus closest to 1 (ties: closest
// to the exact value); other numbers are rounded to nearest.
inline float2 round_c64(std::complex<double> c) {
    float re = (float)c.real(), im = (float)c.imag();
    if (std::fabs(std::abs(c) - 1.0) > 1e-9) return make_float2(re, im);
    float best_re = re, best_im = im;
    double best = 1e300;
    for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b) {
            float r = re, i = im;
            if (a) r = std::nextafter(re, a > 0 ? INFINITY : -INFINITY);
            if (b) i = std::nextafter(im, b > 0 ? INFINITY : -INFINITY);
            const double mod = std::fabs((double)r * r + (double)i * i - 1.0);
            const double dist = std::norm(std::complex<double>(r, i) - c);
            const double cost = mod + 1e-3 * dist;
            if (cost < best) {
                best = cost;
                best_re = r;
                best_im = i;
            }
        }
    return make_float2(best_re, best_im);
}

// A dim x dim matrix (row-major) rounded to complex64.  Unitary matrices
// (to 1e-9) are rounded to be as close to unitary as FP32 allows: diagonal
// ones entry by entry (round_c64), others by coordinate descent over one-ulp
// moves of the entries' components, minimising the unitarity defect plus a
// small multiple of the distance to the exact matrix.  Exact zeros stay zero.
inline void round_matrix_c64(const std::complex<double>* m, int dim, float2* out) {
    const int n = dim * dim;
    bool diag = true;
    for (int r = 0; r < dim; ++r)
        for (int c = 0; c < dim; ++c)
            if (r != c && m[dim * r + c] != 0.0) diag = false;
    float x[32];
    for (int e = 0; e < n; ++e) {
        x[2 * e] = (float)m[e].real();
        x[2 * e + 1] = (float)m[e].imag();
    }
    // unitary to 1e-9 in double?
    double defect = 0.0;
    for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) {
            std::complex<double> s = 0.0;
            for (int k = 0; k < dim; ++k) s += std::conj(m[dim * k + i]) * m[dim * k + j];
            if (i == j) s -= 1.0;
            defect += std::norm(s);
        }
    if (defect <= 1e-18) {
        if (diag) {
            for (int e = 0; e < n; ++e) {
                if (e % (dim + 1)) continue;
                const float2 v = round_c64(m[e]);
                x[2 * e] = v.x;
                x[2 * e + 1] = v.y;
            }
        } else {
            auto cost = [&](const float* y) {
                return fp32r::unitarity_defect(y, dim) + 1e-3 * fp32r::distance2(y, m, n);
            };
            double cur = cost(x);
            for (int it = 0; it < 4; ++it) {
                bool moved = false;
                for (int k = 0; k < 2 * n; ++k) {
                    if (x[k] == 0.0f) continue;
                    const float keep = x[k];
                    for (int d = -1; d <= 1; d += 2) {
                        x[k] = std::nextafter(keep, d > 0 ? INFINITY : -INFINITY);
                        const double c = cost(x);
                        if (c < cur) {
                            cur = c;
                            moved = true;
                            break;
                        }
                        x[k] = keep;
                    }
                }
                if (!moved) break;
            }
        }
    }
    for (int e = 0; e < n; ++e) out[e] = make_float2(x[2 * e], x[2 * e + 1]);
}

}  // namespace nqs
