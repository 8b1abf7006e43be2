/*
 * Plain FP64 state-vector step of the oracle (test infrastructure only).
 *
 * The oracle contracts each split network of Algorithm 1 (Sec. IV) as a
 * state-vector sweep; this file is the same textbook operation as
 * oracle/statevector.py -- apply a 2x2 or 4x4 matrix to the amplitudes that
 * differ only in the acted-on qubits -- written in C so that widths up to
 * ~30 qubits finish.  No blocking, fusion or reordering: one pass over the
 * state per operation, in the order given.  Qubit q is bit q of the index;
 * a 4x4 matrix is indexed by 2*b(q0) + b(q1).
 *
 * States are interleaved (re, im) doubles.  OpenMP parallelises each pass.
 */
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } cplx;

static inline cplx cmul(cplx a, cplx b) {
    cplx r = { a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re };
    return r;
}
static inline cplx cadd(cplx a, cplx b) { cplx r = { a.re + b.re, a.im + b.im }; return r; }

static void apply_1q(int n, cplx* s, int q, const cplx* m) {
    const int64_t half = (int64_t)1 << (n - 1);
    const int64_t bit = (int64_t)1 << q;
    #pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < half; ++p) {
        int64_t lo = p & (bit - 1);
        int64_t i0 = ((p - lo) << 1) | lo;
        int64_t i1 = i0 | bit;
        cplx a = s[i0], b = s[i1];
        s[i0] = cadd(cmul(m[0], a), cmul(m[1], b));
        s[i1] = cadd(cmul(m[2], a), cmul(m[3], b));
    }
}

static int64_t insert_zero(int64_t x, int64_t bit) {
    int64_t lo = x & (bit - 1);
    return ((x - lo) << 1) | lo;
}

static void apply_2q(int n, cplx* s, int q0, int q1, const cplx* m) {
    const int64_t quarter = (int64_t)1 << (n - 2);
    const int64_t b0 = (int64_t)1 << q0, b1 = (int64_t)1 << q1;
    const int64_t blo = b0 < b1 ? b0 : b1, bhi = b0 < b1 ? b1 : b0;
    #pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < quarter; ++p) {
        int64_t base = insert_zero(insert_zero(p, blo), bhi);
        int64_t idx[4] = { base, base | b1, base | b0, base | b0 | b1 };
        cplx in[4], out[4];
        for (int k = 0; k < 4; ++k) in[k] = s[idx[k]];
        for (int r = 0; r < 4; ++r) {
            cplx acc = { 0.0, 0.0 };
            for (int c = 0; c < 4; ++c) acc = cadd(acc, cmul(m[4 * r + c], in[c]));
            out[r] = acc;
        }
        for (int k = 0; k < 4; ++k) s[idx[k]] = out[k];
    }
}

/* Apply n_ops operations in order.  arity[k] is 1 or 2; mats holds 16 complex
 * values (32 doubles) per operation, of which a 1-qubit op uses the first 4. */
void nqso_apply_ops(int n, double* state, int n_ops, const int* arity, const int* q0,
                    const int* q1, const double* mats, int threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    cplx* s = (cplx*)state;
    for (int k = 0; k < n_ops; ++k) {
        const cplx* m = (const cplx*)(mats + 32 * (size_t)k);
        if (arity[k] == 1) apply_1q(n, s, q0[k], m);
        else apply_2q(n, s, q0[k], q1[k], m);
    }
}

/* out = <a|b> = sum conj(a_i) b_i, accumulated per thread then summed. */
void nqso_inner(int n, const double* a, const double* b, double* out) {
    const int64_t d = (int64_t)1 << n;
    const cplx* x = (const cplx*)a;
    const cplx* y = (const cplx*)b;
    double re = 0.0, im = 0.0;
    #pragma omp parallel for reduction(+:re, im) schedule(static)
    for (int64_t i = 0; i < d; ++i) {
        re += x[i].re * y[i].re + x[i].im * y[i].im;
        im += x[i].re * y[i].im - x[i].im * y[i].re;
    }
    out[0] = re;
    out[1] = im;
}

int nqso_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
