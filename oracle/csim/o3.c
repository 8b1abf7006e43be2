/*
 * O3: every kept amplitude of the level-l expansion by forward / backward
 * checkpoints, FP64 (oracle; test infrastructure only).
 *
 * What it computes (Sec. IV, Algorithm 1).  A kept assignment sigma puts the
 * factor F_s[sigma_s] at every noise site s, with sigma_s = 0 (the dominant
 * factor) at all but at most l sites.  Its amplitude is
 *     amp(sigma) = sum_i conj(bra_i) (C[F_sigma] psi)_i ,
 * C[F_sigma] being the gate sequence with the factors inserted at the sites.
 * The caller evaluates the two networks of a term by calling this twice
 * (gates U with factors U_i and bra v; gates U^* with factors V_i, psi^*
 * and bra v^*) and multiplies the two amplitudes.
 *
 * How (instead of one sweep per term):
 *   backward: phi_s = (events after site s, with F_t[0] at the later sites)^dagger bra,
 *             stored for every site;
 *   forward:  the state before site s with F_t[0] at the earlier sites;
 *   at site t the reduced matrix R[a][b] = sum_rest conj(phi_t[rest,a]) w[rest,b]
 *   on the site's qubits gives <phi_t| F_t[j] |w> = sum_ab F_t[j][a][b] R[a][b]
 *   for every factor j at once;
 *   an assignment whose first non-dominant site is s starts from
 *   F_s[j] (state before s) and is swept on, depth first, reducing at every later
 *   site, so level u re-sweeps only from its first insertion.
 * Every operation is one plain pass over the state in event order: no
 * fusion, no tiling.  Sites act on one or two qubits (2x2 or 4x4 factors,
 * 4x4 indexed 2*b(q0) + b(q1)); each site has m_s factors, index 0 dominant.
 *
 * Output order is the canonical one of the kept-term records: level u
 * ascending, then the site tuple in lexicographic order, then the factor
 * tuple (indices 1..m_s-1 per site) in lexicographic order.
 *
 * Parallelism (OpenMP): for wide states each pass is split over amplitudes;
 * for narrow ones (n <= 16) the first insertions (s, j) are spread over the
 * threads, each with its own work states.
 */
#define _POSIX_C_SOURCE 199309L
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } cplx;

static inline cplx cmul(cplx a, cplx b) {
    cplx r = { a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re };
    return r;
}
static inline cplx cadd(cplx a, cplx b) { cplx r = { a.re + b.re, a.im + b.im }; return r; }
static inline cplx cconj(cplx a) { cplx r = { a.re, -a.im }; return r; }

typedef struct {
    int n;                 /* qubits */
    int n_ev;              /* events */
    const int* kind;       /* 0 gate, 1 site */
    const int* nq;         /* qubits acted on: 1 or 2 */
    const int* q0;
    const int* q1;
    const int* site;       /* site index of a site event */
    const cplx* mat;       /* 16 complex per event (gate matrix; unused for sites) */
    int n_sites;
    const int* m;          /* factors per site */
    const cplx* fac;       /* per site 16 factors x 16 complex */
    int level;
    int par_amps;          /* 1: split each pass over amplitudes */
    int last_site_ev;      /* event index of the last site */
    int* site_ev;          /* event index of every site */
    cplx** phi;            /* backward checkpoints */
    int64_t** set_off;     /* per level: offset of the first term of each site set (lexicographic rank) */
    int64_t n_terms;
    int64_t* binom;        /* (N+1) x (L+1) binomials */
    cplx* out;
} O3;

static const cplx* factor(const O3* o, int s, int j) { return o->fac + ((size_t)s * 16 + j) * 16; }

/* ------------------------------------------------------------------ passes */

static int64_t insert_zero(int64_t x, int64_t bit) {
    int64_t lo = x & (bit - 1);
    return ((x - lo) << 1) | lo;
}

/* apply a 2x2 (nq = 1) or 4x4 (nq = 2) matrix; mat indexed 2*b(q0) + b(q1) */
static void apply(int n, cplx* s, int nq, int q0, int q1, const cplx* m, int adjoint, int par) {
    cplx mm[16];
    const int d = nq == 1 ? 2 : 4;
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) mm[d * r + c] = adjoint ? cconj(m[d * c + r]) : m[d * r + c];
    if (nq == 1) {
        const int64_t half = (int64_t)1 << (n - 1), bit = (int64_t)1 << q0;
        #pragma omp parallel for schedule(static) if (par)
        for (int64_t p = 0; p < half; ++p) {
            int64_t i0 = insert_zero(p, bit), i1 = i0 | bit;
            cplx a = s[i0], b = s[i1];
            s[i0] = cadd(cmul(mm[0], a), cmul(mm[1], b));
            s[i1] = cadd(cmul(mm[2], a), cmul(mm[3], b));
        }
    } else {
        const int64_t quarter = (int64_t)1 << (n - 2);
        const int64_t b0 = (int64_t)1 << q0, b1 = (int64_t)1 << q1;
        const int64_t lo = b0 < b1 ? b0 : b1, hi = b0 < b1 ? b1 : b0;
        #pragma omp parallel for schedule(static) if (par)
        for (int64_t p = 0; p < quarter; ++p) {
            int64_t base = insert_zero(insert_zero(p, lo), hi);
            int64_t idx[4] = { base, base | b1, base | b0, base | b0 | b1 };
            cplx in[4];
            for (int k = 0; k < 4; ++k) in[k] = s[idx[k]];
            for (int r = 0; r < 4; ++r) {
                cplx acc = { 0.0, 0.0 };
                for (int c = 0; c < 4; ++c) acc = cadd(acc, cmul(mm[4 * r + c], in[c]));
                s[idx[r]] = acc;
            }
        }
    }
}

/* R[a][b] = sum_rest conj(phi[rest,a]) w[rest,b] on the site's qubits */
static void reduced(int n, const cplx* phi, const cplx* w, int nq, int q0, int q1, cplx* R, int par) {
    const int d = nq == 1 ? 2 : 4;
    double acc[32];
    memset(acc, 0, sizeof acc);
    const int64_t b0 = (int64_t)1 << q0, b1 = nq == 2 ? (int64_t)1 << q1 : 0;
    const int64_t lo = (nq == 1 || b0 < b1) ? b0 : b1, hi = (nq == 1 || b0 < b1) ? b1 : b0;
    const int64_t count = (int64_t)1 << (n - nq);
    #pragma omp parallel if (par)
    {
        double loc[32];
        memset(loc, 0, sizeof loc);
        #pragma omp for schedule(static)
        for (int64_t p = 0; p < count; ++p) {
            int64_t base = insert_zero(p, lo);
            if (nq == 2) base = insert_zero(base, hi);
            int64_t idx[4];
            if (nq == 1) {
                idx[0] = base;
                idx[1] = base | b0;
            } else {
                idx[0] = base;
                idx[1] = base | b1;
                idx[2] = base | b0;
                idx[3] = base | b0 | b1;
            }
            for (int a = 0; a < d; ++a) {
                const cplx f = cconj(phi[idx[a]]);
                for (int b = 0; b < d; ++b) {
                    const cplx x = cmul(f, w[idx[b]]);
                    loc[2 * (d * a + b)] += x.re;
                    loc[2 * (d * a + b) + 1] += x.im;
                }
            }
        }
        #pragma omp critical
        for (int k = 0; k < 2 * d * d; ++k) acc[k] += loc[k];
    }
    for (int k = 0; k < d * d; ++k) {
        R[k].re = acc[2 * k];
        R[k].im = acc[2 * k + 1];
    }
}

static cplx contract(const cplx* F, const cplx* R, int d) {
    cplx a = { 0.0, 0.0 };
    for (int k = 0; k < d * d; ++k) a = cadd(a, cmul(F[k], R[k]));
    return a;
}

/* --------------------------------------------------------------- canonical order */

static int64_t bin(const O3* o, int a, int b) {
    if (b < 0 || a < b) return 0;
    return o->binom[(size_t)a * (o->level + 1) + b];
}

/* lexicographic rank of the combination c[0] < ... < c[u-1] of {0..N-1} */
static int64_t lex_rank(const O3* o, const int* c, int u) {
    const int N = o->n_sites;
    int64_t r = 0;
    int prev = -1;
    for (int j = 0; j < u; ++j) {
        for (int x = prev + 1; x < c[j]; ++x) r += bin(o, N - 1 - x, u - 1 - j);
        prev = c[j];
    }
    return r;
}

static int build_offsets(O3* o) {
    const int N = o->n_sites, L = o->level;
    o->binom = (int64_t*)calloc((size_t)(N + 1) * (L + 1), sizeof(int64_t));
    if (!o->binom) return -1;
    for (int a = 0; a <= N; ++a)
        for (int b = 0; b <= L && b <= a; ++b)
            o->binom[(size_t)a * (L + 1) + b] = (b == 0 || b == a) ? 1
                : o->binom[(size_t)(a - 1) * (L + 1) + b - 1] + o->binom[(size_t)(a - 1) * (L + 1) + b];
    o->set_off = (int64_t**)calloc((size_t)L + 1, sizeof(int64_t*));
    int64_t total = 0;
    for (int u = 0; u <= L; ++u) {
        const int64_t cnt = bin(o, N, u);
        o->set_off[u] = (int64_t*)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(int64_t));
        if (!o->set_off[u]) return -1;
        int c[16];
        for (int j = 0; j < u; ++j) c[j] = j;
        for (int64_t r = 0; r < cnt; ++r) {   /* combinations in lexicographic order */
            o->set_off[u][r] = total;
            int64_t per = 1;
            for (int j = 0; j < u; ++j) per *= o->m[c[j]] - 1;
            total += per;
            int j = u - 1;
            while (j >= 0 && c[j] == N - u + j) --j;
            if (j < 0) break;
            ++c[j];
            for (int k = j + 1; k < u; ++k) c[k] = c[k - 1] + 1;
        }
    }
    o->n_terms = total;
    return 0;
}

/* position of the term (sites c[0..u-1], factor indices f[0..u-1] >= 1) */
static int64_t term_pos(const O3* o, const int* c, const int* f, int u) {
    int64_t pos = o->set_off[u][lex_rank(o, c, u)], stride = 1;
    for (int j = u - 1; j >= 0; --j) {
        pos += (f[j] - 1) * stride;
        stride *= o->m[c[j]] - 1;
    }
    return pos;
}

/* --------------------------------------------------------------- the sweeps */

typedef struct {
    cplx** work;   /* one state per depth */
} Bufs;

/* Sweep w (the state before event e0, `depth` factors chosen: c/f) to the
 * last site, reducing at every site and recursing into every non-dominant
 * factor while depth + 1 < level.  At depth 0 the reduction at the last site
 * also gives the level-0 amplitude.  w is overwritten. */
static void expand(const O3* o, cplx* w, int e0, int depth, int* c, int* f, Bufs* B, int par) {
    const int64_t dim = (int64_t)1 << o->n;
    for (int e = e0; e <= o->last_site_ev; ++e) {
        const int nq = o->nq[e], q0 = o->q0[e], q1 = o->q1[e];
        if (o->kind[e] == 0) {
            apply(o->n, w, nq, q0, q1, o->mat + (size_t)e * 16, 0, par);
            continue;
        }
        const int t = o->site[e];
        const int d = nq == 1 ? 2 : 4;
        const int last0 = depth == 0 && e == o->last_site_ev;
        if (depth < o->level || last0) {
            cplx R[16];
            reduced(o->n, o->phi[t], w, nq, q0, q1, R, par);
            if (last0) o->out[0] = contract(factor(o, t, 0), R, d);
            if (depth < o->level) {
                c[depth] = t;
                for (int j = 1; j < o->m[t]; ++j) {
                    f[depth] = j;
                    o->out[term_pos(o, c, f, depth + 1)] = contract(factor(o, t, j), R, d);
                    if (depth + 1 < o->level) {
                        cplx* w2 = B->work[depth + 1];
                        memcpy(w2, w, (size_t)dim * sizeof(cplx));
                        apply(o->n, w2, nq, q0, q1, factor(o, t, j), 0, par);
                        expand(o, w2, e + 1, depth + 1, c, f, B, par);
                    }
                }
            }
        }
        apply(o->n, w, nq, q0, q1, factor(o, t, 0), 0, par);
    }
}

static cplx* new_state(int n) { return (cplx*)malloc(((size_t)1 << n) * sizeof(cplx)); }

/*
 * Entry point.  Events: kind (0 gate, 1 site), nq, q0, q1 (-1 if unused),
 * site index of site events, 32 doubles (16 complex) of gate matrix per event.
 * Sites: m[s] factors (2..16), 16 factors x 32 doubles per site.  psi and bra
 * are 2^n complex (interleaved doubles).  Writes every kept amplitude, in the
 * canonical order, to amps (2 doubles each, room for cap terms) and the term
 * count to *n_terms.  Returns 0, or -1 (bad argument / out of memory), or -2
 * (cap too small: *n_terms still set).
 */
int nqso3_amplitudes(int n, int n_ev, const int* kind, const int* nq, const int* q0, const int* q1,
                     const int* site, const double* mat, int n_sites, const int* m, const double* fac,
                     const double* psi, const double* bra, int level, double* amps, int64_t cap,
                     int64_t* n_terms, int threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
    const int nthr = omp_get_max_threads();
#else
    (void)threads;
    const int nthr = 1;
#endif
    if (n < 1 || n > 40 || level < 0 || !n_terms) return -1;
    if (level > n_sites) level = n_sites;
    O3 o;
    memset(&o, 0, sizeof o);
    o.n = n; o.n_ev = n_ev; o.kind = kind; o.nq = nq; o.q0 = q0; o.q1 = q1; o.site = site;
    o.mat = (const cplx*)mat; o.n_sites = n_sites; o.m = m; o.fac = (const cplx*)fac; o.level = level;
    o.par_amps = n > 16;
    const int64_t dim = (int64_t)1 << n;
    int rc = 0;
    o.site_ev = (int*)calloc((size_t)(n_sites > 0 ? n_sites : 1), sizeof(int));
    for (int e = 0; e < n_ev; ++e)
        if (kind[e] == 1) {
            if (site[e] < 0 || site[e] >= n_sites) return -1;
            o.site_ev[site[e]] = e;
            o.last_site_ev = e;
        }
    if (build_offsets(&o) != 0) return -1;
    *n_terms = o.n_terms;
    if (o.n_terms > cap || !amps) { rc = -2; goto done; }
    o.out = (cplx*)amps;
    memset(amps, 0, (size_t)o.n_terms * sizeof(cplx));

    if (n_sites == 0) {   /* plain amplitude <bra| C |psi> */
        cplx* w = new_state(n);
        memcpy(w, psi, (size_t)dim * sizeof(cplx));
        for (int e = 0; e < n_ev; ++e) apply(n, w, nq[e], q0[e], q1[e], o.mat + (size_t)e * 16, 0, 1);
        double re = 0.0, im = 0.0;
        const cplx* b = (const cplx*)bra;
        #pragma omp parallel for reduction(+:re, im) schedule(static)
        for (int64_t i = 0; i < dim; ++i) {
            re += b[i].re * w[i].re + b[i].im * w[i].im;
            im += b[i].re * w[i].im - b[i].im * w[i].re;
        }
        o.out[0].re = re;
        o.out[0].im = im;
        free(w);
        goto done;
    }

    /* backward checkpoints */
    o.phi = (cplx**)calloc((size_t)n_sites, sizeof(cplx*));
    {
        cplx* p = new_state(n);
        if (!p) { rc = -1; goto done; }
        memcpy(p, bra, (size_t)dim * sizeof(cplx));
        for (int e = n_ev - 1; e >= 0; --e) {
            if (kind[e] == 0) {
                apply(n, p, nq[e], q0[e], q1[e], o.mat + (size_t)e * 16, 1, 1);
            } else {
                const int t = site[e];
                o.phi[t] = new_state(n);
                if (!o.phi[t]) { free(p); rc = -1; goto done; }
                memcpy(o.phi[t], p, (size_t)dim * sizeof(cplx));
                apply(n, p, nq[e], q0[e], q1[e], factor(&o, t, 0), 1, 1);
            }
        }
        free(p);
    }

    if (o.par_amps) {
        /* one depth-first sweep, every pass split over amplitudes */
        Bufs B;
        B.work = (cplx**)calloc((size_t)level + 1, sizeof(cplx*));
        for (int dd = 0; dd <= level; ++dd) B.work[dd] = new_state(n);
        memcpy(B.work[0], psi, (size_t)dim * sizeof(cplx));
        int c[16], f[16];
        expand(&o, B.work[0], 0, 0, c, f, &B, 1);
        for (int dd = 0; dd <= level; ++dd) free(B.work[dd]);
        free(B.work);
    } else {
        /* forward checkpoints, then the first insertions spread over threads */
        cplx** chi = (cplx**)calloc((size_t)n_sites, sizeof(cplx*));
        cplx* w = new_state(n);
        memcpy(w, psi, (size_t)dim * sizeof(cplx));
        for (int e = 0; e <= o.last_site_ev; ++e) {
            if (kind[e] == 0) {
                apply(n, w, nq[e], q0[e], q1[e], o.mat + (size_t)e * 16, 0, 0);
            } else {
                const int t = site[e];
                chi[t] = new_state(n);
                memcpy(chi[t], w, (size_t)dim * sizeof(cplx));
                apply(n, w, nq[e], q0[e], q1[e], factor(&o, t, 0), 0, 0);
            }
        }
        free(w);
        {
            const int e = o.last_site_ev, t = site[e];
            cplx R[16];
            reduced(n, o.phi[t], chi[t], nq[e], q0[e], q1[e], R, 0);
            o.out[0] = contract(factor(&o, t, 0), R, nq[e] == 1 ? 2 : 4);
        }
        if (level >= 1) {
            #pragma omp parallel num_threads(nthr)
            {
                Bufs B;
                B.work = (cplx**)calloc((size_t)level + 1, sizeof(cplx*));
                for (int dd = 0; dd <= level; ++dd) B.work[dd] = new_state(n);
                int c[16], f[16];
                #pragma omp for schedule(dynamic, 1)
                for (int t = 0; t < n_sites; ++t) {
                    const int e = o.site_ev[t], qn = nq[e], a0 = q0[e], a1 = q1[e];
                    const int d = qn == 1 ? 2 : 4;
                    cplx R[16];
                    reduced(n, o.phi[t], chi[t], qn, a0, a1, R, 0);
                    c[0] = t;
                    for (int j = 1; j < m[t]; ++j) {
                        f[0] = j;
                        o.out[term_pos(&o, c, f, 1)] = contract(factor(&o, t, j), R, d);
                        if (level >= 2) {
                            memcpy(B.work[1], chi[t], (size_t)dim * sizeof(cplx));
                            apply(n, B.work[1], qn, a0, a1, factor(&o, t, j), 0, 0);
                            expand(&o, B.work[1], e + 1, 1, c, f, &B, 0);
                        }
                    }
                }
                for (int dd = 0; dd <= level; ++dd) free(B.work[dd]);
                free(B.work);
            }
        }
        for (int t = 0; t < n_sites; ++t) free(chi[t]);
        free(chi);
    }

done:
    if (o.phi) {
        for (int t = 0; t < n_sites; ++t) free(o.phi[t]);
        free(o.phi);
    }
    if (o.set_off) {
        for (int u = 0; u <= o.level; ++u) free(o.set_off[u]);
        free(o.set_off);
    }
    free(o.binom);
    free(o.site_ev);
    return rc;
}

/* Term count of the canonical list (no amplitudes). */
int64_t nqso3_term_count(int n_sites, const int* m, int level) {
    if (level > n_sites) level = n_sites;
    O3 o;
    memset(&o, 0, sizeof o);
    o.n_sites = n_sites;
    o.m = m;
    o.level = level;
    if (build_offsets(&o) != 0) return -1;
    const int64_t t = o.n_terms;
    for (int u = 0; u <= level; ++u) free(o.set_off[u]);
    free(o.set_off);
    free(o.binom);
    return t;
}

/* ------------------------------------------------------------------ chosen site sets */

/* Sweep w from event e0 through the sites of set c[depth..k-1]: gates and the
 * dominant factor at every site not in the set; at site c[depth] every
 * non-dominant factor is inserted in turn (depth first); at the last site the
 * reduced matrix against phi gives all its factors at once.  amps receives
 * prod(m - 1) values per set in lexicographic factor order. */
static void set_expand(const O3* o, cplx* w, int e0, const int* c, int k, int depth, cplx** bufs, cplx* out,
                       int64_t* pos, int par) {
    const int64_t dim = (int64_t)1 << o->n;
    const int target = c[depth];
    const int et = o->site_ev[target];
    for (int e = e0; e < et; ++e) {
        const int nq = o->nq[e], q0 = o->q0[e], q1 = o->q1[e];
        if (o->kind[e] == 0) apply(o->n, w, nq, q0, q1, o->mat + (size_t)e * 16, 0, par);
        else apply(o->n, w, nq, q0, q1, factor(o, o->site[e], 0), 0, par);
    }
    const int nq = o->nq[et], q0 = o->q0[et], q1 = o->q1[et];
    if (depth == k - 1) {
        cplx R[16];
        reduced(o->n, o->phi[target], w, nq, q0, q1, R, par);
        for (int j = 1; j < o->m[target]; ++j) out[(*pos)++] = contract(factor(o, target, j), R, nq == 1 ? 2 : 4);
        return;
    }
    for (int j = 1; j < o->m[target]; ++j) {
        cplx* w2 = bufs[depth + 1];
        memcpy(w2, w, (size_t)dim * sizeof(cplx));
        apply(o->n, w2, nq, q0, q1, factor(o, target, j), 0, par);
        set_expand(o, w2, et + 1, c, k, depth + 1, bufs, out, pos, par);
    }
}

/*
 * Amplitudes of every factor choice on each of m_sets chosen site sets
 * (k sites each, ascending), the dominant factor at all other sites: for set
 * S the prod_{s in S}(m_s - 1) amplitudes in lexicographic factor order, sets
 * one after the other.  Same network arguments as nqso3_amplitudes.  Returns
 * 0, or -1 (bad argument / out of memory).
 */
int nqso3_set_amplitudes(int n, int n_ev, const int* kind, const int* nq, const int* q0, const int* q1,
                         const int* site, const double* mat, int n_sites, const int* m, const double* fac,
                         const double* psi, const double* bra, int k, const int* sets, int64_t m_sets,
                         double* amps, int threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    if (n < 1 || n > 40 || k < 1 || k > 8 || n_sites < k || !amps) return -1;
    O3 o;
    memset(&o, 0, sizeof o);
    o.n = n; o.n_ev = n_ev; o.kind = kind; o.nq = nq; o.q0 = q0; o.q1 = q1; o.site = site;
    o.mat = (const cplx*)mat; o.n_sites = n_sites; o.m = m; o.fac = (const cplx*)fac;
    const int64_t dim = (int64_t)1 << n;
    int rc = 0;
    o.site_ev = (int*)calloc((size_t)n_sites, sizeof(int));
    for (int e = 0; e < n_ev; ++e)
        if (kind[e] == 1) {
            if (site[e] < 0 || site[e] >= n_sites) { free(o.site_ev); return -1; }
            o.site_ev[site[e]] = e;
        }
    for (int64_t a = 0; a < m_sets; ++a)
        for (int j = 0; j < k; ++j) {
            const int s = sets[a * k + j];
            if (s < 0 || s >= n_sites || (j > 0 && s <= sets[a * k + j - 1])) { free(o.site_ev); return -1; }
        }
    /* backward checkpoints for every site, forward ones where a set starts */
    o.phi = (cplx**)calloc((size_t)n_sites, sizeof(cplx*));
    cplx** chi = (cplx**)calloc((size_t)n_sites, sizeof(cplx*));
    char* first = (char*)calloc((size_t)n_sites, 1);
    for (int64_t a = 0; a < m_sets; ++a) first[sets[a * k]] = 1;
    cplx** bufs = (cplx**)calloc((size_t)k, sizeof(cplx*));
    cplx* p = new_state(n);
    if (!p) { rc = -1; goto done; }
    memcpy(p, bra, (size_t)dim * sizeof(cplx));
    for (int e = n_ev - 1; e >= 0; --e) {
        if (kind[e] == 0) {
            apply(n, p, nq[e], q0[e], q1[e], o.mat + (size_t)e * 16, 1, 1);
        } else {
            const int t = site[e];
            o.phi[t] = new_state(n);
            if (!o.phi[t]) { rc = -1; goto done; }
            memcpy(o.phi[t], p, (size_t)dim * sizeof(cplx));
            apply(n, p, nq[e], q0[e], q1[e], factor(&o, t, 0), 1, 1);
        }
    }
    memcpy(p, psi, (size_t)dim * sizeof(cplx));
    for (int e = 0; e < n_ev; ++e) {
        if (kind[e] == 0) {
            apply(n, p, nq[e], q0[e], q1[e], o.mat + (size_t)e * 16, 0, 1);
        } else {
            const int t = site[e];
            if (first[t]) {
                chi[t] = new_state(n);
                if (!chi[t]) { rc = -1; goto done; }
                memcpy(chi[t], p, (size_t)dim * sizeof(cplx));
            }
            apply(n, p, nq[e], q0[e], q1[e], factor(&o, t, 0), 0, 1);
        }
    }
    for (int j = 0; j < k; ++j) {
        bufs[j] = new_state(n);
        if (!bufs[j]) { rc = -1; goto done; }
    }
    {
        int64_t pos = 0;
        for (int64_t a = 0; a < m_sets; ++a) {
            const int* c = sets + a * k;
            memcpy(bufs[0], chi[c[0]], (size_t)dim * sizeof(cplx));
            set_expand(&o, bufs[0], o.site_ev[c[0]], c, k, 0, bufs, (cplx*)amps, &pos, 1);
        }
    }
done:
    free(p);
    for (int t = 0; t < n_sites; ++t) {
        if (o.phi) free(o.phi[t]);
        free(chi[t]);
    }
    free(o.phi);
    free(chi);
    free(first);
    for (int j = 0; j < k; ++j) free(bufs[j]);
    free(bufs);
    free(o.site_ev);
    return rc;
}

/* ------------------------------------------------------------------ timing a bounded part of a call */

/* A pass budget: at most `max` state passes (one application of an operation,
 * a reduction or a state copy, each a sweep over 2^n amplitudes); `dry` only
 * counts them, touching no state. */
typedef struct {
    int64_t max, done;
    int dry, stop;
    int64_t untimed;       /* passes run before the clock starts */
    int started;
    double t0, excluded, excl0;
} Budget;

static double now_s(void);

static int take(Budget* b) {
    if (b->stop) return 0;
    if (b->done >= b->max) {
        b->stop = 1;
        return 0;
    }
    if (!b->started && b->done >= b->untimed) {
        b->started = 1;
        b->t0 = now_s();
        b->excl0 = b->excluded;
    }
    b->done++;
    return !b->dry;
}

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* A state for the timed call, its pages touched at once (zeroed) and the time
 * that takes added to *excluded: the first touch of fresh memory is paid once
 * per state of a complete call, which a short sample would overweight. */
static cplx* new_state_touched(int n, double* excluded_) {
    const double t0 = now_s();
    cplx* p = new_state(n);
    if (p) memset(p, 0, ((size_t)1 << n) * sizeof(cplx));
    *excluded_ += now_s() - t0;
    return p;
}

/* expand() of the wide-state call, pass by pass under a budget */
static void expand_budget(const O3* o, cplx* w, int e0, int depth, Bufs* B, Budget* bu) {
    const int64_t dim = (int64_t)1 << o->n;
    for (int e = e0; e <= o->last_site_ev; ++e) {
        if (bu->stop) return;
        const int nq = o->nq[e], q0 = o->q0[e], q1 = o->q1[e];
        if (o->kind[e] == 0) {
            if (take(bu)) apply(o->n, w, nq, q0, q1, o->mat + (size_t)e * 16, 0, 1);
            continue;
        }
        const int t = o->site[e];
        const int last0 = depth == 0 && e == o->last_site_ev;
        if (depth < o->level || last0) {
            cplx R[16];
            if (take(bu)) reduced(o->n, o->phi[t], w, nq, q0, q1, R, 1);
            if (depth < o->level)
                for (int j = 1; j < o->m[t] && depth + 1 < o->level; ++j) {
                    cplx* w2 = B->work[depth + 1];
                    if (take(bu)) memcpy(w2, w, (size_t)dim * sizeof(cplx));
                    if (take(bu)) apply(o->n, w2, nq, q0, q1, factor(o, t, j), 0, 1);
                    expand_budget(o, w2, e + 1, depth + 1, B, bu);
                    if (bu->stop) return;
                }
        }
        if (take(bu)) apply(o->n, w, nq, q0, q1, factor(o, t, 0), 0, 1);
    }
}

/*
 * The wide-state (n > 16) path of nqso3_amplitudes -- psi = |psi_bits>, the
 * bra given, or |v_bits> (v_bits >= 0), or v = U|psi> computed first
 * (v_bits < 0), backward checkpoints, then
 * the depth-first forward sweep -- executed pass by pass until `max_passes`
 * passes are done (amplitudes are not kept), or, with dry = 1, only counted.
 * Returns the passes executed (or counted) and, in *seconds, the time of the
 * passes after the first `untimed` ones (the single-threaded set-up of the
 * input states), allocation and first touch of each state excluded; the
 * caller scales by the pass count of the complete call.  Returns -1 when a
 * state cannot be allocated.
 */
int64_t nqso3_timed_passes(int n, int n_ev, const int* kind, const int* nq, const int* q0, const int* q1,
                           const int* site, const double* mat, int n_sites, const int* m, const double* fac,
                           int64_t psi_bits, int64_t v_bits, const double* bra, int level, int64_t max_passes,
                           int64_t untimed, int dry, double* seconds, int threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    if (n < 1 || n > 40 || level < 0 || n_sites < 1) return -1;
    if (level > n_sites) level = n_sites;
    O3 o;
    memset(&o, 0, sizeof o);
    o.n = n; o.n_ev = n_ev; o.kind = kind; o.nq = nq; o.q0 = q0; o.q1 = q1; o.site = site;
    o.mat = (const cplx*)mat; o.n_sites = n_sites; o.m = m; o.fac = (const cplx*)fac; o.level = level;
    const int64_t dim = (int64_t)1 << n;
    for (int e = 0; e < n_ev; ++e)
        if (kind[e] == 1) o.last_site_ev = e;
    Budget bu;
    memset(&bu, 0, sizeof bu);
    bu.max = max_passes;
    bu.dry = dry;
    bu.untimed = untimed;
    int64_t rc = 0;
    cplx* psi = dry ? NULL : new_state_touched(n, &bu.excluded);
    cplx* v = dry ? NULL : new_state_touched(n, &bu.excluded);
    cplx* p = dry ? NULL : new_state_touched(n, &bu.excluded);
    Bufs B;
    B.work = (cplx**)calloc((size_t)level + 1, sizeof(cplx*));
    o.phi = (cplx**)calloc((size_t)n_sites, sizeof(cplx*));
    if (!dry && (!psi || !v || !p)) { rc = -1; goto done; }
    if (take(&bu)) {   /* |psi_bits> */
        memset(psi, 0, (size_t)dim * sizeof(cplx));
        psi[psi_bits].re = 1.0;
    }
    if (bra) {
        if (take(&bu)) memcpy(v, bra, (size_t)dim * sizeof(cplx));
    } else if (v_bits >= 0) {
        if (take(&bu)) {
            memset(v, 0, (size_t)dim * sizeof(cplx));
            v[v_bits].re = 1.0;
        }
    } else {           /* v = U |psi> */
        if (take(&bu)) memcpy(v, psi, (size_t)dim * sizeof(cplx));
        for (int e = 0; e < n_ev && !bu.stop; ++e)
            if (kind[e] == 0 && take(&bu)) apply(n, v, nq[e], q0[e], q1[e], o.mat + (size_t)e * 16, 0, 1);
    }
    if (take(&bu)) memcpy(p, v, (size_t)dim * sizeof(cplx));
    for (int e = n_ev - 1; e >= 0 && !bu.stop; --e) {
        if (kind[e] == 0) {
            if (take(&bu)) apply(n, p, nq[e], q0[e], q1[e], o.mat + (size_t)e * 16, 1, 1);
        } else {
            const int t = site[e];
            if (!dry && !bu.stop) {
                o.phi[t] = new_state_touched(n, &bu.excluded);
                if (!o.phi[t]) { rc = -1; goto done; }
            }
            if (take(&bu)) memcpy(o.phi[t], p, (size_t)dim * sizeof(cplx));
            if (take(&bu)) apply(n, p, nq[e], q0[e], q1[e], factor(&o, t, 0), 1, 1);
        }
    }
    if (!dry && !bu.stop)
        for (int dd = 0; dd <= level; ++dd) {
            B.work[dd] = new_state_touched(n, &bu.excluded);
            if (!B.work[dd]) { rc = -1; goto done; }
        }
    if (take(&bu)) memcpy(B.work[0], psi, (size_t)dim * sizeof(cplx));
    expand_budget(&o, B.work[0], 0, 0, &B, &bu);
    rc = bu.done;
    if (seconds) *seconds = bu.started ? now_s() - bu.t0 - (bu.excluded - bu.excl0) : 0.0;
done:
    free(psi);
    free(v);
    free(p);
    for (int dd = 0; dd <= level; ++dd) free(B.work[dd]);
    free(B.work);
    for (int t = 0; t < n_sites; ++t) free(o.phi[t]);
    free(o.phi);
    return rc;
}
