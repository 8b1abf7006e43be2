/*
 * nqs.h -- C ABI of libnqs: level-l SVD noise expansion of a noisy circuit's
 * fidelity, evaluated by complex64 state-vector sweeps on an sm_103a GPU.
 *
 * The quantity (Problem 1, Sec. III): for a noisy circuit E = E_d o ... o E_1
 * with N single-qubit noise channels, an input |psi> and a test state |v>,
 *     F = <v| E(|psi><psi|) |v>.
 * The approximation (Sec. IV, Fig. 3, Algorithm 1): each noise's matrix
 * representation M = sum_k E_k (x) E_k^* is tensor-permuted, factored by SVD
 * into M = sum_{i=0..3} U_i (x) V_i with d_0 the dominant singular value, and
 * A(l) = sum_{u<=l} T_u keeps the assignments with at most l non-dominant
 * factors.  For a CPTP channel the permuted matrix is Hermitian positive
 * semidefinite, so U_i = sqrt(d_i) K_i (x) conj(sqrt(d_i) K_i) with one 2x2
 * K_i per factor and every term is |<v| C[K_sigma] |psi>|^2 >= 0.
 *
 * Conventions
 *   - Qubit q is bit q of a basis index; a state is 2^n complex64 values
 *     (interleaved float re, im), index = sum_q x_q 2^q.
 *   - Two-qubit gate matrices are indexed 2*b(first qubit) + b(second qubit).
 *   - Every function returns NQS_OK (0) or an NQS_ERR_* code and leaves its
 *     outputs untouched on error, unless stated otherwise.  nqs_strerror gives
 *     a message.  Device faults detected after a launch are reported as
 *     NQS_ERR_CUDA.
 *   - A handle is not thread-safe; distinct handles may be used from
 *     different threads.  Streams are cudaStream_t passed as void* (NULL =
 *     the legacy default stream).
 *   - Device memory is obtained through the allocator installed with
 *     nqs_set_allocator (default: cudaMalloc / cudaFree) and owned by the
 *     handle until nqs_destroy.
 */
#ifndef NQS_H
#define NQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
enum {
    NQS_OK = 0,
    NQS_ERR_ARG = 1,            /* invalid argument, size or qubit index */
    NQS_ERR_PARSE = 2,          /* malformed circuit text */
    NQS_ERR_NOT_CPTP = 3,       /* ||sum_k E_k^dag E_k - I||_max > 1e-10 */
    NQS_ERR_NOT_DOMINANT = 4,   /* d_0 - d_1 <= 1e-12 d_0: no unique dominant factor */
    NQS_ERR_NOMEM = 5,          /* allocator returned NULL */
    NQS_ERR_CUDA = 6,           /* a CUDA runtime call or kernel launch failed */
    NQS_ERR_ORDER = 7,          /* call sequence violated (e.g. fidelity before prepare) */
    NQS_ERR_DEVICE_TIMEOUT = 8, /* a bounded device-side wait gave up (reported in result.status) */
    NQS_ERR_UNSUPPORTED = 9,    /* request outside the supported range (documented per call) */
    NQS_ERR_TOO_LARGE = 10,     /* request exceeds a fixed capacity (nqs_reduced_matrix_noalloc) */
    NQS_ERR_COMPILE = 11        /* a generated kernel did not compile (nqs_jit_compile_check) */
};

typedef struct nqs_circuit* nqs_handle;

/* ---- states ------------------------------------------------------------- */
enum {
    NQS_STATE_BASIS = 0,   /* |bits> */
    NQS_STATE_DENSE = 1,   /* caller-owned device buffer of 2^n complex64, read-only,
                              valid until the stream reaches the end of the call */
    NQS_STATE_IDEAL = 2    /* only for v: U|psi>, the noiseless circuit applied to psi */
};

typedef struct {
    int32_t kind;
    uint64_t bits;         /* NQS_STATE_BASIS */
    const void* dev;       /* NQS_STATE_DENSE: device pointer, 16-byte aligned */
} nqs_state;

/* ---- noise sites -------------------------------------------------------- */
typedef struct {
    int32_t after_gate;    /* acts right after this gate index; -1 = before gate 0 */
    uint32_t qubit;
    uint32_t n_kraus;      /* 1..16 */
    const double* kraus;   /* n_kraus x 2x2 complex128, row-major, interleaved re/im:
                              kraus[8*k + 2*(2*a+b) + {0,1}] = (re, im) of E_k[a][b] */
} nqs_noise;

enum {
    NQS_PREP_PRUNE_ZERO_RANK = 1   /* drop factors with d_i < 1e-10 d_0 from the expansion */
};

/* ---- results ------------------------------------------------------------ */
#define NQS_MAX_LEVEL 16

typedef struct {
    double F;                      /* A(l) = sum_{u<=l} T_u (Algorithm 1's Result) */
    double T[NQS_MAX_LEVEL + 1];   /* T_u, u = 0..level; zero above */
    double imag_residual;          /* |Im sum X|: 0 for the single-amplitude form */
    uint64_t n_terms;              /* sum_{u<=l} C(N,u) * (#non-dominant factors)^u */
    double bound;                  /* per-site truncation bound (see nqs_truncation_bound) */
    int32_t level;                 /* level after clamping to N */
    int32_t status;                /* NQS_OK or an asynchronous device error */
} nqs_result;

/* ---- allocator ---------------------------------------------------------- */
typedef void* (*nqs_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*nqs_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

/* Install the device-memory allocator used by every later allocation of
 * every handle (process-wide).  Passing NULL for both restores
 * cudaMalloc/cudaFree.  Memory already held keeps the functions it came from. */
int nqs_set_allocator(nqs_alloc_fn alloc, nqs_free_fn release, void* ctx);

/* ---- circuit and noise -------------------------------------------------- */

/* Parse the circuit text (gates h x y z t rx ry rz u3 cz cx and optional
 * noise records; format in the package documentation) into a new handle.
 * Sec. II: the circuit is the gate sequence U = U_d ... U_1.
 * Errors: NQS_ERR_ARG (NULL pointers), NQS_ERR_PARSE, NQS_ERR_UNSUPPORTED
 * (n_qubits outside 1..34). */
int nqs_load_circuit(const char* ir_text, nqs_handle* out);

/* Factor every noise channel (Sec. IV, Fig. 3): check CPTP, build the
 * permuted matrix M~ = sum_k vec(E_k) vec(E_k)^dag, diagonalise it in FP64
 * (Hermitian Jacobi), sort the singular values d_0 >= ... >= d_3, require a
 * unique dominant value, and keep K_i = sqrt(d_i) reshape(eigenvector_i).
 * sites == NULL and n_sites == 0 use the noise records of the circuit text;
 * otherwise `sites` replaces them (ordered by after_gate, stable).  Copies
 * all inputs.  Errors: NQS_ERR_ARG, NQS_ERR_NOT_CPTP, NQS_ERR_NOT_DOMINANT. */
int nqs_prepare_noise(nqs_handle h, const nqs_noise* sites, size_t n_sites, uint32_t flags);

/* A(l) for <v| E(|psi><psi|) |v> (Algorithm 1), levels above N clamped to N.
 * Runs entirely on the GPU in `stream`: a backward sweep from v storing the
 * states phi_s = (everything after site s)^dag |v>, a forward sweep from psi
 * reducing <phi_s| K_i |chi_s> at every site, and for l >= 2 depth-first
 * re-sweeps from each first insertion.  `out` may be device, pinned host or
 * pageable host memory; it is written with one stream-ordered copy (for
 * pageable memory the call returns after the copy completed).
 * Errors: NQS_ERR_ARG (bad state kind, level < 0, level > NQS_MAX_LEVEL after
 * clamping), NQS_ERR_ORDER (not prepared), NQS_ERR_NOMEM, NQS_ERR_CUDA. */
int nqs_fidelity(nqs_handle h, const nqs_state* psi, const nqs_state* v, int level,
                 nqs_result* out, void* stream);

/* Evaluate `count` distinct handles; entry k uses psis[k], vs[k], levels[k]
 * and writes outs[k] (same results as nqs_fidelity per entry).  The batch runs
 * in rounds: round r executes the r-th launch of every circuit's schedule,
 * one multi-circuit launch per launch kind, so narrow circuits share the GPU.
 * Circuits are packed into waves whose buffers fit in free device memory;
 * a batch that fits in one wave is captured as a CUDA graph and replayed by
 * later calls with the same handles, states and levels (the handles keep
 * their workspaces).  Errors as nqs_fidelity, checked for every entry before
 * anything runs; NQS_ERR_ARG also for a handle listed twice. */
int nqs_batch_fidelity(const nqs_handle* hs, size_t count, const nqs_state* psis,
                       const nqs_state* vs, const int* levels, nqs_result* outs, void* stream);

/* ---- inspection hooks (tests) ------------------------------------------- */

/* Kept assignments of Algorithm 1 in canonical order (level u ascending, site
 * tuple lexicographic, factor tuple lexicographic over {1,2,3}), packed:
 * bits 0-3 = u; for r < u the 14-bit field at bit 4+14r holds the site
 * (low 12 bits) and the factor index (high 2 bits).  Needs level <= 4 and
 * N <= 4096 (else NQS_ERR_UNSUPPORTED).  *count receives the total; at most
 * `cap` records are written. */
int nqs_enumerate_terms(nqs_handle h, int level, uint64_t* rec, size_t cap, size_t* count);

/* Factors of noise site `site` after nqs_prepare_noise: d4[i] = d_i and
 * K[8*i + 2*(2a+b) + {0,1}] = K_i[a][b] (complex128), K_i = sqrt(d_i) A_i. */
int nqs_noise_factors(nqs_handle h, uint32_t site, double* d4, double* K);

/* Factors of site `site` of a circuit with general noises (two-qubit
 * channels, records noise2; noises given by their matrix representation,
 * records superop / superop2): the SVD M~ = S D T^dagger of the
 * tensor-permuted matrix (Sec. IV, Fig. 3 in its general form).  *m receives
 * the factor count d^2 (4 or 16 for one or two qubits), *dim the factor size
 * d; when the arrays are not NULL: sv[m] the singular values (descending),
 * KA and KB m x d x d complex128 (row-major, interleaved re/im) with
 * KA_i = sqrt(d_i) reshape(S|i>), KB_i = sqrt(d_i) reshape(T|i>); a term is
 * <v|C[KA_sigma]|psi> conj(<v|C[KB_sigma]|psi>), and KA = KB for channels.
 * *same = 1 when KA = KB at this site.  Test hook.
 * Errors: NQS_ERR_ARG (site out of range), NQS_ERR_ORDER (not prepared),
 * NQS_ERR_UNSUPPORTED (the circuit has only one-qubit channels: see
 * nqs_noise_factors). */
int nqs_general_factors(nqs_handle h, uint32_t site, int32_t* m, int32_t* dim, int32_t* same, double* sv, double* KA,
                        double* KB);

/* Term values X of the last nqs_fidelity on this handle, in canonical order,
 * copied to host memory `out` (synchronises the stream of that call). */
int nqs_term_values(nqs_handle h, double* out, size_t cap, size_t* count);

/* Truncation bound of level l: sum over site sets S with |S| > l of
 * prod_{s in S} ||M-bar_s|| prod_{s not in S} ||M'_s|| (spectral norms of the
 * dropped and dominant parts, Theorem 1's argument per site). */
int nqs_truncation_bound(nqs_handle h, int level, double* out);

/* Check of the sweep plan (host only, test hook): the largest entry
 * difference between the operator of the plan's operation order (fused
 * gates, the Hadamard-diagonal rewrite, the reordering before segmentation,
 * K_0 at the noise sites) and the operator of the circuit itself with K_0
 * after each noise's gate, both applied to every basis state in FP64 (for
 * n <= 10; 0 above).  +infinity when the plan's structure is broken: noise
 * sites out of their order, or a pass (of the free or the site-cut
 * segmentation) that does not continue where the previous one ended, whose
 * tile is not k distinct ascending qubits holding the low qubits and every
 * dense or site qubit of its operations, or that exceeds the operation or
 * site bounds of a pass.  No counterpart in the paper (the plan is this
 * library's).  Errors: NQS_ERR_ARG, NQS_ERR_ORDER (not prepared),
 * NQS_ERR_UNSUPPORTED (general noises). */
int nqs_plan_check(nqs_handle h, double* max_abs_err);

/* Compile check of the pass-specialised kernels (host only, test hook; no
 * counterpart in the paper): the kernels of the first `max_passes` passes of
 * a forward sweep of the handle's plan over `states` states (1 or 3; with
 * reductions and spawns at every site) and, for one state, of a backward
 * sweep (adjoint operations, checkpoint saves) are generated with the
 * library's current settings and compiled with NVRTC for sm_103a; nothing is
 * loaded or run.  *compiled receives the number of kernels compiled.
 * Errors: NQS_ERR_ARG, NQS_ERR_ORDER (not prepared), NQS_ERR_UNSUPPORTED
 * (NVRTC not found, general noises, or fewer than 13 qubits: no generated
 * kernels), NQS_ERR_COMPILE (a kernel failed; the message goes to stderr). */
int nqs_jit_compile_check(nqs_handle h, int states, int max_passes, int* compiled);

/* The kept terms (canonical order, level `level`) that shard `rank` of
 * `count` evaluates under NQS_OPT_SHARD_RANK / NQS_OPT_SHARD_COUNT: mask[i]
 * = 1 for its terms; *n receives the term count (call with mask = NULL or
 * cap too small for the count only).  Host only.  No counterpart in the
 * paper (Algorithm 1's outer loops over site sets are independent).
 * Errors: NQS_ERR_ARG, NQS_ERR_ORDER, NQS_ERR_UNSUPPORTED (general noises). */
int nqs_shard_mask(nqs_handle h, int level, int rank, int count, uint8_t* mask, size_t cap, size_t* n);

/* Adaptive level selection (Theorem 1 and the level study of Sec. V: the
 * truncation error falls with the level, and a low level usually suffices).
 * The level is raised until the dropped part is below `tol`, judged by
 *   NQS_ADAPT_BOUND     the truncation bound (nqs_truncation_bound): the
 *                       smallest level l with bound(l) <= tol is evaluated
 *                       directly -- the bound needs only the factors' norms;
 *   NQS_ADAPT_OBSERVED  the last level's sum: levels 1, 2, ... are evaluated
 *                       in turn until |T_l| <= tol (the next terms are
 *                       smaller still for weak noise, as the paper observes);
 *   both flags          whichever stops first.
 * Levels never exceed max_level (nor N).  `out` (host memory) receives the
 * result of the last evaluated level, out->level that level.  The call
 * synchronises `stream` after each evaluated level (it reads T_l).
 * Errors: as nqs_fidelity; NQS_ERR_ARG for tol < 0, max_level < 0 or no
 * criterion flag. */
enum { NQS_ADAPT_BOUND = 1, NQS_ADAPT_OBSERVED = 2 };

/* One element <x| E(|psi><psi|) |y> of the output density matrix at level l
 * (Sec. III: every element can be estimated on its own, by the identity
 *   <x|rho|y> = 1/4 [ f(x+y) - f(x-y) - i f(x+iy) + i f(x-iy) ],
 * f(v) = <v|rho|v>).  The level-l approximation is <v|rho_l|v> for one
 * Hermitian rho_l, so the identity holds level by level: four level-l calls
 * with v = x + i^k y (dense, built on the device) and their combination.
 *   x, y: NQS_STATE_BASIS or NQS_STATE_DENSE (not IDEAL).
 *   out: host, 2 doubles (re, im).  parts: NULL or host array of 4 results,
 *        the calls for k = 0..3.
 * One temporary state (8 * 2^n bytes) comes from the allocator; the call
 * synchronises `stream`.  Errors: as nqs_fidelity. */
int nqs_offdiagonal(nqs_handle h, const nqs_state* psi, const nqs_state* x, const nqs_state* y, int level,
                    double* out, nqs_result* parts, void* stream);
int nqs_fidelity_adaptive(nqs_handle h, const nqs_state* psi, const nqs_state* v, double tol, int max_level,
                          uint32_t criteria, nqs_result* out, void* stream);

typedef struct {
    int32_t n_qubits;
    int32_t n_gates;
    int32_t n_sites;
    int32_t n_ops;              /* fused operations of the sweep plan */
    int32_t n_passes;           /* tile passes of one full sweep */
    int32_t tile_qubits;        /* qubits held in shared memory per tile */
    uint64_t workspace_bytes;   /* device bytes held by the handle */
    uint64_t upload_bytes;      /* host-to-device bytes of the last schedule build */
    uint64_t launches_per_call; /* kernels launched by one nqs_fidelity call */
    int32_t ckpt_spacing;       /* sites per checkpoint block of the current schedule (0: every site) */
    int32_t n_states;           /* 2^n-amplitude state buffers held by the current schedule */
    int32_t jit_launches;       /* sweep launches of the current schedule that run pass-specialised kernels */
    int32_t jit_state;          /* 0 not requested, 1 built, -1 requested but NVRTC or a compile failed */
} nqs_info;

int nqs_get_info(nqs_handle h, nqs_info* out);

/* Launch list of the handle's current schedule (the one the last
 * nqs_fidelity call built), for profiling: one record per launch, in launch
 * order.  kind: 0 sweep pass, 1 finisher, 2 state fill, 3 state copy,
 * 4 two-state reduction, 5 level sums, 6 normalisation of the computed
 * v = U|psi> (basis psi).  For sweep passes: states swept
 * together, register qubits per thread (0: shared-memory tile kernel), phases
 * of the register-resident program, grid size, operation counts
 * ops[] = {dense 1-qubit, dense 2-qubit, diagonal 1-qubit, diagonal 2-qubit,
 * noise sites, site reductions, spawned states, checkpoint saves}, whether
 * the pass runs a pass-specialised kernel (NQS_OPT_JIT) and the
 * algorithmic bytes of the launch (see nqs_kernel_stats).  Call with out =
 * NULL (or cap too small) to get the count only.  No counterpart in the paper. */
typedef struct {
    int32_t kind;
    int32_t states;
    int32_t reg_qubits;
    int32_t phases;
    int32_t grid;
    int32_t ops[8];
    int32_t jit;                /* 1: the pass runs a pass-specialised kernel */
    double algorithmic_bytes;
} nqs_launch_info;

int nqs_schedule_launches(nqs_handle h, nqs_launch_info* out, size_t cap, size_t* count);

/* ---- execution options ----------------------------------------------------
 * Choices of this library with no counterpart in the paper; value 0 restores
 * the automatic choice.  A change takes effect at the next call (the schedule
 * is rebuilt).
 *   NQS_OPT_CKPT_SPACING  sites per checkpoint block.  Automatic: phi_s is kept
 *       at every noise site when those states fit in device memory; otherwise
 *       (levels <= 2) it is kept at the last site of each block of k sites and
 *       a block's phi are recomputed from there whenever a sweep enters the
 *       block, with k chosen to hold the fewest states.  1 <= k < N forces
 *       blocks of k sites (levels <= 2, else NQS_ERR_UNSUPPORTED at the call);
 *       k >= N keeps every site.
 *   NQS_OPT_SWEEP_RB      register qubits per thread of multi-state sweep
 *       passes: 3 (512-thread blocks) or 4 (256-thread blocks).
 *   NQS_OPT_MAX_OPS       fused operations per pass, 8..160 (default 96).
 *   NQS_OPT_MAX_SITES     noise sites per pass, 1..8 (default 4).
 *   NQS_OPT_SHARD_RANK, NQS_OPT_SHARD_COUNT   split one call's terms over
 *       `count` shards (one per GPU): shard `rank` evaluates the level-0/1
 *       terms when rank = 0 and every term whose first non-dominant site s
 *       has s mod count = rank; the other terms of its result are zero, so
 *       the shards' T_u add up to the whole call's (nqs_shard_mask lists a
 *       shard's terms).  Each shard runs its own backward and forward sweeps.
 *       0 / 0 (or 1): no split.  A rank >= count is NQS_ERR_ARG at the call.
 *   NQS_OPT_JIT           sweep passes of 12-qubit tiles run kernels generated
 *       for each pass (operations, layouts and matrices compiled in as
 *       constants; NVRTC at schedule build time, cached for the process):
 *       0 automatic (circuits of 26 qubits or more), 1 always, 2 never (the
 *       interpreting kernel).  When NVRTC cannot be loaded the interpreting
 *       kernel runs; nqs_info.jit_launches tells which ran.
 * NQS_ERR_ARG for an unknown option or a value out of range; NQS_ERR_ORDER
 * for the two segmentation options before nqs_prepare_noise. */
#define NQS_OPT_CKPT_SPACING 1
#define NQS_OPT_SWEEP_RB 2
#define NQS_OPT_MAX_OPS 3
#define NQS_OPT_MAX_SITES 4
#define NQS_OPT_JIT 5
#define NQS_OPT_SHARD_RANK 6
#define NQS_OPT_SHARD_COUNT 7

int nqs_set_option(nqs_handle h, int option, int64_t value);
int nqs_get_option(nqs_handle h, int option, int64_t* value);

/* Time candidate execution options on this handle and keep the fastest:
 * register qubits of multi-state passes (3, 4) and operations per pass
 * (64, 96, 128), each candidate timed by CUDA events over `trials` calls of
 * nqs_fidelity(h, psi, v, level) on `stream` after one warm-up call.  The
 * chosen values are readable with nqs_get_option; `out` (may be NULL)
 * receives the result of the last timed call.  Checkpoint spacing is chosen
 * by memory, not time (NQS_OPT_CKPT_SPACING). */
int nqs_autotune(nqs_handle h, const nqs_state* psi, const nqs_state* v, int level, int trials,
                 nqs_result* out, void* stream);

/* Per-kernel timing of the calls made since profiling was switched on:
 * CUDA events recorded around every sweep-pass launch on the call's stream.
 * kind 0 = all gate-sweep passes, 1 = finishers/reductions, 2 = state fills,
 * 3 = sweep passes over several states (branch groups), 4 = single-state
 * sweep passes (kinds 3 and 4 split kind 0). */
typedef struct {
    uint64_t launches;
    double total_ms;
    double algorithmic_bytes;   /* sum over launches of 16 B x 2^n x states per pass
                                   plus 8 B x 2^n per checkpoint read or write */
} nqs_kernel_stats;

int nqs_set_profiling(nqs_handle h, int on);
int nqs_get_kernel_stats(nqs_handle h, int kind, nqs_kernel_stats* out);

/* ---- standalone kernels -------------------------------------------------- */

/* Reduced 2x2 matrix of two states on one qubit:
 *   R[a][b] = sum over all other bits of conj(phi[.., a, ..]) * chi[.., b, ..],
 * so <phi| K |chi> = sum_ab K[a][b] R[a][b] (the level-1 term of Algorithm 1
 * read off checkpoints).  phi, chi: device, 2^n complex64, 16-byte aligned.
 * R_out: 8 doubles (re, im of R00, R01, R10, R11), device or host memory,
 * written stream-ordered.  scratch: device memory of at least
 * nqs_reduced_matrix_scratch_bytes(n) bytes (per-block partial sums).
 * Errors: NQS_ERR_ARG (n outside 1..34, qubit >= n, NULL, small scratch). */
int nqs_reduced_matrix(const void* phi, const void* chi, int n, int qubit, double* R_out,
                       void* scratch, size_t scratch_bytes, void* stream);
size_t nqs_reduced_matrix_scratch_bytes(int n);

/* Allocation-free variant of nqs_reduced_matrix (the paper has no
 * counterpart: this serves callers that cannot allocate device memory --
 * hosts whose device heap is owned by another runtime's pool, latency-bound
 * loops that cannot afford cudaMalloc's implicit device synchronisation,
 * plugin environments that forbid dynamic device allocation).
 *
 * Same result as nqs_reduced_matrix: R_out (8 doubles: re, im of R00, R01,
 * R10, R11) receives the reduced 2x2 matrix of phi and chi on `qubit`.  The
 * per-block partial sums live in one fixed device array of
 * NQS_NOALLOC_MAX_BLOCKS * 8 doubles (64 KiB) compiled into the library;
 * every GPU that loads the library holds it until the process exits.  The
 * call allocates nothing: no cudaMalloc, no cudaFree, no allocator callback.
 *   - phi, chi: memory of the current device (or managed), 2^n complex64
 *     each, 16-byte aligned; n in 1..NQS_NOALLOC_MAX_QUBITS.  Host memory
 *     and another device's memory are rejected with NQS_ERR_ARG.
 *   - R_out: the current device's memory, managed or pinned host memory,
 *     8-byte aligned; written by a kernel in `stream`.  Pageable host
 *     memory is rejected with NQS_ERR_ARG.
 *   - stream: NULL or a stream of the current device (NQS_ERR_ARG otherwise).
 *   - The first call on each device resolves the array's device address
 *     (cudaGetSymbolAddress) with that device current and caches it.
 *   - Every call on a device shares the one array and overwrites the
 *     slots it reads, so sequential calls need no clearing; calls whose
 *     kernels overlap on the GPU (different streams, no ordering between
 *     them) race on the array and must be serialised by the caller.
 * Errors: NQS_ERR_ARG (NULL, misaligned, qubit >= n, a pointer or stream
 * the current device cannot use), NQS_ERR_TOO_LARGE (n > NQS_NOALLOC_MAX_QUBITS),
 * NQS_ERR_CUDA. */
#define NQS_NOALLOC_MAX_BLOCKS 1024
#define NQS_NOALLOC_MAX_QUBITS 34
int nqs_reduced_matrix_noalloc(const void* phi, const void* chi, int n, int qubit, double* R_out, void* stream);

/* ---- chosen site sets ------------------------------------------------------
 * W(S) for a set of noise sites S = {s_1 < ... < s_k}, k <= 3: the sum of the
 * term values X over every choice of kept non-dominant factor at the sites of
 * S (dominant factor elsewhere) -- the summand of T_k grouped by site set
 * (Sec. IV, Algorithm 1's inner loop over factor tuples).
 * nqs_prepare_sets runs the backward sweep from v and a forward sweep from
 * psi, keeping phi_s and chi_s for every site (2N + 14 device states); it must
 * precede nqs_eval_sets and be repeated after nqs_prepare_noise.
 * nqs_eval_sets: `sets` is m x k site indices (ascending within a set),
 * W_out receives m doubles on the host (the call synchronises `stream`).
 * Errors: NQS_ERR_ARG (bad k, unordered or out-of-range sites),
 * NQS_ERR_ORDER (not prepared), NQS_ERR_NOMEM, NQS_ERR_CUDA. */
int nqs_prepare_sets(nqs_handle h, const nqs_state* psi, const nqs_state* v, void* stream);
int nqs_eval_sets(nqs_handle h, int k, const int32_t* sets, size_t m, double* W_out, void* stream);

/* ---- proposal network (learned importance sampling) --------------------
 * A multilayer perceptron: n_in inputs, `hidden_layers` ReLU layers of
 * `hidden` units, one linear output.  Weights are stored in fp32 (masters)
 * and used in bf16 by the forward and backward kernels, with fp32
 * accumulation; training is Adam on the mean squared error.  The paper has
 * no counterpart: the network proposes which higher-level site sets an
 * importance-sampled estimate of a level's sum evaluates.
 * Parameters flatten as, per layer, W (out x in, row-major) then b (out).
 * X is row-major [batch x n_in] fp32, y is [batch] fp32, device memory. */
typedef struct nqs_mlp_s* nqs_mlp;
int nqs_mlp_create(int n_in, int hidden, int hidden_layers, uint64_t seed, nqs_mlp* out);
size_t nqs_mlp_param_count(nqs_mlp m);
int nqs_mlp_get_params(nqs_mlp m, float* host, size_t cap);          /* fp32 masters */
int nqs_mlp_set_params(nqs_mlp m, const float* host, size_t count);
int nqs_mlp_forward(nqs_mlp m, const float* X, int batch, float* y, void* stream);
/* loss and gradient (w.r.t. the fp32 masters) of one batch, copied to host */
int nqs_mlp_loss_grad(nqs_mlp m, const float* X, const float* y, int batch, double* loss, float* grad_host,
                      size_t cap, void* stream);
/* `steps` Adam steps on batches drawn (counter-based generator, `seed`)
 * from the n rows of (X, y); *final_loss = loss of the last batch */
int nqs_mlp_train(nqs_mlp m, const float* X, const float* y, int n, int batch, int steps, float lr, uint64_t seed,
                  double* final_loss, void* stream);
void nqs_mlp_destroy(nqs_mlp m);

/* ---- importance-sampled level sums ------------------------------------------
 * Site features for the proposal network (host, N x 4 floats, each column
 * standardised over the sites): the noise's position in the gate sequence,
 * its qubit, log10 of its noise rate ||M - I||, log10 of its level-1 weight
 * W1[s] = sum of its level-1 term values. */
int nqs_site_features(nqs_handle h, const double* W1, float* out);
/* Training rows for pair scores: for every pair s < t (lexicographic), X row =
 * features of s then of t (8 floats), y = ln W2[s*N + t] (W2: host N x N,
 * the level-2 weight of the pair).  *count = N(N-1)/2; nothing is written
 * when cap < count. */
int nqs_pair_training_data(nqs_handle h, const float* feats, const double* W2, float* X, float* y, size_t cap,
                           size_t* count);

typedef struct {
    double estimate;      /* unbiased estimate of T_level */
    double stderr_;       /* its standard error (sample variance / samples) */
    double ess;           /* effective sample size of the proposal weights */
    uint64_t samples;
    uint64_t distinct;    /* distinct site sets evaluated */
    uint64_t n_sets;      /* C(N, level) */
    double alpha;         /* weight of the uniform part of the proposal */
    int32_t level;
    int32_t status;
} nqs_is_result;

/* Importance-sampled estimate of T_level (level 2 or 3) of the expansion
 * (Sec. IV's T_u summed by site sets).  The proposal scores a site set by
 * the network's pair scores (a triple by its three pairs minus the level-1
 * log weights of its sites), takes the softmax over all C(N, level) sets and
 * mixes it with the uniform law: q = (1 - alpha) softmax + alpha / C(N, level).
 * mlp == NULL gives the uniform proposal.  Sets are drawn by inverse-CDF
 * lookup of SplitMix64 uniforms (seed + draw index), each distinct set is
 * evaluated once on the GPU (nqs_eval_sets, which needs nqs_prepare_sets),
 * and estimate = mean of W(S_j) / q(S_j).  feats: host N x 4 from
 * nqs_site_features; W1: host N level-1 weights.  Synchronises `stream`. */
int nqs_is_estimate(nqs_handle h, nqs_mlp mlp, int level, uint64_t samples, double alpha, uint64_t seed,
                    const float* feats, const double* W1, nqs_is_result* out, void* stream);

/* The proposal nqs_is_estimate draws from: q[i] for every site set of the
 * level in canonical (lexicographic) order, summing to 1 (same arguments as
 * nqs_is_estimate).  With the exact per-set weights W (from a full
 * enumeration) the estimator's variance per draw is sum W^2/q - T^2, which
 * judges a proposal without sampling noise.  q_out: host, cap doubles; call
 * with q_out = NULL to get the count.  No counterpart in the paper. */
int nqs_is_proposal(nqs_handle h, nqs_mlp mlp, int level, double alpha, const float* feats, const double* W1,
                    double* q_out, size_t cap, size_t* count, void* stream);

void nqs_destroy(nqs_handle h);
const char* nqs_strerror(int code);
/* Failure-detection self-test (no counterpart in the paper): runs the sweep
 * kernels' bounded mbarrier wait on a barrier that nothing arrives at.  The
 * wait gives up after about two seconds; *status_out receives the status word
 * the kernel wrote (NQS_ERR_DEVICE_TIMEOUT when the bound works).  Returns
 * NQS_OK when the probe ran; the context stays usable afterwards. */
int nqs_selftest_bounded_wait(int* status_out, void* stream);

const char* nqs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NQS_H */
