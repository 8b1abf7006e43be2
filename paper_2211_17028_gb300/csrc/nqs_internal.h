// Internal types of libnqs shared by the host planner (C++) and the sweep
// engine (CUDA).  Nothing here is part of the C ABI.
#pragma once

#include <array>
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/nqs.h"

namespace nqs {

using cd = std::complex<double>;
using Mat2 = std::array<cd, 4>;    // row-major 2x2
using Mat4 = std::array<cd, 16>;   // row-major 4x4, index 2*b(q0)+b(q1)

// ---------------------------------------------------------------- circuit IR
enum GateKind : int { G_H, G_X, G_Y, G_Z, G_T, G_RX, G_RY, G_RZ, G_U3, G_CZ, G_CX };

struct Gate {
    GateKind kind;
    int q0 = -1, q1 = -1;
    double p[3] = {0, 0, 0};
};

struct NoiseSite {
    int after_gate = -1;               // -1: before gate 0
    int qubit = 0;
    std::vector<Mat2> kraus;
    // general noises (IR records noise2 / superop / superop2): a second qubit,
    // d x d Kraus operators (d = 4), or the matrix representation M itself
    int qubit2 = -1;
    std::vector<std::vector<cd>> kraus_d;   // row-major d x d
    std::vector<cd> superop;                // row-major d^2 x d^2
    bool general() const { return qubit2 >= 0 || !superop.empty(); }
    int dim() const { return qubit2 >= 0 ? 4 : 2; }
};

struct Circuit {
    int n = 0;
    std::vector<Gate> gates;
    std::vector<NoiseSite> noises;     // ordered by after_gate (stable)
};

// Parse the text format; returns NQS_OK or NQS_ERR_PARSE / NQS_ERR_UNSUPPORTED.
int parse_circuit(const char* text, Circuit& out, std::string& err);
bool gate_is_two_qubit(GateKind k);
Mat2 gate_matrix_1q(const Gate& g);
Mat4 gate_matrix_2q(const Gate& g);

// ------------------------------------------------------------ noise factors
struct Factors {
    double d[4];            // singular values of M~, descending
    Mat2 K[4];              // K_i = sqrt(d_i) A_i, A_i = reshape of the i-th singular vector
    int m = 3;              // number of non-dominant factors kept in the expansion
    int keep[3] = {1, 2, 3};// their factor indices
    double norm_dom;        // ||U_0 (x) V_0||_2 = d_0 * ... (spectral norm of M')
    double norm_rest;       // ||sum_{i>=1} U_i (x) V_i||_2
    double rate;            // noise rate ||M - I||_2 (Sec. IV)
};

// Returns NQS_OK, NQS_ERR_NOT_CPTP or NQS_ERR_NOT_DOMINANT.
int factor_noise(const NoiseSite& s, bool prune_zero_rank, Factors& out);
// Hermitian 4x4 eigen-decomposition by cyclic complex Jacobi rotations.
void hermitian_jacobi4(const Mat4& a, double evals[4], Mat4& evecs_columns);

// --------------------------------------------------------------- enumeration
struct TermIndex {
    int N = 0;
    int level = 0;
    std::vector<int> m;                          // kept factors per site
    std::vector<std::vector<uint64_t>> E;        // E[j][a] = e_j(m_a .. m_{N-1})
    std::vector<uint64_t> level_offset;          // first rank of each level
    uint64_t total = 0;
    void build(const std::vector<int>& m_per_site, int level);
    // rank of a kept term; sites ascending, factor positions 0..m_s-1
    uint64_t rank(int k, const int* sites, const int* fpos) const;
};

// --------------------------------------------------------------------- plan
enum OpType : int { OP_G1 = 1, OP_G2 = 2, OP_D1 = 3, OP_D2 = 4, OP_SITE = 5 };

struct HostOp {
    OpType type;
    int q0 = -1, q1 = -1;
    int site = -1;                 // OP_SITE
    std::array<cd, 16> m{};        // G1/D1: 4 (D1 uses m[0], m[3]); G2/D2: 16; SITE: K_0
    bool diag = false;             // SITE: K_0 is diagonal
};

struct PassSpec {
    std::vector<int> local;        // tile qubits, ascending (low `c` qubits always included)
    int op_begin = 0, op_end = 0;  // range in the linear op list
};

struct Plan {
    int n = 0, k = 0, c = 0;       // qubits, tile qubits, always-local low qubits
    std::vector<HostOp> ops;       // linear op order used by every sweep
    std::vector<int> site_pos;     // op index of each site's OP_SITE
    std::vector<PassSpec> free_passes;     // cuts only where locality forces them
    std::vector<PassSpec> sitecut_passes;  // additionally cut after every OP_SITE
    std::vector<PassSpec> grouped_passes;  // the reordering's own passes (at most 4 sites, 96 operations)
};

void build_plan(const Circuit& c, const std::vector<Factors>& f, int tile_qubits, Plan& out);
// Cut the linear op order into passes whose operations fit one tile of k
// qubits; cut after every site (cut_after_sites), after the sites flagged in
// `cut_after` (indexed by site), and after max_sites_per_pass sites or
// max_ops_per_pass operations.
std::vector<PassSpec> segment(const Plan& p, bool cut_after_sites, int max_sites_per_pass, int max_ops_per_pass,
                              const std::vector<char>* cut_after = nullptr);
// Largest entry difference between the plan's operator product and the
// circuit's (gates, K_0 at the noise sites), on every basis state (n <= 10).
double plan_product_error(const Circuit& c, const std::vector<Factors>& f, const Plan& p);

// ------------------------------------------ general noises (generic.cu)
// Factors of a one- or two-qubit noise given by Kraus operators or by its
// matrix representation: M~ = S D T^dagger (one-sided Jacobi SVD, FP64),
// KA_i = sqrt(d_i) reshape(S|i>), KB_i = sqrt(d_i) reshape(T|i>); a term is
// X = <v|C[KA_sigma]|psi> conj(<v|C[KB_sigma]|psi>).  For a channel M~ is PSD
// and KA = KB.
struct GFactors {
    int nq = 1, q0 = 0, q1 = -1;       // site qubits
    int m = 4;                         // factors (d^2), index 0 dominant
    std::vector<double> d;             // singular values, descending
    std::vector<cd> KA, KB;            // m x (dim x dim), row-major
    bool same = true;                  // KA == KB (one network per term)
    double norm_dom = 0, norm_rest = 0;
};
int factor_general(const NoiseSite& s, GFactors& out);
// complex one-sided Jacobi SVD of a square n x n matrix (row-major):
// a = U diag(sv) V^dagger, singular values descending; U, V column-major
// as u[col * n + row]
void svd_jacobi(const std::vector<cd>& a, int n, std::vector<double>& sv, std::vector<cd>& u, std::vector<cd>& v);

// ------------------------------------------------------------------- handle
struct Engine;     // device-side state (engine.cu)
struct GEngine;    // general-noise path state (generic.cu)
struct SetsState;  // checkpoints for site-set evaluation (sets.cu)

struct Handle {
    Circuit circ;
    bool prepared = false;
    std::vector<Factors> factors;
    Plan plan;
    Engine* eng = nullptr;
    SetsState* sets = nullptr;
    bool profiling = false;
    nqs_kernel_stats stats[5] = {};
    // execution options (nqs_set_option): 0 = automatic
    int opt_spacing = 0;           // sites per checkpoint block
    int opt_rb_multi = 0;          // register qubits of multi-state sweeps (3 or 4)
    int opt_max_ops = 0;           // operations per pass (segmentation)
    int opt_max_sites = 0;         // sites per pass (segmentation)
    int opt_jit = 0;               // pass-specialised kernels: 0 auto, 1 always, 2 never
    int opt_shard_rank = 0;        // this shard of the terms (multi-GPU split of one call)
    int opt_shard_count = 0;       // 0 or 1: no split
    // general noises: the circuit is evaluated by the general-noise path
    bool general = false;
    std::vector<GFactors> gfac;
    GEngine* geng = nullptr;
};
int general_fidelity(Handle& h, const nqs_state* psi, const nqs_state* v, int level, nqs_result* out,
                     void* stream);
int general_term_values(Handle& h, double* out, size_t cap, size_t* count);
void general_destroy(Handle& h);

// engine entry points (engine.cu)
int engine_fidelity(Handle& h, const nqs_state* psi, const nqs_state* v, int level,
                    nqs_result* out, void* stream);
int engine_term_values(Handle& h, double* out, size_t cap, size_t* count);
int engine_batch_fidelity(Handle** hs, size_t count, const nqs_state* psis, const nqs_state* vs, const int* levels,
                          nqs_result* outs, void* stream);
void engine_batch_forget(Handle* h);   // drop a cached batch plan that uses h
int engine_prepare_sets(Handle& h, const nqs_state* psi, const nqs_state* v, void* stream);
int engine_eval_sets(Handle& h, int k, const int* sets, size_t m, double* W_out, void* stream);
void sets_destroy(Handle& h);
// learned importance sampling (is.cpp)
struct Mlp;
int site_features(const Handle& h, const double* W1, float* out);
int pair_training_data(const Handle& h, const float* feats, const double* W2, float* X, float* y, size_t cap,
                       size_t* count);
int is_estimate(Handle& h, Mlp* mlp, int level, unsigned long long samples, double alpha, unsigned long long seed,
                const float* feats, const double* W1, nqs_is_result* out, void* stream);
int is_proposal_values(Handle& h, Mlp* mlp, int level, double alpha, const float* feats, const double* W1,
                       double* q_out, size_t cap, size_t* count, void* stream);
void engine_destroy(Handle& h);
void engine_invalidate(Handle& h);     // rebuild the schedule at the next call
int engine_spacing(const Handle& h, int* n_states);
int engine_launch_list(const Handle& h, nqs_launch_info* out, size_t cap, size_t* count);
uint64_t engine_workspace_bytes(const Handle& h);
uint64_t engine_upload_bytes(const Handle& h);
uint64_t engine_launches_per_call(const Handle& h);
int engine_jit_info(const Handle& h, int* state);
// generate and compile (no device) the kernels of a forward sweep's first passes
int engine_jit_compile_check(Handle& h, int states, int max_passes, int* compiled);
// bounded-wait self-test (kernels_sweep.cu): status word into `status` (device)
int selftest_bounded_wait(int* status, void* stream);
int engine_reduced_matrix(const void* phi, const void* chi, int n, int qubit, double* R_out,
                          void* scratch, size_t scratch_bytes, void* stream);
size_t engine_reduced_matrix_scratch_bytes(int n);
// out = x + (cre + i cim) y on the device (kernels_reduce.cu); kind 1: dense, 0: |bits>
cudaError_t launch_combine(float2* out, long long dim, int xk, unsigned long long xb, const float2* xd, int yk,
                           unsigned long long yb, const float2* yd, float cre, float cim, int grid, cudaStream_t st);

// proposal network (mlp.cu)
struct Mlp;
int mlp_create(int n_in, int hidden, int layers, unsigned long long seed, Mlp** out);
void mlp_destroy(Mlp* m);
size_t mlp_n_params(const Mlp* m);
int mlp_n_in(const Mlp* m);
int mlp_get_params(Mlp* m, float* host, size_t cap);
int mlp_set_params(Mlp* m, const float* host, size_t count);
int mlp_forward(Mlp* m, const float* X, int B, float* y, void* stream);
int mlp_loss_grad(Mlp* m, const float* X, const float* y, int B, double* loss, float* grad_host, size_t cap,
                  void* stream);
int mlp_train(Mlp* m, const float* X, const float* y, int n, int batch, int steps, float lr, unsigned long long seed,
              double* final_loss, void* stream);

// allocator (capi.cpp)
void* dev_alloc(size_t bytes, void* stream);
void dev_free(void* p, size_t bytes, void* stream);

}  // namespace nqs
