// Schedule and engine state shared by the single-circuit engine (engine.cu)
// and the batch executor (batch.cu).  Internal to libnqs.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "fp32_round.h"
#include "jit.h"
#include "nqs_internal.h"
#include "sweep_types.h"

namespace nqs {


struct RunPass {
    int op_off = 0, n_ops = 0;       // in the device op buffer
    int k = 0, c = 0;
    int local[kTileSlots] = {};
    int nonlocal[kMaxQ] = {};
    std::vector<int> lin;            // linear op index of each device op
    std::vector<int> ev_site;        // site of reduction event e
    int spawn_site = -1;             // site that spawns in this pass (at most one)
    int phase_off = 0, n_phases = 0; // register-resident phases (device phase buffer)
};

struct Run {
    std::vector<RunPass> passes;     // in execution order
};

enum LaunchKind { L_PASS, L_FINISH, L_FILL, L_COPY, L_REDUCE2, L_SUM, L_NORMALIZE };

struct Launch {
    LaunchKind kind;
    int S = 1;
    PassArgs args{};
    int op_index = 0;                // offset of the first device op (rebased onto the device table)
    int prog_index = 0;              // offset (16-byte words) of the launch's program
    bool rt = false;                 // register-resident kernel
    int rb = 4;                      // its register qubits
    int grid = 0;
    size_t smem = 0;
    // finisher
    int n_red = 0, fin_grid = 0;
    size_t desc_off = 0;
    // fill / copy
    float2* dst = nullptr;
    const float2* src = nullptr;
    unsigned long long bits = 0;
    double bytes = 0;                // algorithmic bytes (pass kernels)
    bool bd_table = false;           // pass saves through the block-boundary checkpoint table
    int op_counts[8] = {};           // pass: G1, G2, D1, D2, sites, reductions, spawned states, saves
    JitPass* jit = nullptr;          // pass-specialised kernel (owned by the engine), or the interpreter
    bool seq = false;                // multi-state pass-specialised kernel sweeps its states one at a time
};

struct Engine {
    int sm_count = 0;
    size_t smem_optin = 0;           // largest dynamic shared memory per block
    int device = -1;
    // persistent device buffers
    void* buf = nullptr;             // one allocation for states
    size_t buf_bytes = 0;
    void* aux = nullptr;             // ops, mats, tables, partials, term values, result
    size_t aux_bytes = 0;
    // schedule cache key
    int level = -1, psi_kind = -1, v_kind = -1;
    unsigned long long psi_bits = 0, v_bits = 0;
    const void* psi_dev = nullptr;
    const void* v_dev = nullptr;
    std::vector<Launch> launches;
    double bound = 0;
    long long n_terms = 0;
    int eff_level = 0;
    long long* level_off_dev = nullptr;
    double* term_vals = nullptr;
    nqs_result* res_dev = nullptr;
    FinishDesc* desc_dev = nullptr;
    double* partials = nullptr;
    double* kmats_dev = nullptr;
    int* err_dev = nullptr;
    // profiling
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    struct EvUse {
        int kind, sub;   // stats slot; second slot for sweep passes (3: several states, 4: one), -1 none
        double bytes;
    };
    std::vector<EvUse> ev_used;
    size_t ev_next = 0;
    cudaStream_t last_stream = nullptr;
    bool has_result = false;
    uint64_t upload_bytes = 0;
    uint64_t gen = 0;                // bumped whenever the schedule is rebuilt
    int spacing = 0;                 // sites per checkpoint block of the current schedule (0: every site)
    size_t n_states = 0;             // state buffers of the current schedule
    std::vector<std::unique_ptr<JitPass>> jit;   // pass-specialised kernels of the current schedule
    int jit_launches = 0;
    int jit_state = 0;               // 0 not requested, 1 built, -1 failed (interpreter runs)
    Plan wide_plan;                  // the plan re-cut for 13-qubit tiles (generated kernels)
    bool wide = false;               // the current schedule runs on wide_plan
    bool wide_failed = false;        // a wide schedule's kernels could not be built: 12-qubit tiles
};


// Matrix table builder (float2 for sweeps, complex128 for finishers).
struct Tables {
    std::vector<float2> mats;
    std::vector<double> kmats;     // per site: K_0..K_3, 8 doubles each
    // unitary matrices are rounded to stay as unitary as FP32 allows (fp32_round.h)
    int add(const cd* m, int cnt, bool adjoint, int dim) {
        int off = (int)mats.size();
        cd v[16];
        for (int r = 0; r < dim; ++r)
            for (int c = 0; c < dim; ++c) v[dim * r + c] = adjoint ? std::conj(m[dim * c + r]) : m[dim * r + c];
        float2 f[16];
        round_matrix_c64(v, dim, f);
        for (int e = 0; e < dim * dim; ++e) mats.push_back(f[e]);
        (void)cnt;
        return off;
    }
};

enum RunType { RT_IDEAL, RT_BWD, RT_FWD };

struct ProgInfo {
    int words_begin = 0, n_words = 0, ops_word = 0, mats_word = 0, n_phases = 0;
};

int cuda_err(cudaError_t e);
ProgInfo build_program(const std::vector<DevOp>& dops, int off, int n, int RB, const Tables& tab,
                       std::vector<uint4>& prog, int k = kMaxTileQ);
// Device ops of one sweep direction over the passes `segs`.  Backward runs
// save phi at every site, or only at the sites flagged in `save_only`.
Run make_run(const Plan& plan, const std::vector<PassSpec>& segs, RunType rt, bool reduce, bool spawn,
             bool level0_only, const std::vector<Factors>& fac, Tables& tab, std::vector<DevOp>& dops,
             const std::vector<char>* save_only = nullptr);

// schedule construction and execution (engine.cu)
int engine_init(Engine& E);
void engine_release(Engine& E, void* stream);
// allow_jit: the schedule may use pass-specialised kernels (the batch executor
// launches passes through its own multi-circuit kernel and passes false)
int build_schedule(Handle& h, Engine& E, const nqs_state* psi, const nqs_state* v, int level, void* stream,
                   bool allow_jit = true);
int run_schedule(Handle& h, Engine& E, cudaStream_t st);
int run_launch(Handle& h, Engine& E, const Launch& l, cudaStream_t st);
int launch_pass(const Launch& l, cudaStream_t st);

}  // namespace nqs
