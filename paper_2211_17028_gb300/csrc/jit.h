// Pass-specialised sweep kernels compiled at run time (jit.cpp).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "sweep_types.h"

namespace nqs {

// Everything the generator needs from one register-resident launch.
struct JitPass {
    int S = 1, RB = 4, n = 0;
    int k = kMaxTileQ;        // tile qubits (12, or 13 with 512-thread blocks)
    bool pp = false;          // one-state kernels: two re-layout buffers, one barrier per re-layout
    int hint = 0;             // L2 policies: 1 state tiles evict-first, 2 phi kept for the other states
    int rv = 1;               // site reduction form: 1 conj-multiply-add, 2 split accumulators
    int db = 1;               // staging buffers of one-state kernels (1 or 2)
    bool seq = false;         // multi-state pass swept one state at a time (2 blocks per SM)
    int local[kTileSlots] = {};
    int nonlocal[kMaxQ] = {};
    int n_events = 0;
    int err_timeout = NQS_ERR_DEVICE_TIMEOUT;
    std::vector<DevPhase> phases;
    std::vector<OpRec> ops;
    std::vector<float2> mats;
    std::string source;       // generated CUDA source (cache key)
    void* kernel = nullptr;   // cudaKernel_t once built
    size_t smem_bytes() const;
};

// Host mirror of the kernels' argument block (same layout).
struct JitArgsHost {
    const float2* in[3];
    float2* out[3];
    float2* const* ckpt;
    float2* const* ckpt_fwd;
    float2* spawn[9];
    double* partials;
    int* err;
    long long n_tiles;
};

std::string jit_source(const JitPass& p);
bool jit_available();
int jit_blocks_per_sm();      // resident blocks per SM of one-state-in-registers kernels
long long jit_compile_count();
// Generate, compile (distinct sources in parallel, cached for the process)
// and load every pass; 0 on success, -1 with a message otherwise.
int jit_build(std::vector<JitPass*>& passes, std::string* error);
// Generate and compile only (no device needed); 0 when every pass compiled.
int jit_compile(std::vector<JitPass*>& passes, std::string* error);
cudaError_t jit_launch(const JitPass& p, int grid, const PassArgs& a, cudaStream_t st);

}  // namespace nqs
