// Device-side types shared by the sweep kernels and the schedule builder.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/nqs.h"

namespace nqs {

constexpr int kMaxTileQ = 12;          // 4096 amplitudes = 32 KB per state tile
constexpr int kWideTileQ = 13;         // generated kernels: 8192 amplitudes, 512-thread blocks
constexpr int kTileSlots = 13;         // tile-qubit slots of the pass records
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxEvents = 8;          // reductions per pass (the planner cuts passes accordingly)
constexpr int kMaxQ = 34;
constexpr int kRegBits = 4;            // register-resident qubits per thread (16 amplitudes)
constexpr int kRegElems = 1 << kRegBits;

// OP_SITE flags
enum : int {
    FL_REDUCE = 1,    // accumulate the 2x2 reduced matrix against phi_site
    FL_SPAWN = 2,     // write K_i x for the kept non-dominant factors
    FL_SAVE = 4,      // store the state as phi_site (before K_0^dagger)
    FL_APPLY = 8,     // apply the site's K_0 (K_0^dagger backwards) after the other actions
    FL_SAVE_FWD = 16, // store the state as chi_site (forward checkpoint, before K_0)
    FL_KDIAG = 32     // K_0 is diagonal
};

// location of a qubit inside the register-resident layout of a phase
//   0..3   register bit i (amplitude index r within the thread)
//   8..15  thread bit (threadIdx.x bit l - 8)
//   -1     outside the tile (bit read from the tile's base index)
enum : int { LOC_NONLOCAL = -1, LOC_THREAD = 8 };

struct DevOp {
    int type;        // OP_*
    int a, b;        // tile positions of q0, q1 (-1 when outside the tile)
    int qa, qb;      // qubits
    int mat;         // offset (in float2) of the matrix in the matrix table
    int site;
    int flags;       // site flags | event << 8 | spawn count << 16
    int la, lb;      // locations of q0, q1 in the phase layout (register-resident kernel)
};

// One phase of a pass in the register-resident kernel: which tile positions
// sit in registers (R), in the lane bits (L) and in the warp bits (W).
struct DevPhase {
    signed char R[kRegBits];
    signed char L[5];
    signed char W[4];
    signed char pad[3];
    int op_begin, op_end;   // indices into the launch's op records
    int pad2[2];
};

// Compact operation record of the register-resident kernel (16 bytes).
struct OpRec {
    unsigned char type, la, lb, flags;   // la, lb: location codes (register bit, LOC_THREAD + bit, 0xff outside)
    unsigned char qa, qb, ev, nspawn;    // qubits; reduction event; spawned factors
    unsigned short site, mat;            // site index; matrix offset (float2) in the program
    unsigned int pad;
};

struct PassArgs {
    const DevOp* ops;
    int n_ops;
    const DevPhase* phases;   // shared-memory tile kernel: unused
    int n_phases;
    const uint4* prog;        // register-resident kernel: phases, op records, matrices
    int prog_words, ops_word, mats_word;
    const float2* mats;
    int n, k, c;
    int n_events;
    int local[kTileSlots];
    int nonlocal[kMaxQ];
    long long n_tiles;
    const float2* in[3];
    float2* out[3];
    float2* const* ckpt;   // phi_s slots
    float2* const* ckpt_fwd;   // chi_s slots (forward checkpoints)
    float2* spawn[9];
    double* partials;      // [(event * S + state) * grid + block][8]
    int* err;              // device status word (bounded waits that gave up)
};

struct FinishDesc {
    long long rank;   // -1: no term
    int kmat;         // offset (doubles) of the 2x2 complex128 factor
    int pad;
};

// batched bookkeeping units (one per circuit of a batch round)
struct FinishUnit {
    const double* partials;
    const FinishDesc* desc;
    const double* kmats;
    double* vals;
    int grid;
    int pad;
};

struct FillUnit {
    float2* dst;
    long long dim;
    unsigned long long bits;
};

struct SumUnit {
    const double* vals;
    const long long* level_off;
    nqs_result* res;
    nqs_result* copy;    // gathered copy of the result (batch output array)
    const int* err;
    double bound;
    long long n_terms;
    int level;
    int pad;
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {   // a*b + c
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ int insert0(int p, int pos) {
    return ((p >> pos) << (pos + 1)) | (p & ((1 << pos) - 1));
}

// ---------------------------------------------------------------- launchers
// shared-memory tile kernel (any tile width up to 12 qubits)
int tile_pass_blocks_per_sm(int S, size_t smem);
cudaError_t launch_tile_pass(int S, int grid, size_t smem, const PassArgs& P, cudaStream_t st);
// register-resident kernel with TMA prefetch (tile width exactly 12 qubits)
int sweep_reg_bits(int S);
int sweep_blocks_per_sm(int S, int RB, size_t smem);
size_t sweep_smem_bytes(int S, int RB, int prog_words, int n_events);
cudaError_t launch_sweep(int S, int RB, int grid, const PassArgs& P, cudaStream_t st);
cudaError_t launch_bounded_wait_probe(int* status, cudaStream_t st);
// the passes of many circuits in one launch: unit u runs on blocks
// [cta_begin[u], cta_begin[u+1]) (device arrays); all units share S and RB
cudaError_t launch_sweep_batched(int S, int RB, const PassArgs* units, const int* cta_begin, int n_units,
                                 int total_ctas, size_t smem, cudaStream_t st);
// reductions, finishers, fills
cudaError_t launch_reduce2x2(const float2* phi, const float2* chi, int n, int q, double* partials, int grid,
                             cudaStream_t st);
cudaError_t launch_finish(const double* partials, int grid, const FinishDesc* desc, const double* kmats,
                          double* vals, int n_red, cudaStream_t st);
cudaError_t launch_partials_sum(const double* part, int grid, double* R, cudaStream_t st);
cudaError_t launch_normalize(float2* v, long long dim, const double* partials, int red_grid, int grid,
                             cudaStream_t st);
cudaError_t launch_combine(float2* out, long long dim, int xk, unsigned long long xb, const float2* xd, int yk,
                           unsigned long long yb, const float2* yd, float cre, float cim, int grid, cudaStream_t st);
cudaError_t launch_level_sum(const double* vals, const long long* level_off, int level, nqs_result* res,
                             double bound, long long n_terms, const int* err, cudaStream_t st);
cudaError_t launch_basis_fill(float2* out, long long dim, unsigned long long bits, int grid, cudaStream_t st);
cudaError_t launch_finish_batched(const FinishUnit* units, const int* blk_begin, int n_units, int total_blocks,
                                  cudaStream_t st);
cudaError_t launch_level_sum_batched(const SumUnit* units, int n_units, cudaStream_t st);
cudaError_t launch_fill_batched(const FillUnit* units, int n_units, cudaStream_t st);

}  // namespace nqs
