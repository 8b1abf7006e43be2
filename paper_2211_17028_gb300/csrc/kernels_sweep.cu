// Register-resident tile sweep for sm_103a: dispatch by state count and
// register qubits to the kernels instantiated in kernels_sweep_s*.cu (the
// kernel itself is described in kernels_sweep_body.cuh), occupancy and
// shared-memory sizes, and the bounded-wait self-test.
#include "kernels_sweep_body.cuh"

namespace nqs {

namespace {

// Failure-detection self-test: the sweep kernels' bounded mbarrier wait on a
// barrier that nothing ever arrives at.  The wait must give up (after about
// two seconds) and report it through the status word, leaving the context usable.
__global__ void bounded_wait_probe_kernel(int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0);
    if (threadIdx.x == 0) *status = ok ? NQS_OK : NQS_ERR_DEVICE_TIMEOUT;
}


}  // namespace

// Register qubits per thread for an S-state launch.  Three states with four
// register qubits need ~96 registers of amplitudes per thread (8 warps per
// SM); with three register qubits the block has 512 threads (16 warps) but
// a pass needs more phases.  NQS_SWEEP_RB (3 or 4) overrides the choice for
// multi-state launches.
int sweep_reg_bits(int S) {
    static int forced = -1;
    if (forced < 0) {
        const char* e = getenv("NQS_SWEEP_RB");
        forced = (e && (e[0] == '3' || e[0] == '4')) ? e[0] - '0' : 0;
    }
    if (S == 1) return 4;
    return forced ? forced : 3;
}

int sweep_blocks_per_sm(int S, int RB, size_t smem) {
    if (S == 1) return sweep_occupancy_1_4(smem);
    if (S == 2) return RB == 4 ? sweep_occupancy_2_4(smem) : sweep_occupancy_2_3(smem);
    return RB == 4 ? sweep_occupancy_3_4(smem) : sweep_occupancy_3_3(smem);
}

size_t sweep_smem_bytes(int S, int RB, int prog_words, int n_events) {
    if (S == 1) return smem_for<1, 4>(prog_words, n_events);
    if (S == 2) return RB == 4 ? smem_for<2, 4>(prog_words, n_events) : smem_for<2, 3>(prog_words, n_events);
    return RB == 4 ? smem_for<3, 4>(prog_words, n_events) : smem_for<3, 3>(prog_words, n_events);
}

cudaError_t launch_bounded_wait_probe(int* status, cudaStream_t st) {
    bounded_wait_probe_kernel<<<1, 32, 0, st>>>(status);
    return cudaGetLastError();
}

int selftest_bounded_wait(int* status, void* stream) {
    return launch_bounded_wait_probe(status, (cudaStream_t)stream) == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
}

cudaError_t launch_sweep(int S, int RB, int grid, const PassArgs& P, cudaStream_t st) {
    if (S == 1) return sweep_launch_1_4(grid, P, st);
    if (S == 2) return RB == 4 ? sweep_launch_2_4(grid, P, st) : sweep_launch_2_3(grid, P, st);
    return RB == 4 ? sweep_launch_3_4(grid, P, st) : sweep_launch_3_3(grid, P, st);
}

cudaError_t launch_sweep_batched(int S, int RB, const PassArgs* units, const int* cta_begin, int n_units,
                                 int total_ctas, size_t smem, cudaStream_t st) {
    if (S == 1) return sweep_launch_batched_1_4(units, cta_begin, n_units, total_ctas, smem, st);
    if (S == 2)
        return RB == 4 ? sweep_launch_batched_2_4(units, cta_begin, n_units, total_ctas, smem, st)
                       : sweep_launch_batched_2_3(units, cta_begin, n_units, total_ctas, smem, st);
    return RB == 4 ? sweep_launch_batched_3_4(units, cta_begin, n_units, total_ctas, smem, st)
                   : sweep_launch_batched_3_3(units, cta_begin, n_units, total_ctas, smem, st);
}


}  // namespace nqs
