// nqs_reduced_matrix_noalloc: the reduced-matrix reduction of
// nqs_reduced_matrix with its per-block scratch in a fixed device array
// instead of caller-provided or allocated memory.
//
// Some callers cannot allocate device memory at the point where they need
// this reduction: hosts that hand the whole device heap to another runtime's
// pool, latency-critical loops where cudaMalloc's implicit device-wide
// synchronisation is not acceptable, and plugin environments that forbid
// dynamic device allocation.  For them the scratch lives in a file-scope
// __device__ array of fixed size that every GPU loading the library holds
// until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "nqs_internal.h"
#include "sweep_types.h"

namespace nqs {

namespace {

// scratch: per-block partial sums (8 doubles per block) of at most
// NQS_NOALLOC_MAX_BLOCKS blocks
static __device__ __align__(256) double g_noalloc_scratch[NQS_NOALLOC_MAX_BLOCKS * 8];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device

// Once per device, with that device current: resolve the array's device
// address (its host-side name is only a stand-in for the symbol).
int scratch_address(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NQS_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return NQS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return NQS_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return NQS_OK;
}

// Memory a kernel on device `dev` may use: device memory of that device,
// managed memory, or (when allowed, for the result) pinned host memory.
int check_pointer(const void* p, int dev, bool pinned_host_ok) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return NQS_ERR_ARG;
    }
    switch (a.type) {
        case cudaMemoryTypeDevice: return a.device == dev ? NQS_OK : NQS_ERR_ARG;
        case cudaMemoryTypeManaged: return NQS_OK;
        case cudaMemoryTypeHost: return pinned_host_ok ? NQS_OK : NQS_ERR_ARG;
        default: return NQS_ERR_ARG;   // pageable host memory
    }
}

}  // namespace

}  // namespace nqs

extern "C" int nqs_reduced_matrix_noalloc(const void* phi, const void* chi, int n, int qubit, double* R_out,
                                          void* stream) {
    using namespace nqs;
    if (!phi || !chi || !R_out || n < 1 || qubit < 0 || qubit >= n) return NQS_ERR_ARG;
    if (n > NQS_NOALLOC_MAX_QUBITS) return NQS_ERR_TOO_LARGE;
    if (((uintptr_t)phi & 15u) || ((uintptr_t)chi & 15u) || ((uintptr_t)R_out & 7u)) return NQS_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NQS_ERR_CUDA;
    // the kernels run on the current device: the states must live there (or
    // be managed), the result may also be pinned host memory, and the stream
    // must belong to that device (the cached scratch address is this device's)
    if (check_pointer(phi, dev, false) != NQS_OK || check_pointer(chi, dev, false) != NQS_OK ||
        check_pointer(R_out, dev, true) != NQS_OK)
        return NQS_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (st) {
        int sdev = -1;
        if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
            cudaGetLastError();
            return NQS_ERR_ARG;
        }
        if (sdev != dev) return NQS_ERR_ARG;
    }
    double* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != NQS_OK) return rc;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NQS_ERR_CUDA;
    // same grid rule as nqs_reduced_matrix (about 16 pairs per thread per
    // round, at most 4 blocks per SM), capped by the scratch capacity
    long long npairs = 1ll << (n - 1);
    long long g = (npairs + 16ll * kThreads - 1) / (16ll * kThreads);
    g = std::min<long long>(g, (long long)sms * 4);
    g = std::min<long long>(g, 2048);
    g = std::min<long long>(g, NQS_NOALLOC_MAX_BLOCKS);
    const int grid = (int)std::max<long long>(1, g);
    // every block overwrites its 8 partial slots before the sum reads them,
    // so nothing left by an earlier call is read
    if (launch_reduce2x2((const float2*)phi, (const float2*)chi, n, qubit, scratch, grid, st) != cudaSuccess)
        return NQS_ERR_CUDA;
    if (launch_partials_sum(scratch, grid, R_out, st) != cudaSuccess) return NQS_ERR_CUDA;
    return NQS_OK;
}
