// Instantiation of the register-resident sweep kernels (kernels_sweep_body.cuh)
// for 1 states with 4 register qubits, in a translation unit of its own so that the pairs compile in parallel.
#include "kernels_sweep_body.cuh"

namespace nqs {

NQS_SWEEP_PAIR(1, 4)

}  // namespace nqs
