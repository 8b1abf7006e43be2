// Instantiation of the register-resident sweep kernels (kernels_sweep_body.cuh)
// for 3 states with 4 register qubits, in a translation unit of its own so that the pairs compile in parallel.
#include "kernels_sweep_body.cuh"

namespace nqs {

NQS_SWEEP_PAIR(3, 4)

}  // namespace nqs
