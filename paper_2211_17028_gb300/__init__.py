"""GB300 (sm_103a) level-l SVD noise expansion of noisy-circuit fidelities.

The compute path is libnqs.so (CUDA kernels behind a C ABI, include/nqs.h);
``paper_2211_17028_gb300.nqs`` is its ctypes binding.
"""

from . import nqs  # noqa: F401
