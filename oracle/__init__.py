"""FP64 CPU oracle for the level-l noise expansion -- TEST INFRASTRUCTURE ONLY.

This package is the independent checker of the CUDA path.  Only the test
suite, the smoke check and the CPU-baseline leg of the benchmark may import
it; the library itself never does, and it shares no code, tables or helpers
with the library (the two meet only through the seeded inputs of the
top-level ``workloads`` package).

Contents (each function cites the passage of the paper it follows):

* ``ir``             -- reader of the circuit/noise text format
* ``gates``          -- gate matrices (Table I, controlled gates of Sec. II, U3)
* ``statevector``    -- plain FP64 state-vector application of gate matrices
* ``density_matrix`` -- O1: exact F = <v|E(|psi><psi|)|v> by Kraus maps (Sec. II, Problem 1)
* ``expansion``      -- O2/O4: the level-l expansion of Sec. IV (matrix
                        representation M = sum_k E_k (x) E_k^*, tensor
                        permutation, SVD, level-l substitution, two networks
                        per term, one sweep per network) and the canonical
                        enumeration of kept terms
* ``o3``             -- O3: the same terms from forward/backward FP64
                        checkpoints in C with OpenMP (csim/o3.c), for wide
                        circuits and large term counts
* ``bounds``         -- Theorem 1, the level-1 corollary, Lemmas 1-2 helpers
* ``csim``           -- the same plain state-vector step in C (FP64, OpenMP)
                        for widths where numpy is too slow

Parity status: every function here is pinned by tests in tests/test_oracle_*.py
against closed forms, brute force and the paper's worked values.
"""
