"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package only draws inputs (circuits, noise placements, channels, states);
it holds none of the noisy-simulation arithmetic.
"""

from .rng import SplitMix64
from . import channels
from .circuits import (Workload, Noise, c1_line6, c2_grid20, c3_qaoa30, c4_circuit, c4_batch,
                       c5_grid, c5_twin, c5_twin_hot, qaoa_workload, random_circuit, identity_workload)
from .ir_text import to_ir_text

__all__ = ["SplitMix64", "channels", "Workload", "Noise", "c1_line6", "c2_grid20", "c3_qaoa30",
           "c4_circuit", "c4_batch", "c5_grid", "c5_twin", "c5_twin_hot", "qaoa_workload", "random_circuit",
           "identity_workload", "to_ir_text"]
