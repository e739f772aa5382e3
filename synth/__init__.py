"""Seeded synthetic inputs shaped like the paper's bulk-silicon workloads.

This package only draws random numbers and lays them out; it holds none of the
method's arithmetic (no neighbour search, no products, no traces).  Both the
CPU oracle and the CUDA library are fed from here.
"""
from .si import (  # noqa: F401
    SI_A,
    si_diamond_positions,
    sym_block_values,
    diag_block,
    si_workload,
    batch_cell_counts,
)
