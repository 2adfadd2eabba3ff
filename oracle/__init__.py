"""CPU FP64 oracle for the S_N source-iteration solve.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py. The product library never imports it, and the
two share no code. See dts_oracle.c for what is computed and which passages
of the paper each part follows.
"""
from .oracle import (  # noqa: F401
    build, load, quadrature, real_sh, sh_tables, subsweep_size, subsweep_cells,
    dd_cell, sweep_dir, uncollided_voxel, solve, solve_workload, adjoint, OracleResult, dose,
    MEV_PER_G_TO_GY,
)
