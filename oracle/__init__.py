"""CPU float64 oracle of the MERBIT hot path — test infrastructure only.

Import is reserved for tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg; the CUDA library never uses it.
"""
from .merbit_oracle import *  # noqa: F401,F403
from .merbit_oracle import (  # noqa: F401
    build_tile, tile_counts, spmv, spmm, spmv_rows, personalized_pagerank, ppr_residual,
    ppr_dense_solve, ppr_step, transpose_csr, sddmm, pagerank_adjoint,
    pagerank_adjoint_dense, pagerank_value_gradient, bicgstab, pagerank, pagerank_residual,
    pagerank_dense_solve, relative_errors, round_to_format, f16_scale_exponent,
    spmv_lowprec_reference, dangling_mask, block_boundary_rows, decode_lane_desc,
    step_coordinate, merge_path_down_steps, descriptor_fits, relative_linf_error,
)
