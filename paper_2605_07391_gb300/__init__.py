"""MERBIT SpMV / PageRank for GB300 (sm_103a): CUDA library + thin Python binding."""
from .merbit import (  # noqa: F401
    BF16, Batch, EXPORTS, F16, F32, F64, IR_BF16, IR_F16, IR_F32, MODES, PLAIN, MerbitError, Plan,
    PlanInfo, TileArrays, Transpose, autotune, autotune_sigma, bicgstab, gather, library_path, load, pagerank, pagerank_adjoint, plan, ppr,
    sddmm, spmm, spmv, spmv_host, transpose, vals_convert, version,
)
from . import autograd  # noqa: F401,E402
