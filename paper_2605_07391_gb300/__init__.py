"""MERBIT SpMV / PageRank for GB300 (sm_103a): CUDA library + thin Python binding."""
from .merbit import (  # noqa: F401
    BF16, EXPORTS, F16, F32, F64, IR_BF16, IR_F16, IR_F32, MODES, PLAIN, MerbitError, Plan,
    PlanInfo, TileArrays, library_path, load, pagerank, plan, ppr, spmm, spmv, spmv_host, vals_convert,
    version,
)
