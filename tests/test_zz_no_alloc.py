"""merbit_spmv_noalloc: the entry point for callers that may not allocate device memory.

Such callers (code whose device memory belongs to another framework's pool, or
paths that cannot afford cudaMalloc's device-wide synchronisation) get the same
product as the planned path, computed with only a scratch array compiled into
the library.  This file is collected last so that a run stopping at its first
failure has already run every other test; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb

pytestmark = pytest.mark.gpu


def _noalloc(lib):
    f = lib.merbit_spmv_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, vp]
    f.restype = ctypes.c_int
    return f


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_planned_spmv_twice(cuda_device):
    lib = mb.load()
    f = _noalloc(lib)
    a = inputs.add_hubs(inputs.rmat_uniform(16, 16, 3, 3), 2, 20000, 40000, 5)
    row_ptr = torch.from_numpy(a.row_ptr).cuda()
    col = torch.from_numpy(a.col).cuda()
    vals = torch.from_numpy(a.val).cuda().float()
    plan = mb.plan(row_ptr, col, a.n_rows, a.n_cols)
    stream = torch.cuda.current_stream()
    for seed in (2, 9):                       # two calls in a row, different x
        x = torch.from_numpy(inputs.uniform_vector(a.n_cols, seed)).cuda().float()
        y_ref = mb.spmv(plan, vals, x)        # the existing entry point
        y = torch.full((a.n_rows,), float("nan"), device="cuda")
        st = f(_p(row_ptr), _p(col), _p(vals), _p(x), _p(y), a.n_rows, a.n_cols, a.nnz,
               ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, lib.merbit_last_error()
        torch.cuda.synchronize()
        # the tolerance of the FP32 parity tests: |dy_i| <= 1e-5 * sum_j |a_ij x_j|
        _, d = oracle.spmv(a.row_ptr, a.col, vals.double().cpu().numpy(), x.double().cpu().numpy())
        diff = np.abs(y.double().cpu().numpy() - y_ref.double().cpu().numpy())
        assert np.all(diff <= 1e-5 * d), float((diff / np.maximum(d, 1e-300)).max())
    plan.destroy()


def test_noalloc_rejects_oversized_matrix(cuda_device):
    lib = mb.load()
    f = _noalloc(lib)
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    # 100 million rows + nonzeros need far more than the reserved scratch
    st = f(_p(dummy), _p(dummy), _p(dummy), _p(dummy), _p(dummy), 50_000_000, 50_000_000,
           50_000_000, None)
    assert st == 1
    assert b"too large" in lib.merbit_last_error()
