"""Kernel-side error path: a stage wait that gives up.

Every mbarrier wait of the SpMV block kernels is bounded.  The test hook
merbit_plan_set_wait_limit(plan, 0) makes each launch give up at its first stage wait,
without any fault: the kernel records the error bit, waits (with the default limit) for
its own bulk copies to land and returns.  The host must report MERBIT_EDEVICE, reset the
plan's device state, and the next call on the same plan must be correct again."""
import numpy as np
import pytest
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb
from tests.gpu_helpers import TOL, as_f64, check_rel

pytestmark = pytest.mark.gpu
ALPHA = 0.85
EDEVICE = 6


def _setup(kernel, hot):
    a = inputs.rmat_transition(15, 16, 2)
    rp, col = torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col).cuda()
    p = mb.plan(rp, col, a.n_rows, a.n_cols)
    p.set_kernel(kernel)
    if hot:
        assert p.set_hot_columns(2000)[0] > 0
    return a, p, col


@pytest.mark.parametrize("hot", [False, True])
@pytest.mark.parametrize("kernel", ["split", "split2", "classic"])
def test_expired_wait_then_recovery_spmv(cuda_device, kernel, hot):
    a, p, _ = _setup(kernel, hot)
    for dtype in (torch.float32, torch.float64):
        vals = torch.from_numpy(a.val).to("cuda", dtype)
        x = torch.from_numpy(inputs.uniform_vector(a.n_cols, 3)).to("cuda", dtype)
        p.set_wait_limit(0)
        mb.spmv(p, vals, x)                       # asynchronous: the launch itself succeeds
        with pytest.raises(mb.MerbitError) as e:
            p.sync()
        assert e.value.status == EDEVICE
        p.sync()                                  # the state was cleared: no error left
        p.set_wait_limit(-1)
        y = mb.spmv(p, vals, x)
        p.sync()
        y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(vals), as_f64(x))
        check_rel(as_f64(y), y_ref, d, TOL[dtype], f"after recovery {kernel} {dtype}")


@pytest.mark.parametrize("kernel", ["split", "split2", "classic"])
def test_expired_wait_then_recovery_pagerank(cuda_device, kernel):
    a, p, _ = _setup(kernel, True)
    v64 = torch.from_numpy(a.val).cuda()
    for mode in ("plain", "ir_bf16"):
        p.set_wait_limit(0)
        with pytest.raises(mb.MerbitError) as e:
            mb.pagerank(p, v64, ALPHA, tol=1e-10, mode=mode, inner_sweeps=8, max_iter=40)
        assert e.value.status == EDEVICE
        p.set_wait_limit(-1)
        pi, info = mb.pagerank(p, v64, ALPHA, tol=1e-10, mode=mode, inner_sweeps=12, max_iter=400)
        assert info["converged"], (mode, info)
        r = oracle.pagerank_residual(a.row_ptr, a.col, a.val, as_f64(pi), ALPHA)
        assert r < 1.2e-10, (mode, r)


def test_wait_limit_rejects_null_plan(cuda_device):
    lib = mb.merbit.load()
    assert lib.merbit_plan_set_wait_limit(None, 0) == 1
