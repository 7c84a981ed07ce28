"""Kernel-side error path: a stage wait that gives up.

Every mbarrier wait of the SpMV and SpMM block kernels is bounded.  The test hook
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


@pytest.mark.parametrize("k", [3, 8, 32])
def test_expired_wait_then_recovery_spmm(cuda_device, k):
    # the SpMM's warps move through its block ring without block barriers: a warp that
    # gives up drains the ring on its own, and the warps left waiting run out in turn
    a, p, _ = _setup("auto", False)
    vals = torch.from_numpy(a.val).cuda().float()
    X = torch.from_numpy(np.random.default_rng(k).random((a.n_cols, k))).cuda().float()
    p.set_wait_limit(0)
    mb.spmm(p, vals, X)
    with pytest.raises(mb.MerbitError) as e:
        p.sync()
    assert e.value.status == EDEVICE
    p.sync()
    p.set_wait_limit(-1)
    Y = mb.spmm(p, vals, X)
    p.sync()
    Y_ref, d = oracle.spmm(a.row_ptr, a.col, as_f64(vals), as_f64(X))
    Yg = as_f64(Y)
    for c in range(k):
        check_rel(Yg[:, c], Y_ref[:, c], d[:, c], TOL[torch.float32], f"SpMM after recovery k={k} column {c}")


def test_expired_wait_then_recovery_ppr(cuda_device):
    a, p, _ = _setup("auto", False)
    vals = torch.from_numpy(a.val).cuda().float()
    seeds = inputs.ppr_seeds(a, 8, 5)
    p.set_wait_limit(0)
    with pytest.raises(mb.MerbitError) as e:
        mb.ppr(p, vals, seeds, ALPHA, tol=1e-6, max_iter=50)
    assert e.value.status == EDEVICE
    p.set_wait_limit(-1)
    r = mb.ppr(p, vals, seeds, ALPHA, tol=1e-6, max_iter=300)
    assert r["converged"]
    Pi = r["pi"][:, [0, 7]].double().cpu().numpy()
    rr = oracle.ppr_residual(a.row_ptr, a.col, a.val, Pi, [int(seeds[0]), int(seeds[7])], ALPHA)
    assert max(rr) < 1e-5, rr
