"""Personalised PageRank (merbit_ppr, one column per seed on the batched product)
against the float64 oracle: the same number of updates, converged vectors against
closed forms and dense solves, and the oracle's own FP64 residual of the result."""
import numpy as np
import pytest
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb
from tests.gpu_helpers import as_f64, make_plan

pytestmark = pytest.mark.gpu

ALPHA = 0.85


def _ppr(a, seeds, **kw):
    p, _ = make_plan(a)
    vals = torch.from_numpy(a.val).to("cuda", torch.float32)
    r = mb.ppr(p, vals, seeds, ALPHA, **kw)
    return as_f64(r["pi"]), r


def _converged_matches(a, seeds, ref_cols, atol):
    """300 updates (alpha^300 < 1e-21: what is left is f32 rounding), then entries against
    the exact fixed point; the last update's size is at the f32 rounding level."""
    Pi, r = _ppr(a, seeds, tol=0.0, max_iter=300)
    assert r["iters"] == 300
    assert max(r["resid"]) < 2e-6, r["resid"]
    for c, ref in enumerate(ref_cols):
        np.testing.assert_allclose(Pi[:, c], ref, rtol=0, atol=atol, err_msg=f"{a.name} col {c}")


def test_ppr_cycle_closed_form(cuda_device):
    n = 64
    a = inputs.cycle_graph(n)
    seeds = [0, 5, 63]
    refs = []
    for s in seeds:
        ref = np.zeros(n)
        for j in range(n):
            ref[(s + j) % n] = (1 - ALPHA) * ALPHA ** j / (1 - ALPHA ** n)
        refs.append(ref)
    _converged_matches(a, seeds, refs, 2e-6)


def test_ppr_chain_dangling_end(cuda_device):
    L = 7
    a = inputs.from_edges(L, [(i, i + 1) for i in range(L - 1)], "chain7")
    seeds = [0, 3, 6, 1]                              # 6 is the dangling end
    refs = []
    for m in seeds:
        ref = np.zeros(L)
        for j in range(L - m):
            ref[m + j] = (1 - ALPHA) * ALPHA ** j / (1 - ALPHA ** (L - m))
        refs.append(ref)
    _converged_matches(a, seeds, refs, 2e-6)


def test_ppr_star_closed_form(cuda_device):
    k = 9
    a = inputs.bidirected_star(k)
    c = ALPHA / (1 + ALPHA)
    leaf = ALPHA * c / k
    refs = [np.array([c, 1 - ALPHA + leaf] + [leaf] * (k - 1)),
            np.array([1 / (1 + ALPHA)] + [ALPHA / ((1 + ALPHA) * k)] * k)]
    _converged_matches(a, [1, 0] * 4, refs * 4, 2e-6)   # k = 8 columns: the 16-byte path


@pytest.mark.parametrize("seed", range(3))
def test_ppr_dense_solve(cuda_device, seed):
    a = inputs.random_graph_transition(40 + 11 * seed, 0.06, seed)
    dang = oracle.dangling_mask(a.n_rows, a.col)
    dense = np.zeros((a.n_rows, a.n_cols))
    for r in range(a.n_rows):
        dense[r, a.col[a.row_ptr[r]:a.row_ptr[r + 1]]] = a.val[a.row_ptr[r]:a.row_ptr[r + 1]]
    seeds = list(range(0, a.n_rows, max(1, a.n_rows // 8)))[:8]
    if dang.any():
        seeds[-1] = int(np.flatnonzero(dang)[0])          # one dangling seed
    _converged_matches(a, seeds, [oracle.ppr_dense_solve(dense, s, ALPHA) for s in seeds], 2e-6)


@pytest.mark.parametrize("k", [1, 3, 8, 12, 32, 40])
def test_ppr_fixed_updates_rmat14(cuda_device, k):
    """30 updates on the device and in the oracle: L1 difference per column."""
    a = inputs.rmat_transition(14, 16, 1)
    seeds = inputs.ppr_seeds(a, k, 5 + k)
    Pi, r = _ppr(a, seeds, tol=0.0, max_iter=30)
    assert r["iters"] == 30
    ref = oracle.personalized_pagerank(a.row_ptr, a.col, a.val, seeds, ALPHA, fixed_iters=30)
    err = np.abs(Pi - ref["pi"]).sum(axis=0)
    assert err.max() < 2e-5, err
    np.testing.assert_allclose(r["resid"], ref["last"], rtol=1e-3, atol=1e-6)
    np.testing.assert_allclose(r["hist"], ref["resid"], rtol=1e-3, atol=1e-6)


def test_ppr_tolerance_stop_rmat14(cuda_device):
    a = inputs.rmat_transition(14, 16, 1)
    seeds = inputs.ppr_seeds(a, 8, 11)
    Pi, r = _ppr(a, seeds, tol=1e-6, max_iter=500)
    ref = oracle.personalized_pagerank(a.row_ptr, a.col, a.val, seeds, ALPHA, tol=1e-6)
    assert r["converged"] and abs(r["iters"] - ref["iters"]) <= 1
    assert max(r["resid"]) < 1e-6
    # the oracle's own FP64 residual of the device's answer, and its distance to the fixed point
    res = oracle.ppr_residual(a.row_ptr, a.col, a.val, Pi, seeds, ALPHA)
    assert res.max() < 3e-6, res
    exact = oracle.personalized_pagerank(a.row_ptr, a.col, a.val, seeds, ALPHA, tol=1e-13)["pi"]
    assert np.abs(Pi - exact).sum(axis=0).max() <= (res.max() + 1e-6) / (1 - ALPHA)


def test_ppr_errors(cuda_device):
    a = inputs.rmat_transition(10, 8, 2)
    p, _ = make_plan(a)
    vals = torch.from_numpy(a.val).cuda().float()
    with pytest.raises(mb.MerbitError, match="EINVAL"):
        mb.ppr(p, vals, [a.n_rows])
    with pytest.raises(mb.MerbitError, match="EINVAL"):
        mb.ppr(p, vals, [0], alpha=1.0)
    r = mb.ppr(p, vals, [1, 2], tol=1e-12, max_iter=3)
    assert not r["converged"] and r["iters"] == 3
    rect = inputs.random_sparse(50, 40, 0.1, 1)
    q, _ = make_plan(rect)
    with pytest.raises(mb.MerbitError, match="EINVAL"):
        mb.ppr(q, torch.from_numpy(rect.val).cuda().float(), [0])


@pytest.mark.parametrize("k", [8, 32])
def test_ppr_full_rmat22(cuda_device, k):
    """The batched personalised PageRank workload at full size: R-MAT scale 22, k seeds
    over non-dangling vertices, to L1 residual 1e-6 per column."""
    a = inputs.rmat_transition(22, 16, 7)
    seeds = inputs.ppr_seeds(a, k, 22)
    Pi, r = _ppr(a, seeds, tol=1e-6, max_iter=300)
    assert r["converged"], r["hist"][-3:]
    sums = Pi.sum(axis=0)
    np.testing.assert_allclose(sums, 1.0, atol=1e-4)
    assert Pi.min() >= 0.0
    assert np.all(Pi[seeds, np.arange(k)] >= 1 - ALPHA - 1e-6)
    cols = [0, k - 1]
    res = oracle.ppr_residual(a.row_ptr, a.col, a.val, Pi[:, cols], [int(seeds[c]) for c in cols],
                              ALPHA)
    assert res.max() < 5e-6, res


@pytest.mark.parametrize("k", [300, 516])
def test_ppr_many_seeds(cuda_device, k):
    """Wide batches: k = 300 takes the scalar path with one row of 300 threads per block of
    the streaming pass, k = 516 the 16-byte path with 129 column vectors per row."""
    a = inputs.rmat_transition(10, 16, 4)
    seeds = inputs.ppr_seeds(a, k, 9)
    Pi, r = _ppr(a, seeds, tol=0.0, max_iter=12)
    ref = oracle.personalized_pagerank(a.row_ptr, a.col, a.val, seeds, ALPHA, fixed_iters=12)
    assert np.abs(Pi - ref["pi"]).sum(axis=0).max() < 2e-5
    np.testing.assert_allclose(r["resid"], ref["last"], rtol=1e-3, atol=1e-6)
