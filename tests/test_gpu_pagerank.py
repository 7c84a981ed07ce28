"""PageRank on the MERBIT SpMV (Sec. 5.5.1): power method and mixed-precision refinement."""
import numpy as np
import pytest
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb
from tests.gpu_helpers import as_f64, make_plan

pytestmark = pytest.mark.gpu
ALPHA = 0.85


def _pr(a, dtype=torch.float64, **kw):
    p, _ = make_plan(a)
    vals = torch.from_numpy(a.val).to("cuda", dtype)
    pi, info = mb.pagerank(p, vals, ALPHA, **kw)
    return as_f64(pi), info


@pytest.mark.parametrize("dtype,rtol", [(torch.float64, 1e-12), (torch.float32, 2e-6)])
def test_closed_forms(cuda_device, dtype, rtol):
    tol = 1e-13 if dtype == torch.float64 else 1e-7
    for n in (1, 5, 64, 1000):
        pi, info = _pr(inputs.cycle_graph(n), dtype, tol=tol)
        np.testing.assert_allclose(pi, 1.0 / n, rtol=rtol)
    for k in (3, 40, 5000):
        pi, _ = _pr(inputs.bidirected_star(k), dtype, tol=tol)
        c = (1 + ALPHA * k) / ((k + 1) * (1 + ALPHA))
        leaf = (k + ALPHA) / (k * (k + 1) * (1 + ALPHA))
        np.testing.assert_allclose(pi, [c] + [leaf] * k, rtol=rtol * 10)
        pi, _ = _pr(inputs.in_star(k), dtype, tol=tol)
        den = 1 + k * (1 + ALPHA)
        np.testing.assert_allclose(pi, [(1 + ALPHA * k) / den] + [1 / den] * k, rtol=rtol * 10)
    pi, _ = _pr(inputs.from_edges(3, [(0, 1), (1, 2)], "chain3"), dtype, tol=tol)
    np.testing.assert_allclose(pi, np.array([1, 1 + ALPHA, 1 + ALPHA + ALPHA ** 2])
                               / (3 + 2 * ALPHA + ALPHA ** 2), rtol=rtol)


@pytest.mark.parametrize("seed", range(3))
def test_dense_solve(cuda_device, seed):
    a = inputs.random_graph_transition(40 + 10 * seed, 0.07, seed)
    dense = np.zeros((a.n_rows, a.n_cols))
    for r in range(a.n_rows):
        dense[r, a.col[a.row_ptr[r]:a.row_ptr[r + 1]]] = a.val[a.row_ptr[r]:a.row_ptr[r + 1]]
    pi, info = _pr(a, torch.float64, tol=1e-14)
    np.testing.assert_allclose(pi, oracle.pagerank_dense_solve(dense, ALPHA), rtol=1e-11)
    assert info["converged"]


@pytest.mark.parametrize("dtype,rtol", [(torch.float64, 1e-11), (torch.float32, 2e-5)])
def test_rmat14_100_iterations(cuda_device, dtype, rtol):
    """Configuration 1: exactly 100 updates from pi_0 = 1/n."""
    a = inputs.rmat_transition(14, 16, 1)
    vals_r = as_f64(torch.from_numpy(a.val).to(dtype))
    ref = oracle.pagerank(a.row_ptr, a.col, vals_r, ALPHA, fixed_iters=100)
    pi, info = _pr(a, dtype, tol=0.0, max_iter=100, history=True)
    assert info["iters"] == 100 and info["converged"]
    np.testing.assert_allclose(pi, ref["pi"], rtol=rtol)
    # residual histories agree until they reach the rounding floor of the dtype
    floor = 1e-13 if dtype == torch.float64 else 1e-6
    np.testing.assert_allclose(info["hist"], ref["resid"], rtol=1e-3 if dtype == torch.float32 else 1e-9,
                               atol=floor)
    n = a.n_rows
    assert abs(pi.sum() - 1) < (1e-12 if dtype == torch.float64 else 1e-5)
    assert pi.min() >= (1 - ALPHA) / n * (1 - 1e-6)


def test_rmat14_tolerance_stop(cuda_device):
    a = inputs.rmat_transition(14, 16, 1)
    ref = oracle.pagerank(a.row_ptr, a.col, a.val, ALPHA, tol=1e-10)
    pi, info = _pr(a, torch.float64, tol=1e-10, history=True)
    assert info["converged"] and abs(info["iters"] - ref["iters"]) <= 1
    assert info["resid"] < 1e-10
    h = info["hist"]
    assert np.all(h[1:] <= ALPHA * h[:-1] * (1 + 1e-6) + 1e-15)     # L1 contraction
    r = oracle.pagerank_residual(a.row_ptr, a.col, a.val, pi, ALPHA)
    assert r < 1.2e-10 * ALPHA


@pytest.mark.parametrize("mode", ["ir_bf16", "ir_f16", "ir_f32"])
def test_mixed_precision_rmat14(cuda_device, mode):
    a = inputs.rmat_transition(14, 16, 1)
    star = oracle.pagerank(a.row_ptr, a.col, a.val, ALPHA, tol=1e-15, max_iter=400)["pi"]
    pi, info = _pr(a, torch.float64, tol=1e-10, mode=mode, inner_sweeps=12, max_iter=50,
                   history=True)
    assert info["converged"], info
    assert info["resid"] < 1e-10
    r = oracle.pagerank_residual(a.row_ptr, a.col, a.val, pi, ALPHA)
    assert r < 1.1e-10, r                                  # the oracle agrees on the residual
    assert np.abs(pi - star).sum() <= r / (1 - ALPHA) + 1e-13   # ||pi - pi*||_1 <= ||r||_1/(1-alpha)
    assert info["iters"] < 20


def test_plain_fp32_floor(cuda_device):
    """All-FP32 power iteration cannot reach an L1 residual of 1e-10: its iterates may stop
    changing in FP32, but each update, measured before it is rounded to FP32, stays about
    one rounding (u ||pi||_1, u = 2^-24) from the iterate, so the solver must report that it
    did not converge; the FP64 residual of its answer, computed by the oracle with the
    master values, stays at the FP32 rounding floor too (Sec. 5.5.1 iteration)."""
    a = inputs.rmat_transition(14, 16, 1)
    pi, info = _pr(a, torch.float32, tol=1e-10, max_iter=300)
    assert not info["converged"] and info["iters"] == 300
    assert 1e-9 < info["resid"] < 1e-6, info["resid"]
    r = oracle.pagerank_residual(a.row_ptr, a.col, a.val, pi, ALPHA)
    assert 1e-9 < r < 1e-5, r


def test_pagerank_errors(cuda_device):
    a = inputs.random_sparse(50, 60, 0.1, 1)
    p, _ = make_plan(a)
    vals = torch.from_numpy(a.val).cuda()
    with pytest.raises(mb.MerbitError) as e:
        mb.pagerank(p, vals)
    assert e.value.status == 1
    b = inputs.rmat_transition(10, 8, 1)
    q, _ = make_plan(b)
    with pytest.raises(mb.MerbitError):
        mb.pagerank(q, torch.from_numpy(b.val).cuda(), mode="ir_bf16", inner_sweeps=0)
    with pytest.raises(mb.MerbitError):
        mb.pagerank(q, torch.from_numpy(b.val).cuda().float(), mode="ir_bf16")
    pi, info = mb.pagerank(q, torch.from_numpy(b.val).cuda(), tol=1e-10, max_iter=5)
    assert not info["converged"] and info["iters"] == 5


def test_full_rmat24_mixed_precision(cuda_device):
    """Configuration 3 at full size: R-MAT scale 24 transition matrix, IR with bf16 inner
    sweeps to L1 residual 1e-10; the oracle's own FP64 residual of the result must agree."""
    a = inputs.rmat_transition(24, 16, 7)
    pi, info = _pr(a, torch.float64, tol=1e-10, mode="ir_bf16", inner_sweeps=16, max_iter=60)
    assert info["converged"]
    r = oracle.pagerank_residual(a.row_ptr, a.col, a.val, pi, ALPHA)
    assert r < 1.1e-10, r
    assert abs(pi.sum() - 1) < 1e-9
