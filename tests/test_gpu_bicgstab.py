"""BiCGSTAB on the device (merbit_bicgstab, one CUDA-graph launch) against the float64
oracle: the same recurrence step for step on well-conditioned systems, the residual
history's first iterations on the graph workloads, and the oracle's own residual
||b - A x||_2 / ||b||_2 of the device's answer."""
import numpy as np
import pytest
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb
from tests.gpu_helpers import as_f64

pytestmark = pytest.mark.gpu


def _solve(a, b, tol=1e-10, max_iter=20000, x0=None, sigma=14):
    p = mb.plan(torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col).cuda(), a.n_rows,
                a.n_cols, sigma=sigma)
    vals = torch.from_numpy(a.val).cuda()
    x = None if x0 is None else torch.from_numpy(np.asarray(x0, np.float64)).cuda()
    x, info = mb.bicgstab(p, vals, torch.from_numpy(b).cuda(), x, tol=tol, max_iter=max_iter)
    return as_f64(x), info


def _true_resid(a, b, x):
    return np.linalg.norm(b - oracle.spmv(a.row_ptr, a.col, a.val, x)[0]) / np.linalg.norm(b)


def _diag_dominant(n, seed):
    """A strictly diagonally dominant nonsymmetric matrix: a random sparse -B plus a
    diagonal larger than B's row sums."""
    base = inputs.random_sparse(n, n, 0.003, seed)
    d = np.zeros(n)
    rows = np.repeat(np.arange(n), np.diff(base.row_ptr))
    np.add.at(d, rows, np.abs(base.val))
    # strictly diagonally dominant: A = B - D' with |diag| > row sums
    keys = {(int(r), int(c)): -v for r, c, v in zip(rows, base.col, base.val)}
    for r in range(n):
        keys[(r, r)] = keys.get((r, r), 0.0) + d[r] + 1.0
    rr = np.array([k[0] for k in keys]); cc = np.array([k[1] for k in keys])
    vv = np.array(list(keys.values()))
    order = np.lexsort((cc, rr))
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rr, minlength=n), out=rp[1:])
    return inputs.CSR(n, n, rp.astype(np.int32), cc[order].astype(np.int32), vv[order], "diagdom")


@pytest.mark.parametrize("seed", range(3))
def test_bicgstab_well_conditioned(cuda_device, seed):
    rng = np.random.default_rng(seed)
    a = _diag_dominant(3000, seed)
    b = rng.standard_normal(a.n_rows)
    x, info = _solve(a, b, tol=1e-12)
    ref = oracle.bicgstab(a.row_ptr, a.col, a.val, b, tol=1e-12)
    assert info["converged"] and info["status"] == 1
    assert abs(info["iters"] - ref["iters"]) <= 1
    np.testing.assert_allclose(info["hist"][:5], ref["resid"][:5], rtol=1e-9)
    np.testing.assert_allclose(x, ref["x"], rtol=1e-9, atol=1e-12)
    assert _true_resid(a, b, x) <= 2e-12


@pytest.mark.parametrize("make", [lambda: inputs.road_grid(60, 50, 0.6, 1),
                                  lambda: inputs.kmer_chains(4000, 32, 0.02, 2),
                                  lambda: inputs.hub_graph(12, 2, 3)])
def test_bicgstab_graph_workloads(cuda_device, make):
    """A = adjacency (values 1), b = A x_true with x_true ~ U[-1, 1].  These indefinite
    systems make BiCGSTAB erratic (near-zero denominators amplify the rounding of a
    different summation order within a few iterations), so only the first residuals are
    compared step for step; the device's answer must meet the tolerance in the oracle's
    own FP64 residual (with slack for the drift of the recurrence's residual from the true
    one over thousands of iterations) in a similar number of iterations."""
    a = make()
    xt = np.random.default_rng(1).uniform(-1, 1, a.n_rows)
    b = oracle.spmv(a.row_ptr, a.col, a.val, xt)[0]
    x, info = _solve(a, b)
    ref = oracle.bicgstab(a.row_ptr, a.col, a.val, b, tol=1e-10, max_iter=20000)
    assert info["converged"], info["resid"]
    np.testing.assert_allclose(info["hist"][:3], ref["resid"][:3], rtol=1e-6)
    assert _true_resid(a, b, x) <= 1e-9
    assert 0.5 * ref["iters"] <= info["iters"] <= 2 * ref["iters"]


def test_bicgstab_edge_cases(cuda_device):
    a = inputs.road_grid(30, 30, 0.6, 4)
    xt = np.random.default_rng(2).uniform(-1, 1, a.n_rows)
    b = oracle.spmv(a.row_ptr, a.col, a.val, xt)[0]
    # the exact solution as initial guess: converged before the first iteration
    x, info = _solve(a, b, x0=xt)
    assert info["converged"] and info["iters"] == 0
    np.testing.assert_array_equal(x, xt)
    # b = 0 with x0 = 0
    x, info = _solve(a, np.zeros(a.n_rows))
    assert info["converged"] and info["iters"] == 0 and not x.any()
    # max_iter reached, on a system where the recurrence is stable step for step
    d = _diag_dominant(2000, 7)
    bd = np.random.default_rng(3).standard_normal(d.n_rows)
    ref = oracle.bicgstab(d.row_ptr, d.col, d.val, bd, tol=1e-30, max_iter=6)
    for sigma in (14, 7):
        x, info = _solve(d, bd, tol=1e-30, max_iter=6, sigma=sigma)
        assert not info["converged"] and info["status"] == 2 and info["iters"] == 6
        np.testing.assert_allclose(info["hist"], ref["resid"], rtol=1e-9)
        np.testing.assert_allclose(x, ref["x"], rtol=1e-9, atol=1e-12)


def test_bicgstab_pattern_only_matches_unit_values(cuda_device):
    """vals = NULL (all values 1, no value stream) runs the same recurrence as explicit
    unit values."""
    a = inputs.road_grid(50, 40, 0.6, 5)
    xt = np.random.default_rng(6).uniform(-1, 1, a.n_rows)
    b = oracle.spmv(a.row_ptr, a.col, a.val, xt)[0]
    p = mb.plan(torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col).cuda(), a.n_rows, a.n_cols)
    bt = torch.from_numpy(b).cuda()
    x1, i1 = mb.bicgstab(p, torch.from_numpy(a.val).cuda(), bt, tol=1e-30, max_iter=4)
    x0, i0 = mb.bicgstab(p, None, bt, tol=1e-30, max_iter=4)
    np.testing.assert_allclose(i0["hist"], i1["hist"], rtol=1e-12)
    np.testing.assert_allclose(as_f64(x0), as_f64(x1), rtol=1e-11, atol=1e-13)
    xc, ic = mb.bicgstab(p, None, bt)
    assert ic["converged"] and _true_resid(a, b, as_f64(xc)) <= 1e-9
