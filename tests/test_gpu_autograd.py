"""Differentiation through the C ABI against the float64 oracle: the transpose (bit-exact),
the per-nonzero products, SpMV gradients, and PageRank value gradients by the implicit
adjoint (against the oracle's gradient and against central finite differences)."""
import numpy as np
import pytest
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb
from paper_2605_07391_gb300 import autograd as ag
from tests.gpu_helpers import as_f64

pytestmark = pytest.mark.gpu

ALPHA = 0.85


def _dev(a):
    return torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col).cuda()


def _cases():
    return [inputs.rmat_transition(14, 16, 1),
            inputs.random_sparse(3001, 257, 0.05, 7, empty_frac=0.3),
            inputs.random_sparse(50, 4000, 0.02, 3),
            inputs.row_lengths_csr([0, 0, 3000, 0, 1, 0, 0, 2000, 0], 4000, 2, "hubs_and_empties"),
            inputs.row_lengths_csr([0] * 40, 10, 0, "all_empty"),
            inputs.rmat_uniform(18, 8, 3, 3)]          # 2^18 columns: three radix passes


def test_transpose_bit_exact(cuda_device):
    for a in _cases():
        rp, col = _dev(a)
        t = mb.transpose(rp, col, a.n_rows, a.n_cols)
        ref_rp, ref_ct, ref_perm = oracle.transpose_csr(a.row_ptr, a.col, a.n_cols)
        torch.cuda.synchronize()
        assert np.array_equal(t.row_ptr_t.cpu().numpy(), ref_rp), a.name
        assert np.array_equal(t.col_t.cpu().numpy(), ref_ct), a.name
        assert np.array_equal(t.perm.cpu().numpy(), ref_perm), a.name
        t.destroy()


def test_gather_and_transposed_spmv(cuda_device):
    a = inputs.random_sparse(2000, 700, 0.03, 5, empty_frac=0.2)
    rp, col = _dev(a)
    t = mb.transpose(rp, col, a.n_rows, a.n_cols)
    for dt in (torch.float32, torch.float64):
        vals = torch.from_numpy(a.val).to("cuda", dt)
        vt = mb.gather(vals, t.perm)
        assert torch.equal(vt.cpu(), vals.cpu()[t.perm.cpu().long()])
    pt = t.plan()
    g = torch.rand(a.n_rows, device="cuda", dtype=torch.float64)
    y = mb.spmv(pt, mb.gather(torch.from_numpy(a.val).cuda(), t.perm), g)
    rt, ct, perm = oracle.transpose_csr(a.row_ptr, a.col, a.n_cols)
    ref, d = oracle.spmv(rt, ct, a.val[perm], as_f64(g))
    assert np.all(np.abs(as_f64(y) - ref) <= 1e-12 * d + 1e-300)


def test_sddmm(cuda_device):
    a = inputs.rmat_transition(14, 16, 2)
    p = mb.plan(*_dev(a), a.n_rows, a.n_cols)
    rng = np.random.default_rng(3)
    g, x = rng.standard_normal(a.n_rows), rng.standard_normal(a.n_cols)
    out = mb.sddmm(p, torch.from_numpy(g).cuda(), torch.from_numpy(x).cuda(), 0.85)
    ref = oracle.sddmm(a.row_ptr, a.col, g, x, 0.85)
    assert np.array_equal(as_f64(out), ref)                     # same two FP64 roundings
    out32 = mb.sddmm(p, torch.from_numpy(g).cuda().float(), torch.from_numpy(x).cuda().float())
    np.testing.assert_allclose(as_f64(out32), oracle.sddmm(a.row_ptr, a.col, g, x), rtol=3e-7, atol=0)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_spmv_autograd(cuda_device, dt):
    a = inputs.add_hubs(inputs.rmat_uniform(13, 16, 4, 3), 2, 3000, 5000, 6)
    A = ag.Matrix(*_dev(a), a.n_rows, a.n_cols)
    rng = np.random.default_rng(4)
    vals = torch.from_numpy(a.val).to("cuda", dt).requires_grad_()
    x = torch.from_numpy(rng.random(a.n_cols)).to("cuda", dt).requires_grad_()
    w = torch.from_numpy(rng.standard_normal(a.n_rows)).to("cuda", dt)
    (ag.spmv(A, vals, x) * w).sum().backward()
    gv_ref = oracle.sddmm(a.row_ptr, a.col, as_f64(w), as_f64(x))
    rt, ct, perm = oracle.transpose_csr(a.row_ptr, a.col, a.n_cols)
    gx_ref, d = oracle.spmv(rt, ct, as_f64(vals)[perm], as_f64(w))
    tol = 1e-12 if dt == torch.float64 else 1e-5
    assert np.all(np.abs(as_f64(vals.grad) - gv_ref) <= tol * np.abs(gv_ref) + 1e-300)
    assert np.all(np.abs(as_f64(x.grad) - gx_ref) <= tol * d + 1e-300)


def _pr_grad(a, dt, w):
    A = ag.Matrix(*_dev(a), a.n_rows, a.n_cols)
    vals = torch.from_numpy(a.val).to("cuda", dt).requires_grad_()
    pi = ag.pagerank(A, vals, ALPHA)
    (pi * torch.from_numpy(w).to("cuda", dt)).sum().backward()
    return as_f64(vals.grad), as_f64(pi.detach())


@pytest.mark.parametrize("dt, bound", [(torch.float64, 1e-9), (torch.float32, 1e-4)])
def test_pagerank_gradient_rmat14(cuda_device, dt, bound):
    """Relative L1 distance to the FP64 oracle's gradient alpha lambda[row] pi[col]:
    FP64 at 1e-9; FP32 within 1e-4 (tolerances 1e-7 on pi and 1e-6 relative on lambda,
    amplified by at most 1/(1 - alpha) each)."""
    a = inputs.rmat_transition(14, 16, 1)
    w = np.random.default_rng(7).standard_normal(a.n_rows)
    g, _ = _pr_grad(a, dt, w)
    ref = oracle.pagerank_value_gradient(a.row_ptr, a.col, a.val, w, ALPHA)["grad"]
    rel = np.abs(g - ref).sum() / np.abs(ref).sum()
    assert rel <= bound, rel


def test_pagerank_gradient_finite_differences(cuda_device):
    """64 random values of an R-MAT scale 10 transition matrix: the device's FP64 gradient
    against central differences of the FP64 oracle's loss, step 1e-3."""
    a = inputs.rmat_transition(10, 16, 2)
    rng = np.random.default_rng(5)
    w = rng.standard_normal(a.n_rows)
    g, _ = _pr_grad(a, torch.float64, w)
    h = 1e-3
    for k in rng.choice(a.nnz, 64, replace=False):
        e = np.zeros(a.nnz)
        e[k] = h
        lp = float(w @ oracle.pagerank(a.row_ptr, a.col, a.val + e, ALPHA, tol=1e-15, max_iter=100000)["pi"])
        lm = float(w @ oracle.pagerank(a.row_ptr, a.col, a.val - e, ALPHA, tol=1e-15, max_iter=100000)["pi"])
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-4 * abs(g[k]) + 1e-9, (k, fd, g[k])


def test_pagerank_adjoint_errors(cuda_device):
    a = inputs.rmat_transition(8, 8, 1)
    A = ag.Matrix(*_dev(a), a.n_rows, a.n_cols)
    t, pt = A.transposed()
    vals = torch.from_numpy(a.val).cuda()
    w = torch.ones(a.n_rows, device="cuda", dtype=torch.float64)
    with pytest.raises(mb.MerbitError, match="EINVAL"):
        mb.pagerank_adjoint(A.plan, pt, A.transposed_values(vals), w, alpha=1.0)
    rect = inputs.random_sparse(30, 20, 0.2, 1)
    R = ag.Matrix(*_dev(rect), rect.n_rows, rect.n_cols)
    with pytest.raises(mb.MerbitError, match="EINVAL"):
        mb.pagerank_adjoint(R.plan, R.transposed()[1], R.transposed_values(torch.from_numpy(rect.val).cuda()),
                            torch.ones(20, device="cuda", dtype=torch.float64))
    lam, info = mb.pagerank_adjoint(A.plan, pt, A.transposed_values(vals), w, tol=1e-30, max_iter=3)
    assert not info["converged"] and info["iters"] == 3


def test_pagerank_gradient_rmat20(cuda_device):
    """The differentiation workload: R-MAT scale 20, FP32 values, L = sum_i w_i pi_i with
    w ~ N(0, 1); the device gradient of every value against the FP64 oracle's, and 64
    random values against central differences (step 1e-3) of the device's FP64 PageRank."""
    a = inputs.rmat_transition(20, 16, 3)
    rng = np.random.default_rng(20)
    w = rng.standard_normal(a.n_rows)
    g32, _ = _pr_grad(a, torch.float32, w)
    ref = oracle.pagerank_value_gradient(a.row_ptr, a.col, a.val, w, ALPHA, tol=1e-11)["grad"]
    rel = np.abs(g32 - ref).sum() / np.abs(ref).sum()
    assert rel <= 1e-4, rel
    A = ag.Matrix(*_dev(a), a.n_rows, a.n_cols)
    v64 = torch.from_numpy(a.val).cuda()
    wt = torch.from_numpy(w).cuda()
    h = 1e-3
    for k in rng.choice(a.nnz, 64, replace=False):
        vp, vm = v64.clone(), v64.clone()
        vp[k] += h
        vm[k] -= h
        lp = float((mb.pagerank(A.plan, vp, ALPHA, tol=1e-14, max_iter=2000)[0] * wt).sum())
        lm = float((mb.pagerank(A.plan, vm, ALPHA, tol=1e-14, max_iter=2000)[0] * wt).sum())
        fd = (lp - lm) / (2 * h)
        assert abs(fd - ref[k]) <= 2e-3 * abs(ref[k]) + 1e-10, (k, fd, ref[k])
        assert abs(g32[k] - ref[k]) <= 1e-2 * abs(ref[k]) + 1e-10, (k, g32[k], ref[k])


def test_gradcheck_spmv_and_pagerank(cuda_device):
    """torch.autograd.gradcheck of both wrappers in FP64 on small graphs: the analytic
    backward (transpose SpMV, per-nonzero products, adjoint solve) against torch's own
    central differences of the forward."""
    a = inputs.random_graph_transition(24, 0.15, 8)
    A = ag.Matrix(*_dev(a), a.n_rows, a.n_cols)
    rng = np.random.default_rng(8)
    vals = torch.from_numpy(a.val).cuda().requires_grad_()
    x = torch.from_numpy(rng.random(a.n_cols)).cuda().requires_grad_()
    assert torch.autograd.gradcheck(lambda v, xx: ag.spmv(A, v, xx), (vals, x), eps=1e-6, atol=1e-8)
    w = torch.from_numpy(rng.standard_normal(a.n_rows)).cuda()
    assert torch.autograd.gradcheck(lambda v: (ag.pagerank(A, v, 0.85, tol=1e-14) * w).sum(), (vals,),
                                    eps=1e-6, atol=1e-8)
