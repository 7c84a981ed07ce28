"""Both block kernels of the product against the float64 oracle, through every family of
epilogue that multiplies by a plan's matrix.  MERBIT_KERNEL_CLASSIC forms the products of
a block with all 256 threads and then reduces it; MERBIT_KERNEL_SPLIT gathers with 256
producer threads while 256 consumer threads reduce the previous block.  Each result must
meet the same bound whichever kernel the plan uses."""
import numpy as np
import pytest
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb
from tests.gpu_helpers import TOL, as_f64, check_rel, make_plan

pytestmark = pytest.mark.gpu
KERNELS = ["classic", "split", "split2"]
DTYPES = [torch.float32, torch.float64]
ALPHA = 0.85


def _plan(a, kernel, sigma=14):
    p, col = make_plan(a, sigma)
    p.set_kernel(kernel)
    return p, col


def _spmv(a, dtype, kernel, sigma=14, calls=2, seed=2):
    p, _ = _plan(a, kernel, sigma)
    vals = torch.from_numpy(a.val).to("cuda", dtype)
    x = torch.from_numpy(inputs.uniform_vector(a.n_cols, seed)).to("cuda", dtype)
    y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(vals), as_f64(x))
    y = torch.full((a.n_rows,), float("nan"), dtype=dtype, device="cuda")
    for _ in range(calls):
        mb.spmv(p, vals, x, y)
    p.sync()
    check_rel(as_f64(y), y_ref, d, TOL[dtype], f"{a.name} {kernel} sigma={sigma}")


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("dtype", DTYPES)
def test_structures_sizes_and_sigma(cuda_device, kernel, dtype):
    """Empty rows and matrices, hub rows longer than a block, rows of exactly tile and
    block size, ragged row counts around the block size, non-square shapes, and the
    plan's sigma at 14, 7 and 1."""
    cases = [inputs.row_lengths_csr([0] * 50, 10, 0, "all_empty"),
             inputs.row_lengths_csr([5000], 8000, 1, "one_hub_row"),
             inputs.row_lengths_csr([0, 0, 3000, 0, 1, 0, 0, 2000, 0], 4000, 2, "hubs_and_empties"),
             inputs.row_lengths_csr([14] * 300 + [448] * 20 + [447, 449, 3583, 3584, 3585], 4000, 4,
                                    "tile_sized_rows"),
             inputs.row_lengths_csr([0] * 3000 + [1] + [0] * 3000, 10, 5, "lone_entry"),
             inputs.random_sparse(700, 20000, 0.001, 3),
             inputs.random_sparse(9000, 40, 0.05, 4)]
    cases += [inputs.random_sparse(n, 257, 0.05, n, empty_frac=0.25) for n in (1, 31, 449, 3585, 20001)]
    for a in cases:
        _spmv(a, dtype, kernel)
    r = inputs.rmat_transition(14, 16, 1)
    for sigma in (14, 7, 1):
        _spmv(r, dtype, kernel, sigma=sigma)


@pytest.mark.parametrize("kernel", KERNELS)
def test_stress_scale16(cuda_device, kernel):
    base = inputs.rmat_uniform(16, 16, 3, 3)
    for a in (base, inputs.empty_rows(base, 0.3, 4), inputs.add_hubs(base, 4, 20000, 60000, 5),
              inputs.erdos_renyi(1 << 16, 16, 6)):
        for dtype in DTYPES:
            _spmv(a, dtype, kernel, calls=3)


@pytest.mark.parametrize("kernel", KERNELS)
def test_reduced_precision_values(cuda_device, kernel):
    """bf16 and scaled f16 values with f32 x and f32 accumulation (products in the slots
    of the column indices)."""
    a = inputs.rmat_transition(14, 16, 1)
    p, _ = _plan(a, kernel)
    x = torch.from_numpy(inputs.uniform_vector(a.n_cols, 2)).to("cuda", torch.float32)
    for fmt, tdt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        lo, k = mb.vals_convert(torch.from_numpy(a.val).cuda(), tdt, auto_scale=(fmt == "f16"))
        y = mb.spmv(p, lo, x, scale_exp=k)
        y_ref, d, _ = oracle.spmv_lowprec_reference(a.row_ptr, a.col, a.val, as_f64(x), fmt)
        check_rel(as_f64(y), y_ref, d, 1e-5, f"{fmt} {kernel}")


@pytest.mark.parametrize("kernel", KERNELS)
def test_pagerank_plain_and_refinement(cuda_device, kernel):
    a = inputs.rmat_transition(14, 16, 1)
    p, _ = _plan(a, kernel)
    v64 = torch.from_numpy(a.val).cuda()
    # 100 FP32 updates from 1/n
    v32 = v64.float()
    ref = oracle.pagerank(a.row_ptr, a.col, as_f64(v32), ALPHA, fixed_iters=100)
    pi, info = mb.pagerank(p, v32, ALPHA, tol=0.0, max_iter=100)
    assert info["iters"] == 100
    np.testing.assert_allclose(as_f64(pi), ref["pi"], rtol=2e-5)
    # FP64 to 1e-10: the oracle's iteration count and residual
    ref = oracle.pagerank(a.row_ptr, a.col, a.val, ALPHA, tol=1e-10)
    pi, info = mb.pagerank(p, v64, ALPHA, tol=1e-10)
    assert info["converged"] and abs(info["iters"] - ref["iters"]) <= 1
    assert oracle.pagerank_residual(a.row_ptr, a.col, a.val, as_f64(pi), ALPHA) < 1.2e-10 * ALPHA
    # refinement with bf16 and f32 inner values
    for mode in ("ir_bf16", "ir_f32"):
        pi, info = mb.pagerank(p, v64, ALPHA, tol=1e-10, mode=mode, inner_sweeps=12, max_iter=50)
        assert info["converged"], (mode, info)
        assert oracle.pagerank_residual(a.row_ptr, a.col, a.val, as_f64(pi), ALPHA) < 1.1e-10


@pytest.mark.parametrize("kernel", KERNELS)
def test_many_graphs(cuda_device, kernel):
    """The block-list epilogue: converged graphs' blocks are skipped."""
    a, off = inputs.rmat_batch(12, 9, scales=(5, 11), edge_factors=(4, 24), threads=4)
    b = mb.Batch(torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col).cuda(), off)
    b.set_kernel(kernel)
    pi, info = b.pagerank(torch.from_numpy(a.val).cuda(), ALPHA, tol=1e-10)
    assert info["converged"]
    pin = as_f64(pi)
    for g in range(off.size - 1):
        lo, hi = int(off[g]), int(off[g + 1])
        k0, k1 = a.row_ptr[lo], a.row_ptr[hi]
        rp = (a.row_ptr[lo:hi + 1] - k0).astype(np.int32)
        col = (a.col[k0:k1] - lo).astype(np.int32)
        ref = oracle.pagerank(rp, col, a.val[k0:k1], ALPHA, tol=1e-10)
        assert abs(int(info["iters"][g]) - ref["iters"]) <= 1
        assert np.abs(pin[lo:hi] - ref["pi"]).sum() <= 1e-10 * ALPHA / (1 - ALPHA) * 1.01 + 1e-13
    b.destroy()


@pytest.mark.parametrize("kernel", KERNELS)
def test_bicgstab_explicit_and_pattern_values(cuda_device, kernel):
    """Epilogue-fused dot products; all-ones values with and without a value stream."""
    a = inputs.road_grid(50, 40, 0.6, 5)
    xt = np.random.default_rng(6).uniform(-1, 1, a.n_rows)
    b = oracle.spmv(a.row_ptr, a.col, a.val, xt)[0]
    ref = oracle.bicgstab(a.row_ptr, a.col, a.val, b, tol=1e-30, max_iter=3)
    p, _ = _plan(a, kernel)
    bt = torch.from_numpy(b).cuda()
    for vals in (torch.from_numpy(a.val).cuda(), None):
        x, info = mb.bicgstab(p, vals, bt, tol=1e-30, max_iter=3)
        np.testing.assert_allclose(info["hist"], ref["resid"], rtol=1e-6)
        x, info = mb.bicgstab(p, vals, bt, tol=1e-10, max_iter=20000)
        assert info["converged"]
        r = np.linalg.norm(b - oracle.spmv(a.row_ptr, a.col, a.val, as_f64(x))[0]) / np.linalg.norm(b)
        assert r <= 1e-9


@pytest.mark.parametrize("kernel", KERNELS)
def test_adjoint(cuda_device, kernel):
    """The adjoint solve multiplies by A^T through its own plan."""
    a = inputs.rmat_transition(12, 16, 3)
    A = mb.autograd.Matrix(torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col).cuda(),
                           a.n_rows, a.n_cols)
    _, pt = A.transposed()
    A.plan.set_kernel(kernel)
    pt.set_kernel(kernel)
    vals = torch.from_numpy(a.val).cuda()
    w = np.random.default_rng(4).standard_normal(a.n_rows)
    lam, info = mb.pagerank_adjoint(A.plan, pt, A.transposed_values(vals), torch.from_numpy(w).cuda(),
                                    alpha=ALPHA, tol=1e-13)
    assert info["converged"]
    ref = oracle.pagerank_adjoint(a.row_ptr, a.col, a.val, w, ALPHA, tol=1e-14)["lambda"]
    # the device stops at ||delta||_1 <= 1e-13 ||w||_1: distance <= that * alpha / (1 - alpha)
    assert np.abs(as_f64(lam) - ref).sum() <= 1e-13 * np.abs(w).sum() * ALPHA / (1 - ALPHA) * 1.01 + 1e-12


def test_kernels_agree_rmat20(cuda_device):
    """R-MAT scale 20: both kernels within the oracle's bound on every row, and the
    global identity sum_i y_i = sum_j x_j colsum_j."""
    a = inputs.rmat_transition(20, 16, 7)
    x64 = inputs.uniform_vector(a.n_cols, 2)
    for dtype in DTYPES:
        vals = torch.from_numpy(a.val).to("cuda", dtype)
        x = torch.from_numpy(x64).to("cuda", dtype)
        y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(vals), as_f64(x))
        colsum = np.bincount(a.col, weights=as_f64(vals), minlength=a.n_cols)
        tot = float(np.dot(colsum, as_f64(x)))
        for kernel in KERNELS:
            p, _ = _plan(a, kernel)
            y = mb.spmv(p, vals, x)
            y = mb.spmv(p, vals, x, y)
            p.sync()
            check_rel(as_f64(y), y_ref, d, TOL[dtype], f"rmat20 {kernel} {dtype}")
            assert abs(float(y.double().sum()) - tot) <= 1e-5 * tot


def test_set_kernel_rejects_unknown(cuda_device):
    a = inputs.rmat_transition(8, 8, 1)
    p, _ = make_plan(a)
    lib = mb.merbit.load()
    assert lib.merbit_plan_set_kernel(p.handle, 4) == 1
    assert lib.merbit_plan_set_kernel(p.handle, -1) == 1
    assert lib.merbit_plan_set_kernel(None, 1) == 1
    p.set_kernel("auto")
