"""Batched product Y = A X (merbit_spmm) against the float64 oracle, per entry
|dY_ij| <= 1e-5 * sum_k |a_ik X_kj|."""
import numpy as np
import pytest
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb
from tests.gpu_helpers import as_f64, check_rel, make_plan

pytestmark = pytest.mark.gpu


def _run(a, k, ldx=None, seed=3, calls=1):
    p, _ = make_plan(a)
    vals = torch.from_numpy(a.val).to("cuda", torch.float32)
    rng = np.random.default_rng(seed)
    ldx = ldx or k
    Xfull = torch.from_numpy(rng.random((a.n_cols, ldx))).to("cuda", torch.float32)
    X = Xfull[:, :k]
    Y = torch.full((a.n_rows, k), float("nan"), device="cuda")
    for _ in range(calls):
        mb.spmm(p, vals, X, Y)
    p.sync()
    Yr, D = oracle.spmm(a.row_ptr, a.col, as_f64(vals), as_f64(X))
    check_rel(as_f64(Y).ravel(), Yr.ravel(), D.ravel(), 1e-5, f"{a.name} k={k}")
    return Y


@pytest.mark.parametrize("k", [1, 2, 3, 4, 8, 12, 13, 16, 32, 36, 40])
def test_spmm_rmat14(cuda_device, k):
    _run(inputs.rmat_transition(14, 16, 1), k)


def test_spmm_structures(cuda_device):
    cases = [inputs.row_lengths_csr([0] * 50, 10, 0, "all_empty"),
             inputs.row_lengths_csr([5000], 8000, 1, "one_hub_row"),
             inputs.row_lengths_csr([0, 0, 3000, 0, 1, 0, 0, 2000, 0], 4000, 2, "hubs_and_empties"),
             inputs.row_lengths_csr([14] * 300 + [448] * 20 + [447, 449, 3583, 3584, 3585], 4000, 4),
             inputs.random_sparse(3001, 257, 0.05, 7, empty_frac=0.3)]
    for a in cases:
        for k in (8, 32):
            _run(a, k)


def test_spmm_strided_and_repeated(cuda_device):
    a = inputs.add_hubs(inputs.rmat_uniform(14, 16, 3, 3), 2, 5000, 9000, 5)
    _run(a, 24, ldx=37, calls=3)
    _run(a, 8, ldx=8, calls=2, seed=9)


def test_spmm_matches_spmv_columns(cuda_device):
    """Column j of A X equals the SpMV of column j (both through the device)."""
    a = inputs.rmat_transition(13, 16, 2)
    p, _ = make_plan(a)
    vals = torch.from_numpy(a.val).cuda().float()
    X = torch.rand(a.n_cols, 8, device="cuda")
    Y = mb.spmm(p, vals, X)
    for j in range(8):
        y = mb.spmv(p, vals, X[:, j].contiguous())
        torch.testing.assert_close(Y[:, j], y, rtol=2e-5, atol=1e-6)


@pytest.mark.parametrize("k", [8, 32])
def test_spmm_full_rmat22(cuda_device, k):
    """Configuration 4(a) size: R-MAT scale 22 transition matrix; every row of every column
    against the oracle."""
    a = inputs.rmat_transition(22, 16, 7)
    p, _ = make_plan(a)
    vals = torch.from_numpy(a.val).cuda().float()
    X = torch.rand(a.n_cols, k, device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    Y = mb.spmm(p, vals, X)
    torch.cuda.synchronize()
    Xh = as_f64(X)
    vh = as_f64(vals)
    Yh = as_f64(Y)
    for j in range(k):
        yr, d = oracle.spmv(a.row_ptr, a.col, vh, Xh[:, j])
        check_rel(Yh[:, j], yr, d, 1e-5, f"col {j}")
    # every column's total equals sum_j colsum_j * X_j (all entries written)
    colsum = np.bincount(a.col, weights=vh, minlength=a.n_cols)
    tot = colsum @ Xh
    assert np.allclose(Yh.sum(axis=0), tot, rtol=1e-5)


def test_spmm_wide(cuda_device):
    """k = 300: nine 32-column chunks and a 12-column remainder in a 16-column chunk."""
    _run(inputs.rmat_transition(11, 16, 5), 300)


@pytest.mark.parametrize("k,ldx,shift", [(16, 16, 0), (16, 16, 4), (32, 36, 0), (24, 24, 0), (48, 56, 8)])
def test_spmm_slice_widths(cuda_device, k, ldx, shift):
    # 32-byte slices need k and ldx multiples of 8 and X 32-byte aligned; a 16-byte shift
    # of X, or ldx = 36, takes the 16-byte slices, and k = 24 mixes both (chunks 16 + 8)
    a = inputs.add_hubs(inputs.rmat_uniform(13, 16, 3, 3), 2, 3000, 6000, 5)
    p, _ = make_plan(a)
    vals = torch.from_numpy(a.val).to("cuda", torch.float32)
    rng = np.random.default_rng(k + ldx + shift)
    buf = torch.from_numpy(rng.random(a.n_cols * ldx + 64)).to("cuda", torch.float32)
    X = buf[shift:shift + a.n_cols * ldx].view(a.n_cols, ldx)[:, :k]
    Y = torch.full((a.n_rows, k), float("nan"), device="cuda")
    mb.spmm(p, vals, X, Y)
    p.sync()
    Yr, D = oracle.spmm(a.row_ptr, a.col, as_f64(vals), as_f64(X))
    check_rel(as_f64(Y).ravel(), Yr.ravel(), D.ravel(), 1e-5, f"k={k} ldx={ldx} shift={shift}")
