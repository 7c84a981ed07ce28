"""Plans of 4, 8 and 16 tiles per block (the block size W of Sec. 4.2, a tuning parameter).

The TILE arrays do not depend on W; the block rows do (row of the first coordinate of
every block of W tiles), and every block kernel must give the same product for any W:
the plan is compared bit for bit with the oracle, and every row of the SpMV with the
oracle's within the parity bound."""
import numpy as np
import pytest
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb
from tests.gpu_helpers import TOL, as_f64, check_rel

pytestmark = pytest.mark.gpu
ALPHA = 0.85
CASES = {
    "rmat15_hubs": lambda: inputs.add_hubs(inputs.rmat_uniform(15, 16, 3, 3), 2, 10000, 30000, 5),
    "ragged": lambda: inputs.row_lengths_csr([0, 1, 4000, 0, 0, 3, 448, 447, 449, 0, 13, 14, 15] * 37, 5000, 2),
    "empty30": lambda: inputs.empty_rows(inputs.rmat_uniform(14, 16, 4, 4), 0.3, 4),
}


def _plan(a, sigma, W, kernel="auto"):
    rp = torch.from_numpy(a.row_ptr).cuda()
    col = torch.from_numpy(a.col).cuda()
    p = mb.plan(rp, col, a.n_rows, a.n_cols, sigma=sigma, tiles_per_block=W)
    p.set_kernel(kernel)
    return p, col


@pytest.mark.parametrize("W", [4, 16])
@pytest.mark.parametrize("sigma", [14, 7])
@pytest.mark.parametrize("case", sorted(CASES))
def test_plan_block_rows_bit_exact(cuda_device, case, sigma, W):
    a = CASES[case]()
    p, _ = _plan(a, sigma, W)
    t = p.tiles()
    ref = oracle.build_tile(a.row_ptr, sigma)
    assert np.array_equal(t.tile_x, ref["tile_x"]) and np.array_equal(t.tile_y, ref["tile_y"])
    assert np.array_equal(t.lane_desc, ref["lane_desc"])
    br = oracle.block_boundary_rows(ref["tile_y"], ref["tile_num"], W)
    assert np.array_equal(t.block_row.astype(np.int64), br)
    assert p.info().tiles_per_block == W


@pytest.mark.parametrize("kernel", ["classic", "split", "split2"])
@pytest.mark.parametrize("W", [4, 8, 16])
@pytest.mark.parametrize("case", sorted(CASES))
def test_spmv_every_block_size(cuda_device, case, W, kernel):
    a = CASES[case]()
    for sigma in (14, 9):
        p, _ = _plan(a, sigma, W, kernel)
        for dtype in (torch.float32, torch.float64):
            vals = torch.from_numpy(a.val).to("cuda", dtype)
            x = torch.from_numpy(inputs.uniform_vector(a.n_cols, 6)).to("cuda", dtype)
            y = torch.full((a.n_rows,), float("nan"), dtype=dtype, device="cuda")
            for _ in range(2):
                mb.spmv(p, vals, x, y)
            p.sync()
            y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(vals), as_f64(x))
            check_rel(as_f64(y), y_ref, d, TOL[dtype], f"{case} W={W} sigma={sigma} {kernel} {dtype}")
        p.destroy()


@pytest.mark.parametrize("W", [4, 16])
def test_pagerank_and_hot_table_with_block_size(cuda_device, W):
    a = inputs.rmat_transition(15, 16, 1)
    p, _ = _plan(a, 14, W)
    assert p.set_hot_columns(2000)[0] > 0
    v64 = torch.from_numpy(a.val).cuda()
    ref = oracle.pagerank(a.row_ptr, a.col, a.val, ALPHA, tol=0.0, fixed_iters=40)
    pi, _ = mb.pagerank(p, v64, ALPHA, tol=0.0, max_iter=40)
    np.testing.assert_allclose(as_f64(pi), ref["pi"], rtol=1e-12, atol=0)
    pi, info = mb.pagerank(p, v64, ALPHA, tol=1e-10, mode="ir_f32", inner_sweeps=8, max_iter=40)
    assert info["converged"]
    assert oracle.pagerank_residual(a.row_ptr, a.col, a.val, as_f64(pi), ALPHA) < 1.1e-10


def test_block_size_rejections(cuda_device):
    a = inputs.rmat_transition(10, 8, 1)
    rp = torch.from_numpy(a.row_ptr).cuda()
    col = torch.from_numpy(a.col).cuda()
    for W in (0, 2, 7, 32):
        with pytest.raises(mb.MerbitError) as e:
            mb.plan(rp, col, a.n_rows, a.n_cols, tiles_per_block=W)
        assert e.value.status == 1
    p = mb.plan(rp, col, a.n_rows, a.n_cols, tiles_per_block=4)
    vals = torch.from_numpy(a.val).cuda().float()
    with pytest.raises(mb.MerbitError) as e:
        mb.spmm(p, vals, torch.ones(a.n_cols, 4, device="cuda"))
    assert e.value.status == 1


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64, torch.bfloat16])
def test_autotune_searches_sigma_block_kernel_table(cuda_device, dtype):
    a = inputs.rmat_transition(15, 16, 3)
    rp = torch.from_numpy(a.row_ptr).cuda()
    col = torch.from_numpy(a.col).cuda()
    v64 = torch.from_numpy(a.val).cuda()
    vals = mb.vals_convert(v64, dtype)[0] if dtype == torch.bfloat16 else v64.to(dtype)
    best, table = mb.autotune(rp, col, vals, sigmas=(14, 7), blocks=(4, 8, 16),
                              kernels=("classic", "split", "split2"), hots=(0, 1000), reps=2)
    assert len(table) == 2 * 3 * 3 * 2
    timed = {k: v for k, v in table.items() if v is not None}
    assert timed and all(v > 0 for v in timed.values())
    if dtype != torch.float64:
        assert len(timed) == len(table)          # every 4-byte-product combination launches
    key = (best["sigma"], best["tiles_per_block"], best["kernel"], best["hot"])
    assert table[key] == min(timed.values())
    # the chosen configuration gives the oracle's product
    p = mb.plan(rp, col, a.n_rows, a.n_cols, sigma=best["sigma"], tiles_per_block=best["tiles_per_block"])
    p.set_kernel(best["kernel"])
    p.set_hot_columns(best["hot"])
    xdt = torch.float64 if dtype == torch.float64 else torch.float32
    x = torch.from_numpy(inputs.uniform_vector(a.n_cols, 2)).to("cuda", xdt)
    y = mb.spmv(p, vals, x)
    y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(vals), as_f64(x))
    check_rel(as_f64(y), y_ref, d, 1e-12 if dtype == torch.float64 else 1e-5, f"autotuned {best}")


# ---------------------------------------------------------------- 64-bit lane descriptors

@pytest.mark.parametrize("sigma", [15, 21, 28, 42])
@pytest.mark.parametrize("case", sorted(CASES))
def test_plan_64bit_descriptors_bit_exact(cuda_device, case, sigma):
    a = CASES[case]()
    p, _ = _plan(a, sigma, 8)
    assert p.info().desc_bytes == 8
    t = p.tiles()
    ref = oracle.build_tile(a.row_ptr, sigma)
    assert ref["lane_desc"].dtype == np.uint64
    assert np.array_equal(t.tile_x, ref["tile_x"]) and np.array_equal(t.tile_y, ref["tile_y"])
    assert np.array_equal(t.lane_desc, ref["lane_desc"])
    assert np.array_equal(t.block_row.astype(np.int64), oracle.block_boundary_rows(ref["tile_y"], ref["tile_num"], 8))


def _fits_one_cta(sigma, W, value_bytes):
    """Two stages of a block (values, column indices) fit one CTA's 227 KB of shared memory."""
    return 2 * (value_bytes + 4) * (W * 32 * sigma + 32) <= 227 * 1024 - 4096


@pytest.mark.parametrize("kernel", ["classic", "split", "split2"])
@pytest.mark.parametrize("W", [4, 8])
@pytest.mark.parametrize("sigma", [17, 28, 42])
def test_spmv_64bit_descriptors(cuda_device, sigma, W, kernel):
    for case in ("rmat15_hubs", "ragged"):
        a = CASES[case]()
        p, _ = _plan(a, sigma, W, kernel)
        for dtype in (torch.float32, torch.float64):
            vals = torch.from_numpy(a.val).to("cuda", dtype)
            x = torch.from_numpy(inputs.uniform_vector(a.n_cols, 7)).to("cuda", dtype)
            y = torch.full((a.n_rows,), float("nan"), dtype=dtype, device="cuda")
            if not _fits_one_cta(sigma, W, vals.element_size()):
                # no block kernel can hold this plan's stages: a clear EINVAL, nothing launched
                with pytest.raises(mb.MerbitError) as e:
                    mb.spmv(p, vals, x, y)
                assert e.value.status == 1 and "shared memory" in str(e.value)
                continue
            for _ in range(2):
                mb.spmv(p, vals, x, y)
            p.sync()
            y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(vals), as_f64(x))
            check_rel(as_f64(y), y_ref, d, TOL[dtype], f"{case} sigma={sigma} W={W} {kernel} {dtype}")
        p.destroy()


def test_pagerank_and_gradient_on_64bit_plan(cuda_device):
    a = inputs.rmat_transition(14, 16, 1)
    p, _ = _plan(a, 28, 4)
    v64 = torch.from_numpy(a.val).cuda()
    pi, info = mb.pagerank(p, v64, ALPHA, tol=1e-10, mode="ir_bf16", inner_sweeps=12, max_iter=40)
    assert info["converged"]
    assert oracle.pagerank_residual(a.row_ptr, a.col, a.val, as_f64(pi), ALPHA) < 1.1e-10
    # per-nonzero products g[row] x[col] walk the 64-bit descriptors
    g = torch.from_numpy(inputs.uniform_vector(a.n_rows, 3)).cuda()
    x = torch.from_numpy(inputs.uniform_vector(a.n_cols, 4)).cuda()
    out = mb.sddmm(p, g, x, 1.0)
    np.testing.assert_array_equal(as_f64(out), oracle.sddmm(a.row_ptr, a.col, as_f64(g), as_f64(x)))


def test_64bit_plans_rejected_where_unsupported(cuda_device):
    a = inputs.rmat_transition(12, 8, 1)
    rp = torch.from_numpy(a.row_ptr).cuda()
    col = torch.from_numpy(a.col).cuda()
    p = mb.plan(rp, col, sigma=20)
    vals = torch.from_numpy(a.val).cuda().float()
    with pytest.raises(mb.MerbitError):
        mb.spmm(p, vals, torch.ones(a.n_cols, 4, device="cuda"))
    with pytest.raises(mb.MerbitError):
        mb.Batch(rp, col, np.array([0, a.n_rows]), sigma=20)
    with pytest.raises(mb.MerbitError):
        mb.plan(rp, col, sigma=43)
