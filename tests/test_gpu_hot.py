"""The plan's hot-column table (x values of the most used columns in shared memory).

The products taken from the table must match the plain gather: every row of the SpMV
against the oracle within the parity bound, for each block kernel and value type, with
tables that fit every kernel, tables too large for some kernels (those launches stream the
plain column array) and degenerate tables.  The selection rule is checked exactly against
a recount of the column uses."""
import numpy as np
import pytest
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb
from tests.gpu_helpers import TOL, as_f64, check_rel

pytestmark = pytest.mark.gpu
ALPHA = 0.85


def _expected_table(a, max_hot, min_cover=0.0):
    """The selection rule: the smallest threshold t >= 2 such that at most max_hot columns
    are used t times or more; those columns form the table if they hold min_cover of the
    nonzeros."""
    cnt = np.bincount(a.col, minlength=a.n_cols)
    if max_hot <= 0 or a.nnz == 0:
        return 0, 0.0
    top = 65535
    capped = np.minimum(cnt, top)
    t = top
    while t > 2 and np.count_nonzero(capped >= t - 1) <= max_hot:
        t -= 1
    sel = cnt[capped >= t]
    if sel.size == 0:
        return 0, 0.0
    sel = np.sort(sel)[::-1][:max_hot]
    cover = float(sel.sum()) / a.nnz
    return (int(sel.size), cover) if cover >= min_cover else (0, 0.0)


def _plan(a, sigma=14, kernel="auto"):
    rp = torch.from_numpy(a.row_ptr).cuda()
    col = torch.from_numpy(a.col).cuda()
    p = mb.plan(rp, col, a.n_rows, a.n_cols, sigma=sigma)
    p.set_kernel(kernel)
    return p, col


def _spmv_check(p, a, dtype, seed=2, what=""):
    vals = torch.from_numpy(a.val).to("cuda", dtype)
    x = torch.from_numpy(inputs.uniform_vector(a.n_cols, seed)).to("cuda", dtype)
    y = torch.full((a.n_rows,), float("nan"), dtype=dtype, device="cuda")
    for _ in range(2):
        mb.spmv(p, vals, x, y)
    p.sync()
    y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(vals), as_f64(x))
    check_rel(as_f64(y), y_ref, d, TOL[dtype], what)


@pytest.mark.parametrize("max_hot", [1, 64, 1000, 7000])
def test_selection_rule_exact(cuda_device, max_hot):
    a = inputs.rmat_uniform(16, 16, 3, 3)
    p, _ = _plan(a)
    n, cover = p.set_hot_columns(max_hot)
    en, ecover = _expected_table(a, max_hot)
    assert n == en and abs(cover - ecover) < 1e-12
    assert n <= max_hot
    assert p.set_hot_columns(max_hot, min_cover=min(1.0, ecover + 1e-6)) == (0, 0.0)
    assert p.set_hot_columns(0) == (0, 0.0)


@pytest.mark.parametrize("kernel", ["split", "split2", "classic"])
@pytest.mark.parametrize("sigma", [14, 10, 7])
def test_spmv_with_table_both_kernels(cuda_device, kernel, sigma):
    a = inputs.add_hubs(inputs.rmat_uniform(16, 16, 3, 3), 2, 20000, 40000, 5)
    p, _ = _plan(a, sigma, kernel)
    for max_hot in (4000, 1):
        n, cover = p.set_hot_columns(max_hot)
        assert 0 < n <= max_hot and cover > 0
        for dtype in (torch.float32, torch.float64):
            _spmv_check(p, a, dtype, what=f"{kernel} sigma={sigma} hot={n} {dtype}")


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_spmv_16bit_values_with_table(cuda_device, dtype):
    a = inputs.rmat_uniform(15, 16, 7, 7)
    p, _ = _plan(a)
    assert p.set_hot_columns(3000)[0] > 0
    v64 = torch.from_numpy(a.val).cuda()
    lo, k = mb.vals_convert(v64, dtype)
    x = torch.from_numpy(inputs.uniform_vector(a.n_cols, 5)).cuda().float()
    y = mb.spmv(p, lo, x, scale_exp=k) if k else mb.spmv(p, lo, x)
    y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(lo) * 2.0 ** -k, as_f64(x))
    check_rel(as_f64(y), y_ref, d, 1e-5, f"{dtype} values")


def test_table_larger_than_any_kernel_fits(cuda_device):
    """A table of 2^17 columns fits no block kernel's shared memory: every launch streams
    the plain column array and the products stay exact."""
    a = inputs.rmat_uniform(18, 4, 9, 9)
    p, _ = _plan(a)
    n, _ = p.set_hot_columns(1 << 17)
    assert n > 60000
    for dtype in (torch.float32, torch.float64):
        _spmv_check(p, a, dtype, what=f"oversized table {dtype}")


def test_degenerate_tables(cuda_device):
    # every nonzero in one of three columns: the table holds all of them
    lens = [0, 3, 1, 0, 2, 3, 3, 0, 1, 2] * 500
    rng = np.random.default_rng(3)
    row_ptr = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    col = np.concatenate([np.sort(rng.choice(3, size=l, replace=False)) for l in lens if l]).astype(np.int32)
    a = inputs.CSR(len(lens), 3, row_ptr.astype(np.int32), col, 1.0 - rng.random(col.size), "three_cols")
    p, _ = _plan(a)
    n, cover = p.set_hot_columns(16)
    assert n == 3 and cover == 1.0
    for kernel in ("split", "split2", "classic"):
        p.set_kernel(kernel)
        _spmv_check(p, a, torch.float32, what=f"three columns {kernel}")
    # every column used once: no column qualifies
    b = inputs.from_dense(np.eye(300) * 2.0)
    q, _ = _plan(b)
    assert q.set_hot_columns(100) == (0, 0.0)
    _spmv_check(q, b, torch.float32, what="identity")


def test_pagerank_and_refinement_with_table(cuda_device):
    a = inputs.rmat_transition(16, 16, 1)
    p, _ = _plan(a)
    assert p.set_hot_columns(4000)[0] > 0
    v64 = torch.from_numpy(a.val).cuda()
    ref = oracle.pagerank(a.row_ptr, a.col, a.val, ALPHA, tol=0.0, fixed_iters=60)
    pi, info = mb.pagerank(p, v64, ALPHA, tol=0.0, max_iter=60)
    np.testing.assert_allclose(as_f64(pi), ref["pi"], rtol=1e-12, atol=0)
    for mode in ("ir_bf16", "ir_f32"):
        pi, info = mb.pagerank(p, v64, ALPHA, tol=1e-10, mode=mode, inner_sweeps=12, max_iter=50)
        assert info["converged"], (mode, info)
        r = oracle.pagerank_residual(a.row_ptr, a.col, a.val, as_f64(pi), ALPHA)
        assert r < 1.1e-10, (mode, r)


def test_full_rmat24_f32_with_table(cuda_device):
    """The bench's product at full size with the table: every row against the oracle."""
    a = inputs.rmat_transition(24, 16, 7)
    p, _ = _plan(a)
    n, cover = p.set_hot_columns(8192)
    assert n > 1000 and cover > 0.1, (n, cover)
    _spmv_check(p, a, torch.float32, what="rmat24 f32 with table")


@pytest.mark.parametrize("kernel", ["split", "split2"])
@pytest.mark.parametrize("max_hot", [0, 3000])
def test_gather_probe_sums_every_gather(cuda_device, max_hot, kernel):
    """The gather probe loads x[col[k]] once per nonzero (from the table for hot columns):
    its per-CTA sums add up to sum_c uses(c) x[c]."""
    a = inputs.rmat_uniform(16, 16, 3, 3)
    p, _ = _plan(a, 14, kernel)
    p.set_hot_columns(max_hot)
    cnt = np.bincount(a.col, minlength=a.n_cols).astype(np.float64)
    for dtype, tol in ((torch.float32, 1e-5), (torch.float64, 1e-12)):
        x = torch.from_numpy(inputs.uniform_vector(a.n_cols, 8)).to("cuda", dtype)
        sink = p.gather_probe(x)
        torch.cuda.synchronize()
        want = float(cnt @ as_f64(x))
        assert abs(float(sink.double().sum()) - want) <= tol * want

