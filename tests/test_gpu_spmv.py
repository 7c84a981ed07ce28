"""MERBIT SpMV (Sec. 4.2) against the float64 oracle: |dy_i| <= tol * sum_j |a_ij x_j|."""
import numpy as np
import pytest
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb
from tests.gpu_helpers import TOL, as_f64, check_rel, make_plan

pytestmark = pytest.mark.gpu
DTYPES = [torch.float32, torch.float64]


def _run(a, dtype, x=None, sigma=14, calls=1, seed=2):
    p, col = make_plan(a, sigma)
    vals = torch.from_numpy(a.val).to("cuda", dtype)
    if x is None:
        x = inputs.uniform_vector(a.n_cols, seed)
    xd = torch.from_numpy(np.asarray(x)).to("cuda", dtype)
    # the oracle sees exactly the rounded inputs the device sees
    vr, xr = as_f64(vals), as_f64(xd)
    y_ref, d = oracle.spmv(a.row_ptr, a.col, vr, xr)
    y = torch.full((a.n_rows,), float("nan"), dtype=dtype, device="cuda")
    for _ in range(calls):
        mb.spmv(p, vals, xd, y)
    torch.cuda.synchronize()
    p.sync()
    return check_rel(as_f64(y), y_ref, d, TOL[dtype], a.name)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("seed", range(4))
def test_spmv_small_dense(cuda_device, dtype, seed):
    rng = np.random.default_rng(seed)
    n_rows, n_cols = [(1, 1), (7, 64), (64, 64), (33, 5)][seed]
    a = inputs.random_sparse(n_rows, n_cols, 0.3, seed, empty_frac=0.2)
    _run(a, dtype, x=rng.standard_normal(n_cols))


@pytest.mark.parametrize("dtype", DTYPES)
def test_spmv_special(cuda_device, dtype):
    rng = np.random.default_rng(7)
    n = 1000
    x = rng.standard_normal(n)
    perm = rng.permutation(n)
    P = np.zeros((n, n))
    P[np.arange(n), perm] = 1.0
    mats = [inputs.from_dense(np.eye(n), "eye"), inputs.from_dense(P, "perm"),
            inputs.from_dense(np.diag(rng.random(n) + 0.5), "diag")]
    for a in mats:
        _run(a, dtype, x=x)
    # identity is exact
    a = mats[0]
    p, _ = make_plan(a)
    xd = torch.from_numpy(x).to("cuda", dtype)
    y = mb.spmv(p, torch.from_numpy(a.val).to("cuda", dtype), xd)
    assert torch.equal(y, xd)


@pytest.mark.parametrize("dtype", DTYPES)
def test_spmv_structures(cuda_device, dtype):
    cases = [
        inputs.row_lengths_csr([0] * 50, 10, 0, "all_empty"),
        inputs.row_lengths_csr([5000], 8000, 1, "one_hub_row"),
        inputs.row_lengths_csr([0, 0, 3000, 0, 1, 0, 0, 2000, 0], 4000, 2, "hubs_and_empties"),
        inputs.row_lengths_csr([1, 2, 3] * 700, 500, 3, "short_rows"),
        inputs.row_lengths_csr([14] * 300 + [448] * 20 + [447, 449, 3583, 3584, 3585], 4000, 4,
                               "tile_sized_rows"),
        inputs.row_lengths_csr([0] * 3000 + [1] + [0] * 3000, 10, 5, "lone_entry"),
    ]
    for a in cases:
        _run(a, dtype)
    # all-empty matrix gives exact zeros
    a = cases[0]
    p, _ = make_plan(a)
    y = mb.spmv(p, torch.zeros(0, dtype=dtype, device="cuda"),
                torch.ones(10, dtype=dtype, device="cuda"))
    assert torch.count_nonzero(y) == 0


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n_rows", [1, 31, 449, 3585, 20001])
def test_spmv_ragged_sizes(cuda_device, dtype, n_rows):
    a = inputs.random_sparse(n_rows, 257, 0.05, n_rows, empty_frac=0.25)
    _run(a, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("sigma", [14, 7, 1])
def test_spmv_rmat14(cuda_device, dtype, sigma):
    a = inputs.rmat_transition(14, 16, 1)
    _run(a, dtype, sigma=sigma)


@pytest.mark.parametrize("dtype", DTYPES)
def test_spmv_stress_scale16(cuda_device, dtype):
    base = inputs.rmat_uniform(16, 16, 3, 3)
    for a in (base, inputs.empty_rows(base, 0.3, 4), inputs.add_hubs(base, 4, 20000, 60000, 5),
              inputs.erdos_renyi(1 << 16, 16, 6)):
        _run(a, dtype)


def test_spmv_non_square(cuda_device):
    for a in (inputs.random_sparse(700, 20000, 0.001, 3), inputs.random_sparse(9000, 40, 0.05, 4)):
        for dt in DTYPES:
            _run(a, dt)


@pytest.mark.parametrize("dtype", DTYPES)
def test_spmv_repeated_calls(cuda_device, dtype):
    """Back-to-back calls reuse the boundary accumulators: each result must be exact again."""
    a = inputs.add_hubs(inputs.rmat_uniform(15, 16, 8, 8), 3, 30000, 60000, 9)
    p, _ = make_plan(a)
    vals = torch.from_numpy(a.val).to("cuda", dtype)
    ys = [torch.empty(a.n_rows, dtype=dtype, device="cuda") for _ in range(2)]
    xs = [torch.from_numpy(inputs.uniform_vector(a.n_cols, s)).to("cuda", dtype) for s in range(5)]
    for i, x in enumerate(xs):
        mb.spmv(p, vals, x, ys[i % 2])
        y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(vals), as_f64(x))
        check_rel(as_f64(ys[i % 2]), y_ref, d, TOL[dtype], f"call {i}")


@pytest.mark.parametrize("fmt,tdt", [("bf16", torch.bfloat16), ("f16", torch.float16)])
def test_lowprec_values(cuda_device, fmt, tdt):
    a = inputs.rmat_transition(14, 16, 1)
    v64 = torch.from_numpy(a.val).cuda()
    lo, k = mb.vals_convert(v64, tdt, auto_scale=(fmt == "f16"))
    ref_k = oracle.f16_scale_exponent(float(a.val.max())) if fmt == "f16" else 0
    assert k == ref_k
    # conversion is bit-exact against the oracle's round-to-nearest-even
    assert np.array_equal(as_f64(lo), oracle.round_to_format(np.ldexp(a.val, k), fmt))
    # wide-range values, subnormals and ties
    rng = np.random.default_rng(3)
    w = np.concatenate([np.ldexp(rng.random(5000) + 0.5, rng.integers(-140, 20, 5000)),
                        np.ldexp(1.0 + 3 * 2.0 ** -12, np.arange(-20, 10)), [0.0, 1e-300, 7e4]])
    wl, _ = mb.vals_convert(torch.from_numpy(w).cuda(), tdt)
    assert np.array_equal(as_f64(wl), oracle.round_to_format(w, fmt))
    # SpMV with the reduced values, f32 x, f32 accumulation
    p, _ = make_plan(a)
    x = torch.from_numpy(inputs.uniform_vector(a.n_cols, 2)).to("cuda", torch.float32)
    y = mb.spmv(p, lo, x, scale_exp=k)
    y_ref, d, _ = oracle.spmv_lowprec_reference(a.row_ptr, a.col, a.val, as_f64(x), fmt)
    check_rel(as_f64(y), y_ref, d, 1e-5, fmt)


@pytest.mark.parametrize("dtype", DTYPES)
def test_spmv_host_buffers(cuda_device, dtype):
    a = inputs.rmat_transition(14, 16, 1)
    p, _ = make_plan(a)
    vals = torch.from_numpy(a.val).to("cuda", dtype)
    x = torch.from_numpy(inputs.uniform_vector(a.n_cols, 4)).to(dtype).pin_memory()
    y = mb.spmv_host(p, vals, x)
    y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(vals), x.double().numpy())
    check_rel(y.double().numpy(), y_ref, d, TOL[dtype], "host")


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_spmv_host_async_overlapping_calls(cuda_device, dtype):
    """merbit_spmv_host_async: six calls in flight with different host x and y buffers (the
    two staging slots are reused three times each), then one sync; also a pageable pair."""
    a = inputs.rmat_transition(14, 16, 2)
    p, _ = make_plan(a)
    vals = torch.from_numpy(a.val).to("cuda", dtype)
    xs = [torch.from_numpy(inputs.uniform_vector(a.n_cols, 10 + i)).to(dtype).pin_memory() for i in range(6)]
    ys = [torch.full((a.n_rows,), float("nan"), dtype=dtype).pin_memory() for _ in range(6)]
    for x, y in zip(xs, ys):
        mb.spmv_host(p, vals, x, y, wait=False)
    p.sync()
    for x, y in zip(xs, ys):
        y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(vals), x.double().numpy())
        check_rel(y.double().numpy(), y_ref, d, TOL[dtype], "host async")
    xp = torch.from_numpy(inputs.uniform_vector(a.n_cols, 30)).to(dtype)
    yp = torch.empty(a.n_rows, dtype=dtype)
    mb.spmv_host(p, vals, xp, yp, wait=False)
    p.sync()
    y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(vals), xp.double().numpy())
    check_rel(yp.double().numpy(), y_ref, d, TOL[dtype], "host async pageable")
    p.destroy()


def test_spmv_argument_errors(cuda_device):
    a = inputs.rmat_transition(10, 8, 1)
    p, _ = make_plan(a)
    vals = torch.from_numpy(a.val).to("cuda", torch.float32)
    x = torch.ones(a.n_cols, device="cuda")
    big = torch.zeros(a.nnz + 1, device="cuda")
    with pytest.raises(mb.MerbitError) as e:
        mb.spmv(p, big[1:], x)          # 4-byte offset: not 16-byte aligned
    assert e.value.status == 1
    with pytest.raises(mb.MerbitError):
        mb.spmv(p, vals, x.double())    # mixed dtypes
    p.destroy()
    with pytest.raises(mb.MerbitError):
        mb.spmv(p, vals, x)


# ---------------------------------------------------------------- full size

@pytest.mark.parametrize("variant", ["a", "b", "c", "d"])
def test_spmv_full_config2(cuda_device, variant):
    """Configuration 2 at full size (R-MAT scale 22 stress variants, ER 2^22), FP32 and FP64,
    plan reused over 3 calls; every row against the oracle, plus global properties."""
    base = inputs.rmat_uniform(22, 16, 3, 3) if variant != "d" else None
    a = {"a": lambda: base, "b": lambda: inputs.empty_rows(base, 0.3, 4),
         "c": lambda: inputs.add_hubs(base, 16, 1_000_000, 4_000_000, 5),
         "d": lambda: inputs.erdos_renyi(1 << 22, 16, 6)}[variant]()
    p, _ = make_plan(a)
    x64 = inputs.uniform_vector(a.n_cols, 2)
    for dtype in DTYPES:
        vals = torch.from_numpy(a.val).to("cuda", dtype)
        x = torch.from_numpy(x64).to("cuda", dtype)
        y = torch.empty(a.n_rows, dtype=dtype, device="cuda")
        for _ in range(3):
            mb.spmv(p, vals, x, y)
        p.sync()
        y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(vals), as_f64(x))
        check_rel(as_f64(y), y_ref, d, TOL[dtype], f"config2{variant} {dtype}")
        # property at any size: sum_i y_i = sum_j x_j * colsum_j
        colsum = np.bincount(a.col, weights=as_f64(vals), minlength=a.n_cols)
        tot = float(np.dot(colsum, as_f64(x)))
        assert abs(float(y.double().sum()) - tot) <= 1e-5 * tot
        # rows with no entries are exactly zero
        empty = np.diff(a.row_ptr) == 0
        assert np.count_nonzero(as_f64(y)[empty]) == 0


@pytest.mark.parametrize("dtype", DTYPES)
def test_spmv_plans_of_different_sigma_interleaved(cuda_device, dtype):
    """Plans with small and large sigma used alternately by the same kernel (the larger
    stage size must stay launchable after a smaller one)."""
    a = inputs.rmat_uniform(13, 16, 5, 5)
    for sigma in (7, 14, 1, 14, 7):
        _run(a, dtype, sigma=sigma)


def test_spmv_full_rmat24_bench_configuration(cuda_device):
    """The product bench.py times, at full size: R-MAT scale 24 transition matrix, x ~ U[0,1)
    (seed 2), plan reused over 3 calls.  f32 on the sigma-14 plan (the split kernel) and
    f64 on the sigma-14 (classic kernel) and sigma-10 (split kernel) plans: every row
    against the oracle, the column-sum identity, and exact zeros in empty rows."""
    a = inputs.rmat_transition(24, 16, 7)
    x64 = inputs.uniform_vector(a.n_cols, 2)
    empty = np.diff(a.row_ptr) == 0
    for dtype, sigma in ((torch.float32, 14), (torch.float64, 14), (torch.float64, 10)):
        p, _ = make_plan(a, sigma)
        vals = torch.from_numpy(a.val).to("cuda", dtype)
        x = torch.from_numpy(x64).to("cuda", dtype)
        y = torch.empty(a.n_rows, dtype=dtype, device="cuda")
        for _ in range(3):
            mb.spmv(p, vals, x, y)
        p.sync()
        yh = as_f64(y)
        y_ref, d = oracle.spmv(a.row_ptr, a.col, as_f64(vals), as_f64(x))
        check_rel(yh, y_ref, d, TOL[dtype], f"rmat24 {dtype} sigma={sigma}")
        colsum = np.bincount(a.col, weights=as_f64(vals), minlength=a.n_cols)
        tot = float(np.dot(colsum, as_f64(x)))
        assert abs(float(yh.sum()) - tot) <= 1e-5 * tot
        assert np.count_nonzero(yh[empty]) == 0
        p.destroy()
        del vals, x, y
