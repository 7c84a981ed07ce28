"""merbit_spmv_noalloc: the entry point for callers that may not allocate device memory.

Such callers (code whose device memory belongs to another framework's pool, or
paths that cannot afford cudaMalloc's device-wide synchronisation) get the same
product as the planned path, computed with only a scratch array compiled into
the library.  This file is collected last so that a run stopping at its first
failure has already run every other test; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb

SCRATCH_BYTES = 8 << 20


def _up256(b: int) -> int:
    return (b + 255) // 256 * 256


def scratch_needed(steps: int) -> int:
    """Scratch bytes a matrix with n_rows + nnz = steps needs (the formula of the header)."""
    lane_num = -(-steps // 14)
    tile_num = -(-steps // 448)
    nb = -(-tile_num // 8)
    return (66816 + _up256(4 * lane_num) + 2 * _up256(4 * (tile_num + 1))
            + 2 * _up256(4 * (nb + 1)) + _up256(8 * (nb + 1)))


def max_steps() -> int:
    """Largest n_rows + nnz whose scratch fits the library's array."""
    lo, hi = 1, 1 << 31
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if scratch_needed(mid) <= SCRATCH_BYTES:
            lo = mid
        else:
            hi = mid - 1
    return lo


def _noalloc(lib):
    return lib.merbit_spmv_noalloc


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _call(lib, a_dev, x, y, a, stream):
    row_ptr, col, vals = a_dev
    return _noalloc(lib)(_p(row_ptr), _p(col), _p(vals), _p(x), _p(y), a.n_rows, a.n_cols, a.nnz,
                         ctypes.c_void_p(stream.cuda_stream))


def _check_oracle(a, vals, x, y):
    """Per-element bound of the FP32 parity tests, |dy_i| <= 1e-5 * sum_j |a_ij x_j|, with
    rows whose bound is 0 (empty rows) required to be exactly 0."""
    y_ref, d = oracle.spmv(a.row_ptr, a.col, vals.double().cpu().numpy(), x.double().cpu().numpy())
    err = oracle.relative_errors(y.double().cpu().numpy(), y_ref, d)
    assert err.max() <= 1e-5, float(err.max())
    return y_ref


@pytest.mark.gpu
def test_noalloc_matches_oracle_and_planned_spmv_twice(cuda_device):
    lib = mb.load()
    a = inputs.add_hubs(inputs.rmat_uniform(16, 16, 3, 3), 2, 20000, 40000, 5)
    a_dev = (torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col).cuda(),
             torch.from_numpy(a.val).cuda().float())
    plan = mb.plan(a_dev[0], a_dev[1], a.n_rows, a.n_cols)
    stream = torch.cuda.current_stream()
    for seed in (2, 9):                       # two calls in a row, different x
        x = torch.from_numpy(inputs.uniform_vector(a.n_cols, seed)).cuda().float()
        y_ref = mb.spmv(plan, a_dev[2], x)    # the existing entry point
        y = torch.full((a.n_rows,), float("nan"), device="cuda")
        st = _call(lib, a_dev, x, y, a, stream)
        assert st == 0, lib.merbit_last_error()
        assert lib.merbit_spmv_noalloc_status(ctypes.c_void_p(stream.cuda_stream)) == 0
        _check_oracle(a, a_dev[2], x, y)
        # against the planned product: the same tolerance, scaled by sum_j |a_ij x_j|
        _, d = oracle.spmv(a.row_ptr, a.col, a_dev[2].double().cpu().numpy(), x.double().cpu().numpy())
        diff = np.abs(y.double().cpu().numpy() - y_ref.double().cpu().numpy())
        assert np.all(diff <= 1e-5 * d), float((diff / np.maximum(d, 1e-300)).max())
    plan.destroy()


@pytest.mark.gpu
def test_noalloc_at_the_size_limit(cuda_device):
    """A matrix with exactly the largest n_rows + nnz the scratch holds: the last carved
    region ends at the array's end.  Every row is compared with the oracle; the rows left
    empty at the end must be exactly 0."""
    lib = mb.load()
    s_max = max_steps()
    assert scratch_needed(s_max) <= SCRATCH_BYTES < scratch_needed(s_max + 1)
    base = inputs.erdos_renyi(1 << 21, 12, 6, 6)
    nnz = s_max - base.n_rows
    assert 0 < nnz <= base.nnz
    row_ptr = np.minimum(base.row_ptr.astype(np.int64), nnz).astype(np.int32)
    a = inputs.CSR(base.n_rows, base.n_cols, row_ptr, base.col[:nnz].copy(), base.val[:nnz].copy(),
                   "er2^21_truncated")
    assert a.n_rows + a.nnz == s_max and (np.diff(a.row_ptr) == 0).sum() > 1000
    a_dev = (torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col).cuda(),
             torch.from_numpy(a.val).cuda().float())
    x = torch.from_numpy(inputs.uniform_vector(a.n_cols, 2)).cuda().float()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        y = torch.full((a.n_rows,), float("nan"), device="cuda")
        assert _call(lib, a_dev, x, y, a, stream) == 0, lib.merbit_last_error()
        assert lib.merbit_spmv_noalloc_status(ctypes.c_void_p(stream.cuda_stream)) == 0
        y_ref = _check_oracle(a, a_dev[2], x, y)
        empty = np.diff(a.row_ptr) == 0
        assert np.all(y.cpu().numpy()[empty] == 0.0) and np.all(y_ref[empty] == 0.0)


def test_noalloc_rejects_one_step_above_the_limit():
    """Rejected on the host before any device work (no GPU needed)."""
    lib = mb.load()
    s = max_steps() + 1
    f = _noalloc(lib)
    fake = ctypes.c_void_p(256)
    st = f(fake, fake, fake, fake, fake, 1000, 1000, s - 1000, None)
    assert st == 1 and b"too large" in lib.merbit_last_error()
    st = f(fake, fake, fake, fake, fake, 50_000_000, 50_000_000, 50_000_000, None)
    assert st == 1 and b"too large" in lib.merbit_last_error()


def test_noalloc_rejects_misaligned_vectors():
    """x or y off their 4-byte alignment: EINVAL on the host, nothing launched."""
    lib = mb.load()
    f = _noalloc(lib)
    ok, odd = ctypes.c_void_p(256), ctypes.c_void_p(258)
    assert f(ok, ok, ok, odd, ok, 100, 100, 100, None) == 1
    assert b"4-byte" in lib.merbit_last_error()
    assert f(ok, ok, ok, ok, odd, 100, 100, 100, None) == 1
    assert b"4-byte" in lib.merbit_last_error()
