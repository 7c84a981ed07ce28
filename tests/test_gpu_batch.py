"""Many graphs in one CUDA-graph launch (merbit_batch_pagerank) against the float64
oracle's PageRank of every graph on its own."""
import numpy as np
import pytest
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb
from tests.gpu_helpers import as_f64

pytestmark = pytest.mark.gpu

ALPHA = 0.85


def _batch(a, off, sigma=14):
    rp = torch.from_numpy(a.row_ptr).cuda()
    col = torch.from_numpy(a.col).cuda()
    return mb.Batch(rp, col, off, sigma=sigma), col


def _parts(a, off):
    for g in range(off.size - 1):
        lo, hi = int(off[g]), int(off[g + 1])
        rp = a.row_ptr[lo:hi + 1] - a.row_ptr[lo]
        k0, k1 = a.row_ptr[lo], a.row_ptr[hi]
        yield g, lo, hi, inputs.CSR(hi - lo, hi - lo, rp.astype(np.int32),
                                    (a.col[k0:k1] - lo).astype(np.int32), a.val[k0:k1])


def _check(a, off, dt, tol, max_err, sigma=14, max_iter=1000):
    b, _ = _batch(a, off, sigma)
    vals = torch.from_numpy(a.val).to("cuda", dt)
    pi, info = b.pagerank(vals, ALPHA, tol=tol, max_iter=max_iter)
    assert info["converged"], info
    pin = as_f64(pi)
    for g, lo, hi, part in _parts(a, off):
        ref = oracle.pagerank(part.row_ptr, part.col, part.val, ALPHA, tol=tol, max_iter=max_iter)
        # same stopping rule: the same number of updates up to a tie at the threshold
        assert abs(int(info["iters"][g]) - ref["iters"]) <= 1, (g, info["iters"][g], ref["iters"])
        assert info["resid"][g] < tol
        exact = oracle.pagerank(part.row_ptr, part.col, part.val, ALPHA, tol=1e-15, max_iter=5000)["pi"]
        err = np.abs(pin[lo:hi] - exact).sum()
        assert err <= max_err, (g, err)
        assert abs(pin[lo:hi].sum() - 1.0) <= max_err
    assert info["rounds"] == int(np.max(info["iters"]))
    b.destroy()
    return pi, info


def test_batch_rmat_f64(cuda_device):
    a, off = inputs.rmat_batch(24, 7, scales=(5, 12), edge_factors=(4, 24), threads=4)
    # ||pi_k - pi*||_1 <= ||pi_k - pi_{k-1}||_1 * alpha / (1 - alpha) for the power method
    _check(a, off, torch.float64, 1e-10, 1e-10 * ALPHA / (1 - ALPHA) * 1.01 + 1e-13)


def test_batch_rmat_f32(cuda_device):
    a, off = inputs.rmat_batch(16, 9, scales=(6, 11), edge_factors=(8, 16), threads=4)
    _check(a, off, torch.float32, 1e-6, 1e-5)


def test_batch_special_graphs(cuda_device):
    """Tiny and degenerate graphs mixed with R-MAT ones: one vertex, a cycle, an in-star
    (dangling centre), a chain, and empty graphs of several vertices (all dangling)."""
    parts = [inputs.cycle_graph(1), inputs.rmat_transition(8, 8, 3), inputs.cycle_graph(7),
             inputs.in_star(5), inputs.from_edges(4, [(0, 1), (1, 2), (2, 3)], "chain4"),
             inputs.row_lengths_csr([0] * 9, 9, 0, "empty9"), inputs.rmat_transition(10, 16, 4),
             inputs.bidirected_star(30)]
    a, off = inputs.block_diagonal(parts)
    _check(a, off, torch.float64, 1e-12, 1e-11)
    _check(a, off, torch.float64, 1e-12, 1e-11, sigma=7)


def test_batch_single_graph_matches_pagerank(cuda_device):
    a = inputs.rmat_transition(12, 16, 2)
    b, _ = _batch(a, np.array([0, a.n_rows]))
    vals = torch.from_numpy(a.val).cuda()
    pi, info = b.pagerank(vals, ALPHA, tol=1e-10)
    p = mb.plan(torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col).cuda())
    ref, rinfo = mb.pagerank(p, vals, ALPHA, tol=1e-10)
    assert info["iters"][0] == rinfo["iters"]
    np.testing.assert_allclose(as_f64(pi), as_f64(ref), rtol=1e-12, atol=1e-18)


def test_batch_relaunch_and_rerecord(cuda_device):
    a, off = inputs.rmat_batch(10, 4, scales=(6, 10), edge_factors=(8, 16), threads=4)
    b, _ = _batch(a, off)
    vals = torch.from_numpy(a.val).cuda()
    out = torch.empty(a.n_rows, dtype=torch.float64, device="cuda")
    _, i1 = b.pagerank(vals, ALPHA, tol=1e-9, pi=out)
    pi1 = out.clone()
    out.fill_(-1.0)
    _, i2 = b.pagerank(vals, ALPHA, tol=1e-9, pi=out)           # the same recorded graph
    # per-graph FP64 sums are atomics in arbitrary order: equal up to rounding, not bitwise
    np.testing.assert_allclose(as_f64(out), as_f64(pi1), rtol=1e-12, atol=1e-18)
    assert np.all(np.abs(i1["iters"] - i2["iters"]) <= 1)
    pi3, i3 = b.pagerank(vals, ALPHA, tol=1e-11)                # recorded again
    assert np.all(i3["iters"] >= i2["iters"]) and i3["converged"]
    _, i4 = b.pagerank(vals, ALPHA, tol=1e-30, max_iter=5)      # no graph converges
    assert not i4["converged"] and np.all(i4["iters"] == 5) and i4["rounds"] == 5


def test_batch_rejects_links_between_graphs(cuda_device):
    a, off = inputs.block_diagonal([inputs.cycle_graph(4), inputs.cycle_graph(5)])
    col = a.col.copy()
    col[0] = 6                                                  # row 0 of graph 0 -> graph 1
    rp = torch.from_numpy(a.row_ptr).cuda()
    with pytest.raises(mb.MerbitError, match="EINVAL"):
        mb.Batch(rp, torch.from_numpy(col).cuda(), off)
    with pytest.raises(mb.MerbitError, match="EINVAL"):
        mb.Batch(rp, torch.from_numpy(a.col).cuda(), np.array([0, 4, 4, 9]))


def test_autotune_sigma(cuda_device):
    a = inputs.rmat_transition(14, 16, 3)
    rp, col = torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col).cuda()
    for dt in (torch.float32, torch.float64):
        vals = torch.from_numpy(a.val).to("cuda", dt)
        best, ms = mb.autotune_sigma(rp, col, vals, candidates=(14, 10, 7, 4), reps=3)
        assert best in (14, 10, 7, 4) and ms[best] == min(ms.values()) and all(t > 0 for t in ms.values())
    with pytest.raises(mb.MerbitError, match="EINVAL"):
        mb.autotune_sigma(rp, col, vals, candidates=(15,))
