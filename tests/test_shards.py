"""Splitting the merge path by diagonal ranges (the partition a multi-GPU split of the
product would use; this project runs replicas only).  Shard g takes the steps
[d_g, d_{g+1}) of the path, i.e. the nonzeros [x_g, x_{g+1}) and the rows
[y_g, y_{g+1}]; a row cut by a shard boundary gets one partial sum from each side.
Checked on the CPU with the oracle: every nonzero falls into exactly one shard, the
shards' partial products add up to the whole product, and equal diagonal ranges give
shards whose work (nonzeros + rows) differs by at most one row end."""
import numpy as np
import pytest

import inputs
import oracle


def _coordinate(row_ptr, d):
    """(x, y) after d steps of the path: y = down steps among the first d."""
    down = oracle.merge_path_down_steps(row_ptr)
    y = int(down[:d].sum())
    return d - y, y


def _shard_product(a, x, d0, d1):
    """The partial products of the nonzeros on steps [d0, d1), as (first row, sums)."""
    x0, y0 = _coordinate(a.row_ptr, d0)
    x1, y1 = _coordinate(a.row_ptr, d1)
    last = min(y1, a.n_rows - 1)
    if y0 > last:
        return y0, np.zeros(0), (x0, x1)
    rp = np.clip(a.row_ptr[y0:last + 2].astype(np.int64), x0, x1) - x0
    part, _ = oracle.spmv(rp, a.col[x0:x1], a.val[x0:x1], x)
    return y0, part, (x0, x1)


def _cases():
    return [inputs.random_sparse(500, 300, 0.02, 1, empty_frac=0.3),
            inputs.row_lengths_csr([0, 0, 3000, 0, 1, 0, 0, 2000, 0], 4000, 2, "hubs_and_empties"),
            inputs.rmat_transition(10, 16, 3),
            inputs.row_lengths_csr([0] * 40, 10, 0, "all_empty")]


@pytest.mark.parametrize("G", [1, 2, 3, 7, 64])
def test_diagonal_shards_add_up_to_the_product(G):
    rng = np.random.default_rng(G)
    for a in _cases():
        x = rng.standard_normal(a.n_cols)
        y_ref, d = oracle.spmv(a.row_ptr, a.col, a.val, x)
        steps = a.nnz + a.n_rows
        # random cut diagonals, and the equal split a launch over G GPUs would take
        for cuts in (np.sort(rng.integers(0, steps + 1, G - 1)),
                     np.array([steps * g // G for g in range(1, G)], np.int64)):
            bounds = np.concatenate([[0], cuts, [steps]]).astype(np.int64)
            y = np.zeros(a.n_rows)
            covered = np.zeros(a.nnz, np.int64)
            for g in range(G):
                y0, part, (x0, x1) = _shard_product(a, x, int(bounds[g]), int(bounds[g + 1]))
                y[y0:y0 + part.size] += part
                covered[x0:x1] += 1
            assert np.all(covered == 1)
            err = oracle.relative_errors(y, y_ref, d)
            assert err.size == 0 or err.max() <= 1e-13


@pytest.mark.parametrize("G", [2, 5, 152])
def test_equal_diagonal_ranges_balance_the_work(G):
    """Equal step ranges: each shard's nonzeros + row ends differ by at most one,
    however skewed the row lengths (one hub row of 3000 among empty rows)."""
    for a in _cases():
        steps = a.nnz + a.n_rows
        bounds = [steps * g // G for g in range(G + 1)]
        work = []
        for g in range(G):
            x0, y0 = _coordinate(a.row_ptr, bounds[g])
            x1, y1 = _coordinate(a.row_ptr, bounds[g + 1])
            work.append((x1 - x0) + (y1 - y0))
        assert sum(work) == steps
        assert max(work) - min(work) <= 1
