import pytest
"""Seeded input generators: determinism and the structure the configurations state."""
import numpy as np

import inputs


def test_rmat_transition_structure():
    a = inputs.rmat_transition(12, 16, 1).check()
    b = inputs.rmat_transition(12, 16, 1)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
    assert np.array_equal(a.val, b.val)
    rows = np.repeat(np.arange(a.n_rows), np.diff(a.row_ptr))
    assert not np.any(rows == a.col)                       # self loops dropped
    key = rows.astype(np.int64) * a.n_cols + a.col
    assert np.all(np.diff(key) > 0)                        # sorted, no duplicates
    colsum = np.bincount(a.col, weights=a.val, minlength=a.n_cols)
    present = np.bincount(a.col, minlength=a.n_cols) > 0
    assert np.allclose(colsum[present], 1.0, rtol=0, atol=1e-12)   # column stochastic
    assert (~present).any()                                # dangling vertices kept
    assert 0.8 * 16 * 4096 < a.nnz < 16 * 4096


def test_rmat_seed_changes_graph():
    a = inputs.rmat_transition(10, 8, 1)
    b = inputs.rmat_transition(10, 8, 2)
    assert a.nnz != b.nnz or not np.array_equal(a.col, b.col)


def test_stress_variants():
    base = inputs.rmat_uniform(12, 16, 3, 3).check()
    assert np.all((base.val > 0) & (base.val <= 1))
    e = inputs.empty_rows(base, 0.3, 4).check()
    frac = (np.diff(e.row_ptr) == 0).mean() - (np.diff(base.row_ptr) == 0).mean()
    assert 0.2 < frac < 0.35
    h = inputs.add_hubs(base, 4, 1000, 3000, 5).check()
    lens = np.diff(h.row_ptr)
    assert sorted(lens[h.meta["hub_rows"]].tolist()) == sorted(h.meta["hub_lens"])
    assert min(h.meta["hub_lens"]) > 700
    er = inputs.erdos_renyi(1 << 12, 16, 6).check()
    assert 15 * 4096 < er.nnz <= 16 * 4096


def test_vectors():
    x = inputs.uniform_vector(1000, 2)
    assert np.all((x >= 0) & (x < 1)) and np.array_equal(x, inputs.uniform_vector(1000, 2))
    u = inputs.uniform_open0(1000, 2)
    assert np.all((u > 0) & (u <= 1))


def test_rmat_batch_is_block_diagonal():
    a, off = inputs.rmat_batch(6, 3, scales=(4, 9), edge_factors=(4, 12), threads=3)
    a.check()
    assert off[0] == 0 and off[-1] == a.n_rows and np.all(np.diff(off) > 0)
    sc, ef = a.meta["scales"], a.meta["edge_factors"]
    assert all(4 <= s <= 9 for s in sc) and all(4 <= f <= 12 for f in ef)
    rows = np.repeat(np.arange(a.n_rows), np.diff(a.row_ptr))
    g_row = np.searchsorted(off, rows, side="right") - 1
    g_col = np.searchsorted(off, a.col, side="right") - 1
    assert np.array_equal(g_row, g_col)
    for g in range(6):
        assert off[g + 1] - off[g] == 1 << sc[g]
    b, off2 = inputs.rmat_batch(6, 3, scales=(4, 9), edge_factors=(4, 12), threads=1)
    assert np.array_equal(b.col, a.col) and np.array_equal(b.val, a.val) and np.array_equal(off, off2)


def test_block_diagonal_of_small_graphs():
    parts = [inputs.cycle_graph(3), inputs.in_star(2), inputs.cycle_graph(1)]
    a, off = inputs.block_diagonal(parts)
    assert off.tolist() == [0, 3, 6, 7]
    dense = np.zeros((7, 7))
    for r in range(7):
        dense[r, a.col[a.row_ptr[r]:a.row_ptr[r + 1]]] = a.val[a.row_ptr[r]:a.row_ptr[r + 1]]
    assert dense[1, 0] == 1.0 and dense[3, 4] == 1.0 and dense[6, 6] == 1.0


@pytest.mark.parametrize("make", [lambda: inputs.road_grid(40, 30, 0.6, 1),
                                  lambda: inputs.kmer_chains(5000, 32, 0.02, 2),
                                  lambda: inputs.hub_graph(12, 2, 3)])
def test_undirected_graphs_are_symmetric_unit(make):
    a = make().check()
    assert np.all(a.val == 1.0)
    dense = np.zeros((a.n_rows, a.n_cols), bool)
    rows = np.repeat(np.arange(a.n_rows), np.diff(a.row_ptr))
    dense[rows, a.col] = True
    assert np.array_equal(dense, dense.T) and not dense.diagonal().any()
    for r in range(a.n_rows):
        seg = a.col[a.row_ptr[r]:a.row_ptr[r + 1]]
        assert np.all(np.diff(seg) > 0)
