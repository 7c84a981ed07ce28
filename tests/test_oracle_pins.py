"""Pins of the CPU oracle against facts that do not come from the oracle itself."""
import math
import os

import numpy as np
import pytest

import inputs
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        out[k] = v
    return out


# --------------------------------------------------------------------------
# Plan (Sec. 4.1)
# --------------------------------------------------------------------------

def test_worked_example_counts():
    g = _golden()
    m, n, omega, sigma = (int(g[k][0]) for k in ("m", "n", "omega", "sigma"))
    assert oracle.tile_counts(n, m, sigma, omega) == (int(g["tile_num"][0]), int(g["lane_num"][0]))


def test_worked_example_step_arithmetic():
    """Coordinate formula of Sec. 4.1.1 on the printed tile-1 data."""
    g = _golden()
    tx, ty = (int(v) for v in g["tile1_start"])
    xo = [int(v) for v in g["tile1_x_offset"]]
    yo = [int(v) for v in g["tile1_y_offset"]]
    starts = [int(v) for v in g["tile1_lane_starts"]]
    starts = list(zip(starts[0::2], starts[1::2]))
    flags = sum((1 << k) for k, b in enumerate(g["tile1_lane0_bit_flag"]) if b == "T")
    for j in range(4):
        desc = (0 << 18) | (yo[j] << 9) | xo[j]
        assert oracle.step_coordinate((tx, ty), desc, 0) == starts[j]
    desc0 = (flags << 18) | (yo[0] << 9) | xo[0]
    assert oracle.step_coordinate((tx, ty), desc0, 1) == (12, 4)
    # after its 4 steps lane 0 arrives exactly where lane 1 starts
    assert oracle.step_coordinate((tx, ty), desc0, 4) == starts[1]


def test_descriptor_fit_condition():
    # sigma = 14 fills the 32-bit word exactly (Sec. 4.1.1); sigma = 15 does not fit.
    assert oracle.descriptor_fits(14) and oracle.descriptor_fits(7)
    assert not oracle.descriptor_fits(15)
    assert 2 * math.ceil(math.log2(32 * 14)) + 14 == 32
    # the 64-bit word (Sec. 5.3.4): 2 * 11 offset bits + sigma flag bits, sigma up to 42
    assert oracle.descriptor_fits(42, bits=64) and not oracle.descriptor_fits(43, bits=64)
    assert oracle.descriptor_layout(14) == (32, 9) and oracle.descriptor_layout(15) == (64, 11)
    assert oracle.descriptor_layout(42) == (64, 11)
    for bad in (0, 43):
        with pytest.raises(ValueError):
            oracle.descriptor_layout(bad)


def _walk_tile(row_ptr, sigma, omega):
    """Literal merge-path walk of Sec. 4.1.2: one step at a time, plain Python.  The
    descriptor packs bit_flag, y_off, x_off with 9-bit offset fields up to sigma = 14 (the
    32-bit word of Sec. 4.1.1) and 11-bit fields above (the 64-bit word)."""
    w = 9 if sigma <= 14 else 11
    row_ptr = [int(v) for v in row_ptr]
    n, m = len(row_ptr) - 1, row_ptr[-1]
    total = m + n
    coords, downs = [(0, 0)], []
    x = y = 0
    for _ in range(total):
        if x < row_ptr[y + 1]:
            x += 1
            downs.append(0)
        else:
            y += 1
            downs.append(1)
        coords.append((x, y))
    assert (x, y) == (m, n)
    lane_num = -(-total // sigma)
    tile_num = -(-total // (omega * sigma))
    tile_x, tile_y, desc = [], [], []
    for i in range(tile_num):
        sx, sy = coords[i * omega * sigma]
        lo, hi = i * omega * sigma, min((i + 1) * omega * sigma, total)
        tile_x.append(sx)
        tile_y.append(sy | (0x80000000 if sum(downs[lo:hi]) == 0 else 0))
    for j in range(lane_num):
        lx, ly = coords[j * sigma]
        sx, sy = coords[(j // omega) * omega * sigma]
        f = 0
        for k in range(sigma):
            s = j * sigma + k
            if s < total and downs[s]:
                f |= 1 << k
        desc.append((f << (2 * w)) | ((ly - sy) << w) | (lx - sx))
    return tile_x + [m], tile_y + [n], desc


CASES = [
    ("single_row", [0, 500]),
    ("all_empty", [0] * 40),
    ("one_row_empty", [0, 0]),
    ("n1_m1", [0, 1]),
    ("sigma_rows", list(np.cumsum([0] + [14] * 70))),
    ("tile_rows", list(np.cumsum([0] + [448] * 5 + [447, 449]))),
]


@pytest.mark.parametrize("name,row_ptr", CASES)
@pytest.mark.parametrize("sigma", [14, 7, 4, 1, 15, 28, 42])
def test_build_tile_matches_walk_special(name, row_ptr, sigma):
    _check_against_walk(np.asarray(row_ptr, np.int64), sigma)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("sigma", [14, 7, 3, 17, 42])
def test_build_tile_matches_walk_random(seed, sigma):
    a = inputs.random_sparse(300 + 37 * seed, 200, 0.03 * (seed + 1), seed, empty_frac=0.3)
    _check_against_walk(a.row_ptr, sigma)


def _check_against_walk(row_ptr, sigma, omega=32):
    t = oracle.build_tile(row_ptr, sigma, omega)
    tx, ty, desc = _walk_tile(row_ptr, sigma, omega)
    assert t["tile_x"].tolist() == tx
    assert t["tile_y"].tolist() == ty
    assert t["lane_desc"].tolist() == desc
    n, m = len(row_ptr) - 1, int(row_ptr[-1])
    assert (t["tile_num"], t["lane_num"]) == oracle.tile_counts(n, m, sigma, omega)
    assert len(t["tile_x"]) == t["tile_num"] + 1 and len(t["lane_desc"]) == t["lane_num"]


def _walk_block_rows(row_ptr, sigma, omega, W):
    """Row of the merge-path coordinate at the start of every block of W tiles, plus the
    end row n, from the literal walk: block b starts at step b*W*omega*sigma (Sec. 4.2's
    y_bs; the last block's end y_be is the path's end, row n)."""
    row_ptr = [int(v) for v in row_ptr]
    n, m = len(row_ptr) - 1, row_ptr[-1]
    total = m + n
    rows_at, x, y = [0], 0, 0
    for _ in range(total):
        if x < row_ptr[y + 1]:
            x += 1
        else:
            y += 1
        rows_at.append(y)
    per_block = W * omega * sigma
    nb = -(-total // per_block)
    return [rows_at[min(b * per_block, total)] for b in range(nb + 1)]


@pytest.mark.parametrize("W", [8, 4, 16, 3])
@pytest.mark.parametrize("sigma", [14, 7, 2, 28])
@pytest.mark.parametrize("case", range(5))
def test_block_boundary_rows_match_walk(case, sigma, W):
    if case < 3:
        a = inputs.random_sparse(900 + 211 * case, 400, 0.02 * (case + 1), 40 + case,
                                 empty_frac=0.25)
        row_ptr = a.row_ptr
    elif case == 3:
        row_ptr = np.asarray(CASES[5][1], np.int64)           # rows of one tile each
    else:
        row_ptr = np.asarray([0] + [0] * 30 + [5000] * 3 + list(range(5001, 5101)), np.int64)
    t = oracle.build_tile(row_ptr, sigma)
    got = oracle.block_boundary_rows(t["tile_y"], t["tile_num"], W)
    assert got.tolist() == _walk_block_rows(row_ptr, sigma, 32, W)


@pytest.mark.parametrize("sigma", [14, 28])
def test_build_tile_invariants_rmat14(sigma):
    a = inputs.rmat_transition(14, 16, 1)
    t = oracle.build_tile(a.row_ptr, sigma)
    w = 9 if sigma <= 14 else 11
    desc = t["lane_desc"].astype(np.uint64)
    flags = desc >> np.uint64(2 * w)
    xo = (desc & np.uint64((1 << w) - 1)).astype(np.int64)
    yo = ((desc >> np.uint64(w)) & np.uint64((1 << w) - 1)).astype(np.int64)
    pop = np.array([bin(int(f)).count("1") for f in flags])
    assert pop.sum() == a.n_rows                        # one down step per row
    total = a.nnz + a.n_rows
    lane_len = np.minimum(sigma, total - np.arange(t["lane_num"]) * sigma)
    assert (lane_len - pop).sum() == a.nnz              # one right step per nonzero
    tx = t["tile_x"].astype(np.int64)
    ty = (t["tile_y"] & 0x7FFFFFFF).astype(np.int64)
    tile = np.arange(t["lane_num"]) // 32
    lane_x, lane_y = tx[tile] + xo, ty[tile] + yo
    assert np.array_equal(lane_x + lane_y, np.arange(t["lane_num"]) * sigma)   # start on diagonal j*sigma
    assert (tx[-1], ty[-1]) == (a.nnz, a.n_rows)
    # a marked tile has no down step: it starts and ends in the same row
    marked = (t["tile_y"][:-1] & 0x80000000) != 0
    assert np.all(ty[:-1][marked] == ty[1:][marked])
    tile_flags = np.zeros(t["tile_num"], np.int64)
    np.add.at(tile_flags, tile, pop)
    assert np.array_equal(marked, tile_flags == 0)
    assert marked.any() and (~marked).any()
    # the row pointer is recovered from the walk: row r ends at its down step
    down = oracle.merge_path_down_steps(a.row_ptr)
    pos = np.nonzero(down)[0]
    assert np.array_equal(pos - np.arange(a.n_rows), a.row_ptr[1:])


# --------------------------------------------------------------------------
# SpMV (Sec. 3.1)
# --------------------------------------------------------------------------

def _dense_bruteforce(dense, x):
    out = []
    for i in range(dense.shape[0]):
        s = 0.0
        for j in range(dense.shape[1]):
            if dense[i, j] != 0.0:
                s += float(dense[i, j]) * float(x[j])
        out.append(s)
    return np.array(out)


@pytest.mark.parametrize("seed", range(5))
def test_spmv_dense_bruteforce(seed):
    rng = np.random.default_rng(seed)
    n_rows, n_cols = 1 + seed * 13, 64 - seed * 7
    a = inputs.random_sparse(n_rows, n_cols, 0.2, seed, empty_frac=0.2)
    dense = np.zeros((n_rows, n_cols))
    for r in range(n_rows):
        for k in range(a.row_ptr[r], a.row_ptr[r + 1]):
            dense[r, a.col[k]] = a.val[k]
    x = rng.standard_normal(n_cols)
    y, d = oracle.spmv(a.row_ptr, a.col, a.val, x)
    np.testing.assert_allclose(y, _dense_bruteforce(dense, x), rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(d, _dense_bruteforce(np.abs(dense), np.abs(x)), rtol=1e-14)


def test_spmm_dense_bruteforce():
    rng = np.random.default_rng(11)
    a = inputs.random_sparse(40, 30, 0.2, 11, empty_frac=0.2)
    dense = np.zeros((40, 30))
    for r in range(40):
        for k in range(a.row_ptr[r], a.row_ptr[r + 1]):
            dense[r, a.col[k]] = a.val[k]
    X = rng.standard_normal((30, 5))
    Y, D = oracle.spmm(a.row_ptr, a.col, a.val, X)
    ref = np.array([[sum(dense[i, j] * X[j, c] for j in range(30)) for c in range(5)] for i in range(40)])
    np.testing.assert_allclose(Y, ref, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(D, np.abs(dense) @ np.abs(X), rtol=1e-13)


def test_spmv_special_matrices():
    rng = np.random.default_rng(7)
    x = rng.standard_normal(50)
    eye = inputs.from_dense(np.eye(50))
    assert np.array_equal(oracle.spmv(eye.row_ptr, eye.col, eye.val, x)[0], x)
    perm = rng.permutation(50)
    P = np.zeros((50, 50))
    P[np.arange(50), perm] = 1.0
    p = inputs.from_dense(P)
    assert np.array_equal(oracle.spmv(p.row_ptr, p.col, p.val, x)[0], x[perm])
    diag = rng.random(50) + 0.5
    dg = inputs.from_dense(np.diag(diag))
    assert np.array_equal(oracle.spmv(dg.row_ptr, dg.col, dg.val, x)[0], diag * x)
    empty = inputs.CSR(50, 50, np.zeros(51, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert np.array_equal(oracle.spmv(empty.row_ptr, empty.col, empty.val, x)[0], np.zeros(50))


def test_spmv_long_row_exact_sum():
    # one row of 10^5 entries summing exactly: x = 1, values 2^-17 -> y = 10^5 * 2^-17
    n_cols = 100_000
    a = inputs.CSR(3, n_cols, np.array([0, 0, n_cols, n_cols], np.int32),
                   np.arange(n_cols, dtype=np.int32), np.full(n_cols, 2.0 ** -17))
    y, d = oracle.spmv(a.row_ptr, a.col, a.val, np.ones(n_cols))
    assert y.tolist() == [0.0, n_cols * 2.0 ** -17, 0.0]
    y2, _ = oracle.spmv_rows(a.row_ptr, a.col, a.val, np.ones(n_cols), [1, 0])
    assert y2.tolist() == [n_cols * 2.0 ** -17, 0.0]


def test_spmv_matches_scipy():
    sp = pytest.importorskip("scipy.sparse")
    a = inputs.rmat_uniform(12, 16, 3, 3)
    x = inputs.uniform_vector(a.n_cols, 2)
    A = sp.csr_matrix((a.val, a.col, a.row_ptr), shape=(a.n_rows, a.n_cols))
    y, d = oracle.spmv(a.row_ptr, a.col, a.val, x)
    assert np.all(np.abs(y - A @ x) <= 1e-14 * d)


def test_relative_errors_rules():
    d = np.array([1.0, 0.0, 0.0, 2.0])
    e = oracle.relative_errors(np.array([1.5, 0.0, 1e-30, 2.0]), np.array([1.0, 0.0, 0.0, 1.0]), d)
    assert e.tolist() == [0.5, 0.0, np.inf, 0.5]


# --------------------------------------------------------------------------
# PageRank (Sec. 5.5.1)
# --------------------------------------------------------------------------

ALPHA = 0.85


def _pr(a, **kw):
    return oracle.pagerank(a.row_ptr, a.col, a.val, ALPHA, **kw)


@pytest.mark.parametrize("n", [1, 2, 7, 64])
def test_pagerank_cycle_uniform(n):
    a = inputs.cycle_graph(n)
    r = _pr(a, tol=1e-14)
    np.testing.assert_allclose(r["pi"], np.full(n, 1.0 / n), rtol=1e-13)


@pytest.mark.parametrize("k", [1, 3, 10, 40])
def test_pagerank_bidirected_star_closed_form(k):
    a = inputs.bidirected_star(k)
    pi = _pr(a, tol=1e-15)["pi"]
    c = (1 + ALPHA * k) / ((k + 1) * (1 + ALPHA))
    leaf = (k + ALPHA) / (k * (k + 1) * (1 + ALPHA))
    np.testing.assert_allclose(pi, [c] + [leaf] * k, rtol=1e-12)


@pytest.mark.parametrize("k", [1, 5, 30])
def test_pagerank_in_star_closed_form(k):
    a = inputs.in_star(k)
    assert oracle.dangling_mask(k + 1, a.col).tolist() == [True] + [False] * k
    pi = _pr(a, tol=1e-15)["pi"]
    den = 1 + k * (1 + ALPHA)
    np.testing.assert_allclose(pi, [(1 + ALPHA * k) / den] + [1 / den] * k, rtol=1e-12)


def test_pagerank_chain_orientation():
    """0 -> 1 -> 2 with vertex 2 dangling: pi = (1, 1+a, 1+a+a^2) / (3+2a+a^2)."""
    a = inputs.from_edges(3, [(0, 1), (1, 2)], "chain3")
    pi = _pr(a, tol=1e-15)["pi"]
    al = ALPHA
    np.testing.assert_allclose(pi, np.array([1, 1 + al, 1 + al + al * al]) / (3 + 2 * al + al * al),
                               rtol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_pagerank_matches_dense_solve(seed):
    a = inputs.random_graph_transition(24 + 10 * seed, 0.08, seed)
    dense = np.zeros((a.n_rows, a.n_cols))
    for r in range(a.n_rows):
        for k in range(a.row_ptr[r], a.row_ptr[r + 1]):
            dense[r, a.col[k]] = a.val[k]
    ref = oracle.pagerank_dense_solve(dense, ALPHA)
    pi = _pr(a, tol=1e-15)["pi"]
    np.testing.assert_allclose(pi, ref, rtol=1e-11)
    assert oracle.pagerank_residual(a.row_ptr, a.col, a.val, ref, ALPHA) < 1e-14


def test_pagerank_invariants_rmat14():
    a = inputs.rmat_transition(14, 16, 1)
    r = _pr(a, fixed_iters=100)
    pi = r["pi"]
    n = a.n_rows
    assert r["iters"] == 100
    assert abs(pi.sum() - 1.0) < 1e-12
    assert np.all(pi >= (1 - ALPHA) / n * (1 - 1e-12))
    h = np.array(r["resid"])
    assert np.all(h[1:] <= ALPHA * h[:-1] * (1 + 1e-9) + 1e-15)   # L1 contraction
    # mass conservation of the column-stochastic operator: sum(P^T pi) + D = sum(pi)
    y, _ = oracle.spmv(a.row_ptr, a.col, a.val, pi)
    D = pi[oracle.dangling_mask(n, a.col)].sum()
    assert abs(y.sum() + D - pi.sum()) < 1e-12
    # residual definition agrees with the size of the next power step
    assert abs(oracle.pagerank_residual(a.row_ptr, a.col, a.val, pi, ALPHA)
               - np.abs(oracle.pagerank_step(a.row_ptr, a.col, a.val, pi, ALPHA,
                                              oracle.dangling_mask(n, a.col)) - pi).sum()) < 1e-15


# Personalised PageRank (one column per seed; teleport and dangling mass go to the seed)

def _ppr(a, seeds, **kw):
    return oracle.personalized_pagerank(a.row_ptr, a.col, a.val, seeds, ALPHA, **kw)


@pytest.mark.parametrize("n", [1, 5, 16])
def test_ppr_cycle_closed_form(n):
    """Directed n-cycle: pi_s[s + j] = (1 - a) a^j / (1 - a^n)."""
    a = inputs.cycle_graph(n)
    seeds = [0, 2 % n, n - 1]
    Pi = _ppr(a, seeds, tol=1e-15)["pi"]
    for c, s in enumerate(seeds):
        ref = np.zeros(n)
        for j in range(n):
            ref[(s + j) % n] = (1 - ALPHA) * ALPHA ** j / (1 - ALPHA ** n)
        np.testing.assert_allclose(Pi[:, c], ref, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("L", [2, 6])
def test_ppr_chain_with_dangling_end(L):
    """0 -> 1 -> ... -> L-1, the last vertex dangling: its mass returns to the seed, so
    from seed m the chain behaves like a cycle of length L - m and vertices before m get 0."""
    a = inputs.from_edges(L, [(i, i + 1) for i in range(L - 1)], f"chain{L}")
    assert oracle.dangling_mask(L, a.col).tolist() == [False] * (L - 1) + [True]
    seeds = list(range(L))
    Pi = _ppr(a, seeds, tol=1e-15)["pi"]
    for c, m in enumerate(seeds):
        ref = np.zeros(L)
        for j in range(L - m):
            ref[m + j] = (1 - ALPHA) * ALPHA ** j / (1 - ALPHA ** (L - m))
        np.testing.assert_allclose(Pi[:, c], ref, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("k", [1, 4, 9])
def test_ppr_bidirected_star_closed_form(k):
    """Centre 0 and leaves 1..k linked both ways.  Seed = leaf 1: centre a/(1+a), seed
    (1-a) + a^2/((1+a)k), other leaves a^2/((1+a)k).  Seed = centre: 1/(1+a), leaves a/((1+a)k)."""
    a = inputs.bidirected_star(k)
    Pi = _ppr(a, [1, 0], tol=1e-15)["pi"]
    c = ALPHA / (1 + ALPHA)
    leaf = ALPHA * c / k
    np.testing.assert_allclose(Pi[:, 0], [c, 1 - ALPHA + leaf] + [leaf] * (k - 1), rtol=1e-12)
    np.testing.assert_allclose(Pi[:, 1], [1 / (1 + ALPHA)] + [ALPHA / ((1 + ALPHA) * k)] * k,
                               rtol=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_ppr_matches_dense_solve(seed):
    a = inputs.random_graph_transition(20 + 9 * seed, 0.07, seed)
    dense = np.zeros((a.n_rows, a.n_cols))
    for r in range(a.n_rows):
        for k in range(a.row_ptr[r], a.row_ptr[r + 1]):
            dense[r, a.col[k]] = a.val[k]
    dang = oracle.dangling_mask(a.n_rows, a.col)
    seeds = [0, int(np.flatnonzero(dang)[0]) if dang.any() else 1, a.n_rows - 1]
    Pi = _ppr(a, seeds, tol=1e-15)["pi"]
    for c, s in enumerate(seeds):
        ref = oracle.ppr_dense_solve(dense, s, ALPHA)
        np.testing.assert_allclose(Pi[:, c], ref, rtol=1e-10, atol=1e-15)
        assert oracle.ppr_residual(a.row_ptr, a.col, a.val, ref[:, None], [s], ALPHA)[0] < 1e-14


def test_ppr_invariants_rmat14():
    a = inputs.rmat_transition(14, 16, 1)
    seeds = inputs.ppr_seeds(a, 8, 3)
    dang = oracle.dangling_mask(a.n_rows, a.col)
    assert len(set(seeds.tolist())) == 8 and not dang[seeds].any()
    r = _ppr(a, seeds, fixed_iters=40)
    Pi = r["pi"]
    np.testing.assert_allclose(Pi.sum(axis=0), 1.0, atol=1e-12)     # mass conservation
    assert Pi.min() >= 0.0
    assert np.all(Pi[seeds, np.arange(8)] >= 1 - ALPHA)              # teleport lands on the seed
    h = np.array(r["resid"])
    assert np.all(h[1:] <= ALPHA * h[:-1] * (1 + 1e-9) + 1e-15)       # L1 contraction
    np.testing.assert_allclose(oracle.ppr_residual(a.row_ptr, a.col, a.val, Pi, seeds, ALPHA),
                               np.abs(oracle.ppr_step(a.row_ptr, a.col, a.val, Pi, ALPHA, dang, seeds)
                                      - Pi).sum(axis=0), rtol=1e-14)


# Differentiation: transpose, value gradients, PageRank adjoint

def _dense_of(a):
    dense = np.zeros((a.n_rows, a.n_cols))
    for r in range(a.n_rows):
        dense[r, a.col[a.row_ptr[r]:a.row_ptr[r + 1]]] = a.val[a.row_ptr[r]:a.row_ptr[r + 1]]
    return dense


@pytest.mark.parametrize("seed", range(3))
def test_transpose_matches_dense(seed):
    a = inputs.random_sparse(40 + 7 * seed, 23 + 11 * seed, 0.15, seed, empty_frac=0.2)
    rt, ct, perm = oracle.transpose_csr(a.row_ptr, a.col, a.n_cols)
    t = inputs.CSR(a.n_cols, a.n_rows, rt.astype(np.int32), ct.astype(np.int32), a.val[perm], "t")
    np.testing.assert_array_equal(_dense_of(t), _dense_of(a).T)
    for r in range(t.n_rows):
        assert np.all(np.diff(ct[rt[r]:rt[r + 1]]) > 0)


def test_sddmm_is_the_gradient_of_the_bilinear_form():
    """d(g^T A x)/d val_k = g[row_k] x[col_k] (central differences, exact for a linear form),
    and d(g^T A x)/dx = A^T g."""
    a = inputs.random_sparse(30, 20, 0.2, 4)
    rng = np.random.default_rng(1)
    g, x = rng.standard_normal(a.n_rows), rng.standard_normal(a.n_cols)

    def L(v, xx):
        return float(g @ oracle.spmv(a.row_ptr, a.col, v, xx)[0])
    grad = oracle.sddmm(a.row_ptr, a.col, g, x)
    h = 1e-3
    for k in range(a.nnz):
        e = np.zeros(a.nnz)
        e[k] = h
        fd = (L(a.val + e, x) - L(a.val - e, x)) / (2 * h)
        assert abs(fd - grad[k]) < 1e-10
    np.testing.assert_allclose(oracle.sddmm(a.row_ptr, a.col, g, x, 0.5), 0.5 * grad, rtol=1e-15)
    rt, ct, perm = oracle.transpose_csr(a.row_ptr, a.col, a.n_cols)
    gx = oracle.spmv(rt, ct, a.val[perm], g)[0]
    np.testing.assert_allclose(gx, _dense_of(a).T @ g, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_pagerank_adjoint_matches_dense_solve(seed):
    a = inputs.random_graph_transition(25 + 9 * seed, 0.08, seed)
    w = np.random.default_rng(seed).standard_normal(a.n_rows)
    lam = oracle.pagerank_adjoint(a.row_ptr, a.col, a.val, w, ALPHA, tol=1e-14)["lambda"]
    np.testing.assert_allclose(lam, oracle.pagerank_adjoint_dense(_dense_of(a), w, ALPHA),
                               rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("seed", range(2))
def test_pagerank_gradient_central_differences(seed):
    """L(val) = w^T pi(val): every value's central difference (h = 1e-6) against
    alpha lambda[row] pi[col]; the graph has dangling vertices."""
    a = inputs.random_graph_transition(18 + 5 * seed, 0.12, 10 + seed)
    assert oracle.dangling_mask(a.n_rows, a.col).any()
    w = np.random.default_rng(seed).standard_normal(a.n_rows)
    grad = oracle.pagerank_value_gradient(a.row_ptr, a.col, a.val, w, ALPHA)["grad"]

    def L(v):
        return float(w @ oracle.pagerank(a.row_ptr, a.col, v, ALPHA, tol=1e-15, max_iter=100000)["pi"])
    h = 1e-6
    for k in range(a.nnz):
        e = np.zeros(a.nnz)
        e[k] = h
        fd = (L(a.val + e) - L(a.val - e)) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(grad[k])) * 10, (k, fd, grad[k])


def test_pagerank_gradient_central_differences_rmat():
    """The differentiation workload's check in small: 64 random values of an R-MAT
    transition matrix, central differences with step 1e-3 in FP64."""
    a = inputs.rmat_transition(10, 16, 2)
    rng = np.random.default_rng(5)
    w = rng.standard_normal(a.n_rows)
    grad = oracle.pagerank_value_gradient(a.row_ptr, a.col, a.val, w, ALPHA)["grad"]
    h = 1e-3
    for k in rng.choice(a.nnz, 64, replace=False):
        e = np.zeros(a.nnz)
        e[k] = h
        lp = float(w @ oracle.pagerank(a.row_ptr, a.col, a.val + e, ALPHA, tol=1e-15, max_iter=100000)["pi"])
        lm = float(w @ oracle.pagerank(a.row_ptr, a.col, a.val - e, ALPHA, tol=1e-15, max_iter=100000)["pi"])
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-4 * abs(grad[k]) + 1e-9, (k, fd, grad[k])


# BiCGSTAB

def _csr_of_dense(d):
    return inputs.from_dense(np.asarray(d, np.float64))


@pytest.mark.parametrize("seed", range(3))
def test_bicgstab_matches_dense_solve(seed):
    rng = np.random.default_rng(seed)
    n = 40
    d = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.2) + np.diag(rng.uniform(3, 5, n))
    a = _csr_of_dense(d)
    b = rng.standard_normal(n)
    r = oracle.bicgstab(a.row_ptr, a.col, a.val, b, tol=1e-13, max_iter=500)
    np.testing.assert_allclose(r["x"], np.linalg.solve(d, b), rtol=1e-10, atol=1e-11)
    assert r["resid"][-1] <= 1e-13
    assert abs(np.linalg.norm(b - d @ r["x"]) / np.linalg.norm(b) - r["resid"][-1]) < 1e-13


def test_bicgstab_diagonal_converges_in_one_iteration():
    d = np.diag(np.arange(1.0, 9.0))
    a = _csr_of_dense(d)
    b = np.ones(8)
    r = oracle.bicgstab(a.row_ptr, a.col, a.val, b, tol=1e-12)
    # the first step's minimal-residual correction solves a diagonal system of 8 distinct
    # eigenvalues only approximately; it converges in at most 8 iterations and exactly
    assert r["iters"] <= 8
    np.testing.assert_allclose(r["x"], 1.0 / np.arange(1.0, 9.0), rtol=1e-10)
    e = np.eye(8) * 2.5
    r = oracle.bicgstab(*(lambda c: (c.row_ptr, c.col, c.val))(_csr_of_dense(e)), b, tol=1e-14)
    assert r["iters"] == 1 and np.allclose(r["x"], 0.4)


def test_bicgstab_matches_scipy():
    """The same recurrence as scipy's bicgstab (shadow residual r_0): the same number of
    iterations to the same relative tolerance, and close iterates."""
    spla = pytest.importorskip("scipy.sparse.linalg")
    sp = pytest.importorskip("scipy.sparse")
    a = inputs.road_grid(30, 20, 0.7, 3)
    rng = np.random.default_rng(1)
    xt = rng.uniform(-1, 1, a.n_rows)
    b = oracle.spmv(a.row_ptr, a.col, a.val, xt)[0]
    mine = oracle.bicgstab(a.row_ptr, a.col, a.val, b, tol=1e-8, max_iter=2000)
    A = sp.csr_matrix((a.val, a.col, a.row_ptr), shape=(a.n_rows, a.n_cols))
    count = [0]
    x, info = spla.bicgstab(A, b, rtol=1e-8, atol=0.0, maxiter=2000,
                            callback=lambda _x: count.__setitem__(0, count[0] + 1))
    assert info == 0 and mine["resid"][-1] <= 1e-8
    assert abs(mine["iters"] - count[0]) <= 1
    assert np.linalg.norm(mine["x"] - x) <= 1e-6 * np.linalg.norm(x)


def test_relative_linf_error():
    assert oracle.relative_linf_error([1.0, 2.2], [1.0, 2.0]) == pytest.approx(0.1)


# --------------------------------------------------------------------------
# Reduced-precision rounding helper
# --------------------------------------------------------------------------

def _wide_values(seed, n=20000):
    rng = np.random.default_rng(seed)
    v = np.ldexp(rng.random(n) + 0.5, rng.integers(-30, 18, n)) * rng.choice([-1, 1], n)
    # exact ties of the 11-bit and 8-bit formats
    ties16 = np.ldexp(1.0 + (2 * rng.integers(0, 1024, 200) + 1) * 2.0 ** -11, rng.integers(-10, 10, 200))
    ties8 = np.ldexp(1.0 + (2 * rng.integers(0, 128, 200) + 1) * 2.0 ** -8, rng.integers(-10, 10, 200))
    return np.concatenate([v, ties16, ties8, [0.0, 65504.0, 65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26]])


def test_round_f16_matches_numpy_half():
    v = _wide_values(1)
    assert np.array_equal(oracle.round_to_format(v, "f16"), v.astype(np.float16).astype(np.float64))


def test_round_f32_matches_numpy_single():
    v = _wide_values(2)
    assert np.array_equal(oracle.round_to_format(v, "f32"), v.astype(np.float32).astype(np.float64))


def test_round_bf16_matches_torch_on_float32_values():
    torch = pytest.importorskip("torch")
    v = _wide_values(3).astype(np.float32).astype(np.float64)   # single rounding from float32 == from float64
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_to_format(v, "bf16"), ref)


def test_f16_scale_exponent():
    for vmax in [1.0, 0.75, 1e-3, 3.0, 2.0 ** -20]:
        k = oracle.f16_scale_exponent(vmax)
        assert 2.0 ** 14 <= vmax * 2.0 ** k < 2.0 ** 15
