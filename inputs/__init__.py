"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only PRODUCES matrices and vectors; it contains none of the
SpMV / PageRank arithmetic.  Large generators run in ``gen.cpp`` (OpenMP,
counter-based splitmix64 draws, so the output is identical on any machine and
thread count); small hand-built matrices are written out in numpy here.

Input recipe (R-MAT, Chakrabarti et al. 2004): ``2**scale`` vertices,
``edge_factor * 2**scale`` edge draws with quadrant probabilities
a/b/c/d = 0.57/0.19/0.19/0.05, no noise and no vertex relabelling; self loops
and duplicate edges are dropped.  The stored matrix is the CSR of P^T (rows =
destination vertices, columns = source vertices, columns sorted within a
row), so ``y = P^T x`` is the PageRank propagation step; dangling vertices
(no out-edge, i.e. an empty column) are kept.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmerbit_gen.so")
_lock = threading.Lock()
_lib_handle = None


def build(force: bool = False) -> str:
    """Compile gen.cpp into inputs/_build/libmerbit_gen.so (host code only)."""
    src = os.path.join(_HERE, "gen.cpp")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O3", "-fopenmp", "-shared", "-fPIC", "-std=c++17",
                           src, "-o", tmp])
    os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    with _lock:
        if _lib_handle is None:
            lib = ctypes.CDLL(build())
            i64, u64, i32, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
            lib.gen_rmat_keys.argtypes = [i32, i64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, u64, vp]
            lib.gen_uniform_keys.argtypes = [i64, i64, i32, i64, u64, vp]
            lib.keys_sort_unique.argtypes = [vp, vp, i64, i32, i32, i32]
            lib.keys_sort_unique.restype = i64
            lib.keys_to_csr.argtypes = [vp, i64, i32, i64, vp, vp]
            lib.vals_transition.argtypes = [vp, i64, i64, vp]
            lib.fill_uniform_open0.argtypes = [i64, u64, u64, vp]
            lib.fill_uniform_open1.argtypes = [i64, u64, u64, vp]
            lib.fill_draws.argtypes = [i64, u64, u64, vp]
            lib.gen_num_threads.restype = i32
            _lib_handle = lib
        return _lib_handle


def _p(a: np.ndarray) -> ctypes.c_void_p:
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


@dataclass
class CSR:
    """A CSR matrix: row_ptr int32[n_rows+1], col int32[nnz], val float64[nnz]."""
    n_rows: int
    n_cols: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def check(self) -> "CSR":
        assert self.row_ptr.dtype == np.int32 and self.col.dtype == np.int32
        assert self.row_ptr.shape == (self.n_rows + 1,) and self.row_ptr[0] == 0
        assert self.col.shape == (self.nnz,) and self.val.shape == (self.nnz,)
        assert np.all(np.diff(self.row_ptr) >= 0)
        if self.nnz:
            assert self.col.min() >= 0 and self.col.max() < self.n_cols
        return self


def _bits(n: int) -> int:
    return max(1, int(n - 1).bit_length())


def _from_keys(keys: np.ndarray, n_rows: int, n_cols: int, col_bits: int, row_bits: int,
               drop_diag: bool) -> tuple[np.ndarray, np.ndarray]:
    lib = _lib()
    tmp = np.empty_like(keys)
    nnz = lib.keys_sort_unique(_p(keys), _p(tmp), keys.size, col_bits, row_bits, int(drop_diag))
    del tmp
    row_ptr = np.empty(n_rows + 1, np.int32)
    col = np.empty(nnz, np.int32)
    lib.keys_to_csr(_p(keys), nnz, col_bits, n_rows, _p(row_ptr), _p(col))
    return row_ptr, col


def rmat_pattern(scale: int, edge_factor: int, seed: int,
                 abc: tuple[float, float, float] = (0.57, 0.19, 0.19)) -> tuple[np.ndarray, np.ndarray]:
    """Pattern of A^T for an R-MAT graph (self loops and duplicates dropped)."""
    n = 1 << scale
    n_edges = edge_factor * n
    keys = np.empty(n_edges, np.uint64)
    _lib().gen_rmat_keys(scale, n_edges, abc[0], abc[1], abc[2], seed, _p(keys))
    return _from_keys(keys, n, n, scale, scale, True)


def rmat_transition(scale: int, edge_factor: int = 16, seed: int = 1) -> CSR:
    """CSR of P^T for an R-MAT graph; entry (dst, src) = 1/outdeg(src) in float64."""
    n = 1 << scale
    row_ptr, col = rmat_pattern(scale, edge_factor, seed)
    val = np.empty(col.size, np.float64)
    _lib().vals_transition(_p(col), col.size, n, _p(val))
    return CSR(n, n, row_ptr, col, val, f"rmat{scale}_ef{edge_factor}_transition",
               {"scale": scale, "edge_factor": edge_factor, "seed": seed})


def block_diagonal(parts: list) -> tuple[CSR, np.ndarray]:
    """Square CSR matrices as the diagonal blocks of one CSR; returns (CSR, offsets) with
    offsets[g] the first row / column of block g (int64, len(parts) + 1)."""
    sizes = np.array([p.n_rows for p in parts], np.int64)
    nnzs = np.array([p.nnz for p in parts], np.int64)
    off = np.zeros(len(parts) + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    zoff = np.zeros(len(parts) + 1, np.int64)
    np.cumsum(nnzs, out=zoff[1:])
    n, nnz = int(off[-1]), int(zoff[-1])
    if n + nnz >= 2**31:
        raise ValueError("batch too large for int32 indices")
    row_ptr = np.empty(n + 1, np.int32)
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz, np.float64)
    for g, p in enumerate(parts):
        assert p.n_rows == p.n_cols
        row_ptr[off[g]:off[g + 1]] = p.row_ptr[:-1] + zoff[g]
        col[zoff[g]:zoff[g + 1]] = p.col + off[g]
        val[zoff[g]:zoff[g + 1]] = p.val
    row_ptr[n] = nnz
    return CSR(n, n, row_ptr, col, val, f"blockdiag{len(parts)}"), off


def rmat_batch(num_graphs: int, seed: int, scales: tuple[int, int] = (10, 20),
               edge_factors: tuple[int, int] = (8, 32), threads: int = 8):
    """Many independent R-MAT transition matrices as the diagonal blocks of one CSR.

    Graph g has scale s_g and edge factor f_g drawn uniformly from the inclusive integer
    ranges (vertex counts log-uniform over powers of two) and its own generator seed.
    Returns (CSR, offsets) with offsets[g] the first vertex of graph g (int64, G + 1)."""
    import concurrent.futures as cf
    rng = np.random.default_rng(seed)
    sc = rng.integers(scales[0], scales[1] + 1, num_graphs)
    ef = rng.integers(edge_factors[0], edge_factors[1] + 1, num_graphs)
    seeds = rng.integers(1, 2**31 - 1, num_graphs)
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda g: rmat_transition(int(sc[g]), int(ef[g]), int(seeds[g])),
                            range(num_graphs)))
    csr, off = block_diagonal(parts)
    csr.name = f"rmat_batch{num_graphs}_s{seed}"
    csr.meta = {"scales": sc.tolist(), "edge_factors": ef.tolist()}
    return csr, off


# ---------------------------------------------------------------------------
# Undirected graphs with unit values (the BiCGSTAB workload's matrices)
# ---------------------------------------------------------------------------

def undirected(n: int, u: np.ndarray, v: np.ndarray, name: str, meta: dict | None = None) -> CSR:
    """Adjacency matrix (values 1) of the undirected graph with edges (u_i, v_i) on n
    vertices; self loops and repeated edges dropped."""
    bits = _bits(n)
    u = np.asarray(u, np.uint64)
    v = np.asarray(v, np.uint64)
    b = np.uint64(bits)
    keys = np.concatenate([(u << b) | v, (v << b) | u])
    row_ptr, col = _from_keys(keys, n, n, bits, bits, True)
    return CSR(n, n, row_ptr, col, np.ones(col.size), name, meta or {})


def road_grid(nx: int, ny: int, keep: float = 0.6, seed: int = 11) -> CSR:
    """Road-network stand-in: an nx x ny grid graph whose edges are kept independently
    with probability `keep` (mean degree about 4 keep); vertex ids are row-major, so
    neighbours are close in memory, as in geographically ordered road networks."""
    rng = np.random.default_rng(seed)
    idx = np.arange(nx * ny, dtype=np.int64).reshape(ny, nx)
    u = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    v = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    m = rng.random(u.size) < keep
    return undirected(nx * ny, u[m], v[m], f"road{nx}x{ny}_k{keep}", {"seed": seed})


def kmer_chains(n: int, mean_len: int = 64, extra: float = 0.02, seed: int = 12) -> CSR:
    """k-mer-graph stand-in: the vertices in random order joined into paths of geometric
    length (mean `mean_len`), plus extra*n random edges (mean degree about 2)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n).astype(np.int64)
    keep = rng.random(n - 1) >= 1.0 / mean_len
    u, v = perm[:-1][keep], perm[1:][keep]
    k = int(extra * n)
    eu, ev = rng.integers(0, n, k), rng.integers(0, n, k)
    return undirected(n, np.concatenate([u, eu]), np.concatenate([v, ev]), f"kmer{n}", {"seed": seed})


def hub_graph(scale: int, edge_factor: int = 2, seed: int = 13,
              abc: tuple[float, float, float] = (0.7, 0.1, 0.1)) -> CSR:
    """Traffic-trace stand-in: an undirected R-MAT graph with a strongly skewed degree
    distribution (a few hubs adjacent to a large share of the vertices)."""
    n = 1 << scale
    keys = np.empty(edge_factor * n, np.uint64)
    _lib().gen_rmat_keys(scale, keys.size, abc[0], abc[1], abc[2], seed, _p(keys))
    sh = np.uint64(scale)
    return undirected(n, keys >> sh, keys & np.uint64(n - 1), f"hub{scale}_ef{edge_factor}",
                      {"seed": seed})


def uniform_open0(n: int, seed: int, stream: int = 21) -> np.ndarray:
    """float64 values in (0, 1]."""
    out = np.empty(n, np.float64)
    if n:
        _lib().fill_uniform_open0(n, seed, stream, _p(out))
    return out


def uniform_vector(n: int, seed: int, stream: int = 31) -> np.ndarray:
    """float64 values in [0, 1)."""
    out = np.empty(n, np.float64)
    if n:
        _lib().fill_uniform_open1(n, seed, stream, _p(out))
    return out


def draws(n: int, seed: int, stream: int) -> np.ndarray:
    out = np.empty(n, np.uint64)
    if n:
        _lib().fill_draws(n, seed, stream, _p(out))
    return out


def rmat_uniform(scale: int, edge_factor: int = 16, seed: int = 3, val_seed: int = 3) -> CSR:
    """R-MAT pattern (rows = destinations) with values U(0,1]."""
    n = 1 << scale
    row_ptr, col = rmat_pattern(scale, edge_factor, seed)
    return CSR(n, n, row_ptr, col, uniform_open0(col.size, val_seed),
               f"rmat{scale}_ef{edge_factor}_u01", {"scale": scale, "seed": seed})


def empty_rows(a: CSR, frac: float = 0.30, seed: int = 4) -> CSR:
    """Copy of `a` with each row emptied independently with probability `frac`."""
    u = (draws(a.n_rows, seed, 41) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    keep_row = u >= frac
    lens = np.diff(a.row_ptr).astype(np.int64)
    keep_nz = np.repeat(keep_row, lens)
    new_lens = np.where(keep_row, lens, 0)
    row_ptr = np.zeros(a.n_rows + 1, np.int64)
    np.cumsum(new_lens, out=row_ptr[1:])
    return CSR(a.n_rows, a.n_cols, row_ptr.astype(np.int32), a.col[keep_nz].copy(),
               a.val[keep_nz].copy(), a.name + f"_empty{int(frac * 100)}",
               dict(a.meta, emptied_rows=int((~keep_row).sum())))


def add_hubs(a: CSR, k: int = 16, lo: int = 1_000_000, hi: int = 4_000_000, seed: int = 5,
             val_seed: int = 5) -> CSR:
    """Copy of `a` with k distinct rows replaced by hub rows.

    Hub row h gets a target length L_h ~ U[lo, hi] (capped at n_cols); each
    column is kept independently with probability L_h / n_cols, which yields
    about L_h distinct, sorted columns.  Values are U(0,1].
    """
    d = draws(4 * k + 64, seed, 51)
    rows = []
    for v in d:
        r = int(v % np.uint64(a.n_rows))
        if r not in rows:
            rows.append(r)
        if len(rows) == k:
            break
    hi_eff = min(hi, a.n_cols)
    lo_eff = min(lo, hi_eff)
    lens_target = [lo_eff + int(d[2 * k + i] % np.uint64(hi_eff - lo_eff + 1)) for i in range(k)]
    hub_cols = {}
    for i, r in enumerate(rows):
        u = (draws(a.n_cols, seed, 100 + i) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        hub_cols[r] = np.nonzero(u < lens_target[i] / a.n_cols)[0].astype(np.int32)
    lens = np.diff(a.row_ptr).astype(np.int64)
    new_lens = lens.copy()
    for r, c in hub_cols.items():
        new_lens[r] = c.size
    row_ptr = np.zeros(a.n_rows + 1, np.int64)
    np.cumsum(new_lens, out=row_ptr[1:])
    assert row_ptr[-1] < 2**31
    keep_nz = np.ones(a.nnz, bool)
    for r in hub_cols:
        keep_nz[a.row_ptr[r]:a.row_ptr[r + 1]] = False
    col = np.empty(int(row_ptr[-1]), np.int32)
    is_hub = np.zeros(a.n_rows, bool)
    is_hub[list(hub_cols)] = True
    dst_mask = np.repeat(~is_hub, new_lens)
    col[dst_mask] = a.col[keep_nz]
    for r, c in hub_cols.items():
        col[row_ptr[r]:row_ptr[r + 1]] = c
    val = uniform_open0(col.size, val_seed, 52)
    return CSR(a.n_rows, a.n_cols, row_ptr.astype(np.int32), col, val, a.name + f"_hubs{k}",
               dict(a.meta, hub_rows=sorted(hub_cols), hub_lens=[int(hub_cols[r].size) for r in sorted(hub_cols)]))


def erdos_renyi(n: int, per_row: int = 16, seed: int = 6, val_seed: int = 6) -> CSR:
    """n x n matrix from per_row*n uniform (row, col) draws, deduplicated; values U(0,1]."""
    bits = _bits(n)
    keys = np.empty(per_row * n, np.uint64)
    _lib().gen_uniform_keys(n, n, bits, keys.size, seed, _p(keys))
    row_ptr, col = _from_keys(keys, n, n, bits, bits, False)
    return CSR(n, n, row_ptr, col, uniform_open0(col.size, val_seed), f"er{n}_d{per_row}",
               {"seed": seed})


# ---------------------------------------------------------------------------
# Small hand-built matrices (test fixtures)
# ---------------------------------------------------------------------------

def from_dense(dense: np.ndarray, name: str = "dense") -> CSR:
    dense = np.asarray(dense, np.float64)
    n_rows, n_cols = dense.shape
    rows, cols = np.nonzero(dense)
    row_ptr = np.zeros(n_rows + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n_rows), out=row_ptr[1:])
    return CSR(n_rows, n_cols, row_ptr.astype(np.int32), cols.astype(np.int32),
               dense[rows, cols].copy(), name)


def from_edges(n: int, edges: list[tuple[int, int]], name: str) -> CSR:
    """Transition matrix P^T of a directed graph given as (src, dst) pairs."""
    outdeg = np.zeros(n, np.int64)
    for s, _ in edges:
        outdeg[s] += 1
    dense = np.zeros((n, n))
    for s, t in edges:
        dense[t, s] = 1.0 / outdeg[s]
    return from_dense(dense, name)


def cycle_graph(n: int) -> CSR:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], f"cycle{n}")


def bidirected_star(k: int) -> CSR:
    """Centre 0 linked both ways with leaves 1..k."""
    e = [(0, i) for i in range(1, k + 1)] + [(i, 0) for i in range(1, k + 1)]
    return from_edges(k + 1, e, f"bistar{k}")


def in_star(k: int) -> CSR:
    """Leaves 1..k each point at centre 0; the centre is dangling."""
    return from_edges(k + 1, [(i, 0) for i in range(1, k + 1)], f"instar{k}")


def ppr_seeds(a: CSR, k: int, seed: int) -> np.ndarray:
    """k distinct seed vertices drawn uniformly from the vertices with at least one
    out-edge (non-empty columns of the transition matrix P^T), as int32."""
    has_out = np.zeros(a.n_cols, bool)
    has_out[np.asarray(a.col, np.int64)] = True
    cand = np.flatnonzero(has_out)
    if cand.size < k:
        raise ValueError(f"only {cand.size} vertices have out-edges, {k} seeds asked")
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(cand, size=k, replace=False)).astype(np.int32)


def random_graph_transition(n: int, p: float, seed: int) -> CSR:
    """Small directed graph, each ordered pair (s != t) an edge w.p. p."""
    rng = np.random.default_rng(seed)
    adj = rng.random((n, n)) < p
    np.fill_diagonal(adj, False)
    edges = [(int(s), int(t)) for s, t in zip(*np.nonzero(adj))]
    return from_edges(n, edges, f"randgraph{n}_{seed}")


def random_sparse(n_rows: int, n_cols: int, density: float, seed: int,
                  empty_frac: float = 0.0, name: str = "") -> CSR:
    """Small random matrix with values U(0,1]; a fraction of rows forced empty."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n_rows, n_cols)) < density
    if empty_frac > 0:
        mask[rng.random(n_rows) < empty_frac, :] = False
    dense = np.where(mask, 1.0 - rng.random((n_rows, n_cols)), 0.0)
    return from_dense(dense, name or f"rand{n_rows}x{n_cols}_{seed}")


def row_lengths_csr(lens: list[int], n_cols: int, seed: int, name: str = "") -> CSR:
    """Matrix with prescribed row lengths (columns distinct and sorted), values U(0,1]."""
    rng = np.random.default_rng(seed)
    row_ptr = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    cols = [np.sort(rng.choice(n_cols, size=l, replace=False)) if l else np.zeros(0, np.int64)
            for l in lens]
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    val = 1.0 - rng.random(col.size)
    return CSR(len(lens), n_cols, row_ptr.astype(np.int32), col, val, name or "rowlens")
