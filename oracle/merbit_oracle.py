"""CPU oracle for the MERBIT hot path (plan, SpMV, PageRank) — TEST INFRASTRUCTURE.

This module is a plain, slow, float64 restatement of what the method
computes, written from the paper (Zhang, Yao, Jiang, Zhang, "MERBIT: A
GPU-Based SpMV Method for Iterative Workloads").  Only the tests, the smoke
check of ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA library and never imports it.

Pinned by ``tests/test_oracle_pins.py`` against: the paper's worked-example
counts (Sec. 4.1.1), a literal step-by-step merge-path walk on tiny inputs,
path invariants, dense brute-force SpMV, closed-form PageRank vectors (n-cycle,
bidirected star, in-star, 3-chain), closed-form personalised vectors (n-cycle,
chain ending in a dangling vertex, bidirected star), dense linear solves of both
fixed-point equations and of the adjoint equation, central finite differences of
the PageRank loss and of g^T A x, and BiCGSTAB against a dense solve and scipy's
implementation, and numpy's IEEE half conversion for the rounding helper.

Readings of points the paper leaves open (each is also listed in the design
notes):
  * ``offset`` (the CSR row pointer) has n+1 entries, offset[0]=0, offset[n]=m.
  * At x == offset[y+1] the walk steps down (Sec. 4.1.2, step (2)).
  * Bit k of a lane's bit_flag is its k-th step, least significant bit first;
    1 = down step.  Shifts 18/9 of the 32-bit descriptor are used for every
    sigma <= 14 (Sec. 4.1.1).
  * The long-row mark covers only lanes that exist (j < lane_num).
  * PageRank: uniform teleport, pi_0 = 1/n, dangling vertices are empty
    columns of P^T and their mass is spread uniformly; the iteration is
    pi' = alpha P^T pi + (alpha D + 1 - alpha)/n with D the dangling mass, and
    it stops when ||pi' - pi||_1 < tol (Sec. 5.5.1 leaves the rule open).
  * Personalised PageRank (the batching extension): one column per seed s, the
    teleport vector is e_s and the dangling mass also returns to s; pi_0 = e_s.
  * BiCGSTAB: unpreconditioned, shadow residual r_hat = r_0, stop at
    ||r||_2 <= tol ||b||_2 (Sec. 5.5 gives the tolerance but not the norm).
  * Differentiation (extension): every stored value of P^T is an independent
    parameter and the dangling set is fixed by the pattern; L = w^T pi gives
    dL/dA_ij = alpha lambda_i pi_j with (I - alpha M)^T lambda = w.
"""
from __future__ import annotations

import math

import numpy as np

OMEGA = 32
MSB = np.uint32(0x80000000)
LONG_ROW_SUM_THRESHOLD = 4096


# ---------------------------------------------------------------------------
# Plan: merge path and the TILE arrays (Sec. 3.3, Sec. 4.1)
# ---------------------------------------------------------------------------

def tile_counts(n: int, m: int, sigma: int, omega: int = OMEGA) -> tuple[int, int]:
    """tile_num = ceil((m+n)/(omega*sigma)), lane_num = ceil((m+n)/sigma) (Sec. 4.1.1)."""
    steps = m + n
    return -(-steps // (omega * sigma)), -(-steps // sigma)


def descriptor_fits(sigma: int, omega: int = OMEGA, bits: int = 32) -> bool:
    """Descriptor condition 2*ceil(log2(omega*sigma)) + sigma <= bits (Sec. 4.1.1 states it
    for a 32-bit word; Sec. 5.3.4 names the 64-bit word as the way to larger sigma)."""
    return 2 * math.ceil(math.log2(omega * sigma)) + sigma <= bits


def descriptor_layout(sigma: int, omega: int = OMEGA) -> tuple[int, int]:
    """(word bits, offset field width) of the lane descriptor for a sigma.

    sigma <= 14: the paper's 32-bit word with 9-bit offset fields (flag<<18 | y<<9 | x).
    15 <= sigma <= 42: a 64-bit word with 11-bit offset fields (flag<<22 | y<<11 | x); 11
    bits hold offsets below omega*sigma <= 1344 and 22 + sigma <= 64 bits hold the flags.
    """
    if sigma >= 1 and sigma <= 14 and descriptor_fits(sigma, omega) and omega * sigma <= 512:
        return 32, 9
    if 15 <= sigma <= 42 and omega * sigma <= 2048 and 22 + sigma <= 64:
        return 64, 11
    raise ValueError("lane descriptors cover sigma in [1, 42] (32-bit up to 14, 64-bit above)")


def merge_path_down_steps(row_ptr: np.ndarray) -> np.ndarray:
    """Boolean step sequence of the merge path from (0,0) to (m,n) (Sec. 3.3).

    Walking from (x, y): if x < row_ptr[y+1] the step goes right (consume a
    nonzero of row y), otherwise it goes down (row y is finished).  Row y thus
    contributes row_ptr[y+1]-row_ptr[y] right steps followed by one down step,
    and its down step is step number row_ptr[y+1] + y.
    """
    row_ptr = np.asarray(row_ptr, np.int64)
    n = row_ptr.size - 1
    m = int(row_ptr[-1])
    down = np.zeros(m + n, bool)
    down[row_ptr[1:] + np.arange(n, dtype=np.int64)] = True
    return down


def build_tile(row_ptr: np.ndarray, sigma: int, omega: int = OMEGA) -> dict:
    """TILE = {tile_x, tile_y, lane_desc} of Sec. 4.1 for a CSR row pointer.

    Lane j covers steps [j*sigma, min((j+1)*sigma, m+n)); its start coordinate
    is (number of right steps, number of down steps) before step j*sigma.  Tile
    i = lanes [i*omega, (i+1)*omega) starts where its lane 0 starts.  Offsets
    are lane start minus tile start; lane_desc = bit_flag<<18 | y_off<<9 |
    x_off (a 64-bit word bit_flag<<22 | y_off<<11 | x_off for sigma > 14,
    descriptor_layout); tile_y gets its most significant bit set when the tile has no down
    step at all (a single-row tile, Sec. 4.1.2 step (3)).  The last entry of
    tile_x / tile_y is (m, n).
    """
    bits, w = descriptor_layout(sigma, omega)
    row_ptr = np.asarray(row_ptr, np.int64)
    n = row_ptr.size - 1
    m = int(row_ptr[-1])
    steps = m + n
    tile_num, lane_num = tile_counts(n, m, sigma, omega)
    down = merge_path_down_steps(row_ptr)
    downs_before = np.zeros(steps + 1, np.int64)
    np.cumsum(down, out=downs_before[1:])

    j = np.arange(lane_num, dtype=np.int64)
    start = j * sigma
    lane_y = downs_before[start]
    lane_x = start - lane_y
    tile_of_lane = j // omega
    tile_start_lane = np.arange(tile_num, dtype=np.int64) * omega
    tx = lane_x[tile_start_lane] if tile_num else np.zeros(0, np.int64)
    ty = lane_y[tile_start_lane] if tile_num else np.zeros(0, np.int64)
    x_off = lane_x - tx[tile_of_lane]
    y_off = lane_y - ty[tile_of_lane]

    lane_len = np.minimum(sigma, steps - start)
    flags = np.zeros(lane_num, np.int64)
    for k in range(sigma):
        valid = k < lane_len
        idx = np.where(valid, start + k, 0)
        bit = valid & down[idx] if steps else np.zeros(lane_num, bool)
        flags |= bit.astype(np.int64) << k
    desc = (flags << (2 * w)) | (y_off << w) | x_off

    tile_end = np.minimum((np.arange(tile_num, dtype=np.int64) + 1) * omega * sigma, steps)
    tile_begin = np.arange(tile_num, dtype=np.int64) * omega * sigma
    downs_in_tile = downs_before[tile_end] - downs_before[tile_begin]
    tile_y = ty.astype(np.uint32)
    tile_y[downs_in_tile == 0] |= MSB

    return {
        "tile_num": tile_num,
        "lane_num": lane_num,
        "tile_x": np.concatenate([tx, [m]]).astype(np.uint32),
        "tile_y": np.concatenate([tile_y, np.array([n], np.uint32)]).astype(np.uint32),
        "lane_desc": desc.astype(np.uint32 if bits == 32 else np.uint64),
    }


def decode_lane_desc(desc: int, sigma: int = 14) -> tuple[int, int, int]:
    """(x_offset, y_offset, bit_flag) of a lane descriptor (Sec. 4.1.1)."""
    desc = int(desc)
    _, w = descriptor_layout(sigma)
    mask = (1 << w) - 1
    return desc & mask, (desc >> w) & mask, desc >> (2 * w)


def step_coordinate(tile_start: tuple[int, int], desc: int, k: int, sigma: int = 14) -> tuple[int, int]:
    """Coordinate reached after the first k steps of a lane (Sec. 4.1.1):
    (tile_x + x_offset + k_x, tile_y + y_offset + k_y), where k_y counts the set
    bits among the first k bits of bit_flag and k_x = k - k_y."""
    xo, yo, flags = decode_lane_desc(desc, sigma)
    k_y = bin(flags & ((1 << k) - 1)).count("1")
    return tile_start[0] + xo + (k - k_y), tile_start[1] + yo + k_y


def block_boundary_rows(tile_y: np.ndarray, tile_num: int, tiles_per_block: int) -> np.ndarray:
    """Row of the first coordinate of every block of tiles, plus the end row:
    entry b = ROW(tile_y[min(b*W, tile_num)]) for b = 0..ceil(tile_num/W)
    (the y_bs / y_be values of the SpMV kernel, Sec. 4.2)."""
    nb = -(-tile_num // tiles_per_block)
    idx = np.minimum(np.arange(nb + 1, dtype=np.int64) * tiles_per_block, tile_num)
    return (np.asarray(tile_y, np.uint32)[idx] & np.uint32(0x7FFFFFFF)).astype(np.int64)


# ---------------------------------------------------------------------------
# SpMV y = A x (Sec. 3.1)
# ---------------------------------------------------------------------------

def _row_ids(row_ptr: np.ndarray) -> np.ndarray:
    lens = np.diff(np.asarray(row_ptr, np.int64))
    return np.repeat(np.arange(lens.size, dtype=np.int64), lens)


def spmv(row_ptr, col, val, x) -> tuple[np.ndarray, np.ndarray]:
    """y_i = sum_k val[k] * x[col[k]] over k in [row_ptr[i], row_ptr[i+1]) in float64.

    Returns (y, d) with d_i = sum_k |val[k] * x[col[k]]|, the scale used by the
    parity bound |y_gpu_i - y_i| <= tol * d_i.  Rows are summed in storage
    order; rows longer than LONG_ROW_SUM_THRESHOLD entries use math.fsum
    (correctly rounded) so the oracle's own rounding stays far below the
    float64 parity bound even for rows with millions of entries.
    """
    row_ptr = np.asarray(row_ptr, np.int64)
    n = row_ptr.size - 1
    prod = np.asarray(val, np.float64) * np.asarray(x, np.float64)[np.asarray(col, np.int64)]
    rows = _row_ids(row_ptr)
    y = np.bincount(rows, weights=prod, minlength=n).astype(np.float64)
    d = np.bincount(rows, weights=np.abs(prod), minlength=n).astype(np.float64)
    lens = np.diff(row_ptr)
    for r in np.nonzero(lens > LONG_ROW_SUM_THRESHOLD)[0]:
        seg = prod[row_ptr[r]:row_ptr[r + 1]]
        y[r] = math.fsum(seg.tolist())
        d[r] = math.fsum(np.abs(seg).tolist())
    return y, d


def spmm(row_ptr, col, val, X) -> tuple[np.ndarray, np.ndarray]:
    """Y = A X for a dense X (n_cols x k): column j of Y is spmv() of column j of X.
    Returns (Y, D) with D the per-entry scale sum_k |val[k] * X[col[k], j]|."""
    X = np.asarray(X, np.float64)
    cols = [spmv(row_ptr, col, val, X[:, j]) for j in range(X.shape[1])]
    return (np.stack([c[0] for c in cols], axis=1) if cols else np.zeros((len(row_ptr) - 1, 0)),
            np.stack([c[1] for c in cols], axis=1) if cols else np.zeros((len(row_ptr) - 1, 0)))


def spmv_rows(row_ptr, col, val, x, rows) -> tuple[np.ndarray, np.ndarray]:
    """spmv() evaluated only at the listed rows (for sampled checks at full size)."""
    row_ptr = np.asarray(row_ptr, np.int64)
    x = np.asarray(x, np.float64)
    y = np.empty(len(rows))
    d = np.empty(len(rows))
    for t, r in enumerate(rows):
        lo, hi = int(row_ptr[r]), int(row_ptr[r + 1])
        p = np.asarray(val[lo:hi], np.float64) * x[np.asarray(col[lo:hi], np.int64)]
        y[t] = math.fsum(p.tolist())
        d[t] = math.fsum(np.abs(p).tolist())
    return y, d


def relative_errors(y_test: np.ndarray, y_ref: np.ndarray, d: np.ndarray) -> np.ndarray:
    """|y_test - y_ref| / d per row; rows with d == 0 give 0 if y_test is exactly 0, else inf."""
    y_test = np.asarray(y_test, np.float64)
    diff = np.abs(y_test - y_ref)
    out = np.zeros_like(diff)
    nz = d > 0
    out[nz] = diff[nz] / d[nz]
    out[~nz] = np.where(y_test[~nz] == 0.0, 0.0, np.inf)
    return out


# ---------------------------------------------------------------------------
# PageRank (Sec. 5.5.1)
# ---------------------------------------------------------------------------

def dangling_mask(n: int, col) -> np.ndarray:
    """Vertex j is dangling (out-degree 0) iff column j of P^T holds no entry."""
    mask = np.ones(n, bool)
    mask[np.asarray(col, np.int64)] = False
    return mask


def pagerank_step(row_ptr, col, val, pi, alpha, dangling) -> np.ndarray:
    """One power step pi' = alpha P^T pi + (alpha D + 1 - alpha)/n, D = sum of pi over dangling."""
    n = pi.size
    D = float(np.sum(pi[dangling]))
    y, _ = spmv(row_ptr, col, val, pi)
    return alpha * y + (alpha * D + (1.0 - alpha)) / n


def pagerank(row_ptr, col, val, alpha: float = 0.85, tol: float = 1e-10,
             max_iter: int = 1000, fixed_iters: int | None = None) -> dict:
    """Power method from pi_0 = 1/n; stops when ||pi_{k+1} - pi_k||_1 < tol.

    With ``fixed_iters`` it performs exactly that many updates instead.
    Returns pi, the number of updates and the residual history.
    """
    n = np.asarray(row_ptr).size - 1
    dangling = dangling_mask(n, col)
    pi = np.full(n, 1.0 / n)
    hist = []
    iters = fixed_iters if fixed_iters is not None else max_iter
    for _ in range(iters):
        nxt = pagerank_step(row_ptr, col, val, pi, alpha, dangling)
        r = float(np.sum(np.abs(nxt - pi)))
        hist.append(r)
        pi = nxt
        if fixed_iters is None and r < tol:
            break
    return {"pi": pi, "iters": len(hist), "resid": hist}


def pagerank_residual(row_ptr, col, val, pi, alpha: float = 0.85) -> float:
    """||b - M pi||_1 with M = I - alpha P^T - (alpha/n) 1 d^T, b = (1-alpha)/n 1,
    d the dangling indicator.  When sum(pi) = 1 this equals the L1 size of one
    power step taken from pi."""
    pi = np.asarray(pi, np.float64)
    n = pi.size
    dangling = dangling_mask(n, col)
    y, _ = spmv(row_ptr, col, val, pi)
    r = (1.0 - alpha) / n + alpha * y + (alpha / n) * float(np.sum(pi[dangling])) - pi
    return float(np.sum(np.abs(r)))


def pagerank_dense_solve(dense_pt: np.ndarray, alpha: float = 0.85) -> np.ndarray:
    """Fixed point of the power step as a linear system M pi = b (n <= 64)."""
    dense_pt = np.asarray(dense_pt, np.float64)
    n = dense_pt.shape[0]
    d = ~np.any(dense_pt != 0, axis=0)
    M = np.eye(n) - alpha * dense_pt - (alpha / n) * np.outer(np.ones(n), d.astype(np.float64))
    b = np.full(n, (1.0 - alpha) / n)
    return np.linalg.solve(M, b)


def ppr_step(row_ptr, col, val, Pi, alpha, dangling, seeds) -> np.ndarray:
    """One personalised power step for every column c of Pi (n x k):
    Pi'[:, c] = alpha P^T Pi[:, c] + (alpha D_c + 1 - alpha) e_{seeds[c]},
    D_c the mass of Pi[:, c] on dangling vertices (teleport and dangling mass go to the seed)."""
    Y, _ = spmm(row_ptr, col, val, Pi)
    Y = alpha * Y
    D = Pi[dangling].sum(axis=0)
    for c, s in enumerate(seeds):
        Y[s, c] += alpha * D[c] + (1.0 - alpha)
    return Y


def personalized_pagerank(row_ptr, col, val, seeds, alpha: float = 0.85, tol: float = 1e-10,
                          max_iter: int = 1000, fixed_iters: int | None = None) -> dict:
    """Power method per seed from Pi_0 = [e_s ...]; stops when every column's
    ||pi' - pi||_1 < tol, or after exactly ``fixed_iters`` updates.  Returns Pi (n x k),
    the number of updates, the per-update largest column residual and the last
    per-column residuals."""
    n = np.asarray(row_ptr).size - 1
    seeds = [int(s) for s in seeds]
    dangling = dangling_mask(n, col)
    Pi = np.zeros((n, len(seeds)))
    for c, s in enumerate(seeds):
        Pi[s, c] = 1.0
    hist, last = [], np.zeros(len(seeds))
    iters = fixed_iters if fixed_iters is not None else max_iter
    for _ in range(iters):
        nxt = ppr_step(row_ptr, col, val, Pi, alpha, dangling, seeds)
        last = np.abs(nxt - Pi).sum(axis=0)
        hist.append(float(last.max()))
        Pi = nxt
        if fixed_iters is None and hist[-1] < tol:
            break
    return {"pi": Pi, "iters": len(hist), "resid": hist, "last": last}


def ppr_residual(row_ptr, col, val, Pi, seeds, alpha: float = 0.85) -> np.ndarray:
    """Per column, ||b_s - M_s pi||_1 with M_s = I - alpha P^T - alpha e_s d^T and
    b_s = (1 - alpha) e_s (d the dangling indicator): the L1 size of one personalised
    power step taken from pi."""
    Pi = np.asarray(Pi, np.float64)
    n = Pi.shape[0]
    dangling = dangling_mask(n, col)
    return np.abs(ppr_step(row_ptr, col, val, Pi, alpha, dangling, seeds) - Pi).sum(axis=0)


def ppr_dense_solve(dense_pt: np.ndarray, seed: int, alpha: float = 0.85) -> np.ndarray:
    """Fixed point of the personalised step as a linear system (n <= 64):
    (I - alpha P^T - alpha e_s d^T) pi = (1 - alpha) e_s."""
    dense_pt = np.asarray(dense_pt, np.float64)
    n = dense_pt.shape[0]
    d = ~np.any(dense_pt != 0, axis=0)
    e = np.zeros(n)
    e[seed] = 1.0
    M = np.eye(n) - alpha * dense_pt - alpha * np.outer(e, d.astype(np.float64))
    return np.linalg.solve(M, (1.0 - alpha) * e)


# ---------------------------------------------------------------------------
# Differentiation (extension): transpose, value gradients, PageRank adjoint
# ---------------------------------------------------------------------------

def transpose_csr(row_ptr, col, n_cols: int):
    """CSR of A^T: (row_ptr_t, col_t, perm) with A^T's k-th nonzero = A's nonzero perm[k];
    each row of A^T lists its columns (A's rows) in increasing order."""
    col = np.asarray(col, np.int64)
    perm = np.argsort(col, kind="stable")
    row_ptr_t = np.zeros(n_cols + 1, np.int64)
    np.cumsum(np.bincount(col, minlength=n_cols), out=row_ptr_t[1:])
    return row_ptr_t, _row_ids(row_ptr)[perm], perm


def sddmm(row_ptr, col, g, x, scale: float = 1.0) -> np.ndarray:
    """out[k] = scale * g[row(k)] * x[col(k)]: the value gradient of g^T A x."""
    rows = _row_ids(row_ptr)
    return (scale * np.asarray(g, np.float64)[rows]) * np.asarray(x, np.float64)[np.asarray(col, np.int64)]


def pagerank_adjoint(row_ptr, col, val, w, alpha: float = 0.85, tol: float = 1e-13,
                     max_iter: int = 10000) -> dict:
    """lambda with (I - alpha M)^T lambda = w, M = A + (1/n) 1 d^T the PageRank operator of
    pagerank_step: iterates lambda' = alpha A^T lambda + alpha (sum(lambda)/n) d + w from
    lambda_0 = w until ||lambda' - lambda||_1 < tol."""
    n = np.asarray(row_ptr).size - 1
    d = dangling_mask(n, col)
    rt, ct, perm = transpose_csr(row_ptr, col, n)
    vt = np.asarray(val, np.float64)[perm]
    w = np.asarray(w, np.float64)
    lam = w.copy()
    hist = []
    for _ in range(max_iter):
        y, _ = spmv(rt, ct, vt, lam)
        nxt = alpha * y + w + (alpha * lam.sum() / n) * d
        hist.append(float(np.abs(nxt - lam).sum()))
        lam = nxt
        if hist[-1] < tol:
            break
    return {"lambda": lam, "iters": len(hist), "resid": hist}


def pagerank_adjoint_dense(dense_pt: np.ndarray, w, alpha: float = 0.85) -> np.ndarray:
    """Dense solve of (I - alpha M)^T lambda = w (n <= 64)."""
    dense_pt = np.asarray(dense_pt, np.float64)
    n = dense_pt.shape[0]
    d = ~np.any(dense_pt != 0, axis=0)
    M = dense_pt + (1.0 / n) * np.outer(np.ones(n), d.astype(np.float64))
    return np.linalg.solve((np.eye(n) - alpha * M).T, np.asarray(w, np.float64))


def pagerank_value_gradient(row_ptr, col, val, w, alpha: float = 0.85, tol: float = 1e-13) -> dict:
    """dL/dval for L = w^T pi at the PageRank fixed point, every stored value of A = P^T
    taken as an independent parameter (the dangling set fixed by the pattern):
    dL/dA_ij = alpha lambda_i pi_j with lambda from pagerank_adjoint."""
    pi = pagerank(row_ptr, col, val, alpha, tol=tol, max_iter=100000)["pi"]
    lam = pagerank_adjoint(row_ptr, col, val, w, alpha, tol=tol)["lambda"]
    return {"grad": sddmm(row_ptr, col, lam, pi, alpha), "pi": pi, "lambda": lam}


# ---------------------------------------------------------------------------
# BiCGSTAB on the SpMV (Sec. 5.5: the second iterative workload)
# ---------------------------------------------------------------------------

def bicgstab(row_ptr, col, val, b, x0=None, tol: float = 1e-10, max_iter: int = 20000) -> dict:
    """Unpreconditioned BiCGSTAB (van der Vorst) for A x = b in float64, shadow residual
    r_hat = r_0, stopping when ||r||_2 <= tol ||b||_2 or after max_iter iterations.
    Per iteration: rho = (r_hat, r); beta = (rho / rho_prev)(alpha / omega);
    p = r + beta (p - omega v); v = A p; alpha = rho / (r_hat, v); s = r - alpha v;
    t = A s; omega = (t, s) / (t, t); x += alpha p + omega s; r = s - omega t.
    Returns x, the iterations, and ||r||_2 / ||b||_2 after each iteration."""
    b = np.asarray(b, np.float64)
    n = b.size
    x = np.zeros(n) if x0 is None else np.asarray(x0, np.float64).copy()
    r = b - spmv(row_ptr, col, val, x)[0]
    r_hat = r.copy()
    p = np.zeros(n)
    v = np.zeros(n)
    rho_prev = alpha = omega = 1.0
    bnorm = float(np.linalg.norm(b))
    hist = []
    rho = float(r_hat @ r)
    it = 0
    if np.linalg.norm(r) <= tol * bnorm:
        return {"x": x, "iters": 0, "resid": hist}
    while it < max_iter:
        beta = (rho / rho_prev) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = spmv(row_ptr, col, val, p)[0]
        alpha = rho / float(r_hat @ v)
        s = r - alpha * v
        t = spmv(row_ptr, col, val, s)[0]
        tt = float(t @ t)
        omega = float(t @ s) / tt if tt > 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        it += 1
        rel = float(np.linalg.norm(r)) / bnorm
        hist.append(rel)
        if rel <= tol or omega == 0.0:
            break
        rho_prev, rho = rho, float(r_hat @ r)
        if rho == 0.0:
            break
    return {"x": x, "iters": it, "resid": hist}


def relative_linf_error(pi, pi_star) -> float:
    """ERR = max_i |pi_i - pi*_i| / pi*_i (Sec. 5.5.1)."""
    pi_star = np.asarray(pi_star, np.float64)
    return float(np.max(np.abs(np.asarray(pi, np.float64) - pi_star) / pi_star))


# ---------------------------------------------------------------------------
# Reduced-precision matrix values for the mixed-precision solver
# ---------------------------------------------------------------------------

_FORMATS = {"bf16": (8, -126, 127), "f16": (11, -14, 15), "f32": (24, -126, 127)}


def round_to_format(v, fmt: str) -> np.ndarray:
    """Round float64 values to the nearest value of a binary format, ties to even.

    fmt is 'bf16' (8 significand bits), 'f16' (11) or 'f32' (24).  For |v| in
    [2^e, 2^(e+1)) the spacing is 2^(e-p+1), clamped below by the subnormal
    spacing 2^(emin-p+1); dividing by a power of two is exact and numpy's rint
    rounds half to even, so q*spacing is the correctly rounded value.  Values
    that round above the largest finite value become +-inf.
    """
    p, emin, emax = _FORMATS[fmt]
    v = np.asarray(v, np.float64)
    out = np.zeros_like(v)
    nz = v != 0
    a = np.abs(v[nz])
    _, e2 = np.frexp(a)          # a = f * 2^e2 with f in [0.5, 1) -> exponent e = e2 - 1
    e = np.maximum(e2 - 1, emin)
    spacing = np.ldexp(1.0, (e - p + 1).astype(np.int64))
    q = np.rint(a / spacing) * spacing
    max_finite = (2.0 - 2.0 ** (1 - p)) * 2.0 ** emax
    q = np.where(q > max_finite, np.inf, q)
    out[nz] = np.copysign(q, v[nz])
    return out


def f16_scale_exponent(max_abs: float) -> int:
    """Power-of-two exponent k with max_abs * 2^k in [2^14, 2^15): the largest
    scale that keeps every scaled value below the half-precision maximum."""
    if max_abs <= 0 or not np.isfinite(max_abs):
        return 0
    _, e2 = math.frexp(max_abs)   # max_abs in [2^(e2-1), 2^e2)
    return 15 - e2


def spmv_lowprec_reference(row_ptr, col, val64, x, fmt: str) -> tuple[np.ndarray, np.ndarray, int]:
    """Exact (float64) product of the reduced-precision matrix with x.

    bf16 / f32: values are rounded directly.  f16: values are scaled by 2^k
    (k from f16_scale_exponent) before rounding and the product is scaled back
    by 2^-k.  Returns (y, d, k).
    """
    val64 = np.asarray(val64, np.float64)
    k = 0
    if fmt == "f16":
        k = f16_scale_exponent(float(np.max(np.abs(val64))) if val64.size else 0.0)
    lo = round_to_format(np.ldexp(val64, k), fmt)
    y, d = spmv(row_ptr, col, lo, x)
    return np.ldexp(y, -k), np.ldexp(d, -k), k
