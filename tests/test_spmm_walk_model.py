"""CPU model of the SpMM kernel's row assembly (the lane walk of Sec. 4.2, k values wide).

The kernel walks a tile's 32 lanes in passes of L lanes (L = 32 / threads per lane).  In a
lane, a down step ends a row; rows ended after the lane's first down step lie inside the
lane and are written directly, the lane's first ended row totals the run flowing in plus
the lane's head sum, and the run open after the lane flows on (the linear recurrence
OC_l = a_l + b_l * OC_{l-1}, carried from pass to pass).  A tile's first row and the run
open at its end go to a per-block table that adds up rows spread over several tiles;
the block's first and last rows go to accumulators shared between blocks.

This model replays those rules on the oracle's own plan (no GPU code involved) and checks
that every row is written exactly once and equals the oracle's product, for every pass
width the kernel uses.  Scalar columns suffice: columns never interact."""
import numpy as np
import pytest

import inputs
import oracle

MSB = 0x80000000
W = 8


def _popc(v: int) -> int:
    return bin(v).count("1")


def _model_spmv(a, x, sigma, L):
    t = oracle.build_tile(a.row_ptr, sigma)
    tx, ty = t["tile_x"].astype(np.int64), t["tile_y"].astype(np.int64)
    desc = t["lane_desc"].astype(np.int64)
    n = a.n_rows
    steps = int(a.row_ptr[-1]) + n
    prod = a.val * x[a.col]
    nb = -(-t["tile_num"] // W)
    br = oracle.block_boundary_rows(t["tile_y"], t["tile_num"], W)
    y = np.zeros(n)
    writes = np.zeros(n, np.int64)
    shared = {}
    for v in range(nb):
        y_bs, y_be = int(br[v]), int(br[v + 1])
        table = [(-1, 0.0)] * (2 * W)

        def emit(r, val, last, warp, y_ws):
            if r >= n:
                return
            if r in (y_bs, y_be):
                shared[r] = shared.get(r, 0.0) + val
            elif last or r == y_ws:
                table[2 * warp + (1 if last else 0)] = (r, val)
            else:
                y[r] = val
                writes[r] += 1

        for warp in range(W):
            ti = v * W + warp
            if ti >= t["tile_num"]:
                continue
            x0, x1, y_ws = tx[ti], tx[ti + 1], int(ty[ti] & ~MSB)
            if ty[ti] & MSB:                       # single-row tile
                emit(y_ws, float(prod[x0:x1].sum()), True, warp, y_ws)
                continue
            carry, open_row = 0.0, y_ws
            for p in range(32 // L):
                A, B, head, y0s, dms = [], [], [], [], []
                for gl in range(L):
                    j = ti * 32 + p * L + gl
                    active = j < t["lane_num"]
                    d = int(desc[j]) if active else 0
                    ln = min(sigma, steps - j * sigma) if active else 0
                    dm = (d >> 18) & ((1 << ln) - 1)
                    xo, y0 = d & 511, ((d >> 9) & 511) if active else n - y_ws
                    s, h, nd = 0.0, 0.0, 0
                    for k in range(ln):
                        if (dm >> k) & 1:
                            if nd == 0:
                                h = s
                            else:
                                y[y_ws + y0 + nd] = s
                                writes[y_ws + y0 + nd] += 1
                            s, nd = 0.0, nd + 1
                        else:
                            s += prod[x0 + xo + k - nd]
                    A.append(s)
                    B.append(0 if dm else 1)
                    head.append(h)
                    y0s.append(y0)
                    dms.append(dm)
                if B[0]:
                    A[0] += carry
                B[0] = 0
                dd = 1
                while dd < L:                      # Hillis-Steele scan of the recurrence
                    A = [A[i] + (A[i - dd] if i >= dd and B[i] else 0.0) for i in range(L)]
                    B = [B[i] & B[i - dd] if i >= dd else B[i] for i in range(L)]
                    dd <<= 1
                for gl in range(L):
                    if dms[gl]:
                        emit(y_ws + y0s[gl], head[gl] + (carry if gl == 0 else A[gl - 1]), False, warp, y_ws)
                carry = A[L - 1]
                open_row = y_ws + y0s[L - 1] + _popc(dms[L - 1])
            emit(open_row, carry, True, warp, y_ws)
        for e in range(2 * W):                     # the block's cross-warp table
            r = table[e][0]
            prev = e - 1
            while prev >= 0 and table[prev][0] < 0:
                prev -= 1
            if r < 0 or (prev >= 0 and table[prev][0] == r):
                continue
            tot = 0.0
            for q in range(e, 2 * W):
                if table[q][0] < 0:
                    continue
                if table[q][0] != r:
                    break
                tot += table[q][1]
            y[r] = tot
            writes[r] += 1
    for r, s in shared.items():
        y[r] = s
        writes[r] += 1
    return y, writes


CASES = {
    "rmat9_hubs": lambda: inputs.add_hubs(inputs.rmat_uniform(9, 8, 3, 3), 2, 600, 1500, 5),
    "ragged": lambda: inputs.row_lengths_csr([0, 1, 900, 0, 0, 3, 448, 447, 449, 0, 13, 14, 15] * 3, 1200, 2),
    "empty30": lambda: inputs.empty_rows(inputs.rmat_uniform(8, 16, 4, 4), 0.3, 4),
}


@pytest.mark.parametrize("L", [32, 16, 8, 4, 1])
@pytest.mark.parametrize("sigma", [14, 5])
@pytest.mark.parametrize("case", sorted(CASES))
def test_lane_walk_writes_every_row_once(case, sigma, L):
    a = CASES[case]()
    x = np.random.default_rng(1).random(a.n_cols)
    y, writes = _model_spmv(a, x, sigma, L)
    assert (writes == 1).all(), np.flatnonzero(writes != 1)[:10]
    ref, d = oracle.spmv(a.row_ptr, a.col, a.val, x)
    assert oracle.relative_errors(y, ref, d).max() <= 1e-12
