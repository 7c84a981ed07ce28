"""Shared helpers of the GPU parity tests (upload, tolerance checks)."""
import numpy as np
import torch

import inputs
import oracle
import paper_2605_07391_gb300 as mb

TOL = {torch.float32: 1e-5, torch.float64: 1e-12}


def upload(a: inputs.CSR, dtype=torch.float32, device="cuda"):
    row_ptr = torch.from_numpy(a.row_ptr).to(device)
    col = torch.from_numpy(a.col).to(device)
    vals = torch.from_numpy(a.val).to(device=device, dtype=dtype)
    return row_ptr, col, vals


def make_plan(a: inputs.CSR, sigma=14, device="cuda"):
    row_ptr = torch.from_numpy(a.row_ptr).to(device)
    col = torch.from_numpy(a.col).to(device)
    return mb.plan(row_ptr, col, a.n_rows, a.n_cols, sigma=sigma), col


def as_f64(t: torch.Tensor) -> np.ndarray:
    return t.detach().to("cpu", torch.float64).numpy()


def check_rel(y_gpu: np.ndarray, y_ref: np.ndarray, d: np.ndarray, tol: float, what: str = ""):
    err = oracle.relative_errors(y_gpu, y_ref, d)
    worst = int(np.argmax(err)) if err.size else 0
    assert err.size == 0 or err.max() <= tol, (
        f"{what}: max rel err {err.max():.3e} > {tol:.0e} at row {worst}: gpu {y_gpu[worst]!r} "
        f"ref {y_ref[worst]!r} d {d[worst]!r}")
    return float(err.max()) if err.size else 0.0


def check_tiles(p, a: inputs.CSR, sigma: int):
    t = p.tiles()
    ref = oracle.build_tile(a.row_ptr, sigma)
    assert np.array_equal(t.tile_x, ref["tile_x"]), "tile_x differs"
    assert np.array_equal(t.tile_y, ref["tile_y"]), "tile_y differs"
    assert np.array_equal(t.lane_desc, ref["lane_desc"]), "lane_desc differs"
    if ref["tile_num"]:
        br = oracle.block_boundary_rows(ref["tile_y"], ref["tile_num"], 8)
        assert np.array_equal(t.block_row.astype(np.int64), br), "block rows differ"
    return ref
