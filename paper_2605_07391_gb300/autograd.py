"""torch.autograd wrappers of the MERBIT product and PageRank (the differentiation
extension).  Every forward and backward step is a call into libmerbit.so:

* ``spmv(A, vals, x)``: y = A x.  Backward: dx = A^T g on a plan of the transpose
  (values carried over by the transpose's permutation), dvals[k] = g[row] x[col].
* ``pagerank(A, vals, ...)``: the PageRank fixed point pi of Sec. 5.5.1 as a function of
  the stored values of A = P^T (each an independent parameter; the dangling set is
  fixed by the pattern).  Backward: the adjoint lambda of (I - alpha M)^T lambda = dL/dpi
  by the same SpMV kernel on A^T, then dvals[k] = alpha lambda[row] pi[col].
"""
from __future__ import annotations

import torch

from . import merbit as _mb


class Matrix:
    """A CSR pattern on the device with its plan and, built on first use, its transpose
    and the transpose's plan.  Values are passed per call, so one Matrix serves any
    values on this pattern."""

    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, n_rows: int | None = None,
                 n_cols: int | None = None, sigma: int = 14, stream=None):
        self.row_ptr, self.col_idx = row_ptr, col_idx
        self.n_rows = row_ptr.numel() - 1 if n_rows is None else n_rows
        self.n_cols = self.n_rows if n_cols is None else n_cols
        self.sigma = sigma
        self.plan = _mb.plan(row_ptr, col_idx, self.n_rows, self.n_cols, sigma=sigma, stream=stream)
        self._t = None
        self._pt = None

    def transposed(self, stream=None) -> tuple[_mb.Transpose, _mb.Plan]:
        if self._t is None:
            self._t = _mb.transpose(self.row_ptr, self.col_idx, self.n_rows, self.n_cols, stream=stream)
            self._pt = self._t.plan(sigma=self.sigma, stream=stream)
        return self._t, self._pt

    def transposed_values(self, vals: torch.Tensor, stream=None) -> torch.Tensor:
        t, _ = self.transposed(stream)
        return _mb.gather(vals, t.perm, stream=stream)


class _SpMV(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, x, A):
        ctx.A = A
        ctx.save_for_backward(vals, x)
        return _mb.spmv(A.plan, vals, x)

    @staticmethod
    def backward(ctx, gy):
        vals, x = ctx.saved_tensors
        A = ctx.A
        gy = gy.contiguous().to(x.dtype)
        gvals = gx = None
        if ctx.needs_input_grad[0]:
            gvals = _mb.sddmm(A.plan, gy, x)
        if ctx.needs_input_grad[1]:
            _, pt = A.transposed()
            gx = _mb.spmv(pt, A.transposed_values(vals), gy)
        return gvals, gx, None


def spmv(A: Matrix, vals: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """y = A x, differentiable in vals and x (f32 or f64)."""
    return _SpMV.apply(vals, x, A)


class _PageRank(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, A, alpha, tol, max_iter, adj_tol):
        pi, info = _mb.pagerank(A.plan, vals, alpha, tol=tol, max_iter=max_iter)
        ctx.A, ctx.alpha, ctx.max_iter, ctx.adj_tol = A, alpha, max_iter, adj_tol
        ctx.info = info
        ctx.save_for_backward(vals, pi)
        return pi

    @staticmethod
    def backward(ctx, gpi):
        vals, pi = ctx.saved_tensors
        A = ctx.A
        _, pt = A.transposed()
        lam, info = _mb.pagerank_adjoint(A.plan, pt, A.transposed_values(vals),
                                         gpi.contiguous().to(pi.dtype), ctx.alpha,
                                         tol=ctx.adj_tol, max_iter=ctx.max_iter)
        ctx.adjoint_info = info
        return _mb.sddmm(A.plan, lam, pi, ctx.alpha), None, None, None, None, None


def pagerank(A: Matrix, vals: torch.Tensor, alpha: float = 0.85, tol: float | None = None,
             max_iter: int = 10000, adj_tol: float | None = None) -> torch.Tensor:
    """PageRank vector pi(vals) (plain power method in vals' precision), differentiable in
    vals.  tol: L1 size of the last update (default 1e-12 for f64, 1e-7 for f32); adj_tol:
    adjoint stop relative to ||dL/dpi||_1 (default 1e-12 for f64, 1e-6 for f32)."""
    f64 = vals.dtype == torch.float64
    if tol is None:
        tol = 1e-12 if f64 else 1e-7
    if adj_tol is None:
        adj_tol = 1e-12 if f64 else 1e-6
    return _PageRank.apply(vals, A, alpha, tol, max_iter, adj_tol)
