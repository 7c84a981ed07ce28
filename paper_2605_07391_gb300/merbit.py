"""Python binding of libmerbit.so (argument marshalling only).

Every computation runs in the CUDA library; this module converts torch
tensors to device pointers and streams, calls the C ABI declared in
include/merbit.h and raises MerbitError on a non-OK status.  There is no CPU
path: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

F32, F64, BF16, F16 = 0, 1, 2, 3
PLAIN, IR_BF16, IR_F16, IR_F32 = 0, 1, 2, 3
STATUS = {0: "OK", 1: "EINVAL", 2: "EOVERFLOW", 3: "ENOMEM", 4: "ECUDA", 5: "ENOTCONV",
          6: "EDEVICE"}
KERNELS = {"auto": 0, "classic": 1, "split": 2, "split2": 3}
MODES = {"plain": PLAIN, "ir_bf16": IR_BF16, "ir_f16": IR_F16, "ir_f32": IR_F32}
_TORCH_DT = {torch.float32: F32, torch.float64: F64, torch.bfloat16: BF16, torch.float16: F16}

EXPORTS = ["merbit_plan", "merbit_plan_ex", "merbit_plan_destroy", "merbit_plan_get_info",
           "merbit_plan_sync", "merbit_plan_set_kernel", "merbit_plan_export", "merbit_spmv",
           "merbit_spmv_ex", "merbit_spmm",
           "merbit_ppr", "merbit_spmv_host", "merbit_spmv_host_async",
           "merbit_vals_convert", "merbit_pagerank", "merbit_pagerank_ex", "merbit_spmv_noalloc",
           "merbit_spmv_noalloc_status",
           "merbit_transpose", "merbit_transpose_get", "merbit_transpose_destroy", "merbit_gather",
           "merbit_plan_set_hot_columns", "merbit_gather_probe", "merbit_plan_set_wait_limit",
           "merbit_autotune", "merbit_sddmm", "merbit_pagerank_adjoint", "merbit_batch_plan", "merbit_batch_pagerank",
           "merbit_batch_get_plan", "merbit_batch_destroy", "merbit_autotune_sigma", "merbit_bicgstab",
           "merbit_last_error",
           "merbit_version"]


class MerbitError(RuntimeError):
    def __init__(self, where: str, status: int, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("sigma", ctypes.c_int32), ("omega", ctypes.c_int32),
                ("tiles_per_block", ctypes.c_int32), ("tile_num", ctypes.c_int64),
                ("lane_num", ctypes.c_int64), ("block_num", ctypes.c_int64),
                ("tile_x", ctypes.c_void_p), ("tile_y", ctypes.c_void_p),
                ("lane_desc", ctypes.c_void_p), ("block_row", ctypes.c_void_p),
                ("desc_bytes", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libmerbit.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if path is None:
            path = _build.build()
        if not os.path.exists(path):
            raise MerbitError("load", 4, f"{path} does not exist")
        lib = ctypes.CDLL(path)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "merbit_plan": [vp, vp, i64, i64, ctypes.POINTER(vp)],
            "merbit_plan_ex": [vp, vp, i64, i64, i64, i32, i32, vp, ctypes.POINTER(vp)],
            "merbit_plan_get_info": [vp, ctypes.POINTER(PlanInfo)],
            "merbit_plan_sync": [vp, vp],
            "merbit_plan_set_kernel": [vp, ctypes.c_int],
            "merbit_gather_probe": [vp, i32, vp, vp, vp],
            "merbit_plan_set_wait_limit": [vp, i32],
            "merbit_plan_set_hot_columns": [vp, i32, dbl, vp, ctypes.POINTER(i32), ctypes.POINTER(dbl)],
            "merbit_plan_export": [vp, vp, vp, vp, vp],
            "merbit_spmv": [vp, i32, vp, vp, vp],
            "merbit_spmv_ex": [vp, i32, i32, vp, vp, vp, i32, vp],
            "merbit_spmv_host": [vp, i32, vp, vp, vp, vp],
            "merbit_spmv_host_async": [vp, i32, vp, vp, vp, vp],
            "merbit_spmm": [vp, vp, vp, vp, i64, i64, i64, vp],
            "merbit_ppr": [vp, vp, vp, i64, dbl, dbl, i32, vp, ctypes.POINTER(i32),
                           ctypes.POINTER(dbl), ctypes.POINTER(dbl), vp],
            "merbit_vals_convert": [vp, i32, vp, i32, i64, i32, ctypes.POINTER(i32), vp],
            "merbit_pagerank": [vp, i32, vp, dbl, dbl, vp],
            "merbit_pagerank_ex": [vp, i32, vp, dbl, dbl, i32, i32, i32, dbl, vp,
                                   ctypes.POINTER(i32), ctypes.POINTER(dbl), vp,
                                   ctypes.POINTER(i32), vp],
            "merbit_transpose": [vp, vp, i64, i64, i64, vp, ctypes.POINTER(vp)],
            "merbit_transpose_get": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)],
            "merbit_gather": [i32, vp, vp, vp, i64, vp],
            "merbit_sddmm": [vp, i32, vp, vp, dbl, vp, vp],
            "merbit_pagerank_adjoint": [vp, vp, i32, vp, dbl, vp, dbl, i32, vp, ctypes.POINTER(i32),
                                        ctypes.POINTER(dbl), vp],
            "merbit_batch_plan": [vp, vp, i64, i64, vp, i32, i32, vp, ctypes.POINTER(vp)],
            "merbit_batch_pagerank": [vp, i32, vp, dbl, dbl, i32, vp, vp, vp, ctypes.POINTER(i32), vp],
            "merbit_autotune_sigma": [vp, vp, i64, i64, i64, i32, vp, vp, i32, i32, vp,
                                      ctypes.POINTER(i32), vp],
            "merbit_autotune": [vp, vp, i64, i64, i64, i32, vp, vp, i32, vp, i32, vp, i32, vp, i32, i32,
                                vp, vp, vp],
            "merbit_spmv_noalloc": [vp, vp, vp, vp, vp, i64, i64, i64, vp],
            "merbit_spmv_noalloc_status": [vp],
            "merbit_bicgstab": [vp, vp, vp, vp, dbl, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl),
                                vp, ctypes.POINTER(i32), vp],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = i32
        lib.merbit_plan_destroy.argtypes = [vp]
        lib.merbit_plan_destroy.restype = None
        lib.merbit_transpose_destroy.argtypes = [vp]
        lib.merbit_transpose_destroy.restype = None
        lib.merbit_batch_destroy.argtypes = [vp]
        lib.merbit_batch_destroy.restype = None
        lib.merbit_batch_get_plan.argtypes = [vp]
        lib.merbit_batch_get_plan.restype = vp
        lib.merbit_last_error.restype = ctypes.c_char_p
        lib.merbit_version.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(where: str, status: int, allow: tuple[int, ...] = ()) -> int:
    if status != 0 and status not in allow:
        raise MerbitError(where, status, load().merbit_last_error().decode())
    return status


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if not t.is_contiguous():
        raise ValueError("tensors passed to the MERBIT library must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dt(t: torch.Tensor) -> int:
    try:
        return _TORCH_DT[t.dtype]
    except KeyError:
        raise ValueError(f"unsupported dtype {t.dtype}") from None


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("MERBIT device calls take CUDA tensors")


@dataclass
class TileArrays:
    tile_x: np.ndarray
    tile_y: np.ndarray
    lane_desc: np.ndarray
    block_row: np.ndarray


class Plan:
    """A reusable MERBIT schedule (TILE arrays + block boundary data) of one CSR pattern.

    The plan borrows ``col_idx``: the tensor is kept referenced here and must
    not be modified while the plan lives.
    """

    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, n_rows: int | None = None,
                 n_cols: int | None = None, sigma: int = 14, tiles_per_block: int = 8,
                 stream=None):
        lib = load()
        _need_cuda(row_ptr, col_idx)
        if row_ptr.dtype != torch.int32 or col_idx.dtype != torch.int32:
            raise ValueError("row_ptr and col_idx must be int32")
        n_rows = row_ptr.numel() - 1 if n_rows is None else n_rows
        n_cols = n_rows if n_cols is None else n_cols
        self._col = col_idx
        self._handle = ctypes.c_void_p()
        _check("merbit_plan_ex", lib.merbit_plan_ex(_ptr(row_ptr), _ptr(col_idx), n_rows, n_cols,
                                                   col_idx.numel(), sigma, tiles_per_block,
                                                   _stream(stream), ctypes.byref(self._handle)))
        self.n_rows, self.n_cols, self.nnz = n_rows, n_cols, col_idx.numel()
        self.sigma = sigma
        self.device = row_ptr.device

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._handle:
            raise MerbitError("plan", 1, "plan was destroyed")
        return self._handle

    def info(self) -> PlanInfo:
        inf = PlanInfo()
        _check("merbit_plan_get_info", load().merbit_plan_get_info(self.handle, ctypes.byref(inf)))
        return inf

    def tiles(self) -> TileArrays:
        """Host copies of the TILE arrays and block rows (merbit_plan_export)."""
        inf = self.info()
        t = TileArrays(np.empty(inf.tile_num + 1, np.uint32), np.empty(inf.tile_num + 1, np.uint32),
                       np.empty(inf.lane_num, np.uint64 if inf.desc_bytes == 8 else np.uint32),
                       np.empty(inf.block_num + 1, np.int32))
        _check("merbit_plan_export", load().merbit_plan_export(
            self.handle, *(ctypes.c_void_p(a.ctypes.data) for a in
                           (t.tile_x, t.tile_y, t.lane_desc, t.block_row))))
        return t

    def set_kernel(self, kernel: str):
        """Block kernel for later products (merbit_plan_set_kernel): "auto", "classic",
        "split" (three-stage ring) or "split2" (two-stage ring)."""
        _check("merbit_plan_set_kernel", load().merbit_plan_set_kernel(self.handle, KERNELS[kernel]))

    def set_wait_limit(self, polls: int):
        """merbit_plan_set_wait_limit (test aid): polls of a stage wait before it gives up;
        -1 restores the default."""
        _check("merbit_plan_set_wait_limit", load().merbit_plan_set_wait_limit(self.handle, int(polls)))

    def set_hot_columns(self, max_hot: int, min_cover: float = 0.0, stream=None) -> tuple[int, float]:
        """merbit_plan_set_hot_columns: (re)build the hot-column table (max_hot = 0 drops
        it).  Returns (columns in the table, fraction of the nonzeros they hold)."""
        n = ctypes.c_int(0)
        cov = ctypes.c_double(0.0)
        _check("merbit_plan_set_hot_columns", load().merbit_plan_set_hot_columns(
            self.handle, int(max_hot), float(min_cover), _stream(stream), ctypes.byref(n), ctypes.byref(cov)))
        return n.value, cov.value

    def gather_probe(self, x: torch.Tensor, sink: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """merbit_gather_probe: one pass of the product's x gather alone (a timing aid);
        returns the per-CTA sums (4096 entries of x's dtype)."""
        _need_cuda(x, sink)
        if sink is None:
            sink = torch.zeros(4096, dtype=x.dtype, device=x.device)
        _check("merbit_gather_probe", load().merbit_gather_probe(self.handle, _dt(x), _ptr(x), _ptr(sink),
                                                                 _stream(stream)))
        return sink

    def sync(self, stream=None):
        _check("merbit_plan_sync", load().merbit_plan_sync(self.handle, _stream(stream)))

    def destroy(self):
        if getattr(self, "_handle", None):
            load().merbit_plan_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class _DeviceArray:
    """A library-owned device array seen by torch through __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}
        self._owner = owner


class Transpose:
    """merbit_transpose: the CSR of A^T on the device (row_ptr_t, col_t, perm), owned by
    the library; the tensors below are views that keep this object alive."""

    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, n_rows: int | None = None,
                 n_cols: int | None = None, stream=None):
        lib = load()
        _need_cuda(row_ptr, col_idx)
        if row_ptr.dtype != torch.int32 or col_idx.dtype != torch.int32:
            raise ValueError("row_ptr and col_idx must be int32")
        n_rows = row_ptr.numel() - 1 if n_rows is None else n_rows
        n_cols = n_rows if n_cols is None else n_cols
        self._handle = ctypes.c_void_p()
        _check("merbit_transpose", lib.merbit_transpose(_ptr(row_ptr), _ptr(col_idx), n_rows, n_cols,
                                                       col_idx.numel(), _stream(stream),
                                                       ctypes.byref(self._handle)))
        rp, ct, pm = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check("merbit_transpose_get", lib.merbit_transpose_get(self._handle, ctypes.byref(rp),
                                                               ctypes.byref(ct), ctypes.byref(pm)))
        nnz = col_idx.numel()
        dev = row_ptr.device
        self.row_ptr_t = torch.as_tensor(_DeviceArray(rp.value, n_cols + 1, "<i4", self), device=dev)
        self.col_t = torch.as_tensor(_DeviceArray(ct.value, nnz, "<i4", self), device=dev)
        self.perm = torch.as_tensor(_DeviceArray(pm.value, nnz, "<i4", self), device=dev)
        self.n_rows, self.n_cols, self.nnz = n_cols, n_rows, nnz    # of A^T

    def plan(self, sigma: int = 14, stream=None) -> "Plan":
        """A plan of A^T (borrows col_t)."""
        return Plan(self.row_ptr_t, self.col_t, self.n_rows, self.n_cols, sigma=sigma, stream=stream)

    def destroy(self):
        if getattr(self, "_handle", None):
            load().merbit_transpose_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Batch:
    """merbit_batch_plan: many graphs as the diagonal blocks of one CSR (graph g owns the
    vertices [offsets[g], offsets[g+1])); borrows col_idx."""

    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, offsets, sigma: int = 14,
                 stream=None):
        lib = load()
        _need_cuda(row_ptr, col_idx)
        if row_ptr.dtype != torch.int32 or col_idx.dtype != torch.int32:
            raise ValueError("row_ptr and col_idx must be int32")
        self._offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self.num_graphs = self._offsets.size - 1
        self.n = row_ptr.numel() - 1
        self._col = col_idx
        self._handle = ctypes.c_void_p()
        _check("merbit_batch_plan", lib.merbit_batch_plan(
            _ptr(row_ptr), _ptr(col_idx), self.n, col_idx.numel(),
            self._offsets.ctypes.data_as(ctypes.c_void_p), self.num_graphs, sigma, _stream(stream),
            ctypes.byref(self._handle)))

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._handle:
            raise MerbitError("batch", 1, "batch was destroyed")
        return self._handle

    def set_kernel(self, kernel: str):
        """Block kernel of the batch's plan: "auto", "classic", "split" or "split2" (the
        solve is recorded again at the next call)."""
        h = ctypes.c_void_p(load().merbit_batch_get_plan(self.handle))
        _check("merbit_plan_set_kernel", load().merbit_plan_set_kernel(h, KERNELS[kernel]))

    def set_hot_columns(self, max_hot: int, min_cover: float = 0.0, stream=None) -> tuple[int, float]:
        """Hot-column table of the batch's plan (the solve is recorded again at the next call)."""
        h = ctypes.c_void_p(load().merbit_batch_get_plan(self.handle))
        n = ctypes.c_int(0)
        cov = ctypes.c_double(0.0)
        _check("merbit_plan_set_hot_columns", load().merbit_plan_set_hot_columns(
            h, int(max_hot), float(min_cover), _stream(stream), ctypes.byref(n), ctypes.byref(cov)))
        return n.value, cov.value

    def plan_info(self) -> PlanInfo:
        """merbit_plan_get_info of the batch's plan (owned by the batch)."""
        inf = PlanInfo()
        h = ctypes.c_void_p(load().merbit_batch_get_plan(self.handle))
        _check("merbit_plan_get_info", load().merbit_plan_get_info(h, ctypes.byref(inf)))
        return inf

    def pagerank(self, vals: torch.Tensor, alpha: float = 0.85, tol: float = 1e-8,
                 max_iter: int = 1000, pi: torch.Tensor | None = None, stream=None):
        """merbit_batch_pagerank.  Returns (pi, info) with per-graph iters and resid."""
        _need_cuda(vals, pi)
        if pi is None:
            pi = torch.empty(self.n, dtype=vals.dtype, device=vals.device)
        iters = np.zeros(self.num_graphs, np.int32)
        resid = np.zeros(self.num_graphs, np.float64)
        rounds = ctypes.c_int(0)
        st = _check("merbit_batch_pagerank", load().merbit_batch_pagerank(
            self.handle, _dt(vals), _ptr(vals), alpha, tol, max_iter, _ptr(pi),
            iters.ctypes.data_as(ctypes.c_void_p), resid.ctypes.data_as(ctypes.c_void_p),
            ctypes.byref(rounds), _stream(stream)), allow=(5,))
        return pi, {"iters": iters, "resid": resid, "rounds": rounds.value, "converged": st == 0}

    def destroy(self):
        if getattr(self, "_handle", None):
            load().merbit_batch_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def autotune_sigma(row_ptr: torch.Tensor, col_idx: torch.Tensor, vals: torch.Tensor,
                   n_rows: int | None = None, n_cols: int | None = None,
                   candidates=(14, 12, 10, 8, 7), reps: int = 5, stream=None) -> tuple[int, dict]:
    """merbit_autotune_sigma: the fastest steps-per-lane for this matrix and value type.
    Returns (best sigma, {sigma: ms per SpMV})."""
    _need_cuda(row_ptr, col_idx, vals)
    n_rows = row_ptr.numel() - 1 if n_rows is None else n_rows
    n_cols = n_rows if n_cols is None else n_cols
    cand = np.ascontiguousarray(np.asarray(candidates, dtype=np.int32))
    ms = np.zeros(cand.size, np.float32)
    best = ctypes.c_int(0)
    _check("merbit_autotune_sigma", load().merbit_autotune_sigma(
        _ptr(row_ptr), _ptr(col_idx), n_rows, n_cols, col_idx.numel(), _dt(vals), _ptr(vals),
        cand.ctypes.data_as(ctypes.c_void_p), cand.size, reps, _stream(stream), ctypes.byref(best),
        ms.ctypes.data_as(ctypes.c_void_p)))
    return best.value, {int(c): float(t) for c, t in zip(cand, ms)}


def autotune(row_ptr: torch.Tensor, col_idx: torch.Tensor, vals: torch.Tensor,
             n_rows: int | None = None, n_cols: int | None = None, sigmas=(14, 12, 10),
             blocks=(8,), kernels=("auto",), hots=(0,), reps: int = 5, stream=None) -> tuple[dict, dict]:
    """merbit_autotune: the fastest (sigma, tiles_per_block, kernel, hot) for this matrix and
    value type.  Returns (best, {(sigma, W, kernel, hot): ms per product or None})."""
    _need_cuda(row_ptr, col_idx, vals)
    n_rows = row_ptr.numel() - 1 if n_rows is None else n_rows
    n_cols = n_rows if n_cols is None else n_cols
    arr = [np.ascontiguousarray(np.asarray(v, dtype=np.int32)) for v in
           (sigmas, blocks, [KERNELS[k] for k in kernels], hots)]
    ms = np.zeros(int(np.prod([a.size for a in arr])), np.float32)
    best = np.zeros(4, np.int32)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check("merbit_autotune", load().merbit_autotune(
        _ptr(row_ptr), _ptr(col_idx), n_rows, n_cols, col_idx.numel(), _dt(vals), _ptr(vals),
        vp(arr[0]), arr[0].size, vp(arr[1]), arr[1].size, vp(arr[2]), arr[2].size, vp(arr[3]), arr[3].size,
        reps, _stream(stream), vp(best), vp(ms)))
    names = {v: k for k, v in KERNELS.items()}
    table, i = {}, 0
    for s_ in sigmas:
        for b in blocks:
            for h in hots:
                for k in kernels:
                    table[(int(s_), int(b), k, int(h))] = float(ms[i]) if ms[i] > 0 else None
                    i += 1
    return ({"sigma": int(best[0]), "tiles_per_block": int(best[1]), "kernel": names[int(best[2])],
             "hot": int(best[3])}, table)


def bicgstab(p: "Plan", vals: torch.Tensor | None, b: torch.Tensor, x: torch.Tensor | None = None,
             tol: float = 1e-10, max_iter: int = 20000, stream=None) -> tuple[torch.Tensor, dict]:
    """merbit_bicgstab (FP64): x with ||b - A x||_2 <= tol ||b||_2.  vals None: every value
    of the plan's matrix is 1 (no value stream).  x: initial guess (zeros if None),
    overwritten.  Returns (x, {iters, resid, status, converged, hist})."""
    _need_cuda(vals, b, x)
    if (vals is not None and vals.dtype != torch.float64) or b.dtype != torch.float64:
        raise ValueError("bicgstab takes f64 vals and b")
    if x is None:
        x = torch.zeros_like(b)
    iters, status = ctypes.c_int(0), ctypes.c_int(0)
    resid = ctypes.c_double(0.0)
    hist = np.zeros(max_iter, np.float64)
    st = _check("merbit_bicgstab", load().merbit_bicgstab(
        p.handle, _ptr(vals), _ptr(b), _ptr(x), tol, max_iter, ctypes.byref(iters),
        ctypes.byref(resid), ctypes.c_void_p(hist.ctypes.data), ctypes.byref(status),
        _stream(stream)), allow=(5,))
    return x, {"iters": iters.value, "resid": resid.value, "status": status.value,
               "converged": st == 0, "hist": hist[:iters.value].copy()}


def transpose(row_ptr, col_idx, n_rows=None, n_cols=None, stream=None) -> Transpose:
    return Transpose(row_ptr, col_idx, n_rows, n_cols, stream)


def gather(src: torch.Tensor, idx: torch.Tensor, out: torch.Tensor | None = None,
           stream=None) -> torch.Tensor:
    """merbit_gather: out[i] = src[idx[i]] (f32 or f64, idx int32)."""
    _need_cuda(src, idx, out)
    if idx.dtype != torch.int32:
        raise ValueError("idx must be int32")
    if out is None:
        out = torch.empty(idx.numel(), dtype=src.dtype, device=src.device)
    _check("merbit_gather", load().merbit_gather(_dt(src), _ptr(src), _ptr(idx), _ptr(out), idx.numel(),
                                                _stream(stream)))
    return out


def sddmm(p: "Plan", g: torch.Tensor, x: torch.Tensor, scale: float = 1.0,
          out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """merbit_sddmm: out[k] = scale * g[row(k)] * x[col(k)] over the plan's nonzeros."""
    _need_cuda(g, x, out)
    if g.dtype != x.dtype:
        raise ValueError("g and x must have the same dtype")
    if out is None:
        out = torch.empty(p.nnz, dtype=g.dtype, device=g.device)
    _check("merbit_sddmm", load().merbit_sddmm(p.handle, _dt(g), _ptr(g), _ptr(x), scale, _ptr(out),
                                              _stream(stream)))
    return out


def pagerank_adjoint(p: "Plan", pt: "Plan", vals_t: torch.Tensor, w: torch.Tensor,
                     alpha: float = 0.85, tol: float = 1e-12, max_iter: int = 10000,
                     lam: torch.Tensor | None = None, stream=None) -> tuple[torch.Tensor, dict]:
    """merbit_pagerank_adjoint: lambda with (I - alpha M)^T lambda = w; stops at
    ||lambda' - lambda||_1 <= tol * ||w||_1.  Returns (lambda, {iters, resid, converged})."""
    _need_cuda(vals_t, w, lam)
    if vals_t.dtype != w.dtype:
        raise ValueError("vals_t and w must have the same dtype")
    if lam is None:
        lam = torch.empty_like(w)
    iters = ctypes.c_int(0)
    resid = ctypes.c_double(0.0)
    st = _check("merbit_pagerank_adjoint", load().merbit_pagerank_adjoint(
        p.handle, pt.handle, _dt(vals_t), _ptr(vals_t), alpha, _ptr(w), tol, max_iter, _ptr(lam),
        ctypes.byref(iters), ctypes.byref(resid), _stream(stream)), allow=(5,))
    return lam, {"iters": iters.value, "resid": resid.value, "converged": st == 0}


def plan(row_ptr, col_idx, n_rows=None, n_cols=None, sigma=14, stream=None, tiles_per_block=8) -> Plan:
    """merbit_plan_ex: build the reusable TILE schedule of a CSR pattern."""
    return Plan(row_ptr, col_idx, n_rows, n_cols, sigma=sigma, tiles_per_block=tiles_per_block,
                stream=stream)


def spmv(p: Plan, vals: torch.Tensor, x: torch.Tensor, y: torch.Tensor | None = None,
         scale_exp: int = 0, stream=None) -> torch.Tensor:
    """merbit_spmv_ex: y = A x (y fully overwritten)."""
    _need_cuda(vals, x, y)
    xdt = _dt(x)
    if y is None:
        y = torch.empty(p.n_rows, dtype=x.dtype, device=x.device)
    _check("merbit_spmv_ex", load().merbit_spmv_ex(p.handle, _dt(vals), xdt, _ptr(vals), _ptr(x),
                                                  _ptr(y), scale_exp, _stream(stream)))
    return y


def spmm(p: Plan, vals: torch.Tensor, X: torch.Tensor, Y: torch.Tensor | None = None,
         stream=None) -> torch.Tensor:
    """merbit_spmm: Y = A X for a row-major X (n_cols x k); Y's first k columns overwritten."""
    _need_cuda(vals, X, Y)
    if X.dim() != 2 or X.dtype != torch.float32 or vals.dtype != torch.float32:
        raise ValueError("spmm takes f32 vals and a 2-D f32 X")
    if X.stride(1) != 1:
        raise ValueError("X must be row-major")
    k = X.shape[1]
    if Y is None:
        Y = torch.empty(p.n_rows, k, dtype=torch.float32, device=X.device)
    if Y.stride(1) != 1:
        raise ValueError("Y must be row-major")
    _check("merbit_spmm", load().merbit_spmm(p.handle, _ptr(vals), ctypes.c_void_p(X.data_ptr()),
                                            ctypes.c_void_p(Y.data_ptr()), k, X.stride(0),
                                            Y.stride(0), _stream(stream)))
    return Y


def ppr(p: Plan, vals: torch.Tensor, seeds, alpha: float = 0.85, tol: float = 1e-6,
        max_iter: int = 1000, Pi: torch.Tensor | None = None, stream=None) -> dict:
    """merbit_ppr: personalised PageRank for the given seed vertices (one column each).
    Returns {"pi": n x k tensor, "iters", "resid" (per column), "hist", "converged"}."""
    _need_cuda(vals, Pi)
    if vals.dtype != torch.float32:
        raise ValueError("ppr takes f32 vals")
    seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32))
    k = int(seeds.size)
    if Pi is None:
        Pi = torch.empty(p.n_rows, k, dtype=torch.float32, device=vals.device)
    if Pi.dtype != torch.float32 or tuple(Pi.shape) != (p.n_rows, k) or not Pi.is_contiguous():
        raise ValueError("Pi must be a contiguous f32 n x k tensor")
    iters = ctypes.c_int(0)
    resid = (ctypes.c_double * max(k, 1))()
    hist = (ctypes.c_double * max_iter)()
    st = _check("merbit_ppr", load().merbit_ppr(
        p.handle, _ptr(vals), seeds.ctypes.data_as(ctypes.c_void_p), k, alpha, tol, max_iter,
        ctypes.c_void_p(Pi.data_ptr()), ctypes.byref(iters), resid, hist, _stream(stream)),
        allow=(5,))
    return {"pi": Pi, "iters": iters.value, "resid": [resid[i] for i in range(k)],
            "hist": [hist[i] for i in range(iters.value)], "converged": st == 0}


def spmv_host(p: Plan, vals: torch.Tensor, x_host: torch.Tensor, y_host: torch.Tensor | None = None,
              stream=None, wait: bool = True) -> torch.Tensor:
    """merbit_spmv_host: x and y in host memory (pinned recommended); synchronous.  With
    wait=False, merbit_spmv_host_async: returns at once and consecutive calls overlap;
    call p.sync() before reading y_host or changing x_host."""
    _need_cuda(vals)
    if x_host.is_cuda:
        raise ValueError("x_host must be a CPU tensor")
    if y_host is None:
        y_host = torch.empty(p.n_rows, dtype=x_host.dtype, pin_memory=True)
    name = "merbit_spmv_host" if wait else "merbit_spmv_host_async"
    _check(name, getattr(load(), name)(p.handle, _dt(vals), _ptr(vals), _ptr(x_host), _ptr(y_host),
                                      _stream(stream)))
    return y_host


def vals_convert(src: torch.Tensor, dtype: torch.dtype, auto_scale: bool = False,
                 stream=None) -> tuple[torch.Tensor, int]:
    """merbit_vals_convert: round values to bf16 / f16 / f32 (RNE); returns (dst, scale_exp)."""
    _need_cuda(src)
    dst = torch.empty(src.numel(), dtype=dtype, device=src.device)
    k = ctypes.c_int(0)
    _check("merbit_vals_convert", load().merbit_vals_convert(
        _ptr(src), _dt(src), _ptr(dst), _TORCH_DT[dtype], src.numel(), int(auto_scale),
        ctypes.byref(k), _stream(stream)))
    return dst, k.value


def pagerank(p: Plan, vals: torch.Tensor, alpha: float = 0.85, tol: float = 1e-10,
             max_iter: int = 10000, mode: str = "plain", inner_sweeps: int = 32,
             inner_tol: float = 0.0, pi: torch.Tensor | None = None, stream=None,
             history: bool = False) -> tuple[torch.Tensor, dict]:
    """merbit_pagerank_ex.  Returns (pi, info) with info keys iters, resid, converged[, hist]."""
    _need_cuda(vals, pi)
    m = MODES[mode]
    dtype = vals.dtype if m == PLAIN else torch.float64
    if pi is None:
        pi = torch.empty(p.n_rows, dtype=dtype, device=vals.device)
    iters = ctypes.c_int(0)
    launches = ctypes.c_int(0)
    resid = ctypes.c_double(0.0)
    hist = np.zeros(max_iter + 1, np.float64) if history else None
    st = _check("merbit_pagerank_ex", load().merbit_pagerank_ex(
        p.handle, _dt(vals), _ptr(vals), alpha, tol, max_iter, m, inner_sweeps, inner_tol, _ptr(pi),
        ctypes.byref(iters), ctypes.byref(resid),
        ctypes.c_void_p(hist.ctypes.data) if history else ctypes.c_void_p(0),
        ctypes.byref(launches), _stream(stream)), allow=(5,))
    info = {"iters": iters.value, "resid": resid.value, "converged": st == 0,
            "spmv_launches": launches.value}
    if history:
        n = iters.value if m == PLAIN else iters.value + 1
        info["hist"] = hist[:n].copy()
    return pi, info


def version() -> str:
    return load().merbit_version().decode()
