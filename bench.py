"""Benchmark of the MERBIT hot path on one GB300 (or N independent replicas).

Workload: the R-MAT scale-24 transition matrix P^T (16,777,216 vertices, edge
factor 16, a/b/c/d = .57/.19/.19/.05, seed 7, self loops and duplicates
dropped), synthetic.  One timed step is one FP32 SpMV y = P^T x through the
plan (built once, outside the timed region, its time reported as plan_ms);
x ~ U[0,1).  The same run then times the product with FP64 values (on the sigma the
autotuner picks for them) and bf16 values, PageRank to L1 residual 1e-10 in every
precision mode, the SpMV through host buffers (e2e), the batched, many-graph,
BiCGSTAB and differentiation workloads, and the CPU oracle on a bounded sample
(cpu_baseline).

Prints ONE JSON line on rank 0.  ``--impl reference`` times the CPU oracle
instead (the reference arm of this project is the float64 oracle).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMV Gnnz/s + % HBM roofline; PageRank time to 1e-10, mixed vs plain FP32"
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, nominal (the roofline's peak is the measured copy rate)
WORKLOADS = {
    # name: (scale, edge_factor, seed)
    "rmat24_transition": (24, 16, 7),
    "rmat22_transition": (22, 16, 7),
    "rmat21_transition": (21, 16, 7),
    "rmat18_transition": (18, 16, 7),
    "rmat14_transition": (14, 16, 1),
}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "spmv_f32_rmat24_traffic.txt")
KERNEL_SOURCES = ["paper_2605_07391_gb300/csrc/spmv_kernel.cuh",
                  "paper_2605_07391_gb300/csrc/spmv_f32.cu",
                  "paper_2605_07391_gb300/csrc/merbit_internal.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernel."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    kv = {}
    for line in open(TRAFFIC_FILE):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha") != kernel_hash() or kv.get("workload") != workload:
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.6)

    def mark(self):
        self.marks.append(time.time())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = []
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(f[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                rows.append((ts, float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        lo, hi = (min(self.marks) - 1, max(self.marks) + 1) if self.marks else (-1e18, 1e18)
        inside = [r for r in rows if lo <= r[0] <= hi] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside)}


def max_over_ranks(v: float, device=None) -> float:
    """Maximum of a per-rank scalar over the process group (the value itself without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gnnz(nnz_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank processes nnz_per_rank nonzeros per step."""
    return world * nnz_per_rank / (ms_per_step * 1e-3) / 1e9


def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_sample_rate(a, budget_s: float, x64: np.ndarray, start_row: int = 0,
                       block_nnz: int | None = None):
    """Time the oracle's float64 SpMV on contiguous row blocks until budget_s is spent (at
    least one block): blocks of 1/64 of the rows, or of about block_nnz nonzeros."""
    import oracle

    nnz_done, t_used, r0 = 0, 0.0, start_row
    block = max(1, a.n_rows // 64)
    while True:
        if block_nnz is None:
            r1 = min(a.n_rows, r0 + block)
        else:
            r1 = int(np.searchsorted(a.row_ptr, a.row_ptr[r0] + block_nnz, side="right")) - 1
            r1 = min(a.n_rows, max(r0 + 1, r1))
        lo, hi = int(a.row_ptr[r0]), int(a.row_ptr[r1])
        rp = (a.row_ptr[r0:r1 + 1] - lo).astype(np.int64)
        t0 = time.perf_counter()
        oracle.spmv(rp, a.col[lo:hi], a.val[lo:hi], x64)
        t_used += time.perf_counter() - t0
        nnz_done += hi - lo
        r0 = r1 if r1 < a.n_rows else 0
        if t_used >= budget_s:
            return nnz_done, t_used


def oracle_timed(fn, unit_count: float, unit: str, sample: str, budget_s: float = 3.0) -> dict:
    """Run fn() (one bounded piece of oracle work worth unit_count units) until budget_s is
    spent; the rate is units per second on one host core (numpy is single-threaded)."""
    done, t_used = 0.0, 0.0
    while t_used < budget_s:
        t0 = time.perf_counter()
        fn()
        t_used += time.perf_counter() - t0
        done += unit_count
    return {"value": done / t_used, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample}


# ---- the oracle on all host cores: worker processes (spawned, never forked after CUDA is
# initialised) attach to the matrix in shared memory and multiply contiguous row blocks

_SHARED = {}


def _attach(spec):
    from multiprocessing import shared_memory
    for name, (shm_name, dtype, shape) in spec.items():
        shm = shared_memory.SharedMemory(name=shm_name)
        _SHARED[name] = (shm, np.ndarray(shape, dtype=dtype, buffer=shm.buf))


def _oracle_block(bounds):
    import oracle
    r0, r1 = bounds
    rp = _SHARED["row_ptr"][1]
    lo, hi = int(rp[r0]), int(rp[r1])
    oracle.spmv((rp[r0:r1 + 1] - lo).astype(np.int64), _SHARED["col"][1][lo:hi], _SHARED["val"][1][lo:hi],
                _SHARED["x"][1])
    return hi - lo


def oracle_all_cores(a, x64: np.ndarray, budget_s: float, block_nnz: int = 4_000_000) -> dict:
    """Float64 oracle SpMV on every host core: one spawned worker process per core, each
    multiplying contiguous row blocks of about block_nnz nonzeros of the shared matrix;
    blocks are handed out until budget_s of wall time is spent."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    cores = os.cpu_count() or 1
    arrays = {"row_ptr": a.row_ptr, "col": a.col, "val": a.val, "x": x64}
    shms, spec = [], {}
    try:
        for name, arr in arrays.items():
            shm = shared_memory.SharedMemory(create=True, size=max(1, arr.nbytes))
            np.ndarray(arr.shape, dtype=arr.dtype, buffer=shm.buf)[...] = arr
            shms.append(shm)
            spec[name] = (shm.name, arr.dtype.str, arr.shape)
        bounds, r0 = [], 0
        while r0 < a.n_rows:
            r1 = int(np.searchsorted(a.row_ptr, a.row_ptr[r0] + block_nnz, side="right")) - 1
            r1 = min(a.n_rows, max(r0 + 1, r1))
            bounds.append((r0, r1))
            r0 = r1
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores, initializer=_attach, initargs=(spec,)) as pool:
            pool.map(_oracle_block, bounds[:cores])          # warm the workers
            done, t0, i = 0, time.perf_counter(), 0
            while time.perf_counter() - t0 < budget_s:
                batch = [bounds[(i + j) % len(bounds)] for j in range(cores)]
                done += sum(pool.map(_oracle_block, batch))
                i += cores
            wall = time.perf_counter() - t0
        return {"value": done / wall / 1e9, "unit": "Gnnz/s", "cores": cores, "kind": "oracle",
                "sample": f"float64 oracle SpMV, {cores} spawned processes on row blocks of about "
                          f"{block_nnz} nnz, {done} nnz in {wall:.1f} s wall"}
    finally:
        for shm in shms:
            shm.close()
            shm.unlink()


def run_reference(args, rank, world):
    """Reference arm: the float64 CPU oracle on bounded samples of the same workload."""
    if rank != 0:
        return
    import inputs

    scale, ef, seed = WORKLOADS[args.workload]
    a = inputs.rmat_transition(scale, ef, seed)
    x64 = inputs.uniform_vector(a.n_cols, 2)
    per_step = max(0.01, args.ref_budget / (args.steps + args.warmup))
    # a step runs at least one block: blocks of about the nonzeros the oracle multiplies
    # in half a step's budget, from its rate on one block of 1/64 of the rows taken from
    # the middle of the matrix
    n_, t_ = oracle_sample_rate(a, 0.0, x64, start_row=a.n_rows // 2)
    block_nnz = max(1000, int(n_ / max(t_, 1e-9) * per_step / 2))
    for _ in range(args.warmup):
        oracle_sample_rate(a, per_step, x64, block_nnz=block_nnz)
    nnz_done, t_used, row = 0, 0.0, 0
    for i in range(args.steps):
        n_, t_ = oracle_sample_rate(a, per_step, x64, start_row=(i * a.n_rows // 7) % a.n_rows,
                                    block_nnz=block_nnz)
        nnz_done += n_
        t_used += t_
    value = nnz_done / t_used / 1e9
    line = {"metric": METRIC, "impl": "reference", "value": value, "unit": "Gnnz/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_used / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "scale": scale, "edge_factor": ef, "seed": seed,
                       "n": a.n_rows, "nnz": a.nnz, "parallelism": "host cores, 1 thread"},
            "cpu_baseline": {"value": value, "unit": "Gnnz/s", "cores": 1, "kind": "oracle",
                             "sample": f"contiguous row blocks of about {block_nnz} nonzeros, "
                                       f"{per_step * 1e3:.0f} ms of oracle SpMV per step"},
            "e2e": {"value": value, "unit": "Gnnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def algorithmic_bytes_f32(a, tiles) -> tuple[int, dict]:
    """Algorithmic DRAM bytes of one FP32 SpMV: vals + col (8 m), x and y once (4 n each),
    descriptors of the non-single-row tiles (4 per lane), tile_x and tile_y (8 per tile)."""
    marked = (tiles.tile_y[:-1] & 0x80000000) != 0
    tile_num = tiles.tile_y.size - 1
    lane_num = tiles.lane_desc.size
    lanes_in_normal = lane_num - 32 * int(marked.sum())
    if marked.size and marked[-1]:
        lanes_in_normal += 32 * tile_num - lane_num     # the last tile may be partial
    parts = {"vals_col": 8 * a.nnz, "x": 4 * a.n_cols, "y": 4 * a.n_rows,
             "lane_desc": 4 * max(0, lanes_in_normal), "tile_xy": 8 * (tile_num + 1)}
    return sum(parts.values()), {"r_f": float(marked.mean()) if marked.size else 0.0, **parts}


def default_plan(rp, col, args, stream, sigma: int | None = None):
    """The bench's plan: merbit_plan at the given sigma, then (with --hot H > 0) the plan's
    hot-column table of up to H columns, kept if they hold --hot-min-cover of the
    nonzeros.  The Plan gets hot_n and hot_cover attributes."""
    import paper_2605_07391_gb300 as mb
    p = mb.plan(rp, col, sigma=sigma or args.sigma, stream=stream)
    p.hot_n, p.hot_cover = p.set_hot_columns(args.hot, args.hot_min_cover, stream=stream) if args.hot > 0 else (0, 0.0)
    return p


def algorithmic_bytes(a, tiles, val_bytes: int, vec_bytes: int) -> int:
    """Algorithmic DRAM bytes of one product with the given value and vector widths: the
    FP32 model of algorithmic_bytes_f32 with vals at val_bytes and x, y at vec_bytes."""
    _, parts = algorithmic_bytes_f32(a, tiles)
    return (val_bytes + 4) * a.nnz + vec_bytes * (a.n_cols + a.n_rows) + parts["lane_desc"] + parts["tile_xy"]


def time_calls(fn, reps: int, stream) -> float:
    """Mean ms per call of fn over reps calls (CUDA events on `stream`, after 5 warm-ups)."""
    import torch
    for _ in range(5):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def run_config1(args, dev, stream) -> dict:
    """Configuration 1 (the small case): R-MAT scale 14 transition matrix, one SpMV in FP32
    and FP64 (mean of 1000 calls) and the 100-update PageRank (alpha 0.85) in FP32 and FP64,
    with the oracle's own times for the same work and the paper's ERR (relative l_inf error
    against pi* = 210 oracle power updates, Sec. 5.5.1) of each 100-update result."""
    import torch

    import inputs
    import oracle
    import paper_2605_07391_gb300 as mb
    scale, ef, seed = WORKLOADS["rmat14_transition"]
    a = inputs.rmat_transition(scale, ef, seed)
    x64 = inputs.uniform_vector(a.n_cols, 2)
    rp, col = torch.from_numpy(a.row_ptr).to(dev), torch.from_numpy(a.col).to(dev)
    p = mb.plan(rp, col, stream=stream)
    tiles = p.tiles()
    hbm = peaks()[0]
    star = oracle.pagerank(a.row_ptr, a.col, a.val, 0.85, tol=0.0, fixed_iters=210)["pi"]
    res = {"workload": "rmat14_transition", "n": a.n_rows, "nnz": a.nnz}
    for name, dt, vb in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
        vals = torch.from_numpy(a.val).to(dev, dt)
        x = torch.from_numpy(x64).to(dev, dt)
        y = torch.empty(a.n_rows, dtype=dt, device=dev)
        ms = time_calls(lambda: mb.spmv(p, vals, x, y, stream=stream), 1000, stream)
        alg = algorithmic_bytes(a, tiles, vb, vb)
        mb.pagerank(p, vals, 0.85, tol=0.0, max_iter=100, stream=stream)          # warm
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        pi, info = mb.pagerank(p, vals, 0.85, tol=0.0, max_iter=100, stream=stream)
        torch.cuda.synchronize(dev)
        pr_ms = (time.perf_counter() - t0) * 1e3
        res[name] = {"spmv_ms": ms, "gnnz_s": a.nnz / (ms * 1e-3) / 1e9, "roofline_frac": alg / (ms * 1e-3) / 1e9 / hbm,
                     "pagerank_100_ms": pr_ms,
                     "pagerank_err_vs_pi_star": oracle.relative_linf_error(pi.double().cpu().numpy(), star)}
    t0 = time.perf_counter()
    oracle.spmv(a.row_ptr, a.col, a.val, x64)
    res["oracle_spmv_ms"] = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    oracle.pagerank(a.row_ptr, a.col, a.val, 0.85, tol=0.0, fixed_iters=100)
    res["oracle_pagerank_100_ms"] = (time.perf_counter() - t0) * 1e3
    res["oracle_cores"] = 1
    p.destroy()
    return res


def run_config2(args, dev, stream) -> dict:
    """Configuration 2 (irregular-structure stress, the degree question of Sec. 5.2.2):
    the R-MAT scale 22 matrix with values U(0,1] as is (a), with 30 % of its rows emptied
    (b), with 16 hub rows of 1M-4M nonzeros (c), and the Erdos-Renyi 2^22 matrix with 16
    nonzeros per row (d); FP32 and FP64 SpMV, each the mean of --config2-calls calls with the
    plan reused (plan built as the bench's default plan)."""
    import torch

    import inputs
    import paper_2605_07391_gb300 as mb
    hbm = peaks()[0]
    base = inputs.rmat_uniform(22, 16, 3, 3)
    makers = {"a_rmat22": lambda: base, "b_empty30": lambda: inputs.empty_rows(base, 0.3, 4),
              "c_hubs16": lambda: inputs.add_hubs(base, 16, 1_000_000, 4_000_000, 5),
              "d_er22": lambda: inputs.erdos_renyi(1 << 22, 16, 6)}
    x64 = inputs.uniform_vector(1 << 22, 2)
    res = {"calls": args.config2_calls}
    for name, make in makers.items():
        a = make()
        rp, col = torch.from_numpy(a.row_ptr).to(dev), torch.from_numpy(a.col).to(dev)
        p = default_plan(rp, col, args, stream)
        tiles = p.tiles()
        rec = {"nnz": a.nnz, "hot_columns": p.hot_n}
        for dname, dt, vb in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
            vals = torch.from_numpy(a.val).to(dev, dt)
            x = torch.from_numpy(x64[:a.n_cols]).to(dev, dt)
            y = torch.empty(a.n_rows, dtype=dt, device=dev)
            ms = time_calls(lambda: mb.spmv(p, vals, x, y, stream=stream), args.config2_calls, stream)
            alg = algorithmic_bytes(a, tiles, vb, vb)
            rec[dname] = {"ms": ms, "gnnz_s": a.nnz / (ms * 1e-3) / 1e9,
                          "roofline_frac": alg / (ms * 1e-3) / 1e9 / hbm}
            del vals, x, y
        p.sync(stream)
        p.destroy()
        res[name] = rec
        del a, rp, col
    return res


def run_batched(args, dev, stream) -> dict:
    """SpMM Y = A X (row-major X, k columns) per call and personalised PageRank (k one-hot
    seeds over vertices with out-edges) to L1 residual 1e-6 per column, R-MAT scale 22."""
    import torch

    import inputs
    import paper_2605_07391_gb300 as mb
    a = inputs.rmat_transition(22, 16, 7)
    rp = torch.from_numpy(a.row_ptr).to(dev)
    col = torch.from_numpy(a.col).to(dev)
    vals = torch.from_numpy(a.val).to(dev, torch.float32)
    p = mb.plan(rp, col, a.n_rows, a.n_cols, stream=stream)
    tiles = p.info()
    hbm = peaks()[0]
    res = {"workload": "rmat22_transition", "nnz": int(a.nnz), "n": int(a.n_rows)}
    for k in args.batched_k:
        X = torch.rand(a.n_cols, k, device=dev)
        Y = torch.empty(a.n_rows, k, device=dev)
        for _ in range(5):
            mb.spmm(p, vals, X, Y, stream=stream)
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        reps = 50
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(reps):
            mb.spmm(p, vals, X, Y, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        alg = 8 * a.nnz + 4 * k * (a.n_cols + a.n_rows) + 4 * tiles.lane_num + 8 * (tiles.tile_num + 1)
        rec = {"spmm_ms": ms, "gnnz_vec_s": a.nnz * k / (ms * 1e-3) / 1e9,
               "spmm_alg_gbs": alg / (ms * 1e-3) / 1e9, "spmm_roofline_frac": alg / (ms * 1e-3) / 1e9 / hbm,
               "spmm_alg_bytes": alg}
        del X, Y
        seeds = inputs.ppr_seeds(a, k, 22)
        mb.ppr(p, vals, seeds, 0.85, tol=0.0, max_iter=2, stream=stream)       # warm
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        r = mb.ppr(p, vals, seeds, 0.85, tol=1e-6, max_iter=300, stream=stream)
        torch.cuda.synchronize(dev)
        pms = (time.perf_counter() - t0) * 1e3
        rec.update({"ppr_ms_to_1e-6": pms, "ppr_updates": r["iters"], "ppr_converged": r["converged"],
                    "ppr_ms_per_update": pms / max(1, r["iters"]), "ppr_max_resid": max(r["resid"])})
        if not args.no_oracle_check:
            import oracle
            Pi = r["pi"][:, [0, k - 1]].double().cpu().numpy()
            rr = oracle.ppr_residual(a.row_ptr, a.col, a.val, Pi, [int(seeds[0]), int(seeds[k - 1])], 0.85)
            rec["ppr_oracle_l1_residual_cols_0_last"] = [float(v) for v in rr]
        if not args.no_oracle_check:
            import oracle
            r1 = a.n_rows // 256
            lo, hi = 0, int(a.row_ptr[r1])
            Xs = np.random.default_rng(3).random((a.n_cols, k))
            rec["oracle"] = oracle_timed(
                lambda: oracle.spmm(a.row_ptr[:r1 + 1].astype(np.int64), a.col[lo:hi], a.val[lo:hi], Xs),
                (hi - lo) * k / 1e9, "Gnnz*vec/s",
                f"float64 oracle SpMM, first 1/256 of the rows ({hi - lo} nnz) x {k} columns")
        res[f"k{k}"] = rec
        del r
    p.destroy()
    return res


def run_many_graphs(args, dev, stream) -> dict:
    """PageRank of many independent R-MAT graphs (scale uniform in 10..20, edge factor in
    8..32, FP64 values) to L1 residual 1e-8 each, as one block-diagonal matrix: sigma
    chosen by the autotuner, then the whole solve as one CUDA-graph launch (recorded on the
    first call, timed on later ones)."""
    import torch

    import inputs
    import paper_2605_07391_gb300 as mb
    t0 = time.perf_counter()
    a, off = inputs.rmat_batch(args.many_graphs, 42, scales=(10, 20), edge_factors=(8, 32),
                               threads=os.cpu_count() or 8)
    gen_s = time.perf_counter() - t0
    rp = torch.from_numpy(a.row_ptr).to(dev)
    col = torch.from_numpy(a.col).to(dev)
    vals = torch.from_numpy(a.val).to(dev)
    res = {"workload": f"rmat_batch{args.many_graphs}_scale10-20_ef8-32", "graphs": args.many_graphs,
           "n": int(a.n_rows), "nnz": int(a.nnz), "dtype": "f64", "tol": 1e-8, "host_generation_s": gen_s}
    # sigma x block kernel by measurement (batches keep 8 tiles per block and 32-bit
    # descriptors; the block size is listed for completeness)
    tune, times = mb.autotune(rp, col, vals, sigmas=(14, 12, 10, 7), blocks=(8,),
                              kernels=("classic", "split", "split2"), hots=(0,), reps=3, stream=stream)
    best = tune["sigma"]
    res["autotune"] = {"best": tune, "ms_per_spmv": {f"s{k[0]}_W{k[1]}_{k[2]}": v for k, v in times.items()}}
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    b = mb.Batch(rp, col, off, sigma=best, stream=stream)
    b.set_kernel(tune["kernel"])
    torch.cuda.synchronize(dev)
    res["plan_ms"] = (time.perf_counter() - t0) * 1e3
    b_plan_info = b.plan_info()
    pi = torch.empty(a.n_rows, dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    _, info = b.pagerank(vals, 0.85, tol=1e-8, max_iter=500, pi=pi, stream=stream)
    res["first_call_ms"] = (time.perf_counter() - t0) * 1e3          # records and instantiates
    runs = []
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    clocks.mark()
    for _ in range(5):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, info = b.pagerank(vals, 0.85, tol=1e-8, max_iter=500, pi=pi, stream=stream)
        runs.append((time.perf_counter() - t0) * 1e3)
    clocks.mark()
    res["clocks"] = clocks.stop()
    ms = statistics.median(runs)
    nnz_g = np.diff(a.row_ptr[off]).astype(np.int64)
    useful = float((info["iters"].astype(np.int64) * nnz_g).sum())
    res.update({"ms": ms, "runs_ms": runs, "min_ms": min(runs), "converged": info["converged"], "rounds": info["rounds"],
                "updates_min_median_max": [int(info["iters"].min()), int(np.median(info["iters"])),
                                           int(info["iters"].max())],
                "useful_gnnz_s": useful / (ms * 1e-3) / 1e9,
                "max_resid": float(info["resid"].max())})
    if not args.no_oracle_check:
        import oracle
        pin = pi.cpu().numpy()
        sizes = np.diff(off)
        checks = {}
        for g in sorted(range(args.many_graphs), key=lambda g: sizes[g])[:2] + \
                [int(np.argsort(sizes)[len(sizes) // 2])]:
            lo, hi = int(off[g]), int(off[g + 1])
            k0, k1 = int(a.row_ptr[lo]), int(a.row_ptr[hi])
            r = oracle.pagerank_residual(a.row_ptr[lo:hi + 1] - a.row_ptr[lo], a.col[k0:k1] - lo,
                                         a.val[k0:k1], pin[lo:hi], 0.85)
            checks[f"graph{g}_n{hi - lo}"] = r
        res["oracle_l1_residual"] = checks
        g0 = int(np.argsort(sizes)[len(sizes) // 2])
        lo, hi = int(off[g0]), int(off[g0 + 1])
        k0, k1 = int(a.row_ptr[lo]), int(a.row_ptr[hi])
        sub = (a.row_ptr[lo:hi + 1] - a.row_ptr[lo], a.col[k0:k1] - lo, a.val[k0:k1])
        upd = int(info["iters"][g0])
        res["oracle"] = oracle_timed(lambda: oracle.pagerank(*sub, 0.85, tol=0.0, fixed_iters=upd),
                                     upd * (k1 - k0) / 1e9, "Gnnz/s",
                                     f"float64 oracle PageRank of graph {g0} ({hi - lo} vertices, "
                                     f"{k1 - k0} nnz, {upd} updates)")
    # algorithmic bytes of one update of graph g: FP64 values and int32 columns (12 B per
    # nonzero), x gathered once, y written, and y and x read by the residual pass (32 B per
    # vertex), plus its share of the plan's lane descriptors and tile coordinates
    hbm = peaks()[0]
    inf = b_plan_info
    n_g = np.diff(off).astype(np.int64)
    plan_b = (4 * inf.lane_num + 8 * (inf.tile_num + 1)) * (nnz_g + n_g) / (a.nnz + a.n_rows)
    useful_bytes = float((info["iters"].astype(np.int64) * (12 * nnz_g + 32 * n_g) + info["iters"] * plan_b).sum())
    res["useful_alg_bytes"] = useful_bytes
    res["roofline"] = {"bound": "hbm", "achieved": useful_bytes / (ms * 1e-3) / 1e9, "peak": hbm,
                       "unit": "GB/s", "frac": useful_bytes / (ms * 1e-3) / 1e9 / hbm}
    b.destroy()
    return res


def run_bicgstab(args, dev, stream) -> dict:
    """BiCGSTAB (FP64) on A x = b, A the unit-valued adjacency of synthetic stand-ins for
    the paper's graphs (a road network, a k-mer graph, a traffic trace with hubs),
    b = A x_true with x_true ~ U[-1, 1], tol 1e-10, capped at --bicgstab-iters iterations.
    Per iteration: two pattern-only SpMVs (no value stream: every value is 1; fused dot
    products) and three vector passes; the algorithmic bytes count each pass's reads and
    writes once.  The same solve with the values read is reported beside it."""
    import torch

    import inputs
    import paper_2605_07391_gb300 as mb
    hbm = peaks()[0]
    cases = [("road_grid_2600x2600_k0.55", lambda: inputs.road_grid(2600, 2600, 0.55, 11)),
             ("kmer_chains_10M", lambda: inputs.kmer_chains(10_000_000, 64, 0.02, 12)),
             ("hub_rmat22_ef2", lambda: inputs.hub_graph(22, 2, 13))]
    res = {"tol": 1e-10, "max_iter": args.bicgstab_iters}
    for name, make in cases:
        a = make()
        n, nnz = a.n_rows, a.nnz
        rp, col = torch.from_numpy(a.row_ptr).to(dev), torch.from_numpy(a.col).to(dev)
        vals = torch.from_numpy(a.val).to(dev)
        # sigma for these FP64 products, by the autotuner (timed with the unit values read)
        sigma, tune = mb.autotune_sigma(rp, col, vals, candidates=(14, 12, 10, 8), reps=3, stream=stream)
        p = mb.plan(rp, col, n, n, sigma=sigma, stream=stream)
        xt = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, n)).to(dev)
        b = mb.spmv(p, vals, xt)
        mb.bicgstab(p, None, b, None, tol=1e-10, max_iter=3, stream=stream)        # warm
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        x, info = mb.bicgstab(p, None, b, None, tol=1e-10, max_iter=args.bicgstab_iters, stream=stream)
        torch.cuda.synchronize(dev)
        ms = (time.perf_counter() - t0) * 1e3
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, info_v = mb.bicgstab(p, vals, b, None, tol=1e-10, max_iter=args.bicgstab_iters, stream=stream)
        torch.cuda.synchronize(dev)
        ms_v = (time.perf_counter() - t0) * 1e3
        inf = p.info()
        spmv_bytes = 4 * nnz + 8 * n + 8 * n + 8 * n + 4 * inf.lane_num + 8 * (inf.tile_num + 1)
        it_bytes = 2 * spmv_bytes + 8 * n * (4 + 3 + 7)
        it = max(1, info["iters"])
        res[name] = {"n": n, "nnz": nnz, "sigma": sigma, "autotune_ms_per_spmv": tune,
                     "iters": info["iters"], "status": info["status"],
                     "rel_resid": info["resid"], "ms": ms, "ms_per_iter": ms / it,
                     "alg_bytes_per_iter": it_bytes, "alg_gbs": it_bytes * it / (ms * 1e-3) / 1e9,
                     "roofline_frac": it_bytes * it / (ms * 1e-3) / 1e9 / hbm,
                     "projected_s_for_20000_iters": ms / it * 20000 / 1e3,
                     "with_values_read": {"iters": info_v["iters"], "ms_per_iter": ms_v / max(1, info_v["iters"])}}
        if name.startswith("road") and args.bicgstab_full:
            # the paper's protocol (Sec. 5.5.2): tol 1e-10 or 20000 iterations, measured
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            _, info_f = mb.bicgstab(p, None, b, None, tol=1e-10, max_iter=20000, stream=stream)
            torch.cuda.synchronize(dev)
            res[name]["paper_protocol_20000"] = {"s": time.perf_counter() - t0, "iters": info_f["iters"],
                                                 "status": info_f["status"], "rel_resid": info_f["resid"],
                                                 "plan_and_autotune_excluded": True}
        del x, b, vals
        p.destroy()
        if not args.no_oracle_check and name.startswith("road"):
            import oracle
            sm = inputs.road_grid(400, 400, 0.55, 11)
            bs = oracle.spmv(sm.row_ptr, sm.col, sm.val, np.random.default_rng(1).uniform(-1, 1, sm.n_rows))[0]
            res["oracle"] = oracle_timed(
                lambda: oracle.bicgstab(sm.row_ptr, sm.col, sm.val, bs, tol=1e-30, max_iter=20),
                20 * sm.n_rows / 1e6, "Mrow-iterations/s",
                f"float64 oracle BiCGSTAB, 20 iterations on a 400x400 road grid ({sm.nnz} nnz)")
    return res


def run_autograd(args, dev, stream) -> dict:
    """dL/dvals for L = sum_i w_i pi_i (w ~ N(0, 1)) at the PageRank fixed point of the R-MAT
    scale 20 transition matrix, FP32: transpose + its plan (once per pattern), forward
    PageRank to 1e-7, backward = gather of the transposed values + adjoint solve to 1e-6
    relative + per-nonzero products; the FP32 gradient compared with the FP64 one."""
    import torch

    import inputs
    import paper_2605_07391_gb300 as mb
    from paper_2605_07391_gb300 import autograd as ag
    a = inputs.rmat_transition(20, 16, 3)
    rp = torch.from_numpy(a.row_ptr).to(dev)
    col = torch.from_numpy(a.col).to(dev)
    w = torch.from_numpy(np.random.default_rng(20).standard_normal(a.n_rows))
    res = {"workload": "rmat20_transition", "nnz": int(a.nnz), "n": int(a.n_rows)}

    def timed(fn):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize(dev)
        return r, (time.perf_counter() - t0) * 1e3

    A, res["plan_ms"] = timed(lambda: ag.Matrix(rp, col, a.n_rows, a.n_cols, stream=stream))
    _, res["transpose_and_plan_ms"] = timed(lambda: A.transposed(stream))
    grads = {}
    for name, dt, tol, adj_tol in (("f32", torch.float32, 1e-7, 1e-6), ("f64", torch.float64, 1e-12, 1e-12)):
        vals = torch.from_numpy(a.val).to(dev, dt)
        wd = w.to(dev, dt)
        mb.pagerank(A.plan, vals, 0.85, tol=0.0, max_iter=2, stream=stream)          # warm
        (pi, info), fwd = timed(lambda: mb.pagerank(A.plan, vals, 0.85, tol=tol, max_iter=5000, stream=stream))
        _, pt = A.transposed()

        def backward():
            vt = A.transposed_values(vals, stream)
            lam, ainfo = mb.pagerank_adjoint(A.plan, pt, vt, wd, 0.85, tol=adj_tol, max_iter=5000,
                                             stream=stream)
            return mb.sddmm(A.plan, lam, pi, 0.85, stream=stream), ainfo
        (g, ainfo), bwd = timed(backward)
        # the same through torch.autograd (what a user calls)
        v_req = vals.clone().requires_grad_()

        def autograd_step():
            v_req.grad = None
            p = ag.pagerank(A, v_req, 0.85, tol=tol, adj_tol=adj_tol)
            (p * wd).sum().backward()
            return v_req.grad
        autograd_step()                      # the autograd engine's first use is not timed
        _, e2e = timed(autograd_step)
        grads[name] = g.double()
        res[name] = {"forward_ms": fwd, "forward_updates": info["iters"], "forward_resid": info["resid"],
                     "backward_ms": bwd, "adjoint_updates": ainfo["iters"], "adjoint_resid": ainfo["resid"],
                     "autograd_forward_backward_ms": e2e}
    res["f32_vs_f64_grad_rel_l1"] = float((grads["f32"] - grads["f64"]).abs().sum() / grads["f64"].abs().sum())
    A.plan.destroy()
    if not args.no_oracle_check:
        import oracle
        s14 = inputs.rmat_transition(14, 16, 3)
        w14 = np.random.default_rng(20).standard_normal(s14.n_rows)
        res["oracle"] = oracle_timed(
            lambda: oracle.pagerank_value_gradient(s14.row_ptr, s14.col, s14.val, w14, 0.85, tol=1e-12),
            1.0, "gradients/s", f"float64 oracle value gradient (forward + adjoint to 1e-12) of the "
            f"R-MAT scale 14 transition matrix ({s14.nnz} nnz)", budget_s=2.0)
    return res


def summarize(out: dict) -> dict:
    """The headline figures in a few hundred bytes, the last key of the line."""
    def r(v, d=4):
        return None if v is None else round(float(v), d)
    rf = out["roofline"]
    sm = {"spmv_f32_ms": r(rf["mean_launch_ms"]), "gnnz_s": r(out["value"], 1), "frac": r(rf["frac"]),
          "plan_ms": r(out["plan_ms"], 2), "hot_cols": out["hot_table"]["columns"],
          "hot_cover": r(out["hot_table"]["cover"], 3)}
    if "gather_floor" in out:
        g = out["gather_floor"]
        sm.update({"floor_ms": r(g["ms"]), "no_hot_ms": r(g["without_hot_table"]["spmv_ms"]),
                   "no_hot_floor_ms": r(g["without_hot_table"]["floor_ms"])})
    if "spmv_other" in out:
        o = out["spmv_other"]
        sm.update({"f64_ms": r(o["f64"]["ms"]), "f64_sigma": o["f64"]["sigma"], "bf16_ms": r(o["bf16_vals"]["ms"])})
    if "pagerank" in out:
        pr = out["pagerank"]
        sm["pagerank"] = {k: [r(v["ms"], 1), v["converged"], v.get("oracle_l1_residual") and float(f"{v['oracle_l1_residual']:.2e}"),
                              float(f"{v['err_vs_pi_star']:.2e}")]
                          for k, v in pr.items() if isinstance(v, dict)}
        sm["mixed_vs_ir_f32"] = r(pr.get("mixed_vs_ir_f32_speedup"), 3)
    if "config2" in out:
        sm["config2_gnnz_f32_f64"] = {k: [r(v["f32"]["gnnz_s"], 1), r(v["f64"]["gnnz_s"], 1)]
                                      for k, v in out["config2"].items() if isinstance(v, dict)}
    if "config1" in out:
        c = out["config1"]
        sm["config1_ms"] = {"spmv_f32": r(c["f32"]["spmv_ms"]), "pr100_f32": r(c["f32"]["pagerank_100_ms"], 2),
                            "pr100_f64": r(c["f64"]["pagerank_100_ms"], 2), "oracle_pr100": r(c["oracle_pagerank_100_ms"], 1)}
    if "cpu_all_cores" in out:
        sm["oracle_gnnz_1core_allcores"] = [r(out["cpu_baseline"]["value"]), r(out["cpu_all_cores"]["value"]),
                                            out["cpu_all_cores"]["cores"]]
    return sm


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="merbit", choices=["merbit", "reference"])
    ap.add_argument("--workload", default="rmat24_transition", choices=sorted(WORKLOADS))
    ap.add_argument("--ref-budget", type=float, default=60.0, help="seconds of oracle work (reference arm)")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work (cpu_baseline)")
    ap.add_argument("--no-pagerank", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched runs (SpMM and personalised PageRank, R-MAT scale 22)")
    ap.add_argument("--no-autograd", action="store_true",
                    help="skip the differentiation run (PageRank value gradient, R-MAT scale 20)")
    ap.add_argument("--no-many-graphs", action="store_true",
                    help="skip the many-graph run (256 R-MAT graphs, scales 10-20, one CUDA-graph launch)")
    ap.add_argument("--many-graphs", type=int, default=256, help="graphs in the many-graph run")
    ap.add_argument("--no-bicgstab", action="store_true",
                    help="skip the BiCGSTAB runs (road / k-mer / hub graph stand-ins)")
    ap.add_argument("--bicgstab-iters", type=int, default=2000, help="iteration cap of the BiCGSTAB runs")
    ap.add_argument("--no-bicgstab-full", dest="bicgstab_full", action="store_false",
                    help="skip the road stand-in's run under the paper's 20000-iteration protocol")
    ap.add_argument("--batched-k", type=int, nargs="+", default=[8, 32],
                    help="numbers of right-hand sides / seeds of the batched runs")
    ap.add_argument("--no-oracle-check", action="store_true")
    ap.add_argument("--inner-sweeps", type=int, default=0,
                    help="max inner sweeps per refinement step (0: the tuned setting of each mode)")
    ap.add_argument("--sigma", type=int, default=14, help="steps per lane of the plan")
    ap.add_argument("--hot", type=int, default=0,
                    help="hot-column table of the plans: up to this many columns (0: none)")
    ap.add_argument("--hot-min-cover", type=float, default=0.05,
                    help="keep a --hot table only if its columns hold this fraction of the nonzeros")
    ap.add_argument("--no-config1", action="store_true", help="skip the R-MAT scale 14 runs")
    ap.add_argument("--no-config2", action="store_true", help="skip the R-MAT scale 22 stress runs")
    ap.add_argument("--config2-calls", type=int, default=1000, help="SpMV calls per stress matrix")
    ap.add_argument("--no-all-cores", action="store_true", help="skip the all-cores oracle leg")
    args = ap.parse_args()
    rank, world, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    import inputs
    import paper_2605_07391_gb300 as mb

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    mb.load()

    scale, ef, seed = WORKLOADS[args.workload]
    t0 = time.perf_counter()
    a = inputs.rmat_transition(scale, ef, seed)
    gen_s = time.perf_counter() - t0
    x64 = inputs.uniform_vector(a.n_cols, 2)
    row_ptr = torch.from_numpy(a.row_ptr).to(dev)
    col = torch.from_numpy(a.col).to(dev)
    v64 = torch.from_numpy(a.val).to(dev)
    v32 = v64.float()
    x = torch.from_numpy(x64).to(dev, torch.float32)
    y = torch.empty(a.n_rows, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # plan (one-time preprocessing), timed on its own
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    p = mb.plan(row_ptr, col, sigma=args.sigma, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    plan_ms = ev0.elapsed_time(ev1)
    # the hot-column table (one-time, like the plan), timed on its own
    t0 = time.perf_counter()
    p.hot_n, p.hot_cover = p.set_hot_columns(args.hot, args.hot_min_cover, stream=stream) if args.hot > 0 else (0, 0.0)
    torch.cuda.synchronize(dev)
    hot_ms = (time.perf_counter() - t0) * 1e3
    tiles = p.tiles()
    alg_bytes, alg_parts = algorithmic_bytes_f32(a, tiles)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier(device_ids=[local])
        torch.cuda.synchronize(dev)

    # ---- timed region: K FP32 SpMV launches (one kernel each)
    for _ in range(args.warmup):
        mb.spmv(p, v32, x, y, stream=stream)
    clocks = ClockSampler(local)
    clocks.start()
    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    total0, total1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    clocks.mark()
    total0.record(stream)
    for i in range(K):
        starts[i].record(stream)
        mb.spmv(p, v32, x, y, stream=stream)
        ends[i].record(stream)
    total1.record(stream)
    barrier()
    clocks.mark()
    clock_info = clocks.stop()
    p.sync(stream)
    elapsed_ms = max_over_ranks(total0.elapsed_time(total1), dev)
    launch_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    mean_launch_ms = statistics.fmean(launch_ms)
    ms_per_step = elapsed_ms / K
    value = whole_job_gnnz(a.nnz, world, ms_per_step)
    hbm_peak, peak_kind = peaks()
    achieved = alg_bytes / (mean_launch_ms * 1e-3) / 1e9
    traffic = measured_traffic(args.workload)

    out = {"metric": METRIC, "value": value, "unit": "Gnnz/s", "n_gpus": world, "steps": K,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": args.workload, "scale": scale, "edge_factor": ef, "seed": seed,
                      "n": a.n_rows, "nnz": a.nnz, "sigma": p.sigma, "omega": 32,
                      "tiles_per_block": 8, "x": "U[0,1) seed 2",
                      "l2": f"inputs larger than L2: {(8 * a.nnz + 8 * a.n_rows) / 1e9:.2f} GB read per step",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                        "frac": achieved / hbm_peak, "traffic": traffic,
                        "peak_kind": peak_kind,
                        "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                        "traffic_bytes_per_nnz": traffic / a.nnz if traffic else None,
                        "algorithmic_bytes_per_launch": alg_bytes,
                        "bytes_per_nnz": alg_bytes / a.nnz, "parts": alg_parts,
                        "kernel": "merbit_spmv_split_kernel<float,float,float,EpiPlain> (the default block "
                                  "kernel for f32 values) + merbit_finalize_kernel",
                        "mean_launch_ms": mean_launch_ms,
                        "median_launch_ms": statistics.median(launch_ms)},
           "plan_ms": plan_ms, "gen_s": gen_s,
           "hot_table": {"max_columns": args.hot, "columns": p.hot_n, "cover": p.hot_cover,
                         "build_ms": hot_ms},
           # each step launches the SpMV kernel and its boundary-row finalize kernel
           "gpu_launches": 2 * K, "clocks": clock_info}

    if rank == 0:
        # ---- the floor of the gathers: the product's x gather alone at the split kernel's
        # shared-memory footprint (merbit_gather_probe), and both without the hot table
        sink = torch.zeros(4096, device=dev)
        floor_ms = time_calls(lambda: p.gather_probe(x, sink, stream=stream), 50, stream)
        q = mb.plan(row_ptr, col, sigma=args.sigma, stream=stream)
        plain_ms = time_calls(lambda: mb.spmv(q, v32, x, y, stream=stream), 50, stream)
        plain_floor_ms = time_calls(lambda: q.gather_probe(x, sink, stream=stream), 50, stream)
        q.destroy()
        out["gather_floor"] = {
            "ms": floor_ms, "spmv_over_floor": mean_launch_ms / floor_ms,
            "frac_at_floor": alg_bytes / (floor_ms * 1e-3) / 1e9 / hbm_peak,
            "without_hot_table": {"spmv_ms": plain_ms, "floor_ms": plain_floor_ms,
                                  "frac": alg_bytes / (plain_ms * 1e-3) / 1e9 / hbm_peak},
            "probe": "merbit_gather_probe: the x[col[k]] loads of every nonzero (hot-table slots from "
                     "shared memory), column stream read coalesced, split kernel's grid and shared memory"}
        mb.spmv(p, v32, x, y, stream=stream)

        # ---- end to end through the host-buffer entry point (pinned buffers)
        xh = x.cpu().pin_memory()
        yh = torch.empty(a.n_rows, dtype=torch.float32).pin_memory()
        for _ in range(3):
            mb.spmv_host(p, v32, xh, yh, stream=stream)
        ke = min(K, 50)
        t0 = time.perf_counter()
        for _ in range(ke):
            mb.spmv_host(p, v32, xh, yh, stream=stream)
        sync_s = (time.perf_counter() - t0) / ke
        # the overlapping entry point: every call still uploads its x and downloads its y
        for _ in range(3):
            mb.spmv_host(p, v32, xh, yh, stream=stream, wait=False)
        p.sync(stream)
        t0 = time.perf_counter()
        for _ in range(ke):
            mb.spmv_host(p, v32, xh, yh, stream=stream, wait=False)
        p.sync(stream)
        e2e_s = (time.perf_counter() - t0) / ke
        ok = torch.allclose(yh, y.cpu(), rtol=1e-5, atol=1e-6)
        out["e2e"] = {"value": a.nnz / e2e_s / 1e9, "unit": "Gnnz/s", "h2d_bytes_per_step": 4 * a.n_cols,
                      "d2h_bytes_per_step": 4 * a.n_rows, "ms_per_step": e2e_s * 1e3,
                      "entry_point": "merbit_spmv_host_async (consecutive calls overlap; pinned buffers)",
                      "result_matches_device": bool(ok),
                      "synchronous_entry_point": {"value": a.nnz / sync_s / 1e9, "ms_per_step": sync_s * 1e3}}

        # ---- other value types of the same product.  FP64 runs on the sigma the autotuner
        # picks for FP64 values (the paper, too, sets sigma per value type); the plan of the
        # FP32 headline is timed with FP64 values as well.
        other = {}
        lo, k = mb.vals_convert(v64, torch.bfloat16)
        x64d = x.double()
        y64 = torch.empty(a.n_rows, dtype=torch.float64, device=dev)
        s64, t64 = mb.autotune_sigma(row_ptr, col, v64, candidates=(14, 12, 10, 8, 7), reps=3,
                                     stream=stream)
        ev0.record(stream)
        p64 = p if s64 == p.sigma else default_plan(row_ptr, col, args, stream, sigma=s64)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        plan64_ms = plan_ms if p64 is p else ev0.elapsed_time(ev1)
        for name, fn in (("f64", lambda: mb.spmv(p64, v64, x64d, y64, stream=stream)),
                         (f"f64_sigma{p.sigma}", lambda: mb.spmv(p, v64, x64d, y64, stream=stream)),
                         ("bf16_vals", lambda: mb.spmv(p, lo, x, y, stream=stream))):
            for _ in range(5):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(100):
                fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / 100
            other[name] = {"gnnz_s": a.nnz / (ms * 1e-3) / 1e9, "ms": ms}
        other["f64"].update({"sigma": s64, "autotune_ms_per_spmv": t64, "plan_ms": plan64_ms,
                             "hot_columns": p64.hot_n})
        out["spmv_other"] = other
        del lo, y64, x64d

        # ---- PageRank to L1 residual 1e-10
        if not args.no_pagerank:
            import oracle
            pr = {}
            # pi* of the paper's ERR (Sec. 5.5.1): 210 updates of the FP64 power method (here on
            # the device), with the oracle's FP64 residual of it beside it
            star, _ = mb.pagerank(p64, v64, 0.85, tol=0.0, max_iter=210, stream=stream)
            star = star.cpu().numpy()
            if not args.no_oracle_check:
                pr["pi_star_oracle_l1_residual"] = oracle.pagerank_residual(a.row_ptr, a.col, a.val, star, 0.85)
            runs = [("ir_bf16", torch.float64), ("ir_f16", torch.float64), ("ir_f32", torch.float64),
                    ("plain_f64", torch.float64), ("plain_f32", torch.float32)]
            # refinement settings (inner stop eta, sweep cap) tuned per mode on this workload:
            # a sweep of the eta x cap grid, both the reduced-precision and the FP32 modes
            tuned = {"ir_bf16": (2.0 ** -4, 12), "ir_f16": (2.0 ** -11, 6), "ir_f32": (2.0 ** -10, 6)}
            for name, dt in runs:
                mode = "plain" if name.startswith("plain") else name
                vals = v64 if dt == torch.float64 else v32
                eta, cap = tuned.get(mode, (0.0, 32))
                if args.inner_sweeps:
                    eta, cap = 0.0, args.inner_sweeps
                kw = dict(tol=1e-10, max_iter=(150 if dt == torch.float32 else 400) if mode == "plain" else 60,
                          mode=mode,
                          inner_sweeps=cap, inner_tol=eta, stream=stream)
                pp, pp_plan_ms = (p64, plan64_ms) if name == "plain_f64" else (p, plan_ms)
                mb.pagerank(pp, vals, 0.85, **dict(kw, max_iter=2, tol=0.0))   # warm
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                pi, info = mb.pagerank(pp, vals, 0.85, **kw)
                torch.cuda.synchronize(dev)
                ms = (time.perf_counter() - t0) * 1e3
                rec = {"ms": ms, "iters": info["iters"], "resid": info["resid"], "sigma": pp.sigma,
                       "converged": info["converged"], "end_to_end_ms": ms + pp_plan_ms,
                       "spmv_launches": info["spmv_launches"]}
                if mode != "plain":
                    rec["inner_sweeps_cap"] = cap
                    rec["inner_eta"] = eta
                pin = pi.double().cpu().numpy()
                rec["err_vs_pi_star"] = oracle.relative_linf_error(pin, star)
                if not args.no_oracle_check:
                    r = oracle.pagerank_residual(a.row_ptr, a.col, a.val, pin, 0.85)
                    rec["oracle_l1_residual"] = r
                    rec["l1_err_bound_vs_fp64_fixed_point"] = r / 0.15
                pr[name] = rec
                del pi
            out["pagerank"] = pr
            if pr["ir_f32"]["converged"] and pr["ir_bf16"]["converged"]:
                out["pagerank"]["mixed_vs_ir_f32_speedup"] = pr["ir_f32"]["ms"] / pr["ir_bf16"]["ms"]
            if pr["plain_f64"]["converged"]:
                out["pagerank"]["mixed_vs_plain_f64_speedup"] = pr["plain_f64"]["ms"] / pr["ir_bf16"]["ms"]

        # ---- configuration 1 (R-MAT scale 14) and configuration 2 (R-MAT scale 22 stress)
        if not args.no_config1:
            out["config1"] = run_config1(args, dev, stream)
        if not args.no_config2:
            out["config2"] = run_config2(args, dev, stream)

        # ---- batching: SpMM and personalised PageRank on R-MAT scale 22, k = 8 and 32
        if not args.no_batched:
            out["batched"] = run_batched(args, dev, stream)

        # ---- many graphs: PageRank of 256 uneven R-MAT graphs in one CUDA-graph launch
        if not args.no_many_graphs:
            out["many_graphs"] = run_many_graphs(args, dev, stream)

        # ---- BiCGSTAB on undirected unit-valued graphs (the paper's second iterative workload)
        if not args.no_bicgstab:
            out["bicgstab"] = run_bicgstab(args, dev, stream)

        # ---- differentiation: PageRank value gradient by the implicit adjoint, R-MAT scale 20
        if not args.no_autograd:
            out["autograd"] = run_autograd(args, dev, stream)

        # ---- CPU baseline: the float64 oracle on a bounded sample
        nnz_done, t_used = oracle_sample_rate(a, args.cpu_budget, x64)
        out["cpu_baseline"] = {"value": nnz_done / t_used / 1e9, "unit": "Gnnz/s", "cores": 1,
                               "kind": "oracle",
                               "sample": f"float64 oracle SpMV on contiguous row blocks of ~1/64 of "
                                         f"the matrix, {nnz_done} nnz in {t_used:.1f} s"}
        out["host"] = {"nproc": os.cpu_count(), "machine": os.uname().machine}
        if not args.no_all_cores:
            out["cpu_all_cores"] = oracle_all_cores(a, x64, args.cpu_budget)
        out["summary"] = summarize(out)
        print(json.dumps(out), flush=True)
        if p64 is not p:
            p64.destroy()
    p.destroy()
    if world > 1:
        import torch.distributed as dist
        dist.barrier(device_ids=[local])
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
