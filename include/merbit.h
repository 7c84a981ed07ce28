/*
 * merbit.h — C ABI of a GB300 (sm_103a) implementation of MERBIT, the
 * merge-path + bit-field-descriptor SpMV of Zhang, Yao, Jiang and Zhang,
 * "MERBIT: A GPU-Based SpMV Method for Iterative Workloads", and of the
 * PageRank power iteration built on it.
 *
 * Conventions for every call
 *   - A CSR matrix is row_ptr (int32, n_rows + 1 entries, row_ptr[0] = 0,
 *     row_ptr[n_rows] = nnz, non-decreasing) and col_idx (int32, nnz entries,
 *     0 <= col < n_cols) as in Sec. 3.1; the row pointer is the paper's
 *     `offset`, read as n_rows + 1 entries.  Columns need not be sorted.
 *   - Unless a parameter says "host", every pointer is a DEVICE pointer of the
 *     current CUDA device, owned by the caller.  `stream` is a cudaStream_t
 *     (NULL = legacy default stream); calls are asynchronous on it unless
 *     stated otherwise.
 *   - `vals` and `col_idx` must be 16-byte aligned (they are staged into
 *     shared memory by bulk copies); x / y / pi must be aligned to their
 *     element size.
 *   - Every call returns a merbit_status; on failure merbit_last_error()
 *     returns a message (per calling thread).  Errors raised inside a kernel
 *     (an expired bounded wait) are reported by the next synchronising call
 *     (merbit_plan_sync, merbit_spmv_host, merbit_pagerank*) as
 *     MERBIT_EDEVICE; that call also clears the plan's device state.
 *   - A plan may be used by one stream at a time: its boundary-row
 *     accumulators and reduction slots are shared by all its calls.
 */
#ifndef MERBIT_H
#define MERBIT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct merbit_plan_s* merbit_plan_t;

typedef enum merbit_status {
  MERBIT_OK = 0,
  MERBIT_EINVAL = 1,     /* invalid argument (message says which)                  */
  MERBIT_EOVERFLOW = 2,  /* n_rows + nnz >= 2^31: merge-path coordinates are int32 */
  MERBIT_ENOMEM = 3,     /* device allocation failed                               */
  MERBIT_ECUDA = 4,      /* a CUDA runtime call failed                             */
  MERBIT_ENOTCONV = 5,   /* PageRank hit max_iter before tol (result still written) */
  MERBIT_EDEVICE = 6     /* a kernel reported an internal error (bounded wait)     */
} merbit_status;

typedef enum merbit_dtype {
  MERBIT_F32 = 0,
  MERBIT_F64 = 1,
  MERBIT_BF16 = 2,
  MERBIT_F16 = 3
} merbit_dtype;

typedef enum merbit_precision {
  MERBIT_PLAIN = 0,    /* power iteration in the dtype of vals / pi                 */
  MERBIT_IR_BF16 = 1,  /* iterative refinement, inner sweeps with bf16 values      */
  MERBIT_IR_F16 = 2,   /* iterative refinement, inner sweeps with scaled f16 values */
  MERBIT_IR_F32 = 3    /* iterative refinement, inner sweeps with f32 values       */
} merbit_precision;

/* Read-only view of a plan (the TILE arrays of Sec. 4.1.1 plus block data). */
typedef struct merbit_plan_info {
  int64_t n_rows, n_cols, nnz;
  int32_t sigma;            /* steps per lane                                   */
  int32_t omega;            /* lanes per tile (32, the warp size)               */
  int32_t tiles_per_block;  /* tiles sharing one output buffer (W)              */
  int64_t tile_num;         /* ceil((nnz + n_rows) / (omega * sigma))            */
  int64_t lane_num;         /* ceil((nnz + n_rows) / sigma)                      */
  int64_t block_num;        /* ceil(tile_num / tiles_per_block)                  */
  const uint32_t* tile_x;   /* device, tile_num + 1: tile start x; last = nnz    */
  const uint32_t* tile_y;   /* device, tile_num + 1: tile start row, MSB = single-row
                               tile; last = n_rows                               */
  const uint32_t* lane_desc;/* device, lane_num: bit_flag<<18 | y_off<<9 | x_off */
  const int32_t* block_row; /* device, block_num + 1: row of each block's first
                               coordinate (ROW(tile_y[b * W])); last = n_rows    */
  int32_t desc_bytes;       /* 4: lane_desc holds 32-bit words (sigma <= 14);
                               8: 64-bit words bit_flag<<22 | y_off<<11 | x_off
                               (sigma 15..42; the pointer above then addresses
                               lane_num 64-bit words)                            */
} merbit_plan_info;

/*
 * merbit_plan — build the reusable TILE schedule of a square n x n CSR matrix
 * (Sec. 4.1, Algorithm generate_tile): merge-path search of every lane start
 * on diagonal j*sigma, sigma-step walk into bit_flag, 32-bit lane descriptors
 * and the single-row (MSB) tile mark.  sigma = 14, omega = 32, 8 tiles per
 * block.  row_ptr is read during the call only; col_idx is BORROWED and must
 * stay alive and unchanged until merbit_plan_destroy.  The plan owns all of
 * its device memory.  Synchronises `stream` once (to read row_ptr[0] and
 * row_ptr[n]).  Errors: EINVAL (NULL pointer, negative size, row_ptr[0] != 0
 * or row_ptr[n] != nnz), EOVERFLOW, ENOMEM, ECUDA.
 */
merbit_status merbit_plan(const int32_t* row_ptr, const int32_t* col_idx, int64_t n,
                          int64_t nnz, merbit_plan_t* out);

/* As merbit_plan for an n_rows x n_cols matrix, with sigma in [1, 42]
 * (32-bit descriptors need 2*ceil(log2(32*sigma)) + sigma <= 32, Sec. 4.1.1, so
 * sigma <= 14; sigma 15..42 uses 64-bit descriptors bit_flag<<22 | y_off<<11 | x_off,
 * the larger word Sec. 5.3.4 names; those plans serve the SpMV and the solvers built on
 * it, not the SpMM, personalised PageRank or batches),
 * tiles_per_block W in {4, 8, 16} (the block of W tiles that shares one
 * shared-memory output buffer, Sec. 4.2; the block kernels keep 8 warps, one per
 * tile for W = 8, warps idle past W = 4, two tiles per warp at W = 16; the SpMM and
 * personalised PageRank need W = 8), on `stream`. */
merbit_status merbit_plan_ex(const int32_t* row_ptr, const int32_t* col_idx, int64_t n_rows,
                             int64_t n_cols, int64_t nnz, int sigma, int tiles_per_block,
                             void* stream, merbit_plan_t* out);

/* Free a plan and everything it owns.  NULL is ignored.  Synchronises the device. */
void merbit_plan_destroy(merbit_plan_t plan);

/* Fill *info (host struct) with the plan's sizes and device array pointers
 * (borrowed, valid until destroy).  Errors: EINVAL. */
merbit_status merbit_plan_get_info(merbit_plan_t plan, merbit_plan_info* info);

/* Copy the TILE arrays and block rows to HOST buffers (sizes as in
 * merbit_plan_info: tile_num + 1, tile_num + 1, lane_num words of desc_bytes each,
 * block_num + 1);
 * any pointer may be NULL to skip that array.  Synchronous (device-wide).
 * Errors: EINVAL, ECUDA. */
merbit_status merbit_plan_export(merbit_plan_t plan, uint32_t* tile_x, uint32_t* tile_y,
                                 uint32_t* lane_desc, int32_t* block_row);

/* Block kernels of the product y = A x (every call that multiplies by a plan's
 * matrix uses one of them; results agree to rounding):
 *   MERBIT_KERNEL_CLASSIC: 256 threads per CTA; all of them gather x and form the
 *     products of a block, then each warp reduces one tile (Sec. 4.2, one block at
 *     a time per CTA, two copy stages).
 *   MERBIT_KERNEL_SPLIT: 512 threads per CTA; 256 producer threads gather x and form
 *     the products of the next blocks while the 256 consumer threads reduce and
 *     commit the current one (three stages), so gathers and scans overlap.
 *   MERBIT_KERNEL_SPLIT2: the split kernel with a ring of two stages instead of three
 *     (less shared memory, so more L1 for x; the copy of block i + 2 then overlaps only
 *     the producers' work on block i + 1).
 *   A split kernel that cannot hold one CTA's stages on an SM (large sigma x block
 *   size with 8-byte values) gives way to CLASSIC.
 *   MERBIT_KERNEL_AUTO (the default): SPLIT while two of its CTAs fit on an SM and
 *     their three stages at the plan's sigma take at most 168 KB of shared memory per
 *     SM, else SPLIT2 while two of those fit, else CLASSIC. */
enum {
  MERBIT_KERNEL_AUTO = 0,
  MERBIT_KERNEL_CLASSIC = 1,
  MERBIT_KERNEL_SPLIT = 2,
  MERBIT_KERNEL_SPLIT2 = 3
};

/* Choose the block kernel for every later call on this plan (host-side setting,
 * takes effect at the next launch).  Errors: EINVAL (NULL plan, unknown kernel). */
merbit_status merbit_plan_set_kernel(merbit_plan_t plan, int kernel);

/*
 * merbit_plan_set_hot_columns — (re)build the plan's hot-column table, or drop it
 * (max_hot = 0).  No counterpart in the paper: it serves the x gather of the SpMV
 * (Sec. 4.2) on GB300.  The columns referenced by the most nonzeros (at most max_hot,
 * each used at least twice) are sorted by use; the plan keeps a copy of col_idx in
 * which each of them is replaced by its table slot, and every product launch copies x
 * at those columns into the shared memory of each CTA once and takes the gathers of
 * those nonzeros from there.  A launch uses the table only when all of it fits beside
 * its block kernel's stages without lowering the resident CTAs per SM (otherwise it
 * streams col_idx as before); results agree with the plain gather bit for bit in the
 * products, to rounding in the sums.  The table is kept only if its columns hold at
 * least min_cover (in [0, 1]) of the nonzeros.  Costs 4 bytes per nonzero of device
 * memory and a few passes over col_idx; synchronises `stream`.  *hot_n_out and
 * *cover_out (host, may be NULL) receive the number of table columns (0: none) and the
 * fraction of the nonzeros they hold.  Errors: EINVAL, ENOMEM, ECUDA.
 */
merbit_status merbit_plan_set_hot_columns(merbit_plan_t plan, int max_hot, double min_cover,
                                          void* stream, int* hot_n_out, double* cover_out);

/*
 * merbit_gather_probe — a measurement aid with no counterpart in the paper: one pass of
 * the SpMV's x gather alone (the x[col[k]] of Sec. 4.2's products) over the plan's
 * nonzeros, with the grid, block size and dynamic shared memory of the plan's
 * split-kernel product launch for x of type xdt (F32 or F64), the hot-column table
 * included when that launch would use it.  The column stream is read coalesced; every
 * gathered value is summed and each CTA writes its sum to sink (device, at least 4096
 * entries of xdt).  Timing it beside the product gives the cost of the gathers at the
 * kernel's shared-memory footprint.  Asynchronous on `stream`.  Errors: EINVAL, ECUDA.
 */
merbit_status merbit_gather_probe(merbit_plan_t plan, merbit_dtype xdt, const void* x, void* sink,
                                  void* stream);

/* Test aid (no counterpart in the paper): the number of polls after which a stage wait
 * of the plan's SpMV and SpMM block kernels gives up (polls < 0 restores the default, 2^22).  A
 * wait that gives up sets the plan's error bit; the kernel then waits, with the default
 * limit, for its own copies in flight and returns, and merbit_plan_sync (or the next
 * solver call) reports MERBIT_EDEVICE and clears the state.  polls = 0 makes every
 * launch give up at its first stage wait, which exercises that path without any fault.
 * Errors: EINVAL (NULL plan). */
merbit_status merbit_plan_set_wait_limit(merbit_plan_t plan, int polls);

/* Synchronise `stream` and report a kernel-side error of this plan's earlier
 * asynchronous calls (EDEVICE; the plan's device state is reset). */
merbit_status merbit_plan_sync(merbit_plan_t plan, void* stream);

/*
 * merbit_spmv — y = A x (Sec. 3.1) with the MERBIT kernel (Sec. 4.2,
 * Algorithms MERBIT SpMV, tile_normal_tackle, WarpSegmentedSum): tile values
 * and column indices staged in shared memory, descriptor-driven lane scan,
 * warp segmented sum, single-row fast path, block commit.  dtype is F32 or F64
 * for vals, x and y alike.  y (n_rows entries) is fully overwritten; the
 * caller never clears it.  x has n_cols entries.  Asynchronous on the legacy
 * default stream.  Errors: EINVAL (NULL, dtype, alignment), ECUDA.
 */
merbit_status merbit_spmv(merbit_plan_t plan, merbit_dtype dtype, const void* vals,
                          const void* x, void* y);

/*
 * merbit_spmv_ex — as merbit_spmv with separate value / vector types and a
 * stream.  Supported (vals_dtype, xy_dtype): (F32, F32), (F64, F64),
 * (BF16, F32), (F16, F32); reduced-precision values are widened to f32 and
 * accumulated in f32.  The result is multiplied by 2^-scale_exp (exact), for
 * values stored pre-scaled by 2^scale_exp (see merbit_vals_convert); pass 0
 * otherwise.
 */
merbit_status merbit_spmv_ex(merbit_plan_t plan, merbit_dtype vals_dtype, merbit_dtype xy_dtype,
                             const void* vals, const void* x, void* y, int scale_exp,
                             void* stream);

/*
 * merbit_spmm — Y = A X for k right-hand sides at once (the batching extension
 * of the method: k personalisation vectors in one pass over the plan).  X is
 * row-major n_cols x k with leading dimension ldx >= k, Y row-major n_rows x k
 * with ldy >= k, all f32 device pointers; vals f32, 16-byte aligned.  The plan
 * must have 8 tiles per block and sigma <= 14.  Columns are processed in chunks of
 * 32, 16, 8 or 4; each nonzero's column index and value are read once per chunk and
 * the gathered row slice X[col, chunk] serves the whole chunk.  When k, ldx and ldy
 * are multiples of 4 and X, Y are 16-byte aligned the slices are read as 16-byte
 * vectors (32-byte ones in chunks of 16 and 32 when k and ldx are also multiples of 8
 * and X is 32-byte aligned), otherwise element by element.  Y's first k columns are
 * fully overwritten (rows of A with no nonzeros get 0).
 * Asynchronous on `stream`; allocates (once per plan) a (block_num + 1) x 32
 * FP64 accumulator for rows shared between blocks.  A stage wait that gives up
 * (bounded; see merbit_plan_set_wait_limit) is reported by merbit_plan_sync as
 * MERBIT_EDEVICE.  Errors: EINVAL (NULL pointers, k < 0, ldx < k, ldy < k,
 * misaligned vals, a plan of other than 8 tiles per block or sigma > 14), ENOMEM,
 * ECUDA.
 */
merbit_status merbit_spmm(merbit_plan_t plan, const float* vals, const float* X, float* Y,
                          int64_t k, int64_t ldx, int64_t ldy, void* stream);

/*
 * merbit_ppr — personalised PageRank for k seed vertices at once, on the batched
 * product (the batching extension of Sec. 5.5.1's power method).  Column c of the
 * row-major n x k result Pi (device, leading dimension k, f32) is the stationary
 * vector of
 *     pi' = alpha P^T pi + (alpha D + 1 - alpha) e_{seeds[c]},
 * D = the mass of pi on dangling vertices (empty columns of the plan's matrix), i.e.
 * teleport and dangling mass both return to the seed.  Starts from pi_0 = e_seed and
 * performs updates until every column's ||pi' - pi||_1 is below tol (tol <= 0: exactly
 * max_iter updates).  The plan must be square; vals (f32 device, 16-byte aligned) are
 * the values of P^T; seeds is a HOST array of k vertex ids, 1 <= k <= 1024.  Outputs (each may be
 * NULL): iters_out = updates performed; resid_out (host, k entries) = each column's
 * last ||pi' - pi||_1; resid_hist (host, max_iter entries) = per update the largest
 * column residual.  Synchronous with respect to the host (it polls the device every 8
 * updates); uses plan-owned device memory for a second n x k iterate.  Errors: EINVAL
 * (bad arguments or seed), ENOTCONV (tol not reached; Pi holds the last iterate),
 * EDEVICE (a kernel's bounded wait expired), ENOMEM, ECUDA.
 */
merbit_status merbit_ppr(merbit_plan_t plan, const float* vals, const int32_t* seeds, int64_t k,
                         double alpha, double tol, int max_iter, float* Pi, int* iters_out,
                         double* resid_out, double* resid_hist, void* stream);

/* ---------------------------------------------------------------- differentiation
 * The backward pass of y = A x needs A^T g and the per-nonzero products g[row] x[col];
 * the backward pass of the PageRank fixed point needs the adjoint solve below.  None of
 * these calls has a counterpart in the paper; they reuse its plan and SpMV on A^T.
 */
typedef struct merbit_transpose_s* merbit_transpose_t;

/*
 * merbit_transpose — the CSR of A^T (n_cols x n_rows) from the CSR of A, on the device:
 * row_ptr_t (n_cols + 1), col_t (nnz; each row of A^T in increasing column order, i.e.
 * the result does not depend on thread timing) and perm (nnz): A^T's k-th nonzero is A's
 * nonzero perm[k], so vals_t = vals[perm] (merbit_gather).  Inputs are device arrays,
 * sorted and duplicate-free per row; the transpose owns its three arrays (read them with
 * merbit_transpose_get) until merbit_transpose_destroy.  A plan of A^T is
 * merbit_plan_ex(row_ptr_t, col_t, n_cols, n_rows, nnz, ...); it borrows col_t.
 * Synchronous.  Errors: EINVAL, EOVERFLOW (sizes beyond int32), ENOMEM, ECUDA.
 */
merbit_status merbit_transpose(const int32_t* row_ptr, const int32_t* col_idx, int64_t n_rows,
                               int64_t n_cols, int64_t nnz, void* stream, merbit_transpose_t* out);
merbit_status merbit_transpose_get(merbit_transpose_t t, const int32_t** row_ptr_t,
                                   const int32_t** col_t, const int32_t** perm);
void merbit_transpose_destroy(merbit_transpose_t t);

/* merbit_gather — dst[i] = src[idx[i]] for i < count; F32 or F64 device arrays. */
merbit_status merbit_gather(merbit_dtype dtype, const void* src, const int32_t* idx, void* dst,
                            int64_t count, void* stream);

/*
 * merbit_sddmm — out[k] = scale * g[row(k)] * x[col(k)] for every nonzero k of the plan's
 * matrix (the value gradient of y = A x is g[row] x[col]).  g has n_rows entries, x has
 * n_cols, out has nnz; F32 or F64 device arrays (the plan's column indices must still
 * be valid).  Asynchronous.  Errors: EINVAL, ECUDA.
 */
merbit_status merbit_sddmm(merbit_plan_t plan, merbit_dtype dtype, const void* g, const void* x,
                           double scale, void* out, void* stream);

/*
 * merbit_pagerank_adjoint — lambda solving (I - alpha M)^T lambda = w, M = A + (1/n) 1 d^T
 * the PageRank operator of merbit_pagerank (A = P^T from `plan`, d its dangling
 * indicator).  For a loss L(pi) at the PageRank fixed point, w = dL/dpi gives
 * dL/dA_ij = alpha * lambda_i * pi_j (merbit_sddmm with scale alpha, g = lambda, x = pi).
 * Iterates lambda' = alpha A^T lambda + alpha (sum(lambda)/n) d + w from lambda_0 = w on
 * `plan_t`, a plan of A^T with values vals_t (F32 or F64, 16-byte aligned), until
 * ||lambda' - lambda||_1 <= tol * ||w||_1 (tol <= 0: exactly max_iter updates); the
 * residual reported in resid_out is absolute.  Synchronous.
 * Errors: EINVAL, ENOTCONV (lambda holds the last iterate), EDEVICE, ENOMEM, ECUDA.
 */
merbit_status merbit_pagerank_adjoint(merbit_plan_t plan, merbit_plan_t plan_t, merbit_dtype dtype,
                                      const void* vals_t, double alpha, const void* w, double tol,
                                      int max_iter, void* lambda, int* iters_out, double* resid_out,
                                      void* stream);

/*
 * merbit_autotune_sigma — picks the plan's steps per lane (sigma, Sec. 4.1.1) for one
 * matrix and value type by measurement: for each of the `count` candidates (each in
 * [1, 14]) it builds a plan, runs one warm-up SpMV and `reps` timed ones (CUDA events on
 * `stream`, x = 0) and frees the plan.  best_sigma = the fastest candidate; ms_out (HOST,
 * count entries, may be NULL) = mean milliseconds per product.  CSR arrays and vals are
 * device pointers as in merbit_plan_ex / merbit_spmv_ex; dtype F32 or F64.  Synchronous.
 * Errors: EINVAL, ENOMEM, ECUDA, and those of merbit_plan_ex / merbit_spmv_ex.
 */
merbit_status merbit_autotune_sigma(const int32_t* row_ptr, const int32_t* col_idx, int64_t n_rows,
                                    int64_t n_cols, int64_t nnz, merbit_dtype dtype, const void* vals,
                                    const int* candidates, int count, int reps, void* stream,
                                    int* best_sigma, float* ms_out);

/*
 * merbit_autotune — picks a plan's parameters for one matrix and value type by
 * measurement: every combination of sigma (sigmas[n_sigma], each in [1, 42]), tiles per
 * block (blocks[n_block], each 4, 8 or 16), block kernel (kernels[n_kernel], each a
 * MERBIT_KERNEL_* value) and hot-column table size (hots[n_hot], each in [0, 2^20];
 * merbit_plan_set_hot_columns with min_cover 0) is built and timed: one warm-up product
 * and `reps` timed ones (CUDA events on `stream`, x = 0).  dtype is the value type (F32,
 * F64, or BF16 / F16 with f32 vectors).  best (HOST, 4 ints) = {sigma, tiles_per_block,
 * kernel, hot} of the fastest; ms_out (HOST, may be NULL, n_sigma * n_block * n_hot *
 * n_kernel entries, row-major in that order) = mean milliseconds per product, -1 for a
 * combination the device cannot launch.  Synchronous.  Errors: EINVAL, ENOMEM, ECUDA
 * (also when no combination can be launched), and those of merbit_plan_ex.
 */
merbit_status merbit_autotune(const int32_t* row_ptr, const int32_t* col_idx, int64_t n_rows,
                              int64_t n_cols, int64_t nnz, merbit_dtype dtype, const void* vals,
                              const int* sigmas, int n_sigma, const int* blocks, int n_block,
                              const int* kernels, int n_kernel, const int* hots, int n_hot, int reps,
                              void* stream, int* best, float* ms_out);

/*
 * merbit_bicgstab — solves A x = b by unpreconditioned BiCGSTAB on the plan's SpMV (the
 * paper's second iterative workload, Sec. 5.5), FP64: vals (16-byte aligned), b and x
 * are device arrays of n; x holds the initial guess on entry and the last iterate on
 * return.  vals NULL means every value is 1 (an adjacency pattern): the products then
 * read no value stream.  Shadow residual r_hat = r_0; stops when ||b - A x||_2 <= tol ||b||_2 (the
 * recurrence's residual), after max_iter iterations, or when a denominator of the
 * recurrence is zero.  The whole solve is one CUDA-graph launch with a device-side loop
 * (two SpMVs and three fused vector passes per iteration).  Outputs (may be NULL):
 * iters_out, resid_out = ||r||_2 / ||b||_2 at the end, resid_hist (HOST, max_iter
 * entries: the same after each iteration), status_out (1 converged, 2 max_iter,
 * 3 breakdown).  Synchronous; allocates 6 n work vectors per call.  Errors: EINVAL,
 * ENOTCONV (statuses 2 and 3; x holds the last iterate), EDEVICE, ENOMEM, ECUDA.
 */
merbit_status merbit_bicgstab(merbit_plan_t plan, const double* vals, const double* b, double* x,
                              double tol, int max_iter, int* iters_out, double* resid_out,
                              double* resid_hist, int* status_out, void* stream);

/* ---------------------------------------------------------------- many graphs
 * PageRank of many independent graphs in one CUDA-graph launch (the batching extension;
 * no counterpart in the paper).  The graphs are the diagonal blocks of one block-diagonal
 * CSR matrix (the transition matrices P^T of each graph, vertex ids offset by
 * graph_offsets), so one MERBIT plan balances the work across all of them.
 */
typedef struct merbit_batch_s* merbit_batch_t;

/*
 * merbit_batch_plan — plan of the block-diagonal matrix (n x n, nnz nonzeros, device
 * CSR; the batch borrows col_idx).  graph_offsets (HOST, num_graphs + 1 entries) gives
 * graph g the vertices [graph_offsets[g], graph_offsets[g+1]); every graph has at least
 * one vertex and every nonzero must stay inside its graph's diagonal block (checked:
 * EINVAL otherwise).  sigma as in merbit_plan_ex.  Synchronous.  Errors: EINVAL,
 * EOVERFLOW, ENOMEM, ECUDA.
 */
merbit_status merbit_batch_plan(const int32_t* row_ptr, const int32_t* col_idx, int64_t n,
                                int64_t nnz, const int64_t* graph_offsets, int num_graphs,
                                int sigma, void* stream, merbit_batch_t* out);

/*
 * merbit_batch_pagerank — for every graph, the PageRank power iteration of
 * merbit_pagerank (pi_0 = 1/n_g, teleport and dangling mass spread over the graph's own
 * vertices) until its ||pi' - pi||_1 < tol, all graphs advancing together one round per
 * SpMV over the whole matrix; a converged graph is left untouched by later rounds.  The
 * whole solve is one CUDA-graph launch with a device-side loop (recorded on first use and
 * kept while dtype, vals, pi, alpha, tol and max_iter stay the same).  vals: F32 or F64
 * device values (16-byte aligned); pi: n entries of that type (graph g's vector in its
 * vertex range).  iters (HOST, num_graphs or NULL): updates of each graph; resid (HOST,
 * num_graphs or NULL): each graph's last ||pi' - pi||_1; rounds_out: rounds run.
 * Synchronous.  Errors: EINVAL, ENOTCONV (some graph did not reach tol in max_iter rounds;
 * pi holds every graph's last iterate), EDEVICE, ENOMEM, ECUDA.
 */
merbit_status merbit_batch_pagerank(merbit_batch_t batch, merbit_dtype dtype, const void* vals,
                                    double alpha, double tol, int max_iter, void* pi, int* iters,
                                    double* resid, int* rounds_out, void* stream);
/* The plan of the block-diagonal matrix (owned by the batch). */
merbit_plan_t merbit_batch_get_plan(merbit_batch_t batch);
void merbit_batch_destroy(merbit_batch_t batch);

/*
 * merbit_spmv_host — y = A x with x and y in HOST memory (pinned or pageable;
 * `vals` stays a device pointer).  x is copied into plan-owned device memory,
 * the product runs on `stream`, y is copied back, and the stream is
 * synchronised before returning.  dtype F32 or F64.  Errors as merbit_spmv,
 * plus ENOMEM and EDEVICE.
 */
merbit_status merbit_spmv_host(merbit_plan_t plan, merbit_dtype dtype, const void* vals,
                               const void* x_host, void* y_host, void* stream);

/*
 * merbit_spmv_host_async — as merbit_spmv_host (F32 or F64, x and y in HOST memory,
 * vals on the device) but without waiting: the call uploads x into one of two plan-owned
 * staging slots and runs the product on `stream`, and an internal copy stream downloads
 * y once the product is done, so consecutive calls overlap one call's download with the
 * next call's upload and product.  With pageable host memory the copies serialise.
 * x_host must stay unchanged and y_host unread until merbit_plan_sync returns (it waits
 * for every pending download of the plan).  Errors: EINVAL, ENOMEM, ECUDA, and those of
 * merbit_spmv_ex.
 */
merbit_status merbit_spmv_host_async(merbit_plan_t plan, merbit_dtype dtype, const void* vals,
                                     const void* x_host, void* y_host, void* stream);

/*
 * merbit_vals_convert — round nnz values (src_dtype F64 or F32) to dst_dtype
 * (BF16, F16 or F32), round-to-nearest-even.  With auto_scale != 0 and dst F16
 * the values are first multiplied by 2^k, k the largest power keeping
 * max|v| * 2^k below 2^15, so that small values of a stochastic matrix stay
 * normal; k is written to *scale_exp_out (host, may be NULL) and must be passed
 * as scale_exp to merbit_spmv_ex.  Synchronises `stream` when auto-scaling.
 */
merbit_status merbit_vals_convert(const void* src, merbit_dtype src_dtype, void* dst,
                                  merbit_dtype dst_dtype, int64_t nnz, int auto_scale,
                                  int* scale_exp_out, void* stream);

/*
 * merbit_pagerank — PageRank by the power method (Sec. 5.5.1) on a square
 * plan whose values form P^T (column j holds 1/outdeg(j) for every edge j->i):
 *   pi_0 = 1/n,  pi_{k+1} = alpha P^T pi_k + (alpha D_k + 1 - alpha)/n,
 * D_k the mass of pi_k on dangling vertices (empty columns).  Stops once
 * ||pi_{k+1} - pi_k||_1 < tol; at most 10000 updates.  dtype F32 or F64 (vals
 * and pi).  pi (n entries) receives the last iterate.  One fused kernel per
 * update (SpMV + update + residual + dangling mass, FP64 reductions).
 * Synchronises the legacy default stream.  Errors: EINVAL (non-square plan,
 * alpha outside [0,1), dtype), ENOTCONV, EDEVICE, ECUDA.
 */
merbit_status merbit_pagerank(merbit_plan_t plan, merbit_dtype dtype, const void* vals,
                              double alpha, double tol, void* pi);

/*
 * merbit_pagerank_ex — as merbit_pagerank with:
 *   max_iter     PLAIN: cap on updates.  IR modes: cap on refinement steps.
 *                With tol <= 0 exactly max_iter updates (steps) run and the
 *                call returns MERBIT_OK.
 *   mode         PLAIN, or IR_BF16 / IR_F16 / IR_F32: mixed-precision
 *                iterative refinement.  vals must be F64 (master values) and
 *                pi F64.  Each step computes r = b - M pi in FP64
 *                (M = I - alpha P^T - (alpha/n) 1 d^T, b = (1-alpha)/n 1), stops
 *                when ||r||_1 < tol, then solves M delta = r approximately by
 *                Richardson sweeps delta <- alpha P~^T delta + (alpha/n)(d^T delta) + r
 *                from delta = r, with reduced-precision values P~, f32 vectors,
 *                f32 accumulation and FP64 dangling sums, and sets pi += delta
 *                (FP64).
 *   inner_sweeps IR modes: maximum sweeps per refinement step (>= 1).
 *   inner_tol    IR modes: the sweeps of a step stop once one sweep changes
 *                delta by less than inner_tol * ||r||_1 (L1); 0 selects the unit
 *                roundoff of the inner values (2^-8 bf16, 2^-11 f16) and 2^-17 for f32.
 *   iters_out    host, may be NULL: updates (PLAIN) or refinement steps (IR).
 *   resid_out    host, may be NULL: the last L1 residual computed.
 *   resid_hist   host, may be NULL: residual per update (PLAIN, max_iter
 *                entries) or per residual evaluation (IR, max_iter + 1 entries).
 *   launches_out host, may be NULL: SpMV launches that did work (PLAIN: the
 *                updates; IR: residual evaluations plus inner sweeps).
 * Synchronises `stream`.
 */
merbit_status merbit_pagerank_ex(merbit_plan_t plan, merbit_dtype dtype, const void* vals,
                                 double alpha, double tol, int max_iter, merbit_precision mode,
                                 int inner_sweeps, double inner_tol, void* pi, int* iters_out,
                                 double* resid_out, double* resid_hist, int* launches_out,
                                 void* stream);

/*
 * merbit_spmv_noalloc — y = A x in f32 for callers that must not allocate
 * device memory (the paper has no counterpart: it is an entry point of this
 * library only).  Some callers cannot call cudaMalloc — code whose device
 * memory belongs to another framework's pool, or paths where cudaMalloc's
 * device-wide synchronisation is not acceptable.  This call builds the MERBIT
 * schedule (sigma = 14) and runs the product without allocating anything: it
 * uses the caller's row_ptr, col_idx, vals, x (n_cols entries) and y (n_rows
 * entries, fully overwritten), all device pointers, plus a fixed scratch array
 * compiled into the library (8 MiB = 8,388,608 bytes; every GPU that loads
 * the library keeps it until the process exits).  A matrix needs
 *     66,816 + up256(4 lane_num) + 2 up256(4 (tile_num + 1))
 *            + 2 up256(4 (block_num + 1)) + up256(8 (block_num + 1))
 * bytes of it, with S = n_rows + nnz, lane_num = ceil(S / 14),
 * tile_num = ceil(S / 448), block_num = ceil(tile_num / 8) and up256 rounding
 * up to a multiple of 256: about 27 million rows plus nonzeros at most.
 * Larger matrices are rejected with MERBIT_EINVAL and a message from
 * merbit_last_error() (use merbit_plan / merbit_spmv).  Every call looks up the
 * scratch array's device address in the current context; make the first call
 * on a device before any stream capture (the lookup may load the module).
 * All calls share the one array: calls that overlap on the GPU (other streams,
 * other threads) race and give wrong results.  Asynchronous on `stream`; vals
 * and col_idx must be 16-byte aligned, x and y 4-byte aligned; row_ptr is
 * trusted (not checked).  Errors: EINVAL, EOVERFLOW, ECUDA.  A kernel that
 * gives up on a bounded wait cannot report it through this asynchronous call:
 * it sets an error word in the scratch array, which stays set until
 * merbit_spmv_noalloc_status reads it.  Callers must check that status before
 * trusting y.
 */
merbit_status merbit_spmv_noalloc(const int32_t* row_ptr, const int32_t* col_idx, const float* vals,
                                  const float* x, float* y, int64_t n_rows, int64_t n_cols,
                                  int64_t nnz, void* stream);

/*
 * merbit_spmv_noalloc_status — synchronises `stream` and reports whether any
 * merbit_spmv_noalloc call since the last status query had a kernel give up on
 * a bounded wait (then the y of that call is incomplete): MERBIT_EDEVICE, with
 * the error word cleared, or MERBIT_OK.  Allocates nothing (a 4-byte copy into
 * a host variable).  No counterpart in the paper.  Errors: EDEVICE, ECUDA.
 */
merbit_status merbit_spmv_noalloc_status(void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* merbit_last_error(void);

/* Library version string. */
const char* merbit_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MERBIT_H */
