// Internal declarations of the MERBIT CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "merbit.h"

namespace merbit {

constexpr int kOmega = 32;          // lanes per tile = warp size (Sec. 4.3)
constexpr int kSigmaMax = 14;       // largest sigma of the 32-bit descriptor (Sec. 4.1.1)
constexpr int kSigmaMax64 = 42;     // largest sigma of the 64-bit descriptor (11-bit offsets)
constexpr int kTilesPerBlock = 8;   // W: tiles that share one shared-memory output buffer (default)
constexpr int kThreads = kTilesPerBlock * kOmega;   // block kernels: 8 warps, one per tile of W = 8
constexpr int kWarps = kThreads / 32;
constexpr int kMaxW = 16;           // largest W a plan may use (W in {4, 8, 16})
constexpr int kMaxTpw = kMaxW / kWarps;             // tiles a warp reduces per block (at most)
constexpr int kRedSlots = 64;       // spread slots of the grid-wide FP64 reductions
constexpr uint32_t kMsb = 0x80000000u;
constexpr uint32_t kSpinLimit = 1u << 22;           // bounded mbarrier waits
constexpr int kMaxParts = 4096;                     // cap on persistent CTAs (partials array)

// Per-plan device state for grid-wide reductions and kernel-side errors.
struct RedState {
  double slot[kRedSlots][2];
  unsigned int arrive;
  int err;        // bit 0: an mbarrier wait expired
  int done;       // PageRank: a fused launch found its residual below tol
  int iters;      // number of launches counted when `done` was set
  int inner_done; // refinement: the inner sweeps of the current step have converged
  int launches;   // SpMV launches that did work since the solve started
  const float* delta;   // refinement: buffer holding the latest inner iterate
};

struct Geometry {
  const uint32_t* tile_x;
  const uint32_t* tile_y;
  const uint32_t* lane_desc;
  const int32_t* col;
  const int32_t* col_stage;   // column stream of the SpMV stages: col, or its hot-tagged copy
  const int32_t* hot_list;    // column of each hot-table slot
  int hot_n;                  // hot columns cached in shared memory by this launch (0: none)
  uint32_t wait_limit;        // polls of a stage wait before it gives up (drains use kSpinLimit)
  const int32_t* bnd_row;
  const int32_t* bnd_slot;
  double* bnd_acc;
  double2* part;   // per-CTA reduction partials of the main kernel
  RedState* red;
  int n_rows;
  int nnz;
  int steps;       // nnz + n_rows
  int sigma;
  int W;           // tiles per block
  int stages;      // split kernel: stages in its ring (2 or 3)
  int desc64;      // lane descriptors are 64-bit words (sigma > 14)
  int fold;        // the block kernel's last CTA finishes the product (few blocks)
  int tile_num;
  int lane_num;
  int nb;          // number of blocks of tiles
};

}  // namespace merbit

struct merbit_plan_s {
  int device = 0;
  int num_sms = 0;
  int64_t n_rows = 0, n_cols = 0, nnz = 0;
  int sigma = 14, tiles_per_block = merbit::kTilesPerBlock;
  int desc_bytes = 4;                    // 4: 32-bit lane descriptors; 8: 64-bit (sigma > 14)
  int spmv_kernel = 0;                   // MERBIT_KERNEL_AUTO / _CLASSIC / _SPLIT
  uint32_t wait_limit = merbit::kSpinLimit;   // polls of a stage wait (test hook lowers it)
  int64_t tile_num = 0, lane_num = 0, nb = 0;
  const int32_t* col = nullptr;          // borrowed
  // hot-column table: col_hot is a copy of col in which a column held in the table is
  // replaced by ~slot; hot_list[slot] is that column (slots by decreasing use)
  int32_t* col_hot = nullptr;
  int32_t* hot_list = nullptr;
  int hot_n = 0;
  double hot_cover = 0.0;                // fraction of the nonzeros in hot columns
  uint32_t* tile_x = nullptr;
  uint32_t* tile_y = nullptr;
  uint32_t* lane_desc = nullptr;
  int32_t* bnd_row = nullptr;
  int32_t* bnd_slot = nullptr;
  double* bnd_acc = nullptr;
  double2* part = nullptr;               // kMaxParts entries
  merbit::RedState* red = nullptr;
  // lazily built PageRank data
  uint32_t* dangling_bits = nullptr;     // (n+31)/32 words, bit set = dangling vertex
  int64_t n_dangling = -1;
  // scratch owned by the plan (grown on demand)
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  double* hist = nullptr;                // per-launch reduction results, [launch][2]
  size_t hist_len = 0;
  void* x_stage = nullptr;               // staging for host-buffer SpMV
  void* y_stage = nullptr;
  size_t x_stage_bytes = 0, y_stage_bytes = 0;
  void* host_pinned = nullptr;           // small pinned block for state read-back
  double* spmm_acc = nullptr;            // (nb + 1) x 32 FP64 boundary accumulators of the SpMM

  merbit::Geometry geom() const {
    merbit::Geometry g;
    g.tile_x = tile_x; g.tile_y = tile_y; g.lane_desc = lane_desc; g.col = col;
    g.col_stage = col; g.hot_list = hot_list; g.hot_n = 0;   // a launch opts in to the table
    g.wait_limit = wait_limit;
    g.bnd_row = bnd_row; g.bnd_slot = bnd_slot;
    g.bnd_acc = bnd_acc; g.part = part; g.red = red;
    g.n_rows = (int)n_rows; g.nnz = (int)nnz; g.steps = (int)(nnz + n_rows);
    g.sigma = sigma; g.W = tiles_per_block; g.stages = 3; g.desc64 = desc_bytes == 8; g.fold = 0;
    g.tile_num = (int)tile_num; g.lane_num = (int)lane_num; g.nb = (int)nb;
    return g;
  }
};

namespace merbit {

// A lane descriptor (Sec. 4.1.1): bit_flag << 2w | y_offset << w | x_offset, with w = 9 in
// the 32-bit word (sigma <= 14) and w = 11 in the 64-bit word (sigma <= 42).
struct LaneDesc {
  int xo, yo;
  uint64_t flags;   // bit k: step k of the lane is a down step
};

__device__ __forceinline__ uint64_t load_desc(const Geometry& g, int64_t j) {
  return g.desc64 ? (uint64_t)__ldg(reinterpret_cast<const unsigned long long*>(g.lane_desc) + j)
                  : (uint64_t)__ldg(g.lane_desc + j);
}

__device__ __forceinline__ LaneDesc decode_lane(const Geometry& g, uint64_t d) {
  if (g.desc64) return LaneDesc{(int)(d & 2047u), (int)((d >> 11) & 2047u), d >> 22};
  return LaneDesc{(int)(d & 511u), (int)((d >> 9) & 511u), d >> 18};
}

// ---- epilogue parameter blocks (device-side behaviour lives in spmv_kernel.cuh) ----

// PageRank power update: out = alpha*s + (alpha*D + 1 - alpha)/n.
struct PRParams {
  void* out;                    // T[n]: pi_{k+1}
  const uint32_t* dang;         // dangling bits
  double alpha, inv_n, tol;
  const double* d_in;           // D_k (dangling mass of pi_k)
  double* s_out;                // [0] = ||pi_{k+1} - pi_k||_1, [1] = D_{k+1}
  int iter;                     // launch index, stored in red->iters on convergence
};

// Mixed-precision refinement: residual r = b - M pi in FP64.
struct ResidParams {
  float* rhs;                   // f32 copy of r (= first inner iterate)
  const uint32_t* dang;
  double alpha, inv_n, tol;
  const double* d_in;           // D of pi
  double* s_out;                // [0] = ||r||_1, [1] = dangling sum of rhs
  int iter;
};

// Mixed-precision refinement: one inner Richardson sweep.
struct SweepParams {
  float* out;                   // next inner iterate
  const float* rhs;
  const uint32_t* dang;
  double alpha, inv_n;
  float scale;                  // 2^-scale_exp of pre-scaled values
  const double* d_in;           // dangling sum of the current inner iterate
  double* s_out;                // [0] = L1 size of this sweep, [1] = dangling sum of `out`
  const double* rnorm;          // ||r||_1 of the current refinement step
  double eta;                   // inner stop: sweep size <= eta * ||r||_1
};

// ---- launchers (one translation unit per value type) ----
cudaError_t spmv_plain_f32(const merbit_plan_s* p, const float* vals, const float* x, float* y,
                           cudaStream_t st);
cudaError_t spmv_plain_f64(const merbit_plan_s* p, const double* vals, const double* x,
                           double* y, cudaStream_t st);
cudaError_t spmv_plain_lo(const merbit_plan_s* p, merbit_dtype vdt, const void* vals,
                          const float* x, float* y, float scale, cudaStream_t st);
cudaError_t spmv_pr_f32(const merbit_plan_s* p, const float* vals, const float* x,
                        const PRParams& prm, cudaStream_t st);
cudaError_t spmv_pr_f64(const merbit_plan_s* p, const double* vals, const double* x,
                        const PRParams& prm, cudaStream_t st);
cudaError_t spmv_resid_f64(const merbit_plan_s* p, const double* vals, const double* pi,
                           const ResidParams& prm, cudaStream_t st);
cudaError_t spmv_sweep(const merbit_plan_s* p, merbit_dtype vdt, const void* vals,
                       const float* x, const SweepParams& prm, cudaStream_t st);
// Y = A X, row-major X (n_cols x k, leading dimension ldx) and Y (n_rows x k, ldy), f32;
// acc: (nb + 1) x 32 zeroed FP64 accumulators (left zeroed)
cudaError_t spmm_plain_f32(const merbit_plan_s* p, const float* vals, const float* X, int64_t k,
                           int64_t ldx, float* Y, int64_t ldy, double* acc, cudaStream_t st);
// Y = scale * A X, skipped once the plan's stop flag is set (iterative drivers)
cudaError_t spmm_scaled_f32(const merbit_plan_s* p, const float* vals, const float* X, int64_t k,
                            int64_t ldx, float* Y, int64_t ldy, float scale, double* acc,
                            cudaStream_t st);
// Personalised PageRank: X = one-hot seed columns (n x k, ld k), d_cur = their dangling mass
cudaError_t ppr_init(const merbit_plan_s* p, float* X, int64_t k, const int32_t* seed,
                     double* d_cur, cudaStream_t st);
// one update Y = alpha P^T X + (alpha D + 1 - alpha) e_seed for all k columns, then the
// finish step (per-column residuals into last_r, D of Y into d_cur, hist[iter] = largest
// residual, stop flag when it is below tol); rd: 2k zeroed FP64 accumulators (left zeroed)
cudaError_t ppr_update(const merbit_plan_s* p, const float* vals, const float* X, float* Y,
                       int64_t k, const int32_t* seed, double* d_cur, double* rd, double* last_r,
                       float alpha, double tol, int iter, double* hist, double* acc,
                       cudaStream_t st);
// pi += delta (FP64) with delta = the refinement's latest inner iterate; s_out[1] = dangling mass
cudaError_t ir_apply(const merbit_plan_s* p, double* pi, double* s_out, cudaStream_t st);

// Launch configuration of the split kernel's plain product (f32 or f64 values and
// vectors) for a plan: grid, dynamic shared memory, geometry (with the hot-column table
// if that launch takes it); false if it cannot be launched.
bool split_config_f32(const merbit_plan_s* p, Geometry& g, int& grid, size_t& smem);
bool split_config_f64(const merbit_plan_s* p, Geometry& g, int& grid, size_t& smem);

// Largest grid worth launching for a kernel (SMs x resident CTAs), cached.
// smem_max: the largest dynamic shared memory any launch of this kernel may use.
int persistent_grid(const void* kernel, int threads, size_t smem, size_t smem_max, int num_sms);

// Dynamic shared memory one CTA of `kernel` may use while `per_sm` of its CTAs stay
// resident on an SM of the current device (0 on error).
size_t smem_room(const void* kernel, int per_sm);

// The same room while the SM's shared memory (per_sm CTAs, each with the reserved block
// share and the kernel's static shared memory) stays at or below shared_per_sm bytes.
size_t smem_room_below(const void* kernel, int per_sm, size_t shared_per_sm);

}  // namespace merbit
