// Autotuners of a plan's parameters for one matrix and value type, by measurement (the
// paper chooses sigma per value type from a measured sweep, Sec. 5.4, and names larger
// sigma and block sizes as the knobs for GPUs with more on-chip memory, Sec. 5.3.4).
// merbit_autotune_sigma searches sigma alone; merbit_autotune searches sigma x tiles per
// block x block kernel x hot-column table size.  Each candidate plan is built, one
// warm-up product and `reps` timed ones run on the caller's stream (CUDA events), and
// the fastest configuration is reported.
#include <cstdio>
#include <vector>

#include "merbit_internal.cuh"

namespace merbit {
void set_last_error(const char* msg);
}  // namespace merbit

using namespace merbit;

namespace {

merbit_status afail(merbit_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

}  // namespace

extern "C" {

merbit_status merbit_autotune_sigma(const int32_t* row_ptr, const int32_t* col_idx, int64_t n_rows,
                                    int64_t n_cols, int64_t nnz, merbit_dtype dtype, const void* vals,
                                    const int* candidates, int count, int reps, void* stream,
                                    int* best_sigma, float* ms_out) {
  set_last_error("");
  if (!candidates || count < 1 || !best_sigma) return afail(MERBIT_EINVAL, "need candidates, count >= 1, best_sigma");
  if (dtype != MERBIT_F32 && dtype != MERBIT_F64) return afail(MERBIT_EINVAL, "dtype must be F32 or F64");
  if (reps < 1) return afail(MERBIT_EINVAL, "reps must be >= 1");
  for (int i = 0; i < count; ++i)
    if (candidates[i] < 1 || candidates[i] > kSigmaMax) return afail(MERBIT_EINVAL, "sigma candidate out of [1, 14]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t es = dtype == MERBIT_F64 ? 8 : 4;
  void *x = nullptr, *y = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&x, es * (size_t)std::max<int64_t>(n_cols, 1));
  if (e == cudaSuccess) e = cudaMalloc(&y, es * (size_t)std::max<int64_t>(n_rows, 1));
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, es * (size_t)std::max<int64_t>(n_cols, 1), st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  merbit_status s = MERBIT_OK;
  float best = 0.f;
  *best_sigma = candidates[0];
  for (int i = 0; i < count && e == cudaSuccess && s == MERBIT_OK; ++i) {
    merbit_plan_t p = nullptr;
    s = merbit_plan_ex(row_ptr, col_idx, n_rows, n_cols, nnz, candidates[i], kTilesPerBlock, stream, &p);
    if (s != MERBIT_OK) break;
    s = merbit_spmv_ex(p, dtype, dtype, vals, x, y, 0, stream);                 // warm-up
    if (s == MERBIT_OK) e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && s == MERBIT_OK && e == cudaSuccess; ++r)
      s = merbit_spmv_ex(p, dtype, dtype, vals, x, y, 0, stream);
    float ms = 0.f;
    if (s == MERBIT_OK && e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (s == MERBIT_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (s == MERBIT_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    merbit_plan_destroy(p);
    ms /= (float)reps;
    if (ms_out) ms_out[i] = ms;
    if (s == MERBIT_OK && e == cudaSuccess && (i == 0 || ms < best)) {
      best = ms;
      *best_sigma = candidates[i];
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  if (s != MERBIT_OK) return s;
  if (e != cudaSuccess) {
    char msg[256];
    std::snprintf(msg, sizeof(msg), "merbit_autotune_sigma: %s", cudaGetErrorString(e));
    return afail(e == cudaErrorMemoryAllocation ? MERBIT_ENOMEM : MERBIT_ECUDA, msg);
  }
  return MERBIT_OK;
}

merbit_status merbit_autotune(const int32_t* row_ptr, const int32_t* col_idx, int64_t n_rows,
                              int64_t n_cols, int64_t nnz, merbit_dtype dtype, const void* vals,
                              const int* sigmas, int n_sigma, const int* blocks, int n_block,
                              const int* kernels, int n_kernel, const int* hots, int n_hot, int reps,
                              void* stream, int* best, float* ms_out) {
  set_last_error("");
  if (!sigmas || !blocks || !kernels || !hots || n_sigma < 1 || n_block < 1 || n_kernel < 1 ||
      n_hot < 1 || !best)
    return afail(MERBIT_EINVAL, "need non-empty candidate lists and best");
  if (reps < 1) return afail(MERBIT_EINVAL, "reps must be >= 1");
  for (int i = 0; i < n_sigma; ++i)
    if (sigmas[i] < 1 || sigmas[i] > kSigmaMax64) return afail(MERBIT_EINVAL, "sigma candidate out of [1, 42]");
  for (int i = 0; i < n_block; ++i)
    if (blocks[i] != 4 && blocks[i] != 8 && blocks[i] != kMaxW)
      return afail(MERBIT_EINVAL, "tiles-per-block candidates must be 4, 8 or 16");
  for (int i = 0; i < n_kernel; ++i)
    if (kernels[i] < MERBIT_KERNEL_AUTO || kernels[i] > MERBIT_KERNEL_SPLIT2)
      return afail(MERBIT_EINVAL, "unknown kernel candidate");
  for (int i = 0; i < n_hot; ++i)
    if (hots[i] < 0 || hots[i] > (1 << 20)) return afail(MERBIT_EINVAL, "hot-table candidate out of [0, 2^20]");
  const bool lo16 = dtype == MERBIT_BF16 || dtype == MERBIT_F16;
  if (dtype != MERBIT_F32 && dtype != MERBIT_F64 && !lo16)
    return afail(MERBIT_EINVAL, "dtype must be F32, F64, BF16 or F16");
  const merbit_dtype xdt = dtype == MERBIT_F64 ? MERBIT_F64 : MERBIT_F32;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t es = xdt == MERBIT_F64 ? 8 : 4;
  void *x = nullptr, *y = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&x, es * (size_t)std::max<int64_t>(n_cols, 1));
  if (e == cudaSuccess) e = cudaMalloc(&y, es * (size_t)std::max<int64_t>(n_rows, 1));
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, es * (size_t)std::max<int64_t>(n_cols, 1), st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  merbit_status s = MERBIT_OK;
  float best_ms = -1.f;
  best[0] = sigmas[0];
  best[1] = blocks[0];
  best[2] = kernels[0];
  best[3] = hots[0];
  int idx = 0;
  for (int a = 0; a < n_sigma && e == cudaSuccess && s == MERBIT_OK; ++a) {
    for (int b = 0; b < n_block && e == cudaSuccess && s == MERBIT_OK; ++b) {
      merbit_plan_t p = nullptr;
      s = merbit_plan_ex(row_ptr, col_idx, n_rows, n_cols, nnz, sigmas[a], blocks[b], stream, &p);
      if (s != MERBIT_OK) break;
      for (int h = 0; h < n_hot && e == cudaSuccess && s == MERBIT_OK; ++h) {
        s = merbit_plan_set_hot_columns(p, hots[h], 0.0, stream, nullptr, nullptr);
        for (int k = 0; k < n_kernel && e == cudaSuccess && s == MERBIT_OK; ++k, ++idx) {
          merbit_plan_set_kernel(p, kernels[k]);
          float ms = -1.f;
          // a configuration the device cannot launch is skipped (ms = -1), not an error
          if (merbit_spmv_ex(p, dtype, xdt, vals, x, y, 0, stream) == MERBIT_OK) {
            e = cudaEventRecord(e0, st);
            merbit_status r = MERBIT_OK;
            for (int i = 0; i < reps && r == MERBIT_OK && e == cudaSuccess; ++i)
              r = merbit_spmv_ex(p, dtype, xdt, vals, x, y, 0, stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (r == MERBIT_OK && e == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
              ms /= (float)reps;
            else
              ms = -1.f;
          } else {
            set_last_error("");
          }
          if (ms_out) ms_out[idx] = ms;
          if (ms > 0.f && (best_ms < 0.f || ms < best_ms)) {
            best_ms = ms;
            best[0] = sigmas[a];
            best[1] = blocks[b];
            best[2] = kernels[k];
            best[3] = hots[h];
          }
        }
      }
      merbit_plan_destroy(p);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  if (s != MERBIT_OK) return s;
  if (e != cudaSuccess) {
    char msg[256];
    std::snprintf(msg, sizeof(msg), "merbit_autotune: %s", cudaGetErrorString(e));
    return afail(e == cudaErrorMemoryAllocation ? MERBIT_ENOMEM : MERBIT_ECUDA, msg);
  }
  if (best_ms < 0.f) return afail(MERBIT_ECUDA, "merbit_autotune: no candidate could be launched");
  return MERBIT_OK;
}

}  // extern "C"
