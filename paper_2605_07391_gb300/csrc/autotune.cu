// Autotuner of the plan's segment length sigma (Sec. 4.1.1: the steps per lane, chosen
// by the paper per value type from a measured sweep).  For a given matrix and value
// type it builds a plan per candidate sigma, times the SpMV with CUDA events on the
// caller's stream (after a warm-up call) and reports the fastest.  The block size (tiles
// per block) is fixed by the kernels' 256-thread CTA and is not searched.
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

}  // extern "C"
