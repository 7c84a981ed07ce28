// Declarations shared by the extension translation units (transpose, differentiation).
#pragma once

#include "merbit_internal.cuh"

struct merbit_transpose_s {
  int device = 0;
  int64_t n_rows = 0, n_cols = 0, nnz = 0;   // of the source matrix A
  int32_t* row_ptr_t = nullptr;              // n_cols + 1: row pointer of A^T
  int32_t* col_t = nullptr;                  // nnz: column indices of A^T (= rows of A)
  int32_t* perm = nullptr;                   // nnz: A^T's k-th nonzero is A's nonzero perm[k]
};

namespace merbit {

// Adjoint of the PageRank fixed point, lambda' = alpha A^T lambda + alpha (S / n) d + w with
// S = sum(lambda) and d the dangling indicator, run on a plan of A^T.
struct AdjParams {
  void* out;                    // T[n]: lambda_{k+1}
  const void* w;                // T[n]: dL/dpi
  const uint32_t* dang;         // dangling bits of the original graph
  double alpha, inv_n, tol;     // stop when ||lambda_{k+1} - lambda_k||_1 <= tol * (*wnorm)
  const double* wnorm;          // ||w||_1
  const double* s_in;           // S_k = sum(lambda_k)
  double* s_out;                // [0] = ||lambda_{k+1} - lambda_k||_1, [1] = S_{k+1}
  int iter;
};

cudaError_t spmv_adj_f32(const merbit_plan_s* p, const float* vals, const float* x,
                         const AdjParams& prm, cudaStream_t st);
cudaError_t spmv_adj_f64(const merbit_plan_s* p, const double* vals, const double* x,
                         const AdjParams& prm, cudaStream_t st);

// out[k] = scale * g[row(k)] * x[col(k)] for every nonzero k of the plan's matrix
cudaError_t sddmm(const merbit_plan_s* p, merbit_dtype dt, const void* g, const void* x,
                  double scale, void* out, cudaStream_t st);

// *out = sum of x[0, n) (or of |x|) in FP64 (f32 or f64 elements)
cudaError_t vec_sum(const void* x, merbit_dtype dt, int64_t n, double* out, bool absolute,
                    int num_sms, cudaStream_t st);

// dst[i] = src[idx[i]], i < count (4- or 8-byte elements)
cudaError_t gather(const void* src, const int32_t* idx, void* dst, int64_t count, size_t elem,
                   cudaStream_t st);

}  // namespace merbit
