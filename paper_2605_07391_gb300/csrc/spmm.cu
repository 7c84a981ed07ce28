// Host side of the batched product Y = scale * A X (row-major X and Y, f32): column
// chunks of 32, 16, 8 or 4 through merbit_spmm_kernel.  A thread's row slice is 4 columns
// (16 bytes) when every slice is 16-byte aligned, 8 columns (one 32-byte load) in chunks
// of 16 and 32 when k and ldx are multiples of 8 and X is 32-byte aligned, and one column
// otherwise.  R-MAT scale 22: 8-column slices took k = 16 from 0.707 to 0.599 ms and
// k = 32 from 1.222 to 1.003 ms, but k = 8 (one lane per thread, a whole tile per pass)
// from 0.456 to 0.490 ms, so 8-column chunks keep 4-column slices.
#include "spmm_kernel.cuh"

namespace merbit {

namespace {

// VW: slice width of 8-column chunks, VWW: of 16- and 32-column chunks
template <int VW, int VWW>
cudaError_t spmm_chunks(const merbit_plan_s* p, const float* vals, const float* X, int64_t k,
                        int64_t ldx, float* Y, int64_t ldy, float scale, bool gated, double* acc,
                        cudaStream_t st) {
  for (int64_t c0 = 0; c0 < k;) {
    const int64_t left = k - c0;
    const int kc = left >= 32 ? 32 : left > 8 ? 16 : left > 4 ? 8 : 4;
    SpmmGeometry sg{acc, (int)std::min<int64_t>(left, kc)};
    EpiSpmmPlain epi{Y + c0, (int)ldy, scale, gated};
    cudaError_t e;
    if (kc == 32) e = launch_spmm<32, VWW>(p, vals, X + c0, (int)ldx, sg, epi, st);
    else if (kc == 16) e = launch_spmm<16, VWW>(p, vals, X + c0, (int)ldx, sg, epi, st);
    else if (kc == 8) e = launch_spmm<8, VW>(p, vals, X + c0, (int)ldx, sg, epi, st);
    else e = launch_spmm<4, VW>(p, vals, X + c0, (int)ldx, sg, epi, st);
    if (e != cudaSuccess) return e;
    c0 += sg.kc;
  }
  return cudaSuccess;
}

cudaError_t spmm_dispatch(const merbit_plan_s* p, const float* vals, const float* X, int64_t k,
                          int64_t ldx, float* Y, int64_t ldy, float scale, bool gated, double* acc,
                          cudaStream_t st) {
  const bool vec = k % 4 == 0 && ldx % 4 == 0 && ldy % 4 == 0 &&
                   (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
  if (!vec) return spmm_chunks<1, 1>(p, vals, X, k, ldx, Y, ldy, scale, gated, acc, st);
  // 8-column slices are read by one 32-byte load, which needs 32-byte alignment
  const bool v8 = k % 8 == 0 && ldx % 8 == 0 && (reinterpret_cast<uintptr_t>(X) & 31) == 0;
  return v8 ? spmm_chunks<4, 8>(p, vals, X, k, ldx, Y, ldy, scale, gated, acc, st)
                    : spmm_chunks<4, 4>(p, vals, X, k, ldx, Y, ldy, scale, gated, acc, st);
}

}  // namespace

cudaError_t spmm_plain_f32(const merbit_plan_s* p, const float* vals, const float* X, int64_t k,
                           int64_t ldx, float* Y, int64_t ldy, double* acc, cudaStream_t st) {
  return spmm_dispatch(p, vals, X, k, ldx, Y, ldy, 1.f, false, acc, st);
}

cudaError_t spmm_scaled_f32(const merbit_plan_s* p, const float* vals, const float* X, int64_t k,
                            int64_t ldx, float* Y, int64_t ldy, float scale, double* acc,
                            cudaStream_t st) {
  return spmm_dispatch(p, vals, X, k, ldx, Y, ldy, scale, true, acc, st);
}

}  // namespace merbit
