// f32 values, f32 vectors: plain SpMV and the fused PageRank update.
#include "spmv_kernel.cuh"

namespace merbit {

cudaError_t spmv_plain_f32(const merbit_plan_s* p, const float* vals, const float* x, float* y,
                           cudaStream_t st) {
  EpiPlain<float, float> epi{y, 1.0f};
  return launch_spmv<float, float, float>(p, vals, x, epi, st);
}

cudaError_t spmv_pr_f32(const merbit_plan_s* p, const float* vals, const float* x,
                        const PRParams& prm, cudaStream_t st) {
  EpiPageRank<float> epi{};
  epi.p = prm;
  epi.xold = x;
  return launch_spmv<float, float, float>(p, vals, x, epi, st);
}

bool split_config_f32(const merbit_plan_s* p, Geometry& g, int& grid, size_t& smem) {
  // the launch the product itself makes (the automatic choice may take a two-stage ring);
  // when the product would fall back to the classic kernel, the split kernel's own launch
  const Geometry g0 = g;
  const int kind = p->spmv_kernel;
  if (kind != MERBIT_KERNEL_CLASSIC &&
      split_config<float, float, float, EpiPlain<float, float>>(p, g, grid, smem, kind != MERBIT_KERNEL_AUTO))
    return true;
  g = g0;
  return split_config<float, float, float, EpiPlain<float, float>>(p, g, grid, smem, true);
}

}  // namespace merbit
