// f64 values, f64 vectors: plain SpMV, fused PageRank update, and the FP64
// residual of the mixed-precision refinement.
#include "spmv_kernel.cuh"

namespace merbit {

cudaError_t spmv_plain_f64(const merbit_plan_s* p, const double* vals, const double* x,
                           double* y, cudaStream_t st) {
  EpiPlain<double, double> epi{y, 1.0};
  return launch_spmv<double, double, double>(p, vals, x, epi, st);
}

cudaError_t spmv_pr_f64(const merbit_plan_s* p, const double* vals, const double* x,
                        const PRParams& prm, cudaStream_t st) {
  EpiPageRank<double> epi{};
  epi.p = prm;
  epi.xold = x;
  return launch_spmv<double, double, double>(p, vals, x, epi, st);
}

cudaError_t spmv_resid_f64(const merbit_plan_s* p, const double* vals, const double* pi,
                           const ResidParams& prm, cudaStream_t st) {
  EpiResid epi{};
  epi.p = prm;
  epi.pi = pi;
  return launch_spmv<double, double, double>(p, vals, pi, epi, st);
}

bool split_config_f64(const merbit_plan_s* p, Geometry& g, int& grid, size_t& smem) {
  // the launch the product itself makes (the automatic choice may take a two-stage ring);
  // when the product would fall back to the classic kernel, the split kernel's own launch
  const Geometry g0 = g;
  const int kind = p->spmv_kernel;
  if (kind != MERBIT_KERNEL_CLASSIC &&
      split_config<double, double, double, EpiPlain<double, double>>(p, g, grid, smem, kind != MERBIT_KERNEL_AUTO))
    return true;
  g = g0;
  return split_config<double, double, double, EpiPlain<double, double>>(p, g, grid, smem, true);
}

}  // namespace merbit
