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
  return split_config<double, double, double, EpiPlain<double, double>>(p, g, grid, smem, true);
}

}  // namespace merbit
