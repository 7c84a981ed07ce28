// Reduced-precision values (bf16, f16) and the f32 inner sweeps of the
// mixed-precision refinement: values widened to f32, f32 accumulation.
#include "spmv_kernel.cuh"

namespace merbit {

cudaError_t spmv_plain_lo(const merbit_plan_s* p, merbit_dtype vdt, const void* vals,
                          const float* x, float* y, float scale, cudaStream_t st) {
  EpiPlain<float, float> epi{y, scale};
  if (vdt == MERBIT_BF16)
    return launch_spmv<__nv_bfloat16, float, float>(p, static_cast<const __nv_bfloat16*>(vals), x,
                                                    epi, st);
  if (vdt == MERBIT_F16)
    return launch_spmv<__half, float, float>(p, static_cast<const __half*>(vals), x, epi, st);
  return cudaErrorInvalidValue;
}

cudaError_t spmv_sweep(const merbit_plan_s* p, merbit_dtype vdt, const void* vals,
                       const float* x, const SweepParams& prm, cudaStream_t st) {
  EpiSweep epi{};
  epi.p = prm;
  epi.xin = x;
  if (vdt == MERBIT_BF16)
    return launch_spmv<__nv_bfloat16, float, float>(p, static_cast<const __nv_bfloat16*>(vals), x,
                                                    epi, st);
  if (vdt == MERBIT_F16)
    return launch_spmv<__half, float, float>(p, static_cast<const __half*>(vals), x, epi, st);
  if (vdt == MERBIT_F32)
    return launch_spmv<float, float, float>(p, static_cast<const float*>(vals), x, epi, st);
  return cudaErrorInvalidValue;
}

}  // namespace merbit
