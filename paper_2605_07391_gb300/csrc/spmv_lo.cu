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

// pi += delta in FP64, delta the refinement's latest inner iterate (recorded on
// the device by the residual / sweep launches); s_out = (||delta||_1, dangling mass of pi).
__global__ void __launch_bounds__(256) ir_apply_kernel(double* __restrict__ pi, int n,
                                                       const uint32_t* __restrict__ dang,
                                                       RedState* red, double* s_out) {
  if (*reinterpret_cast<const volatile int*>(&red->done)) return;
  // the latest inner iterate is published by the finishing pass of the residual or sweep
  // launches; after a kernel gave up (error bit set) it may never have been published
  if (*reinterpret_cast<const volatile int*>(&red->err)) return;
  const float* delta = *reinterpret_cast<const float* const volatile*>(&red->delta);
  if (delta == nullptr) return;
  double p0 = 0.0, p1 = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double d = static_cast<double>(delta[i]);
    const double v = pi[i] + d;
    pi[i] = v;
    p0 += fabs(d);
    if (is_dangling(dang, i)) p1 += v;
  }
  grid_sum2(p0, p1, red, [&](double A, double B) {
    s_out[0] = A;
    s_out[1] = B;
    red->inner_done = 0;
  });
}

cudaError_t ir_apply(const merbit_plan_s* p, double* pi, double* s_out, cudaStream_t st) {
  const int n = (int)p->n_rows;
  const int grid = std::max(1, std::min((n + 255) / 256, p->num_sms * 8));
  ir_apply_kernel<<<grid, 256, 0, st>>>(pi, n, p->dangling_bits, p->red, s_out);
  return cudaGetLastError();
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
