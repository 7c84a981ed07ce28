// merbit_gather_probe: the x gather of the SpMV alone, as a measured floor.
//
// The SpMV's cost on graph matrices is dominated by the random gathers x[col[k]]
// (Sec. 4.2's products val * x[col]).  This kernel does nothing else: it streams
// the column array the plan's products stream (the plain one, or the hot-tagged
// one when the product launch uses the hot-column table), gathers x or the
// table entry for every nonzero and sums what it loads, with the grid, block
// size and dynamic shared memory of the split SpMV kernel's launch.  Reserving
// the same shared memory leaves L1 the same capacity, so its time is the cost of
// the gathers at the kernel's footprint.  A measurement aid: no counterpart in
// the paper.
#include "spmv_kernel.cuh"

namespace merbit {
void set_last_error(const char* msg);
}  // namespace merbit

using namespace merbit;

namespace {

template <typename XT>
__global__ void __launch_bounds__(kSplitThreads, 2)
    gather_probe_kernel(const Geometry g, const XT* __restrict__ x, XT* __restrict__ sink) {
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  XT* tab = reinterpret_cast<XT*>(dyn_smem);
  const uint64_t pol_x = policy_evict_last();
  const uint64_t pol_stream = policy_evict_first();
  if (g.hot_n > 0) {
    fill_hot(g, x, tab, pol_x);
    __syncthreads();
  }
  constexpr int U = 8;   // gathers in flight per thread
  const bool hot = g.hot_n > 0;
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  XT acc = XT(0);
  for (int64_t base = 0; base < g.nnz; base += T * U) {
    XT v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t k = base + t0 + (int64_t)u * T;
      v[u] = XT(0);
      if (k < g.nnz) {
        const int c = (int)ld_stream(reinterpret_cast<const uint32_t*>(g.col_stage) + k, pol_stream);
        v[u] = hot ? gather_x<true>(c, x, tab, pol_x) : gather_x<false>(c, x, tab, pol_x);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) acc += v[u];
  }
  acc = warp_sum(acc);
  __shared__ XT part[kSplitThreads / 32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    XT s = XT(0);
    for (int w = 0; w < kSplitThreads / 32; ++w) s += part[w];
    sink[blockIdx.x] = s;
  }
}

template <typename XT>
cudaError_t launch_probe(const merbit_plan_s* p, const XT* x, XT* sink, cudaStream_t st) {
  // the split SpMV kernel's launch for these types: its grid, its stages' shared memory
  // and, if that launch takes it, the hot-column table
  Geometry g = p->geom();
  int grid = 0;
  size_t smem = 0;
  const bool ok = sizeof(XT) == 4 ? split_config_f32(p, g, grid, smem) : split_config_f64(p, g, grid, smem);
  if (!ok) return cudaErrorInvalidConfiguration;
  auto kern = gather_probe_kernel<XT>;
  const void* kp = reinterpret_cast<const void*>(kern);
  // the probe needs fewer registers than the split kernel, so more of its CTAs could fit
  // and the driver would pick a larger shared-memory carveout (a smaller L1) for it; ask
  // for the carveout that the split kernel's resident CTAs need instead
  int dev = 0, per_sm_total = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm_total, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int per_sm = std::max(1, grid / p->num_sms);
  if (per_sm_total > 0) {
    const size_t need = (size_t)per_sm * (smem + (size_t)reserved + 1024);
    const int pct = (int)std::min<size_t>(100, (need * 100 + per_sm_total - 1) / (size_t)per_sm_total);
    if (cudaFuncSetAttribute(kp, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess)
      cudaGetLastError();   // a hint only
  }
  const int pgrid = persistent_grid(kp, kSplitThreads, smem, smem, p->num_sms);
  if (pgrid <= 0) return cudaErrorInvalidConfiguration;
  grid = std::min(grid, pgrid);
  kern<<<grid, kSplitThreads, smem, st>>>(g, x, sink);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

merbit_status merbit_gather_probe(merbit_plan_t p, merbit_dtype xdt, const void* x, void* sink,
                                  void* stream) {
  set_last_error("");
  if (!p) {
    set_last_error("plan is NULL");
    return MERBIT_EINVAL;
  }
  if (p->nnz > 0 && (!x || !sink)) {
    set_last_error("x or sink is NULL");
    return MERBIT_EINVAL;
  }
  if (p->nnz == 0) return MERBIT_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (xdt == MERBIT_F32)
    e = launch_probe<float>(p, static_cast<const float*>(x), static_cast<float*>(sink), st);
  else if (xdt == MERBIT_F64)
    e = launch_probe<double>(p, static_cast<const double*>(x), static_cast<double*>(sink), st);
  else {
    set_last_error("merbit_gather_probe: x must be F32 or F64");
    return MERBIT_EINVAL;
  }
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return MERBIT_ECUDA;
  }
  return MERBIT_OK;
}

}  // extern "C"
