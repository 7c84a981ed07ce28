// Kernels of the differentiation extension.
//
// * EpiAdjoint: the transposed PageRank fixed point.  With M = A + (1/n) 1 d^T the
//   PageRank operator (A = P^T, d the dangling indicator), pi = alpha M pi + (1-alpha)/n 1,
//   and a loss L(pi), the adjoint lambda of (I - alpha M)^T lambda = dL/dpi is the fixed
//   point of lambda' = alpha A^T lambda + alpha (sum(lambda) / n) d + dL/dpi, iterated here
//   by SpMVs on a plan of A^T (the rows of A^T that are empty are exactly the dangling
//   vertices, so every row is written).  dL/dA_ij = alpha lambda_i pi_j.
// * sddmm: out[k] = scale * g[row(k)] * x[col(k)] for every nonzero, walking the
//   plan's lanes (Sec. 4.1.1 descriptors): the value gradient of y = A x is g[row] x[col].
#include "extensions.cuh"
#include "spmv_kernel.cuh"

namespace merbit {

namespace {

template <typename T>
struct EpiAdjoint {
  static constexpr bool kReduce = true;
  AdjParams p;
  const T* xold;
  T a, c;
  __device__ __forceinline__ void init() {
    a = static_cast<T>(p.alpha);
    c = static_cast<T>(p.alpha * (*p.s_in) * p.inv_n);
  }
  __device__ __forceinline__ bool skip(const RedState* red) const {
    return *reinterpret_cast<const volatile int*>(&red->done) != 0;
  }
  __device__ __forceinline__ void put(int r, T v, double& p0, double& p1) const {
    if (is_dangling(p.dang, r)) v += c;
    static_cast<T*>(p.out)[r] = v;
    p0 += fabs(static_cast<double>(v) - static_cast<double>(xold[r]));
    p1 += static_cast<double>(v);
  }
  __device__ __forceinline__ void row(int r, T s, double& p0, double& p1) const {
    put(r, a * s + static_cast<const T*>(p.w)[r], p0, p1);
  }
  __device__ __forceinline__ void row64(int r, double s, double& p0, double& p1) const {
    put(r, static_cast<T>(p.alpha * s + static_cast<double>(static_cast<const T*>(p.w)[r])), p0, p1);
  }
  __device__ __forceinline__ void finish(double A, double B, RedState* red) const {
    p.s_out[0] = A;
    p.s_out[1] = B;
    ++red->launches;
    if (p.tol > 0.0 && A <= p.tol * (*p.wnorm)) {
      red->iters = p.iter + 1;
      red->done = 1;
    }
  }
};

// One thread per lane: walk its sigma steps; a right step is a nonzero of the current row.
template <typename T>
__global__ void __launch_bounds__(256)
    sddmm_kernel(const Geometry g, const T* __restrict__ gv, const T* __restrict__ x, T scale,
                 T* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < g.lane_num; j += stride) {
    const int ti = (int)(j / kOmega);
    const LaneDesc d = decode_lane(g, load_desc(g, j));
    int xk = (int)__ldg(g.tile_x + ti) + d.xo;
    int row = (int)(__ldg(g.tile_y + ti) & ~kMsb) + d.yo;
    const int64_t left = (int64_t)g.steps - j * g.sigma;
    const int len = left < g.sigma ? (int)left : g.sigma;
    T gr = row < g.n_rows ? scale * gv[row] : T(0);
    for (int k = 0; k < len; ++k) {
      if ((d.flags >> k) & 1u) {
        ++row;
        gr = row < g.n_rows ? scale * gv[row] : T(0);
      } else {
        out[xk] = gr * x[__ldg(g.col + xk)];
        ++xk;
      }
    }
  }
}

template <typename T, bool ABS>
__global__ void vec_sum_kernel(const T* __restrict__ x, int64_t n, double* out) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += ABS ? fabs(static_cast<double>(x[i])) : static_cast<double>(x[i]);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

}  // namespace

cudaError_t spmv_adj_f32(const merbit_plan_s* p, const float* vals, const float* x,
                         const AdjParams& prm, cudaStream_t st) {
  EpiAdjoint<float> epi{};
  epi.p = prm;
  epi.xold = x;
  return launch_spmv<float, float, float>(p, vals, x, epi, st);
}

cudaError_t spmv_adj_f64(const merbit_plan_s* p, const double* vals, const double* x,
                         const AdjParams& prm, cudaStream_t st) {
  EpiAdjoint<double> epi{};
  epi.p = prm;
  epi.xold = x;
  return launch_spmv<double, double, double>(p, vals, x, epi, st);
}

cudaError_t sddmm(const merbit_plan_s* p, merbit_dtype dt, const void* g, const void* x,
                  double scale, void* out, cudaStream_t st) {
  if (p->lane_num == 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((p->lane_num + 255) / 256, (int64_t)p->num_sms * 16);
  if (dt == MERBIT_F64)
    sddmm_kernel<double><<<grid, 256, 0, st>>>(p->geom(), static_cast<const double*>(g),
                                               static_cast<const double*>(x), scale,
                                               static_cast<double*>(out));
  else
    sddmm_kernel<float><<<grid, 256, 0, st>>>(p->geom(), static_cast<const float*>(g),
                                              static_cast<const float*>(x),
                                              static_cast<float>(scale), static_cast<float*>(out));
  return cudaGetLastError();
}

cudaError_t vec_sum(const void* x, merbit_dtype dt, int64_t n, double* out, bool absolute,
                    int num_sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
  if (e != cudaSuccess || n == 0) return e;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8);
  const double* xd = static_cast<const double*>(x);
  const float* xf = static_cast<const float*>(x);
  if (dt == MERBIT_F64 && absolute) vec_sum_kernel<double, true><<<grid, 256, 0, st>>>(xd, n, out);
  else if (dt == MERBIT_F64) vec_sum_kernel<double, false><<<grid, 256, 0, st>>>(xd, n, out);
  else if (absolute) vec_sum_kernel<float, true><<<grid, 256, 0, st>>>(xf, n, out);
  else vec_sum_kernel<float, false><<<grid, 256, 0, st>>>(xf, n, out);
  return cudaGetLastError();
}

}  // namespace merbit
