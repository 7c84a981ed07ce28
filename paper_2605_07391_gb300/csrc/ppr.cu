// Personalised PageRank on the batched product: k seed vertices, one column of a
// row-major n x k iterate per seed (the batching extension of the method's PageRank,
// Sec. 5.5.1 with a one-hot teleport vector per column).  One update is
//   1. the SpMM Y = alpha P^T X (one launch per column chunk, plus its finalize);
//   2. a streaming pass over Y and X: the teleport and dangling mass alpha D_c + 1 - alpha
//      added at each column's seed, and per column ||Y - X||_1 and the dangling mass of Y;
//   3. a one-block finish: D for the next update, the residuals, the stop test.
#include "spmm_kernel.cuh"

namespace merbit {

namespace {

constexpr int kStreamThreads = 256;   // per block when k <= 256 (k threads when k > 256)

// X = [e_{s_0} ... e_{s_{k-1}}] (X zeroed beforehand), D_c = 1 if s_c is dangling else 0.
__global__ void ppr_init_kernel(float* X, int64_t ldx, const int32_t* seed, int k,
                                const uint32_t* dang, double* d_cur) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < k; c += gridDim.x * blockDim.x) {
    const int s = seed[c];
    X[(size_t)s * ldx + c] = 1.f;
    d_cur[c] = is_dangling(dang, s) ? 1.0 : 0.0;
  }
}

// Step 2.  A block's threads cover rpb rows x (k / VW) column vectors of the row-major
// arrays, so a thread keeps VW columns; rows advance by gridDim.x * rpb, four rows per
// round with all their loads issued first.  Partial sums run in f32 over 16 rows and are
// then added in FP64; the block's per-column totals are summed from a per-thread slot array.
// rd[c] += ||Y_c - X_c||_1, rd[k + c] += sum over dangling r of Y[r, c].
template <int VW>
__global__ void __launch_bounds__(VW == 4 ? 256 : 1024)     // k <= 1024: k / 4 <= 256 vectors
    ppr_stream_kernel(float* __restrict__ Y, const float* __restrict__ X, int64_t n, int k,
                      const int32_t* __restrict__ seed, const double* __restrict__ d_cur,
                      const uint32_t* __restrict__ dang, float alpha, double* rd,
                      const RedState* red) {
  using V = SpmmVec<VW>;
  using VT = typename V::T;
  constexpr int R = 4;                           // rows per round
  extern __shared__ double sred[];               // [rpb * kv][VW][2] partials of the threads
  if (*reinterpret_cast<const volatile int*>(&red->done)) return;
  const int kv = k / VW;
  const int rpb = blockDim.x / kv;
  const int t = threadIdx.x;
  if (t < rpb * kv) {
    const int c = (t % kv) * VW;
    int64_t s[VW];
    float tel[VW];
    double res[VW], dm[VW];
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      s[j] = seed[c + j];
      tel[j] = alpha * static_cast<float>(d_cur[c + j]) + (1.f - alpha);
      res[j] = 0.0;
      dm[j] = 0.0;
    }
    const int64_t step = (int64_t)gridDim.x * rpb;
    int64_t r = (int64_t)blockIdx.x * rpb + t / kv;
    while (r < n) {
      float pr[VW], pd[VW];
#pragma unroll
      for (int j = 0; j < VW; ++j) pr[j] = pd[j] = 0.f;
#pragma unroll 1
      for (int q = 0; q < 16 / R && r < n; ++q, r += R * step) {
        VT yv[R], xv[R];
        bool dg[R];
#pragma unroll
        for (int u = 0; u < R; ++u) {
          const int64_t ru = r + u * step;
          yv[u] = V::zero();
          xv[u] = V::zero();
          dg[u] = false;
          if (ru < n) {
            const size_t e = (size_t)ru * k + c;
            yv[u] = V::load_plain(Y + e);
            xv[u] = V::load(X + e);
            dg[u] = is_dangling(dang, (int)ru);
          }
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
          const int64_t ru = r + u * step;
          float y[VW];
#pragma unroll
          for (int j = 0; j < VW; ++j) y[j] = V::get(yv[u], j);
          bool hit = false;
#pragma unroll
          for (int j = 0; j < VW; ++j)
            if (ru == s[j]) {
              y[j] += tel[j];
              hit = true;
            }
          if (hit) V::store(Y + (size_t)ru * k + c, y);
#pragma unroll
          for (int j = 0; j < VW; ++j) {
            pr[j] += fabsf(y[j] - V::get(xv[u], j));
            if (dg[u]) pd[j] += y[j];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < VW; ++j) {
        res[j] += pr[j];
        dm[j] += pd[j];
      }
    }
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      sred[(t * VW + j) * 2] = res[j];
      sred[(t * VW + j) * 2 + 1] = dm[j];
    }
  }
  __syncthreads();
  for (int i = t; i < 2 * k; i += blockDim.x) {
    const int part = i / k, col = i % k, cv = col / VW, j = col % VW;
    double tot = 0.0;
    for (int rho = 0; rho < rpb; ++rho) tot += sred[((rho * kv + cv) * VW + j) * 2 + part];
    atomicAdd(rd + i, tot);
  }
}

// Step 3: D for the next update, the per-column residuals, the largest residual into the
// history, the stop test, and the accumulators cleared.
__global__ void ppr_finish_kernel(double* rd, double* d_cur, double* last_r, int k, double tol,
                                  int iter, double* hist, RedState* red) {
  __shared__ double smax[256];
  if (*reinterpret_cast<const volatile int*>(&red->done)) return;
  double m = 0.0;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const double r = rd[c];
    last_r[c] = r;
    d_cur[c] = rd[k + c];
    rd[c] = 0.0;
    rd[k + c] = 0.0;
    m = fmax(m, r);
  }
  smax[threadIdx.x] = m;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    hist[iter] = smax[0];
    ++red->launches;
    if (tol > 0.0 && smax[0] < tol) {
      red->iters = iter + 1;
      red->done = 1;
    }
  }
}

}  // namespace

cudaError_t ppr_init(const merbit_plan_s* p, float* X, int64_t k, const int32_t* seed,
                     double* d_cur, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(X, 0, sizeof(float) * (size_t)p->n_rows * (size_t)k, st);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<int64_t>((k + 255) / 256, 1024);
  ppr_init_kernel<<<grid, 256, 0, st>>>(X, k, seed, (int)k, p->dangling_bits, d_cur);
  return cudaGetLastError();
}

cudaError_t ppr_update(const merbit_plan_s* p, const float* vals, const float* X, float* Y,
                       int64_t k, const int32_t* seed, double* d_cur, double* rd, double* last_r,
                       float alpha, double tol, int iter, double* hist, double* acc,
                       cudaStream_t st) {
  cudaError_t e = spmm_scaled_f32(p, vals, X, k, k, Y, k, alpha, acc, st);
  if (e != cudaSuccess) return e;
  const bool vec = k % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
  const int kv = vec ? (int)k / 4 : (int)k;                  // column vectors per row
  const int rpb = kv <= kStreamThreads ? kStreamThreads / kv : 1;
  const int threads = rpb * kv;
  const int64_t blocks_needed = (p->n_rows + rpb - 1) / rpb;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(blocks_needed, (int64_t)p->num_sms * 2));
  const size_t sm = 2 * sizeof(double) * (size_t)threads * (vec ? 4 : 1);
  if (vec)
    ppr_stream_kernel<4><<<grid, threads, sm, st>>>(Y, X, p->n_rows, (int)k, seed, d_cur,
                                                    p->dangling_bits, alpha, rd, p->red);
  else
    ppr_stream_kernel<1><<<grid, threads, sm, st>>>(Y, X, p->n_rows, (int)k, seed, d_cur,
                                                    p->dangling_bits, alpha, rd, p->red);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ppr_finish_kernel<<<1, 256, 0, st>>>(rd, d_cur, last_r, (int)k, tol, iter, hist, p->red);
  return cudaGetLastError();
}

}  // namespace merbit
