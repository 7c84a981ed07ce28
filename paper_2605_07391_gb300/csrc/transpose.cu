// Transpose of a CSR pattern on the GPU, for the backward product A^T g.
//
// A stable least-significant-digit radix sort orders the nonzeros of A by column
// (8 bits per pass, as many passes as the column indices need); stability keeps
// each column's nonzeros in row order, so the result is the row-sorted CSR of A^T
// and does not depend on thread timing.  Per pass: a per-tile digit histogram,
// one exclusive scan over (digit, tile), and a scatter that ranks equal digits
// inside a warp with __match_any_sync and across the warps of a tile through
// shared counters.  The sorted columns give A^T's row pointer; the sorted
// original positions are the permutation that carries values over.
#include <algorithm>
#include <cstdio>

#include "extensions.cuh"

namespace merbit {
void set_last_error(const char* msg);
}  // namespace merbit

using namespace merbit;

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;                        // keys per thread
constexpr int kTile = kSortThreads * kSortItems;     // keys per block
constexpr int kRadix = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kSortThreads)
    radix_hist_kernel(const int32_t* __restrict__ keys, int64_t n, int shift, int num_tiles,
                      uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile;
  for (int i = threadIdx.x; i < kTile; i += blockDim.x) {
    const int64_t e = base + i;
    if (e < n) atomicAdd(&cnt[(keys[e] >> shift) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
    hist[(size_t)d * num_tiles + blockIdx.x] = cnt[d];
}

// Exclusive scan of a block of kScanTile values in place; returns the block total.
__device__ uint32_t block_exclusive_scan(uint32_t (&v)[kScanItems], uint32_t* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t t = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint32_t x = v[i];
    v[i] = t;
    t += x;
  }
  uint32_t inc = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;        // exclusive warp offsets
    if (lane == 31) warp_tot[kScanThreads / 32] = wi;             // block total
  }
  __syncthreads();
  const uint32_t off = warp_tot[warp] + inc - t;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) v[i] += off;
  const uint32_t total = warp_tot[kScanThreads / 32];
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(kScanThreads)
    scan_tiles_kernel(uint32_t* a, int64_t n, uint32_t* tile_sums) {
  __shared__ uint32_t warp_tot[kScanThreads / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) v[i] = base + i < n ? a[base + i] : 0u;
  const uint32_t total = block_exclusive_scan(v, warp_tot);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) a[base + i] = v[i];
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// One block: exclusive scan of the tile sums in chunks of kScanTile, carrying the total.
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(uint32_t* s, int64_t n) {
  __shared__ uint32_t warp_tot[kScanThreads / 32 + 1];
  uint32_t carry = 0;
  for (int64_t c0 = 0; c0 < n; c0 += kScanTile) {
    const int64_t base = c0 + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) v[i] = base + i < n ? s[base + i] : 0u;
    const uint32_t total = block_exclusive_scan(v, warp_tot);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
      if (base + i < n) s[base + i] = v[i] + carry;
    carry += total;
  }
}

__global__ void __launch_bounds__(kScanThreads)
    scan_add_kernel(uint32_t* a, int64_t n, const uint32_t* tile_sums) {
  const uint32_t off = tile_sums[blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x)
    if (base + i < n) a[base + i] += off;
}

__global__ void __launch_bounds__(kSortThreads)
    radix_scatter_kernel(const int32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
                         int32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out, int64_t n,
                         int shift, int num_tiles, const uint32_t* __restrict__ offs) {
  __shared__ uint32_t wcnt[kSortWarps][kRadix];
  __shared__ uint32_t base[kRadix];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kSortWarps * kRadix; i += blockDim.x) wcnt[i / kRadix][i % kRadix] = 0;
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t wbase = (int64_t)blockIdx.x * kTile + (int64_t)warp * (32 * kSortItems);
  int32_t key[kSortItems], val[kSortItems];
  uint32_t rank[kSortItems];
  int dig[kSortItems];
  // ranks inside the warp, in key order: item it of lane l is key wbase + 32 it + l
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const int64_t e = wbase + it * 32 + lane;
    const bool ok = e < n;
    key[it] = ok ? keys_in[e] : 0;
    val[it] = ok ? (vals_in ? vals_in[e] : (int32_t)e) : 0;
    const int d = ok ? (key[it] >> shift) & (kRadix - 1) : kRadix;
    dig[it] = d;
    const uint32_t m = __match_any_sync(0xffffffffu, d);
    rank[it] = ok ? wcnt[warp][d] + __popc(m & lt) : 0u;
    __syncwarp();
    if (ok && (m & lt) == 0) wcnt[warp][d] += __popc(m);    // the group's lowest lane
    __syncwarp();
  }
  __syncthreads();
  // warps in order: exclusive offsets per digit; the tile's offset per digit from the scan
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
    uint32_t run = 0;
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t t = wcnt[w][d];
      wcnt[w][d] = run;
      run += t;
    }
    base[d] = offs[(size_t)d * num_tiles + blockIdx.x];
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const int64_t e = wbase + it * 32 + lane;
    if (e < n) {
      const int d = dig[it];
      const uint32_t pos = base[d] + wcnt[warp][d] + rank[it];
      keys_out[pos] = key[it];
      vals_out[pos] = val[it];
    }
  }
}

// row_ptr_t[c] = first position of column c in the sorted column list, c in [0, n_cols].
__global__ void boundaries_kernel(const int32_t* __restrict__ sorted, int64_t nnz, int64_t n_cols,
                                  int32_t* __restrict__ row_ptr_t) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= nnz;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cur = p < nnz ? sorted[p] : n_cols;
    const int64_t prev = p > 0 ? sorted[p - 1] : -1;
    for (int64_t c = prev + 1; c <= cur; ++c) row_ptr_t[c] = (int32_t)p;
  }
}

// row_of[k] = row of nonzero k (one warp per row)
__global__ void expand_rows_kernel(const int32_t* __restrict__ row_ptr, int64_t n_rows,
                                   int32_t* __restrict__ row_of) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows; r += warps)
    for (int64_t k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) row_of[k] = (int32_t)r;
}

template <typename T>
__global__ void gather_kernel(const T* __restrict__ src, const int32_t* __restrict__ idx,
                              T* __restrict__ dst, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

int grid_of(int64_t work, int threads) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads,
                                                     (int64_t)sm_count() * 16));
}

// Exclusive scan of a[0, n) in place (n < 2^31, values summing below 2^32).
cudaError_t exclusive_scan(uint32_t* a, int64_t n, uint32_t* tile_sums, cudaStream_t st) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  scan_tiles_kernel<<<(unsigned)tiles, kScanThreads, 0, st>>>(a, n, tile_sums);
  scan_sums_kernel<<<1, kScanThreads, 0, st>>>(tile_sums, tiles);
  scan_add_kernel<<<(unsigned)tiles, kScanThreads, 0, st>>>(a, n, tile_sums);
  return cudaGetLastError();
}

cudaError_t build_transpose(merbit_transpose_s* t, const int32_t* row_ptr, const int32_t* col,
                            cudaStream_t st) {
  const int64_t nnz = t->nnz;
  int bits = 0;
  while (bits < 31 && ((int64_t)1 << bits) < t->n_cols) ++bits;
  const int passes = std::max(1, (bits + 7) / 8);
  const int64_t num_tiles = std::max<int64_t>(1, (nnz + kTile - 1) / kTile);
  const int64_t hist_n = (int64_t)kRadix * num_tiles;
  const int64_t scan_tiles = (hist_n + kScanTile - 1) / kScanTile;
  int32_t *kb[2] = {nullptr, nullptr}, *vb[2] = {nullptr, nullptr}, *row_of = nullptr;
  uint32_t *hist = nullptr, *sums = nullptr;
  const size_t nb = sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t b) { if (e == cudaSuccess) e = cudaMalloc(p, b); };
  A((void**)&kb[0], nb); A((void**)&kb[1], nb); A((void**)&vb[0], nb); A((void**)&vb[1], nb);
  A((void**)&row_of, nb);
  A((void**)&hist, sizeof(uint32_t) * (size_t)hist_n);
  A((void**)&sums, sizeof(uint32_t) * (size_t)std::max<int64_t>(scan_tiles, 1));
  if (e == cudaSuccess && nnz > 0) {
    const int32_t* kin = col;
    const int32_t* vin = nullptr;              // first pass: values are the positions
    for (int pass = 0; pass < passes && e == cudaSuccess; ++pass) {
      const int out = pass & 1;
      radix_hist_kernel<<<(unsigned)num_tiles, kSortThreads, 0, st>>>(kin, nnz, 8 * pass,
                                                                     (int)num_tiles, hist);
      e = exclusive_scan(hist, hist_n, sums, st);
      if (e != cudaSuccess) break;
      radix_scatter_kernel<<<(unsigned)num_tiles, kSortThreads, 0, st>>>(
          kin, vin, kb[out], vb[out], nnz, 8 * pass, (int)num_tiles, hist);
      e = cudaGetLastError();
      kin = kb[out];
      vin = vb[out];
    }
    if (e == cudaSuccess) {
      const int last = (passes - 1) & 1;
      boundaries_kernel<<<grid_of(nnz + 1, 256), 256, 0, st>>>(kb[last], nnz, t->n_cols,
                                                              t->row_ptr_t);
      expand_rows_kernel<<<grid_of(t->n_rows * 32, 256), 256, 0, st>>>(row_ptr, t->n_rows, row_of);
      gather_kernel<int32_t><<<grid_of(nnz, 256), 256, 0, st>>>(row_of, vb[last], t->col_t, nnz);
      e = cudaMemcpyAsync(t->perm, vb[last], sizeof(int32_t) * (size_t)nnz,
                          cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess) e = cudaGetLastError();
    }
  } else if (e == cudaSuccess) {
    e = cudaMemsetAsync(t->row_ptr_t, 0, sizeof(int32_t) * (size_t)(t->n_cols + 1), st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(kb[0]); cudaFree(kb[1]); cudaFree(vb[0]); cudaFree(vb[1]); cudaFree(row_of);
  cudaFree(hist); cudaFree(sums);
  return e;
}

void free_transpose(merbit_transpose_s* t) {
  if (!t) return;
  cudaFree(t->row_ptr_t);
  cudaFree(t->col_t);
  cudaFree(t->perm);
  delete t;
}

merbit_status tfail(merbit_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

}  // namespace

namespace merbit {

cudaError_t gather(const void* src, const int32_t* idx, void* dst, int64_t count, size_t elem,
                   cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  if (elem == 8)
    gather_kernel<double><<<grid_of(count, 256), 256, 0, st>>>(
        static_cast<const double*>(src), idx, static_cast<double*>(dst), count);
  else
    gather_kernel<float><<<grid_of(count, 256), 256, 0, st>>>(
        static_cast<const float*>(src), idx, static_cast<float*>(dst), count);
  return cudaGetLastError();
}

}  // namespace merbit

extern "C" {

merbit_status merbit_transpose(const int32_t* row_ptr, const int32_t* col_idx, int64_t n_rows,
                               int64_t n_cols, int64_t nnz, void* stream, merbit_transpose_t* out) {
  set_last_error("");
  if (!out) return tfail(MERBIT_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_rows < 0 || n_cols < 0 || nnz < 0) return tfail(MERBIT_EINVAL, "negative size");
  if (!row_ptr || (nnz > 0 && !col_idx)) return tfail(MERBIT_EINVAL, "row_ptr or col_idx is NULL");
  if (n_rows >= INT32_MAX || n_cols >= INT32_MAX || nnz >= INT32_MAX)
    return tfail(MERBIT_EOVERFLOW, "sizes must fit int32");
  if ((int64_t)kRadix * ((nnz + kTile - 1) / kTile) >= ((int64_t)1 << 31))
    return tfail(MERBIT_EOVERFLOW, "too many nonzeros for the radix histogram");
  auto* t = new merbit_transpose_s();
  t->n_rows = n_rows;
  t->n_cols = n_cols;
  t->nnz = nnz;
  cudaGetDevice(&t->device);
  cudaError_t e = cudaMalloc(&t->row_ptr_t, sizeof(int32_t) * (size_t)(n_cols + 1));
  if (e == cudaSuccess) e = cudaMalloc(&t->col_t, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1));
  if (e == cudaSuccess) e = cudaMalloc(&t->perm, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1));
  if (e == cudaSuccess) e = build_transpose(t, row_ptr, col_idx, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    free_transpose(t);
    char msg[256];
    std::snprintf(msg, sizeof(msg), "merbit_transpose: %s", cudaGetErrorString(e));
    return tfail(e == cudaErrorMemoryAllocation ? MERBIT_ENOMEM : MERBIT_ECUDA, msg);
  }
  *out = t;
  return MERBIT_OK;
}

merbit_status merbit_transpose_get(merbit_transpose_t t, const int32_t** row_ptr_t,
                                   const int32_t** col_t, const int32_t** perm) {
  set_last_error("");
  if (!t) return tfail(MERBIT_EINVAL, "transpose is NULL");
  if (row_ptr_t) *row_ptr_t = t->row_ptr_t;
  if (col_t) *col_t = t->col_t;
  if (perm) *perm = t->perm;
  return MERBIT_OK;
}

void merbit_transpose_destroy(merbit_transpose_t t) { free_transpose(t); }

merbit_status merbit_gather(merbit_dtype dtype, const void* src, const int32_t* idx, void* dst,
                            int64_t count, void* stream) {
  set_last_error("");
  if (count < 0) return tfail(MERBIT_EINVAL, "negative count");
  if (count > 0 && (!src || !idx || !dst)) return tfail(MERBIT_EINVAL, "NULL pointer");
  if (dtype != MERBIT_F32 && dtype != MERBIT_F64) return tfail(MERBIT_EINVAL, "dtype must be F32 or F64");
  cudaError_t e = gather(src, idx, dst, count, dtype == MERBIT_F64 ? 8 : 4,
                         static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return tfail(MERBIT_ECUDA, cudaGetErrorString(e));
  return MERBIT_OK;
}

}  // extern "C"
