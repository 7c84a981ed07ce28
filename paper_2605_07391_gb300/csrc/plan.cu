// Plan construction (Sec. 4.1.2, Algorithm generate_tile) and the block
// boundary data used by the SpMV commit.
#include <map>
#include <mutex>
#include <tuple>

#include "merbit_internal.cuh"

namespace merbit {

// Number of down steps among the first d steps of the merge path, i.e. the row
// of the path coordinate on diagonal d (Sec. 3.3, Algorithm merge_search).
// Row y's down step is step row_ptr[y+1] + y, so the answer is the smallest y
// with row_ptr[y+1] + y >= d (or n_rows).  The search is confined to
// [max(d - nnz, 0), min(d, n_rows)] because x = d - y lies in [0, nnz].
__device__ __forceinline__ int rows_before(const int32_t* __restrict__ row_ptr, int n_rows,
                                           int nnz, int d) {
  int lo = max(d - nnz, 0);
  int hi = min(d, n_rows);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(row_ptr + mid + 1) + mid < d)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// One thread per lane j: start coordinate on diagonal j*sigma, sigma-step walk
// into bit_flag, descriptor packing; lane 0 of each warp (= tile) writes the
// tile start, with the MSB set when no lane of the tile takes a down step.
// DT: the descriptor word (uint32_t: offsets of W_ = 9 bits, sigma <= 14; unsigned long long:
// W_ = 11 bits, sigma <= 42).
template <typename DT, int W_>
__global__ void plan_tiles_kernel(const int32_t* __restrict__ row_ptr, int n_rows, int nnz,
                                  int sigma, int lane_num, int tile_num,
                                  uint32_t* __restrict__ tile_x, uint32_t* __restrict__ tile_y,
                                  DT* __restrict__ lane_desc) {
  const int64_t j64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool active = j64 < lane_num;
  const int j = (int)(j64 < (int64_t)lane_num ? j64 : (int64_t)lane_num);
  const int steps = nnz + n_rows;
  int cx = 0, cy = 0;
  if (active) {
    const int d = j * sigma;
    cy = rows_before(row_ptr, n_rows, nnz, d);
    cx = d - cy;
  }
  const int tx = __shfl_sync(0xffffffffu, cx, 0);
  const int ty = __shfl_sync(0xffffffffu, cy, 0);
  int end_y = ty;
  if (active) {
    const int len = min(sigma, steps - j * sigma);
    int x = cx, y = cy;
    int row_end = y < n_rows ? __ldg(row_ptr + y + 1) : nnz;
    DT flags = 0;
    for (int k = 0; k < len; ++k) {
      if (x < row_end) {
        ++x;                       // right step: next nonzero of row y
      } else {
        flags |= DT(1) << k;       // down step: row y is complete
        ++y;
        row_end = y < n_rows ? __ldg(row_ptr + y + 1) : nnz;
      }
    }
    lane_desc[j] = (flags << (2 * W_)) | ((DT)(cy - ty) << W_) | (DT)(cx - tx);
    end_y = y;
  }
  const bool single_row = __all_sync(0xffffffffu, end_y == ty);
  if (active && lane == 0) {
    const int i = j / kOmega;
    tile_x[i] = (uint32_t)tx;
    tile_y[i] = (uint32_t)ty | (single_row ? kMsb : 0u);
  }
  if (j64 == lane_num) {
    tile_x[tile_num] = (uint32_t)nnz;
    tile_y[tile_num] = (uint32_t)n_rows;
  }
}

// bnd_row[b] = ROW(tile_y[min(b*W, tile_num)]) for b = 0..nb.
__global__ void plan_block_rows_kernel(const uint32_t* __restrict__ tile_y, int tile_num, int W,
                                       int nb, int32_t* __restrict__ bnd_row) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > nb) return;
  bnd_row[b] = (int32_t)(tile_y[min(b * W, tile_num)] & ~kMsb);
}

// bnd_slot[b] = first index b' with bnd_row[b'] == bnd_row[b] (bnd_row is sorted).
__global__ void plan_slots_kernel(const int32_t* __restrict__ bnd_row, int nb,
                                  int32_t* __restrict__ bnd_slot) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > nb) return;
  const int key = bnd_row[b];
  int lo = 0, hi = b;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (bnd_row[mid] < key) lo = mid + 1; else hi = mid;
  }
  bnd_slot[b] = lo;
}

__global__ void mark_columns_kernel(const int32_t* __restrict__ col, int nnz,
                                    uint8_t* __restrict__ present) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x)
    present[__ldg(col + k)] = 1;
}

__global__ void dangling_bits_kernel(const uint8_t* __restrict__ present, int n,
                                     uint32_t* __restrict__ bits,
                                     unsigned long long* __restrict__ count) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  const int words = (n + 31) >> 5;
  if (w >= words) return;
  uint32_t b = 0;
  for (int i = 0; i < 32; ++i) {
    const int r = w * 32 + i;
    if (r < n && !present[r]) b |= 1u << i;
  }
  bits[w] = b;
  if (b) atomicAdd(count, (unsigned long long)__popc(b));
}

cudaError_t build_tiles(const merbit_plan_s* p, const int32_t* row_ptr, cudaStream_t st) {
  if (p->lane_num == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t total = p->lane_num + 1;
  const int blocks = (int)((total + threads - 1) / threads);
  if (p->desc_bytes == 8)
    plan_tiles_kernel<unsigned long long, 11><<<blocks, threads, 0, st>>>(
        row_ptr, (int)p->n_rows, (int)p->nnz, p->sigma, (int)p->lane_num, (int)p->tile_num, p->tile_x,
        p->tile_y, reinterpret_cast<unsigned long long*>(p->lane_desc));
  else
    plan_tiles_kernel<uint32_t, 9><<<blocks, threads, 0, st>>>(
        row_ptr, (int)p->n_rows, (int)p->nnz, p->sigma, (int)p->lane_num, (int)p->tile_num, p->tile_x,
        p->tile_y, p->lane_desc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nbt = (int)((p->nb + 1 + threads - 1) / threads);
  plan_block_rows_kernel<<<nbt, threads, 0, st>>>(p->tile_y, (int)p->tile_num, p->tiles_per_block,
                                                  (int)p->nb, p->bnd_row);
  plan_slots_kernel<<<nbt, threads, 0, st>>>(p->bnd_row, (int)p->nb, p->bnd_slot);
  return cudaGetLastError();
}

cudaError_t build_dangling(merbit_plan_s* p, cudaStream_t st, unsigned long long* host_count) {
  const int n = (int)p->n_cols;
  uint8_t* present = nullptr;
  unsigned long long* cnt = nullptr;
  cudaError_t e = cudaMalloc(&present, (size_t)n + 8);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&cnt, sizeof(unsigned long long));
  if (e != cudaSuccess) { cudaFree(present); return e; }
  const size_t words = ((size_t)n + 31) / 32;
  if (!p->dangling_bits) {
    e = cudaMalloc(&p->dangling_bits, words * sizeof(uint32_t) + 4);
    if (e != cudaSuccess) { cudaFree(present); cudaFree(cnt); return e; }
  }
  cudaMemsetAsync(present, 0, (size_t)n, st);
  cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
  if (p->nnz > 0) {
    const int blocks = p->num_sms * 8;
    mark_columns_kernel<<<blocks, 256, 0, st>>>(p->col, (int)p->nnz, present);
  }
  dangling_bits_kernel<<<(int)((words + 255) / 256), 256, 0, st>>>(present, n, p->dangling_bits, cnt);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_count, cnt, sizeof(unsigned long long),
                                            cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(present);
  cudaFree(cnt);
  return e;
}

int persistent_grid(const void* kernel, int threads, size_t smem, size_t smem_max, int num_sms) {
  // cudaFuncSetAttribute and the occupancy answer hold per device, so both
  // caches are keyed by the current device as well as the kernel
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> attr;   // dynamic smem limit set
  static std::map<std::tuple<int, const void*, size_t>, int> cache;   // resident CTAs per SM
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(dev, kernel, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second * num_sms;
  // the limit is raised once to the largest size any plan of this kernel needs, never lowered
  size_t& lim = attr[std::make_pair(dev, kernel)];
  // a refused request (more shared memory than a CTA may have) is an answer, not an error
  // for later calls: the runtime's last-error state is cleared
  if (smem_max > 48 * 1024 && lim < smem_max) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    lim = smem_max;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cache[key] = per_sm;
  return per_sm * num_sms;
}

size_t smem_room(const void* kernel, int per_sm) {
  if (per_sm <= 0) return 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> stat;   // static smem per kernel
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(dev, kernel);
  auto it = stat.find(key);
  if (it == stat.end()) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 0;
    it = stat.emplace(key, fa.sharedSizeBytes).first;
  }
  int per_sm_total = 0, reserved = 0, optin = 0;
  if (cudaDeviceGetAttribute(&per_sm_total, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  const long long share = (long long)per_sm_total / per_sm - reserved - (long long)it->second;
  const long long cap = (long long)optin - (long long)it->second;
  const long long room = share < cap ? share : cap;
  return room > 0 ? (size_t)room : 0;
}

size_t smem_room_below(const void* kernel, int per_sm, size_t shared_per_sm) {
  const size_t room = smem_room(kernel, per_sm);
  if (per_sm <= 0 || room == 0) return 0;
  int dev = 0, reserved = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
    return 0;
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const long long share = (long long)(shared_per_sm / (size_t)per_sm) - reserved - (long long)fa.sharedSizeBytes;
  const size_t below = share > 0 ? (size_t)share : 0;
  return below < room ? below : room;
}

}  // namespace merbit
