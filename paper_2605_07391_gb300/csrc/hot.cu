// Hot-column table of a plan: the columns that the most nonzeros reference.
//
// The SpMV gathers x[col[k]] for every nonzero.  On power-law matrices a few
// thousand columns take a large share of those gathers, and in a graph's
// natural numbering they are scattered over x, one per 128-byte line, so L1
// cannot keep them.  The plan picks up to max_hot such columns, sorts them by
// use, and streams a copy of the column array in which each of them is
// replaced by ~slot (a negative index).  Every launch of the SpMV then copies
// x at those columns into shared memory once per CTA and takes the gathers of
// tagged nonzeros from there (see spmv_kernel.cuh).  The same copy can also
// mark, with bit 30, the columns used only a few times: their gathers skip the
// L1 allocation, so they do not evict the lines of x that are used again.  No
// counterpart in the paper: these are GB300 choices for the x gather of Sec. 4.2.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "merbit_internal.cuh"

namespace merbit {
void set_last_error(const char* msg);
}  // namespace merbit

using namespace merbit;

namespace {

constexpr int kHistBins = 1 << 16;     // use counts >= kHistBins - 1 share the top bin
constexpr int kSmemBins = 4096;        // low counts are binned in shared memory first

__global__ void count_columns_kernel(const int32_t* __restrict__ col, int64_t nnz,
                                     uint32_t* __restrict__ cnt) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + __ldg(col + k), 1u);
}

__global__ void __launch_bounds__(256) count_hist_kernel(const uint32_t* __restrict__ cnt, int64_t n,
                                                         uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kSmemBins];
  for (int i = threadIdx.x; i < kSmemBins; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t v = min(cnt[c], (uint32_t)(kHistBins - 1));
    if (v < kSmemBins) atomicAdd(h + v, 1u);
    else atomicAdd(hist + v, 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kSmemBins; i += blockDim.x)
    if (h[i]) atomicAdd(hist + i, h[i]);
}

// Columns used at least `thr` times, up to `cap` of them (in no particular order).
__global__ void select_kernel(const uint32_t* __restrict__ cnt, int64_t n, uint32_t thr, int cap,
                              int32_t* __restrict__ sel_col, uint32_t* __restrict__ sel_cnt,
                              int* __restrict__ nsel) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t v = cnt[c];
    if (v >= thr) {
      const int s = atomicAdd(nsel, 1);
      if (s < cap) {
        sel_col[s] = (int32_t)c;
        sel_cnt[s] = v;
      }
    }
  }
}

// slot_of[c] = ~slot for every hot column (the other entries keep their non-negative counts)
__global__ void mark_slots_kernel(const int32_t* __restrict__ hot_list, int h,
                                  uint32_t* __restrict__ slot_of) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < h) slot_of[hot_list[s]] = (uint32_t)(~s);
}

// out[k] = ~slot for a hot column, else the column with bit 30 set when it is used at most
// cold_uses times (slot_of holds ~slot for hot columns and the use count otherwise)
__global__ void tag_columns_kernel(const int32_t* __restrict__ col, int64_t nnz,
                                   const uint32_t* __restrict__ slot_of, uint32_t cold_uses,
                                   int32_t* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = __ldg(col + k);
    const int32_t t = (int32_t)__ldg(slot_of + c);
    out[k] = t < 0 ? t : ((uint32_t)t <= cold_uses ? (c | 0x40000000) : c);
  }
}

// the number of nonzeros whose column is used at most cold_uses times
__global__ void count_cold_kernel(const uint32_t* __restrict__ cnt, int64_t n, uint32_t cold_uses,
                                  unsigned long long* __restrict__ total) {
  unsigned long long s = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t v = cnt[c];
    if ((int32_t)v >= 0 && v <= cold_uses) s += v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(total, s);
}

void drop_table(merbit_plan_s* p) {
  cudaFree(p->col_hot);
  cudaFree(p->hot_list);
  p->col_hot = nullptr;
  p->hot_list = nullptr;
  p->hot_n = 0;
  p->hot_cover = 0.0;
  p->cold_cover = 0.0;
}

merbit_status fail_hot(merbit_status s, const char* what, cudaError_t e) {
  char msg[256];
  std::snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
  set_last_error(msg);
  return s;
}

}  // namespace

namespace merbit {

// Build (or drop, max_hot = 0) the plan's hot-column table.  A table is kept only if
// its columns hold at least min_cover of the nonzeros.
merbit_status build_hot_table(merbit_plan_s* p, int max_hot, double min_cover, cudaStream_t st) {
  drop_table(p);
  p->hot_max = max_hot;
  p->hot_min_cover = min_cover;
  // bit 30 can tag a column only while every column index is below 2^30
  const uint32_t cold = p->n_cols <= (int64_t(1) << 30) && p->cold_uses > 0 ? (uint32_t)p->cold_uses : 0u;
  if ((max_hot <= 0 && cold == 0) || p->nnz == 0 || p->n_cols == 0) return MERBIT_OK;
  const int64_t n = p->n_cols, nnz = p->nnz;
  uint32_t* cnt = nullptr;
  uint32_t* hist = nullptr;
  int32_t* sel_col = nullptr;
  uint32_t* sel_cnt = nullptr;
  int* nsel = nullptr;
  auto cleanup = [&]() {
    cudaFree(cnt);
    cudaFree(hist);
    cudaFree(sel_col);
    cudaFree(sel_cnt);
    cudaFree(nsel);
  };
  cudaError_t e = cudaMalloc(&cnt, sizeof(uint32_t) * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&hist, sizeof(uint32_t) * kHistBins);
  if (e == cudaSuccess) e = cudaMalloc(&sel_col, sizeof(int32_t) * (size_t)std::max(max_hot, 1));
  if (e == cudaSuccess) e = cudaMalloc(&sel_cnt, sizeof(uint32_t) * (size_t)std::max(max_hot, 2));
  if (e == cudaSuccess) e = cudaMalloc(&nsel, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kHistBins, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(nsel, 0, sizeof(int), st);
  const int grid = p->num_sms * 8;
  if (e == cudaSuccess) {
    count_columns_kernel<<<grid, 256, 0, st>>>(p->col, nnz, cnt);
    count_hist_kernel<<<grid, 256, 0, st>>>(cnt, n, hist);
    e = cudaGetLastError();
  }
  std::vector<uint32_t> h(kHistBins);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), hist, sizeof(uint32_t) * kHistBins, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cleanup();
    return fail_hot(e == cudaErrorMemoryAllocation ? MERBIT_ENOMEM : MERBIT_ECUDA,
                    "hot-column counts", e);
  }
  // smallest use count thr >= 2 whose columns (count >= thr) number at most max_hot; a
  // top bin holding more than max_hot columns is truncated by the selection's cap
  int thr = kHistBins - 1;
  int64_t above = h[kHistBins - 1];
  while (thr > 2 && above + h[thr - 1] <= max_hot) {
    --thr;
    above += h[thr];
  }
  if (max_hot <= 0) above = 0;
  if (above == 0 && cold == 0) {
    cleanup();
    return MERBIT_OK;
  }
  int ns = 0;
  e = cudaSuccess;
  if (above > 0) {
    select_kernel<<<grid, 256, 0, st>>>(cnt, n, (uint32_t)thr, max_hot, sel_col, sel_cnt, nsel);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, nsel, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    ns = std::min(ns, max_hot);
  }
  std::vector<int32_t> hc((size_t)ns);
  std::vector<uint32_t> hn((size_t)ns);
  if (e == cudaSuccess && ns)
    e = cudaMemcpyAsync(hc.data(), sel_col, sizeof(int32_t) * (size_t)ns, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && ns)
    e = cudaMemcpyAsync(hn.data(), sel_cnt, sizeof(uint32_t) * (size_t)ns, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cleanup();
    return fail_hot(MERBIT_ECUDA, "hot-column selection", e);
  }
  // slots by decreasing use (ties by column), so a smaller table keeps the most used
  std::vector<int> order((size_t)ns);
  for (int i = 0; i < ns; ++i) order[(size_t)i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    return hn[(size_t)a] != hn[(size_t)b] ? hn[(size_t)a] > hn[(size_t)b] : hc[(size_t)a] < hc[(size_t)b];
  });
  std::vector<int32_t> list((size_t)ns);
  double covered = 0.0;
  for (int i = 0; i < ns; ++i) {
    list[(size_t)i] = hc[(size_t)order[(size_t)i]];
    covered += hn[(size_t)order[(size_t)i]];
  }
  double cover = covered / (double)nnz;
  if (cover < min_cover) {   // the table is not worth its shared memory
    ns = 0;
    cover = 0.0;
  }
  if (ns == 0 && cold == 0) {
    cleanup();
    return MERBIT_OK;
  }
  unsigned long long cold_nnz = 0;
  if (ns > 0) e = cudaMalloc(&p->hot_list, sizeof(int32_t) * (size_t)ns);
  if (e == cudaSuccess) e = cudaMalloc(&p->col_hot, sizeof(int32_t) * (size_t)nnz);
  if (e == cudaSuccess && ns > 0)
    e = cudaMemcpyAsync(p->hot_list, list.data(), sizeof(int32_t) * (size_t)ns, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && cold > 0) {
    // reuse the selection counter as the cold total (zeroed first)
    e = cudaMemsetAsync(sel_cnt, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
      count_cold_kernel<<<grid, 256, 0, st>>>(cnt, n, cold, reinterpret_cast<unsigned long long*>(sel_cnt));
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&cold_nnz, sel_cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) {
    if (ns > 0) mark_slots_kernel<<<(ns + 255) / 256, 256, 0, st>>>(p->hot_list, ns, cnt);
    tag_columns_kernel<<<grid, 256, 0, st>>>(p->col, nnz, cnt, cold, p->col_hot);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) {
    drop_table(p);
    return fail_hot(e == cudaErrorMemoryAllocation ? MERBIT_ENOMEM : MERBIT_ECUDA,
                    "hot-column table", e);
  }
  p->hot_n = ns;
  p->hot_cover = cover;
  p->cold_cover = (double)cold_nnz / (double)nnz;
  return MERBIT_OK;
}

void free_hot_table(merbit_plan_s* p) { drop_table(p); }

}  // namespace merbit

extern "C" {

merbit_status merbit_plan_set_hot_columns(merbit_plan_t p, int max_hot, double min_cover,
                                          void* stream, int* hot_n_out, double* cover_out) {
  set_last_error("");
  if (!p) {
    set_last_error("plan is NULL");
    return MERBIT_EINVAL;
  }
  if (max_hot < 0 || max_hot > (1 << 20) || !(min_cover >= 0.0 && min_cover <= 1.0)) {
    set_last_error("max_hot must be in [0, 2^20] and min_cover in [0, 1]");
    return MERBIT_EINVAL;
  }
  const merbit_status s = build_hot_table(p, max_hot, min_cover, static_cast<cudaStream_t>(stream));
  if (hot_n_out) *hot_n_out = p->hot_n;
  if (cover_out) *cover_out = p->hot_cover;
  return s;
}

merbit_status merbit_plan_set_cold_columns(merbit_plan_t p, int max_uses, void* stream,
                                           double* cover_out) {
  set_last_error("");
  if (!p) {
    set_last_error("plan is NULL");
    return MERBIT_EINVAL;
  }
  if (max_uses < 0) {
    set_last_error("max_uses must be >= 0");
    return MERBIT_EINVAL;
  }
  p->cold_uses = max_uses;
  const merbit_status s = build_hot_table(p, p->hot_max, p->hot_min_cover, static_cast<cudaStream_t>(stream));
  if (cover_out) *cover_out = p->cold_cover;
  return s;
}

}  // extern "C"
