// Hot-column table of a plan: the columns that the most nonzeros reference.
//
// The SpMV gathers x[col[k]] for every nonzero.  On power-law matrices a few
// thousand columns take a large share of those gathers, and in a graph's
// natural numbering they are scattered over x, one per 128-byte line, so L1
// cannot keep them.  The plan picks up to max_hot such columns, sorts them by
// use, and streams a copy of the column array in which each of them is
// replaced by ~slot (a negative index).  Every launch of the SpMV then copies
// x at those columns into shared memory once per CTA and takes the gathers of
// tagged nonzeros from there (see spmv_kernel.cuh).  No counterpart in the
// paper: this is a GB300 choice for the x gather of Sec. 4.2.
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

__global__ void tag_columns_kernel(const int32_t* __restrict__ col, int64_t nnz,
                                   const uint32_t* __restrict__ slot_of, int32_t* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = __ldg(col + k);
    const int32_t t = (int32_t)__ldg(slot_of + c);
    out[k] = t < 0 ? t : c;
  }
}

void drop_table(merbit_plan_s* p) {
  cudaFree(p->col_hot);
  cudaFree(p->hot_list);
  p->col_hot = nullptr;
  p->hot_list = nullptr;
  p->hot_n = 0;
  p->hot_cover = 0.0;
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
  if (max_hot <= 0 || p->nnz == 0 || p->n_cols == 0) return MERBIT_OK;
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
  if (e == cudaSuccess) e = cudaMalloc(&sel_col, sizeof(int32_t) * (size_t)max_hot);
  if (e == cudaSuccess) e = cudaMalloc(&sel_cnt, sizeof(uint32_t) * (size_t)max_hot);
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
  if (above == 0) {
    cleanup();
    return MERBIT_OK;
  }
  select_kernel<<<grid, 256, 0, st>>>(cnt, n, (uint32_t)thr, max_hot, sel_col, sel_cnt, nsel);
  int ns = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, nsel, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  ns = std::min(ns, max_hot);
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
  const double cover = covered / (double)nnz;
  if (ns == 0 || cover < min_cover) {
    cleanup();
    return MERBIT_OK;
  }
  e = cudaMalloc(&p->hot_list, sizeof(int32_t) * (size_t)ns);
  if (e == cudaSuccess) e = cudaMalloc(&p->col_hot, sizeof(int32_t) * (size_t)nnz);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->hot_list, list.data(), sizeof(int32_t) * (size_t)ns, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    mark_slots_kernel<<<(ns + 255) / 256, 256, 0, st>>>(p->hot_list, ns, cnt);
    tag_columns_kernel<<<grid, 256, 0, st>>>(p->col, nnz, cnt, p->col_hot);
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

}  // extern "C"
