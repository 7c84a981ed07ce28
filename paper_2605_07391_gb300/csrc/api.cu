// C ABI of the MERBIT library: plan lifecycle, SpMV dispatch, reduced-precision
// value conversion and the PageRank drivers (plain power method and
// mixed-precision iterative refinement).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "extensions.cuh"

namespace merbit {
cudaError_t host_async_wait(const merbit_plan_s* p);
void host_async_release(const merbit_plan_s* p);
cudaError_t build_tiles(const merbit_plan_s* p, const int32_t* row_ptr, cudaStream_t st);
cudaError_t build_dangling(merbit_plan_s* p, cudaStream_t st, unsigned long long* host_count);
void free_hot_table(merbit_plan_s* p);
}  // namespace merbit

using namespace merbit;

namespace {

thread_local char g_err[1024] = "";

merbit_status fail(merbit_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

merbit_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? MERBIT_ENOMEM : MERBIT_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define MB_TRY(call)                                   \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

size_t dtype_size(merbit_dtype d) {
  switch (d) {
    case MERBIT_F32: return 4;
    case MERBIT_F64: return 8;
    case MERBIT_BF16: return 2;
    case MERBIT_F16: return 2;
  }
  return 0;
}

void free_plan(merbit_plan_s* p) {
  if (!p) return;
  host_async_release(p);
  free_hot_table(p);
  cudaFree(p->tile_x);
  cudaFree(p->tile_y);
  cudaFree(p->lane_desc);
  cudaFree(p->bnd_row);
  cudaFree(p->bnd_slot);
  cudaFree(p->bnd_acc);
  cudaFree(p->part);
  cudaFree(p->red);
  cudaFree(p->dangling_bits);
  cudaFree(p->scratch);
  cudaFree(p->hist);
  cudaFree(p->x_stage);
  cudaFree(p->y_stage);
  cudaFree(p->spmm_acc);
  if (p->host_pinned) cudaFreeHost(p->host_pinned);
  delete p;
}

cudaError_t grow(void** buf, size_t* cap, size_t need) {
  if (*cap >= need) return cudaSuccess;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(buf, need);
  if (e == cudaSuccess) *cap = need;
  return e;
}

cudaError_t reset_device_state(merbit_plan_s* p, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(p->red, 0, sizeof(RedState), st);
  if (e == cudaSuccess && p->nb > 0) e = cudaMemsetAsync(p->bnd_acc, 0, sizeof(double) * (p->nb + 1), st);
  return e;
}

// err, done, iters of the plan's RedState, read through pinned memory.
struct StateWord { int err, done, iters, inner_done, launches; };

cudaError_t read_state(merbit_plan_s* p, cudaStream_t st, StateWord* w) {
  cudaError_t e = cudaMemcpyAsync(p->host_pinned, &p->red->err, sizeof(StateWord),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) *w = *static_cast<StateWord*>(p->host_pinned);
  return e;
}

merbit_status check_plan(merbit_plan_t p) {
  if (!p) return fail(MERBIT_EINVAL, "plan is NULL");
  return MERBIT_OK;
}

// ---------------------------------------------------------------- small kernels

template <typename T>
__global__ void fill_kernel(T* a, int64_t n, T v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// hist[0] = 0, hist[1] = D0; PageRank state cleared.
__global__ void pr_state_init_kernel(double* hist, double d0, RedState* red) {
  hist[0] = 0.0;
  hist[1] = d0;
  red->done = 0;
  red->iters = 0;
  red->inner_done = 0;
  red->launches = 0;
  red->delta = nullptr;   // published again by this solve's first residual pass
}

// Correctly rounded (ties to even) float64 -> IEEE binary format with E
// exponent bits and M stored fraction bits, written from the IEEE 754
// encoding: normal results keep the top M fraction bits of the 53-bit
// significand, subnormal results are rounded on the format's subnormal grid,
// overflow gives infinity.  (float64 subnormals are below every target's
// smallest subnormal and round to zero.)
template <int E, int M>
__device__ __forceinline__ uint32_t f64_to_bits(double v) {
  const uint64_t u = static_cast<uint64_t>(__double_as_longlong(v));
  const uint32_t sign = static_cast<uint32_t>(u >> 63) << (E + M);
  const int e = static_cast<int>((u >> 52) & 0x7ff);
  const uint64_t frac = u & ((1ull << 52) - 1);
  const uint32_t inf = ((1u << E) - 1u) << M;
  if (e == 0x7ff) return sign | inf | (frac ? (1u << (M - 1)) : 0u);
  if (e == 0) return sign;
  const int bias = (1 << (E - 1)) - 1;
  int te = e - 1023 + bias;                    // target biased exponent
  const uint64_t mant = (1ull << 52) | frac;   // 53-bit significand
  const int shift = te >= 1 ? 52 - M : 52 - M + (1 - te);
  if (shift >= 54) return sign;                // below half the smallest subnormal
  uint64_t q = mant >> shift;
  const uint64_t rem = mant & ((1ull << shift) - 1);
  const uint64_t half = 1ull << (shift - 1);
  if (rem > half || (rem == half && (q & 1ull))) ++q;
  if (te >= 1) {
    if (q >> (M + 1)) { q >>= 1; ++te; }
    if (te >= (1 << E) - 1) return sign | inf;
    return sign | (static_cast<uint32_t>(te) << M) | static_cast<uint32_t>(q & ((1ull << M) - 1));
  }
  return sign | static_cast<uint32_t>(q);      // q == 2^M encodes the smallest normal
}

template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ src, D* __restrict__ dst, int64_t n,
                               double mul) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = static_cast<double>(src[i]) * mul;
    if constexpr (std::is_same<D, __nv_bfloat16>::value) {
      dst[i] = __ushort_as_bfloat16(static_cast<unsigned short>(f64_to_bits<8, 7>(v)));
    } else if constexpr (std::is_same<D, __half>::value) {
      dst[i] = __ushort_as_half(static_cast<unsigned short>(f64_to_bits<5, 10>(v)));
    } else {
      dst[i] = static_cast<float>(v);
    }
  }
}

template <typename S>
__global__ void max_abs_bits_kernel(const S* __restrict__ src, int64_t n,
                                    unsigned long long* out) {
  unsigned long long m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = fabs(static_cast<double>(src[i]));
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(a));
    m = b > m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

int grid_for(int64_t n, int num_sms) {
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms * 16;
  return (int)std::max<int64_t>(1, std::min(want, cap));
}

template <typename S>
merbit_status convert_typed(const S* src, void* dst, merbit_dtype ddt, int64_t nnz, int auto_scale,
                            int* scale_exp_out, cudaStream_t st, int num_sms) {
  int k = 0;
  if (auto_scale && ddt == MERBIT_F16 && nnz > 0) {
    unsigned long long* d = nullptr;
    MB_TRY(cudaMalloc(&d, sizeof(unsigned long long)));
    unsigned long long bits = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(bits), st);
    if (e == cudaSuccess) {
      max_abs_bits_kernel<S><<<grid_for(nnz, num_sms), 256, 0, st>>>(src, nnz, d);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "max |value| reduction");
    double mx;
    memcpy(&mx, &bits, sizeof(mx));
    if (mx > 0 && std::isfinite(mx)) {
      int e2 = 0;
      std::frexp(mx, &e2);          // mx in [2^(e2-1), 2^e2)
      k = 15 - e2;                  // mx * 2^k in [2^14, 2^15)
    }
  }
  if (scale_exp_out) *scale_exp_out = k;
  if (nnz == 0) return MERBIT_OK;
  const double mul = std::ldexp(1.0, k);
  const int g = grid_for(nnz, num_sms);
  switch (ddt) {
    case MERBIT_BF16:
      convert_kernel<S, __nv_bfloat16><<<g, 256, 0, st>>>(src, static_cast<__nv_bfloat16*>(dst), nnz, mul);
      break;
    case MERBIT_F16:
      convert_kernel<S, __half><<<g, 256, 0, st>>>(src, static_cast<__half*>(dst), nnz, mul);
      break;
    case MERBIT_F32:
      convert_kernel<S, float><<<g, 256, 0, st>>>(src, static_cast<float*>(dst), nnz, mul);
      break;
    default:
      return fail(MERBIT_EINVAL, "merbit_vals_convert: dst_dtype must be BF16, F16 or F32");
  }
  MB_TRY(cudaGetLastError());
  return MERBIT_OK;
}

merbit_status ensure_dangling(merbit_plan_s* p, cudaStream_t st) {
  if (p->n_dangling >= 0) return MERBIT_OK;
  unsigned long long cnt = 0;
  MB_TRY(build_dangling(p, st, &cnt));
  p->n_dangling = (int64_t)cnt;
  return MERBIT_OK;
}

merbit_status ensure_hist(merbit_plan_s* p, size_t launches) {
  const size_t need = 2 * (launches + 2);
  if (p->hist_len >= need) return MERBIT_OK;
  cudaFree(p->hist);
  p->hist = nullptr;
  p->hist_len = 0;
  MB_TRY(cudaMalloc(&p->hist, need * sizeof(double)));
  p->hist_len = need;
  return MERBIT_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// (block_num + 1) x 32 zeroed FP64 accumulators of the SpMM's block-shared rows
merbit_status ensure_spmm_acc(merbit_plan_s* p, cudaStream_t st) {
  if (p->spmm_acc) return MERBIT_OK;
  const size_t bytes = sizeof(double) * 32 * (size_t)(p->nb + 1);
  MB_TRY(cudaMalloc(&p->spmm_acc, bytes));
  MB_TRY(cudaMemsetAsync(p->spmm_acc, 0, bytes, st));
  return MERBIT_OK;
}

}  // namespace

namespace merbit {
void set_last_error(const char* msg) {
  std::snprintf(g_err, sizeof(g_err), "%s", msg);
}
}  // namespace merbit

// ============================================================================
extern "C" {

const char* merbit_last_error(void) { return g_err; }

const char* merbit_version(void) { return "merbit-gb300 0.1 (sm_103a)"; }

merbit_status merbit_plan_ex(const int32_t* row_ptr, const int32_t* col_idx, int64_t n_rows,
                             int64_t n_cols, int64_t nnz, int sigma, int tiles_per_block,
                             void* stream, merbit_plan_t* out) {
  g_err[0] = 0;
  if (!out) return fail(MERBIT_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_rows < 0 || n_cols < 0 || nnz < 0) return fail(MERBIT_EINVAL, "negative size");
  if (!row_ptr) return fail(MERBIT_EINVAL, "row_ptr is NULL");
  if (nnz > 0 && !col_idx) return fail(MERBIT_EINVAL, "col_idx is NULL");
  if (sigma < 1 || sigma > kSigmaMax64)
    return fail(MERBIT_EINVAL, "sigma must be in [1, %d] (32-bit lane descriptors up to %d, 64-bit above)",
                kSigmaMax64, kSigmaMax);
  if (tiles_per_block != 4 && tiles_per_block != 8 && tiles_per_block != kMaxW)
    return fail(MERBIT_EINVAL, "tiles_per_block must be 4, 8 or 16");
  if (n_rows + nnz >= (int64_t)INT32_MAX)
    return fail(MERBIT_EOVERFLOW, "n_rows + nnz = %lld does not fit the int32 merge path",
                (long long)(n_rows + nnz));
  if (n_cols >= (int64_t)INT32_MAX) return fail(MERBIT_EOVERFLOW, "n_cols too large");
  if (nnz > 0 && !aligned(col_idx, 16)) return fail(MERBIT_EINVAL, "col_idx must be 16-byte aligned");
  cudaStream_t st = as_stream(stream);

  int32_t ends[2] = {0, 0};
  MB_TRY(cudaMemcpyAsync(&ends[0], row_ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MB_TRY(cudaMemcpyAsync(&ends[1], row_ptr + n_rows, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MB_TRY(cudaStreamSynchronize(st));
  if (ends[0] != 0 || (int64_t)ends[1] != nnz)
    return fail(MERBIT_EINVAL, "row_ptr[0] = %d and row_ptr[n] = %d; expected 0 and nnz = %lld",
                ends[0], ends[1], (long long)nnz);
  if (const char* v = getenv("MERBIT_VALIDATE")) {
    if (v[0] == '1') {
      std::vector<int32_t> h((size_t)n_rows + 1);
      MB_TRY(cudaMemcpy(h.data(), row_ptr, h.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < n_rows; ++i)
        if (h[i + 1] < h[i]) return fail(MERBIT_EINVAL, "row_ptr decreases at row %lld", (long long)i);
    }
  }

  merbit_plan_s* p = new merbit_plan_s();
  auto bail = [&](merbit_status s) { free_plan(p); return s; };
  cudaGetDevice(&p->device);
  cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
  p->n_rows = n_rows;
  p->n_cols = n_cols;
  p->nnz = nnz;
  p->sigma = sigma;
  p->desc_bytes = sigma > kSigmaMax ? 8 : 4;
  p->tiles_per_block = tiles_per_block;
  p->col = col_idx;
  const int64_t steps = n_rows + nnz;
  p->lane_num = (steps + sigma - 1) / sigma;
  p->tile_num = (steps + (int64_t)kOmega * sigma - 1) / ((int64_t)kOmega * sigma);
  p->nb = (p->tile_num + tiles_per_block - 1) / tiles_per_block;

  cudaError_t e = cudaSuccess;
  const size_t tb = sizeof(uint32_t) * (size_t)(p->tile_num + 1);
  const size_t nbb = sizeof(int32_t) * (size_t)(p->nb + 1);
  if (e == cudaSuccess) e = cudaMalloc(&p->tile_x, tb);
  if (e == cudaSuccess) e = cudaMalloc(&p->tile_y, tb);
  if (e == cudaSuccess)
    e = cudaMalloc(&p->lane_desc, (size_t)p->desc_bytes * (size_t)std::max<int64_t>(p->lane_num, 1));
  if (e == cudaSuccess) e = cudaMalloc(&p->bnd_row, nbb);
  if (e == cudaSuccess) e = cudaMalloc(&p->bnd_slot, nbb);
  if (e == cudaSuccess) e = cudaMalloc(&p->bnd_acc, sizeof(double) * (size_t)(p->nb + 1));
  if (e == cudaSuccess) e = cudaMalloc(&p->part, sizeof(double2) * (size_t)kMaxParts);
  if (e == cudaSuccess) e = cudaMalloc(&p->red, sizeof(RedState));
  if (e == cudaSuccess) e = cudaMallocHost(&p->host_pinned, 256);
  if (e != cudaSuccess) return bail(cuda_fail(e, "plan allocation"));
  if (p->tile_num == 0) {
    // empty path (n_rows = 0): only the terminator
    const uint32_t term[2] = {(uint32_t)nnz, (uint32_t)n_rows};
    e = cudaMemcpyAsync(p->tile_x, &term[0], 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->tile_y, &term[1], 4, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = reset_device_state(p, st);
  if (e == cudaSuccess) e = build_tiles(p, row_ptr, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bail(cuda_fail(e, "plan construction"));
  *out = p;
  return MERBIT_OK;
}

merbit_status merbit_plan(const int32_t* row_ptr, const int32_t* col_idx, int64_t n, int64_t nnz,
                          merbit_plan_t* out) {
  return merbit_plan_ex(row_ptr, col_idx, n, n, nnz, kSigmaMax, kTilesPerBlock, nullptr, out);
}

void merbit_plan_destroy(merbit_plan_t plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  free_plan(plan);
}

merbit_status merbit_plan_get_info(merbit_plan_t p, merbit_plan_info* info) {
  if (merbit_status s = check_plan(p)) return s;
  if (!info) return fail(MERBIT_EINVAL, "info is NULL");
  info->n_rows = p->n_rows;
  info->n_cols = p->n_cols;
  info->nnz = p->nnz;
  info->sigma = p->sigma;
  info->omega = kOmega;
  info->tiles_per_block = p->tiles_per_block;
  info->tile_num = p->tile_num;
  info->lane_num = p->lane_num;
  info->block_num = p->nb;
  info->tile_x = p->tile_x;
  info->tile_y = p->tile_y;
  info->lane_desc = p->lane_desc;
  info->block_row = p->bnd_row;
  info->desc_bytes = p->desc_bytes;
  return MERBIT_OK;
}

merbit_status merbit_plan_export(merbit_plan_t p, uint32_t* tile_x, uint32_t* tile_y,
                                 uint32_t* lane_desc, int32_t* block_row) {
  if (merbit_status s = check_plan(p)) return s;
  MB_TRY(cudaDeviceSynchronize());
  const size_t tb = sizeof(uint32_t) * (size_t)(p->tile_num + 1);
  if (tile_x) MB_TRY(cudaMemcpy(tile_x, p->tile_x, tb, cudaMemcpyDeviceToHost));
  if (tile_y) MB_TRY(cudaMemcpy(tile_y, p->tile_y, tb, cudaMemcpyDeviceToHost));
  if (lane_desc && p->lane_num)
    MB_TRY(cudaMemcpy(lane_desc, p->lane_desc, (size_t)p->desc_bytes * (size_t)p->lane_num,
                      cudaMemcpyDeviceToHost));
  if (block_row && p->nb)
    MB_TRY(cudaMemcpy(block_row, p->bnd_row, sizeof(int32_t) * (size_t)(p->nb + 1), cudaMemcpyDeviceToHost));
  else if (block_row)
    block_row[0] = (int32_t)p->n_rows;
  return MERBIT_OK;
}

merbit_status merbit_plan_set_kernel(merbit_plan_t p, int kernel) {
  if (merbit_status s = check_plan(p)) return s;
  if (kernel < MERBIT_KERNEL_AUTO || kernel > MERBIT_KERNEL_SPLIT2)
    return fail(MERBIT_EINVAL, "kernel must be MERBIT_KERNEL_AUTO, _CLASSIC, _SPLIT or _SPLIT2");
  p->spmv_kernel = kernel;
  return MERBIT_OK;
}

merbit_status merbit_plan_set_wait_limit(merbit_plan_t p, int polls) {
  if (merbit_status s = check_plan(p)) return s;
  p->wait_limit = polls < 0 ? kSpinLimit : (uint32_t)polls;
  return MERBIT_OK;
}

merbit_status merbit_plan_sync(merbit_plan_t p, void* stream) {
  if (merbit_status s = check_plan(p)) return s;
  cudaStream_t st = as_stream(stream);
  MB_TRY(host_async_wait(p));
  StateWord w{};
  MB_TRY(read_state(p, st, &w));
  if (w.err) {
    MB_TRY(reset_device_state(p, st));
    MB_TRY(cudaStreamSynchronize(st));
    return fail(MERBIT_EDEVICE, "a kernel reported error bits 0x%x (bounded wait expired)", w.err);
  }
  return MERBIT_OK;
}

merbit_status merbit_spmv_ex(merbit_plan_t p, merbit_dtype vdt, merbit_dtype xdt,
                             const void* vals, const void* x, void* y, int scale_exp,
                             void* stream) {
  if (merbit_status s = check_plan(p)) return s;
  if (p->n_rows > 0 && !y) return fail(MERBIT_EINVAL, "y is NULL");
  if (p->nnz > 0 && (!vals || !x)) return fail(MERBIT_EINVAL, "vals or x is NULL");
  if (p->nnz > 0 && !aligned(vals, 16)) return fail(MERBIT_EINVAL, "vals must be 16-byte aligned");
  const size_t xs = dtype_size(xdt);
  if ((x && !aligned(x, xs)) || (y && !aligned(y, xs)))
    return fail(MERBIT_EINVAL, "x / y must be aligned to their element size");
  if (scale_exp < -200 || scale_exp > 200) return fail(MERBIT_EINVAL, "scale_exp out of range");
  cudaStream_t st = as_stream(stream);
  cudaError_t e;
  if (vdt == MERBIT_F32 && xdt == MERBIT_F32 && scale_exp == 0) {
    e = spmv_plain_f32(p, static_cast<const float*>(vals), static_cast<const float*>(x),
                       static_cast<float*>(y), st);
  } else if (vdt == MERBIT_F64 && xdt == MERBIT_F64 && scale_exp == 0) {
    e = spmv_plain_f64(p, static_cast<const double*>(vals), static_cast<const double*>(x),
                       static_cast<double*>(y), st);
  } else if ((vdt == MERBIT_BF16 || vdt == MERBIT_F16) && xdt == MERBIT_F32) {
    e = spmv_plain_lo(p, vdt, vals, static_cast<const float*>(x), static_cast<float*>(y),
                      std::ldexp(1.0f, -scale_exp), st);
  } else {
    return fail(MERBIT_EINVAL,
                "unsupported (vals, x/y) dtypes: (F32,F32), (F64,F64), (BF16,F32), (F16,F32); "
                "scale_exp only with 16-bit values");
  }
  if (e == cudaErrorInvalidConfiguration)
    return fail(MERBIT_EINVAL, "spmv launch: a block of this plan (sigma %d x %d tiles) needs more "
                "shared memory than one CTA may use for these value types; use a smaller sigma or "
                "tiles_per_block", p->sigma, p->tiles_per_block);
  if (e != cudaSuccess) return cuda_fail(e, "spmv launch");
  return MERBIT_OK;
}

merbit_status merbit_spmv(merbit_plan_t p, merbit_dtype dtype, const void* vals, const void* x,
                          void* y) {
  if (dtype != MERBIT_F32 && dtype != MERBIT_F64)
    return fail(MERBIT_EINVAL, "merbit_spmv: dtype must be F32 or F64");
  return merbit_spmv_ex(p, dtype, dtype, vals, x, y, 0, nullptr);
}

merbit_status merbit_spmm(merbit_plan_t p, const float* vals, const float* X, float* Y, int64_t k,
                          int64_t ldx, int64_t ldy, void* stream) {
  if (merbit_status s = check_plan(p)) return s;
  if (p->tiles_per_block != kTilesPerBlock || p->sigma > kSigmaMax)
    return fail(MERBIT_EINVAL, "the SpMM needs a plan of %d tiles per block and sigma <= %d",
                kTilesPerBlock, kSigmaMax);
  if (k < 0 || ldx < k || ldy < k) return fail(MERBIT_EINVAL, "need k >= 0, ldx >= k, ldy >= k");
  if (k == 0 || p->n_rows == 0) return MERBIT_OK;
  if (!Y || (p->nnz > 0 && (!vals || !X))) return fail(MERBIT_EINVAL, "vals, X or Y is NULL");
  if (p->nnz > 0 && !aligned(vals, 16)) return fail(MERBIT_EINVAL, "vals must be 16-byte aligned");
  if (!aligned(X, 4) || !aligned(Y, 4)) return fail(MERBIT_EINVAL, "X / Y must be 4-byte aligned");
  if ((int64_t)p->n_cols * ldx >= ((int64_t)1 << 40)) return fail(MERBIT_EINVAL, "X too large");
  cudaStream_t st = as_stream(stream);
  if (merbit_status s = ensure_spmm_acc(p, st)) return s;
  MB_TRY(spmm_plain_f32(p, vals, X, k, ldx, Y, ldy, p->spmm_acc, st));
  return MERBIT_OK;
}

merbit_status merbit_ppr(merbit_plan_t p, const float* vals, const int32_t* seeds, int64_t k,
                         double alpha, double tol, int max_iter, float* Pi, int* iters_out,
                         double* resid_out, double* resid_hist, void* stream) {
  if (merbit_status s = check_plan(p)) return s;
  if (p->n_rows != p->n_cols) return fail(MERBIT_EINVAL, "personalised PageRank needs a square plan");
  if (p->tiles_per_block != kTilesPerBlock || p->sigma > kSigmaMax)
    return fail(MERBIT_EINVAL, "personalised PageRank needs a plan of %d tiles per block and sigma <= %d",
                kTilesPerBlock, kSigmaMax);
  if (!(alpha >= 0.0 && alpha < 1.0)) return fail(MERBIT_EINVAL, "alpha must be in [0, 1)");
  if (max_iter < 1) return fail(MERBIT_EINVAL, "max_iter must be >= 1");
  if (k < 1 || k > 1024) return fail(MERBIT_EINVAL, "k must be in [1, 1024]");
  if (p->n_rows == 0) return fail(MERBIT_EINVAL, "the graph has no vertices");
  if (!seeds || !Pi) return fail(MERBIT_EINVAL, "seeds or Pi is NULL");
  if (p->nnz > 0 && !vals) return fail(MERBIT_EINVAL, "vals is NULL");
  if (p->nnz > 0 && !aligned(vals, 16)) return fail(MERBIT_EINVAL, "vals must be 16-byte aligned");
  if (!aligned(Pi, 4)) return fail(MERBIT_EINVAL, "Pi must be 4-byte aligned");
  const int64_t n = p->n_rows;
  if (n * k >= ((int64_t)1 << 40)) return fail(MERBIT_EINVAL, "n * k too large");
  for (int64_t c = 0; c < k; ++c)
    if (seeds[c] < 0 || seeds[c] >= n) return fail(MERBIT_EINVAL, "seed %lld out of range", (long long)c);
  cudaStream_t st = as_stream(stream);
  if (merbit_status s = ensure_dangling(p, st)) return s;
  if (merbit_status s = ensure_hist(p, (size_t)max_iter)) return s;
  if (merbit_status s = ensure_spmm_acc(p, st)) return s;
  // scratch: second iterate | seeds | D per column | 2k accumulators | last residuals
  const size_t xb = align256(sizeof(float) * (size_t)n * (size_t)k);
  const size_t sb = align256(sizeof(int32_t) * (size_t)k);
  const size_t db = align256(sizeof(double) * (size_t)k);
  MB_TRY(grow(&p->scratch, &p->scratch_bytes, xb + sb + 4 * db));
  char* base = static_cast<char*>(p->scratch);
  float* x1 = reinterpret_cast<float*>(base);
  int32_t* seed_d = reinterpret_cast<int32_t*>(base + xb);
  double* d_cur = reinterpret_cast<double*>(base + xb + sb);
  double* rd = reinterpret_cast<double*>(base + xb + sb + db);
  double* last_r = reinterpret_cast<double*>(base + xb + sb + 3 * db);
  MB_TRY(cudaMemcpyAsync(seed_d, seeds, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, st));
  MB_TRY(reset_device_state(p, st));
  MB_TRY(cudaMemsetAsync(rd, 0, 2 * sizeof(double) * (size_t)k, st));
  MB_TRY(ppr_init(p, Pi, k, seed_d, d_cur, st));
  float* buf[2] = {Pi, x1};
  const int kBatch = 8;
  int it = 0;
  StateWord w{};
  while (it < max_iter) {
    const int stop = std::min(max_iter, it + kBatch);
    for (; it < stop; ++it) {
      cudaError_t e = ppr_update(p, vals, buf[it & 1], buf[(it + 1) & 1], k, seed_d, d_cur, rd,
                                 last_r, (float)alpha, tol, it, p->hist, p->spmm_acc, st);
      if (e != cudaSuccess) return cuda_fail(e, "personalised PageRank launch");
    }
    MB_TRY(read_state(p, st, &w));
    if (w.err || w.done) break;
  }
  if (w.err) {
    MB_TRY(reset_device_state(p, st));
    MB_TRY(cudaStreamSynchronize(st));
    return fail(MERBIT_EDEVICE, "a kernel reported error bits 0x%x", w.err);
  }
  const int iters = w.done ? w.iters : max_iter;
  if (iters & 1)
    MB_TRY(cudaMemcpyAsync(Pi, x1, sizeof(float) * (size_t)n * (size_t)k, cudaMemcpyDeviceToDevice, st));
  std::vector<double> h((size_t)iters);
  MB_TRY(cudaMemcpyAsync(h.data(), p->hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (resid_out)
    MB_TRY(cudaMemcpyAsync(resid_out, last_r, sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost, st));
  MB_TRY(cudaStreamSynchronize(st));
  if (iters_out) *iters_out = iters;
  if (resid_hist)
    for (int i = 0; i < iters; ++i) resid_hist[i] = h[(size_t)i];
  if (tol > 0 && !w.done)
    return fail(MERBIT_ENOTCONV, "personalised PageRank did not reach tol %.3g in %d updates "
                "(largest residual %.3g)", tol, max_iter, iters > 0 ? h[(size_t)iters - 1] : 0.0);
  return MERBIT_OK;
}

merbit_status merbit_spmv_host(merbit_plan_t p, merbit_dtype dtype, const void* vals,
                               const void* x_host, void* y_host, void* stream) {
  if (merbit_status s = check_plan(p)) return s;
  if (dtype != MERBIT_F32 && dtype != MERBIT_F64)
    return fail(MERBIT_EINVAL, "merbit_spmv_host: dtype must be F32 or F64");
  if ((p->n_cols > 0 && !x_host) || (p->n_rows > 0 && !y_host))
    return fail(MERBIT_EINVAL, "x_host or y_host is NULL");
  cudaStream_t st = as_stream(stream);
  const size_t es = dtype_size(dtype);
  const size_t xb = es * (size_t)p->n_cols, yb = es * (size_t)p->n_rows;
  MB_TRY(grow(&p->x_stage, &p->x_stage_bytes, std::max<size_t>(xb, 16)));
  MB_TRY(grow(&p->y_stage, &p->y_stage_bytes, std::max<size_t>(yb, 16)));
  if (xb) MB_TRY(cudaMemcpyAsync(p->x_stage, x_host, xb, cudaMemcpyHostToDevice, st));
  merbit_status s = merbit_spmv_ex(p, dtype, dtype, vals, p->x_stage, p->y_stage, 0, stream);
  if (s != MERBIT_OK) return s;
  if (yb) MB_TRY(cudaMemcpyAsync(y_host, p->y_stage, yb, cudaMemcpyDeviceToHost, st));
  return merbit_plan_sync(p, stream);
}

merbit_status merbit_vals_convert(const void* src, merbit_dtype sdt, void* dst, merbit_dtype ddt,
                                  int64_t nnz, int auto_scale, int* scale_exp_out, void* stream) {
  if (nnz < 0) return fail(MERBIT_EINVAL, "nnz < 0");
  if (nnz > 0 && (!src || !dst)) return fail(MERBIT_EINVAL, "src or dst is NULL");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t st = as_stream(stream);
  if (sdt == MERBIT_F64)
    return convert_typed(static_cast<const double*>(src), dst, ddt, nnz, auto_scale, scale_exp_out, st, sms);
  if (sdt == MERBIT_F32)
    return convert_typed(static_cast<const float*>(src), dst, ddt, nnz, auto_scale, scale_exp_out, st, sms);
  return fail(MERBIT_EINVAL, "merbit_vals_convert: src_dtype must be F64 or F32");
}

}  // extern "C"

// ---------------------------------------------------------------- PageRank

namespace {

template <typename T>
merbit_status pagerank_plain(merbit_plan_s* p, const T* vals, double alpha, double tol,
                             int max_iter, T* pi, int* iters_out, double* resid_out,
                             double* resid_hist, int* launches_out, cudaStream_t st) {
  const int64_t n = p->n_rows;
  MB_TRY(grow(&p->scratch, &p->scratch_bytes, align256(sizeof(T) * (size_t)n)));
  if (merbit_status s = ensure_hist(p, (size_t)max_iter)) return s;
  T* buf[2] = {pi, static_cast<T*>(p->scratch)};
  const double d0 = (double)p->n_dangling / (double)n;
  fill_kernel<T><<<grid_for(n, p->num_sms), 256, 0, st>>>(pi, n, static_cast<T>(1.0 / (double)n));
  pr_state_init_kernel<<<1, 1, 0, st>>>(p->hist, d0, p->red);
  MB_TRY(cudaGetLastError());
  const int kBatch = 8;
  int k = 0;
  StateWord w{};
  while (k < max_iter) {
    const int stop = std::min(max_iter, k + kBatch);
    for (; k < stop; ++k) {
      PRParams prm;
      prm.out = buf[(k + 1) & 1];
      prm.dang = p->dangling_bits;
      prm.alpha = alpha;
      prm.inv_n = 1.0 / (double)n;
      prm.tol = tol;
      prm.d_in = p->hist + 2 * k + 1;
      prm.s_out = p->hist + 2 * (k + 1);
      prm.iter = k;
      cudaError_t e;
      if constexpr (sizeof(T) == 4)
        e = spmv_pr_f32(p, reinterpret_cast<const float*>(vals), reinterpret_cast<const float*>(buf[k & 1]), prm, st);
      else
        e = spmv_pr_f64(p, reinterpret_cast<const double*>(vals), reinterpret_cast<const double*>(buf[k & 1]), prm, st);
      if (e != cudaSuccess) return cuda_fail(e, "pagerank launch");
    }
    MB_TRY(read_state(p, st, &w));
    if (w.err || w.done) break;
  }
  if (w.err) {
    MB_TRY(reset_device_state(p, st));
    MB_TRY(cudaStreamSynchronize(st));
    return fail(MERBIT_EDEVICE, "a kernel reported error bits 0x%x", w.err);
  }
  const int iters = w.done ? w.iters : max_iter;
  if (iters & 1) MB_TRY(cudaMemcpyAsync(pi, buf[1], sizeof(T) * (size_t)n, cudaMemcpyDeviceToDevice, st));
  std::vector<double> h(2 * ((size_t)iters + 1));
  MB_TRY(cudaMemcpyAsync(h.data(), p->hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  MB_TRY(cudaStreamSynchronize(st));
  if (iters_out) *iters_out = iters;
  if (launches_out) *launches_out = iters;
  if (resid_out) *resid_out = iters > 0 ? h[2 * (size_t)iters] : 0.0;
  if (resid_hist)
    for (int i = 0; i < iters; ++i) resid_hist[i] = h[2 * ((size_t)i + 1)];
  if (tol > 0 && !w.done)
    return fail(MERBIT_ENOTCONV, "PageRank did not reach tol %.3g in %d updates (last residual %.3g)",
                tol, max_iter, iters > 0 ? h[2 * (size_t)iters] : 0.0);
  return MERBIT_OK;
}

merbit_status pagerank_ir(merbit_plan_s* p, const double* vals, double alpha, double tol,
                          int max_steps, merbit_precision mode, int max_sweeps, double inner_tol,
                          double* pi, int* iters_out, double* resid_out, double* resid_hist,
                          int* launches_out, cudaStream_t st) {
  const int64_t n = p->n_rows;
  const merbit_dtype ldt = mode == MERBIT_IR_BF16 ? MERBIT_BF16
                           : mode == MERBIT_IR_F16 ? MERBIT_F16 : MERBIT_F32;
  // inner stop: a sweep smaller than eta * ||r||_1 is below the rounding level of the
  // reduced-precision values (unit roundoff 2^-8 and 2^-11), so further sweeps cannot
  // improve the correction; f32 values would allow far more, but a step gaining about
  // five decades already balances sweeps against the FP64 residual evaluations
  const double eta = inner_tol > 0.0 ? inner_tol
                     : ldt == MERBIT_BF16 ? std::ldexp(1.0, -8)
                     : ldt == MERBIT_F16 ? std::ldexp(1.0, -11) : std::ldexp(1.0, -17);
  const size_t lo_bytes = align256(dtype_size(ldt) * (size_t)std::max<int64_t>(p->nnz, 1));
  const size_t vb = align256(sizeof(float) * (size_t)n);
  MB_TRY(grow(&p->scratch, &p->scratch_bytes, lo_bytes + 3 * vb));
  char* base = static_cast<char*>(p->scratch);
  void* lo = base;
  float* rhs = reinterpret_cast<float*>(base + lo_bytes);
  float* dl[2] = {reinterpret_cast<float*>(base + lo_bytes + vb),
                  reinterpret_cast<float*>(base + lo_bytes + 2 * vb)};
  int scale_exp = 0;
  if (merbit_status s = convert_typed(vals, lo, ldt, p->nnz, ldt == MERBIT_F16, &scale_exp, st,
                                      p->num_sms))
    return s;
  const size_t per_step = (size_t)max_sweeps + 2;
  if (merbit_status s = ensure_hist(p, ((size_t)max_steps + 1) * per_step + 1)) return s;
  const double d0 = (double)p->n_dangling / (double)n;
  fill_kernel<double><<<grid_for(n, p->num_sms), 256, 0, st>>>(pi, n, 1.0 / (double)n);
  pr_state_init_kernel<<<1, 1, 0, st>>>(p->hist, d0, p->red);
  MB_TRY(cudaGetLastError());
  const float scale = std::ldexp(1.0f, -scale_exp);
  int L = 0;   // launch counter (hist slot L+1 holds launch L's results)
  std::vector<int> resid_launch;
  StateWord w{};
  int step = 0;
  for (; step <= max_steps; ++step) {
    // r = b - M pi  (FP64); the solve stops once ||r||_1 < tol
    ResidParams rp;
    rp.rhs = rhs;
    rp.dang = p->dangling_bits;
    rp.alpha = alpha;
    rp.inv_n = 1.0 / (double)n;
    rp.tol = tol;
    rp.d_in = p->hist + 2 * L + 1;
    rp.s_out = p->hist + 2 * (L + 1);
    rp.iter = step;
    const double* rnorm = rp.s_out;
    resid_launch.push_back(L);
    cudaError_t e = spmv_resid_f64(p, vals, pi, rp, st);
    if (e != cudaSuccess) return cuda_fail(e, "residual launch");
    ++L;
    if (step >= max_steps) break;   // final residual of the last correction
    // inner Richardson sweeps on M delta = r, from delta = r; launches after the
    // inner stop fired return at once
    for (int s = 1; s <= max_sweeps; ++s) {
      SweepParams sp;
      sp.out = dl[(s + 1) & 1];
      sp.rhs = rhs;
      sp.dang = p->dangling_bits;
      sp.alpha = alpha;
      sp.inv_n = 1.0 / (double)n;
      sp.scale = scale;
      sp.d_in = p->hist + 2 * L + 1;
      sp.s_out = p->hist + 2 * (L + 1);
      sp.rnorm = rnorm;
      sp.eta = eta;
      const float* xin = s == 1 ? rhs : dl[s & 1];
      e = spmv_sweep(p, ldt, lo, xin, sp, st);
      if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
      ++L;
    }
    // pi += delta
    e = ir_apply(p, pi, p->hist + 2 * (L + 1), st);
    if (e != cudaSuccess) return cuda_fail(e, "apply launch");
    ++L;
    MB_TRY(read_state(p, st, &w));
    if (w.err || w.done) break;
  }
  if (!w.err && !w.done) MB_TRY(read_state(p, st, &w));
  if (w.err) {
    MB_TRY(reset_device_state(p, st));
    MB_TRY(cudaStreamSynchronize(st));
    return fail(MERBIT_EDEVICE, "a kernel reported error bits 0x%x", w.err);
  }
  std::vector<double> h(2 * ((size_t)L + 1));
  MB_TRY(cudaMemcpyAsync(h.data(), p->hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  MB_TRY(cudaStreamSynchronize(st));
  // corrections applied = residual evaluations minus the final one
  const int evals = w.done ? w.iters : (int)resid_launch.size();
  const int corrections = w.done ? evals - 1 : std::min<int>(step, max_steps);
  const double last = h[2 * ((size_t)resid_launch[(size_t)evals - 1] + 1)];
  if (iters_out) *iters_out = corrections;
  if (launches_out) *launches_out = w.launches;
  if (resid_out) *resid_out = last;
  if (resid_hist)
    for (int i = 0; i < evals; ++i)
      resid_hist[i] = h[2 * ((size_t)resid_launch[(size_t)i] + 1)];
  if (tol > 0 && !w.done)
    return fail(MERBIT_ENOTCONV, "refinement did not reach tol %.3g in %d steps (residual %.3g)",
                tol, max_steps, last);
  return MERBIT_OK;
}

}  // namespace

extern "C" {

merbit_status merbit_pagerank_ex(merbit_plan_t p, merbit_dtype dtype, const void* vals,
                                 double alpha, double tol, int max_iter, merbit_precision mode,
                                 int inner_sweeps, double inner_tol, void* pi, int* iters_out,
                                 double* resid_out, double* resid_hist, int* launches_out,
                                 void* stream) {
  if (merbit_status s = check_plan(p)) return s;
  if (p->n_rows != p->n_cols) return fail(MERBIT_EINVAL, "PageRank needs a square plan");
  if (!(alpha >= 0.0 && alpha < 1.0)) return fail(MERBIT_EINVAL, "alpha must be in [0, 1)");
  if (max_iter < 1) return fail(MERBIT_EINVAL, "max_iter must be >= 1");
  if (p->n_rows == 0) {
    if (iters_out) *iters_out = 0;
    if (resid_out) *resid_out = 0.0;
    return MERBIT_OK;
  }
  if (!pi) return fail(MERBIT_EINVAL, "pi is NULL");
  if (p->nnz > 0 && !vals) return fail(MERBIT_EINVAL, "vals is NULL");
  if (p->nnz > 0 && !aligned(vals, 16)) return fail(MERBIT_EINVAL, "vals must be 16-byte aligned");
  cudaStream_t st = as_stream(stream);
  if (merbit_status s = ensure_dangling(p, st)) return s;
  if (mode == MERBIT_PLAIN) {
    if (dtype == MERBIT_F32)
      return pagerank_plain<float>(p, static_cast<const float*>(vals), alpha, tol, max_iter,
                                   static_cast<float*>(pi), iters_out, resid_out, resid_hist,
                                   launches_out, st);
    if (dtype == MERBIT_F64)
      return pagerank_plain<double>(p, static_cast<const double*>(vals), alpha, tol, max_iter,
                                    static_cast<double*>(pi), iters_out, resid_out, resid_hist,
                                    launches_out, st);
    return fail(MERBIT_EINVAL, "PLAIN PageRank: dtype must be F32 or F64");
  }
  if (mode != MERBIT_IR_BF16 && mode != MERBIT_IR_F16 && mode != MERBIT_IR_F32)
    return fail(MERBIT_EINVAL, "unknown precision mode %d", (int)mode);
  if (dtype != MERBIT_F64) return fail(MERBIT_EINVAL, "refinement modes need F64 master values and pi");
  if (inner_sweeps < 1) return fail(MERBIT_EINVAL, "inner_sweeps must be >= 1");
  if (inner_tol < 0.0) return fail(MERBIT_EINVAL, "inner_tol must be >= 0");
  return pagerank_ir(p, static_cast<const double*>(vals), alpha, tol, max_iter, mode, inner_sweeps,
                     inner_tol, static_cast<double*>(pi), iters_out, resid_out, resid_hist,
                                    launches_out, st);
}

merbit_status merbit_sddmm(merbit_plan_t p, merbit_dtype dtype, const void* g, const void* x,
                          double scale, void* out, void* stream) {
  if (merbit_status s = check_plan(p)) return s;
  if (dtype != MERBIT_F32 && dtype != MERBIT_F64) return fail(MERBIT_EINVAL, "dtype must be F32 or F64");
  if (p->nnz == 0) return MERBIT_OK;
  if (!g || !x || !out) return fail(MERBIT_EINVAL, "g, x or out is NULL");
  MB_TRY(sddmm(p, dtype, g, x, scale, out, as_stream(stream)));
  return MERBIT_OK;
}

merbit_status merbit_pagerank_adjoint(merbit_plan_t p, merbit_plan_t pt, merbit_dtype dtype,
                                      const void* vals_t, double alpha, const void* w, double tol,
                                      int max_iter, void* lambda, int* iters_out,
                                      double* resid_out, void* stream) {
  if (merbit_status s = check_plan(p)) return s;
  if (merbit_status s = check_plan(pt)) return s;
  if (p->n_rows != p->n_cols) return fail(MERBIT_EINVAL, "PageRank needs a square plan");
  if (pt->n_rows != p->n_cols || pt->n_cols != p->n_rows || pt->nnz != p->nnz)
    return fail(MERBIT_EINVAL, "plan_t is not a plan of the transposed matrix");
  if (dtype != MERBIT_F32 && dtype != MERBIT_F64) return fail(MERBIT_EINVAL, "dtype must be F32 or F64");
  if (!(alpha >= 0.0 && alpha < 1.0)) return fail(MERBIT_EINVAL, "alpha must be in [0, 1)");
  if (max_iter < 1) return fail(MERBIT_EINVAL, "max_iter must be >= 1");
  const int64_t n = p->n_rows;
  if (n == 0) {
    if (iters_out) *iters_out = 0;
    if (resid_out) *resid_out = 0.0;
    return MERBIT_OK;
  }
  if (!w || !lambda) return fail(MERBIT_EINVAL, "w or lambda is NULL");
  if (pt->nnz > 0 && (!vals_t || !aligned(vals_t, 16)))
    return fail(MERBIT_EINVAL, "vals_t must be a 16-byte aligned device array");
  cudaStream_t st = as_stream(stream);
  if (merbit_status s = ensure_dangling(p, st)) return s;
  if (merbit_status s = ensure_hist(pt, (size_t)max_iter)) return s;
  const size_t es = dtype_size(dtype);
  MB_TRY(grow(&pt->scratch, &pt->scratch_bytes, align256(es * (size_t)n) + 256));
  void* buf[2] = {lambda, pt->scratch};
  double* wnorm = reinterpret_cast<double*>(static_cast<char*>(pt->scratch) + align256(es * (size_t)n));
  // lambda_0 = w, S_0 = sum(w); state cleared
  MB_TRY(cudaMemcpyAsync(lambda, w, es * (size_t)n, cudaMemcpyDeviceToDevice, st));
  pr_state_init_kernel<<<1, 1, 0, st>>>(pt->hist, 0.0, pt->red);
  MB_TRY(cudaGetLastError());
  MB_TRY(vec_sum(w, dtype, n, pt->hist + 1, false, pt->num_sms, st));
  MB_TRY(vec_sum(w, dtype, n, wnorm, true, pt->num_sms, st));
  const int kBatch = 8;
  int k = 0;
  StateWord sw{};
  while (k < max_iter) {
    const int stop = std::min(max_iter, k + kBatch);
    for (; k < stop; ++k) {
      AdjParams prm;
      prm.out = buf[(k + 1) & 1];
      prm.w = w;
      prm.dang = p->dangling_bits;
      prm.alpha = alpha;
      prm.inv_n = 1.0 / (double)n;
      prm.tol = tol;
      prm.wnorm = wnorm;
      prm.s_in = pt->hist + 2 * k + 1;
      prm.s_out = pt->hist + 2 * (k + 1);
      prm.iter = k;
      cudaError_t e = dtype == MERBIT_F32
          ? spmv_adj_f32(pt, static_cast<const float*>(vals_t), static_cast<const float*>(buf[k & 1]), prm, st)
          : spmv_adj_f64(pt, static_cast<const double*>(vals_t), static_cast<const double*>(buf[k & 1]), prm, st);
      if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
    }
    MB_TRY(read_state(pt, st, &sw));
    if (sw.err || sw.done) break;
  }
  if (sw.err) {
    MB_TRY(reset_device_state(pt, st));
    MB_TRY(cudaStreamSynchronize(st));
    return fail(MERBIT_EDEVICE, "a kernel reported error bits 0x%x", sw.err);
  }
  const int iters = sw.done ? sw.iters : max_iter;
  if (iters & 1) MB_TRY(cudaMemcpyAsync(lambda, buf[1], es * (size_t)n, cudaMemcpyDeviceToDevice, st));
  double last = 0.0;
  MB_TRY(cudaMemcpyAsync(&last, pt->hist + 2 * (size_t)iters, sizeof(double), cudaMemcpyDeviceToHost, st));
  MB_TRY(cudaStreamSynchronize(st));
  if (iters_out) *iters_out = iters;
  if (resid_out) *resid_out = last;
  if (tol > 0 && !sw.done)
    return fail(MERBIT_ENOTCONV, "adjoint solve did not reach tol %.3g * ||w||_1 in %d updates (residual %.3g)",
                tol, max_iter, last);
  return MERBIT_OK;
}

merbit_status merbit_pagerank(merbit_plan_t p, merbit_dtype dtype, const void* vals, double alpha,
                              double tol, void* pi) {
  return merbit_pagerank_ex(p, dtype, vals, alpha, tol, 10000, MERBIT_PLAIN, 0, 0.0, pi, nullptr,
                            nullptr, nullptr, nullptr, nullptr);
}

}  // extern "C"
