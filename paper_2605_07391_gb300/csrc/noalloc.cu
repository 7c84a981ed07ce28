// merbit_spmv_noalloc: a one-shot y = A x for callers that must not allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// another allocator (a framework's memory pool that must account for every
// byte), or paths where cudaMalloc's implicit device-wide synchronisation and
// latency are not acceptable.  For them this entry point builds the schedule
// (the TILE arrays and block boundary data) and runs the SpMV using only a
// fixed scratch area compiled into the library, plus the inputs and output the
// caller passes.  The scratch is a file-scope device array of
// kNoAllocScratchBytes; every GPU that loads the library keeps it until the
// process exits.
#include <cstdio>
#include <mutex>

#include "merbit_internal.cuh"

namespace merbit {
cudaError_t build_tiles(const merbit_plan_s* p, const int32_t* row_ptr, cudaStream_t st);
void set_last_error(const char* msg);   // the text merbit_last_error() returns
}  // namespace merbit

using namespace merbit;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of the scratch array, looked up once per device with that
// device current.  In host code the array's name is only a host-side handle,
// so the kernels must receive this address instead.
cudaError_t scratch_address(int dev, void** out) {
  static std::mutex mu;
  static void* addr[kMaxDevices] = {};
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = p;
  }
  *out = addr[dev];
  return cudaSuccess;
}

merbit_status noalloc_fail(merbit_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

}  // namespace

extern "C" {

merbit_status merbit_spmv_noalloc(const int32_t* row_ptr, const int32_t* col_idx, const float* vals,
                                  const float* x, float* y, int64_t n_rows, int64_t n_cols,
                                  int64_t nnz, void* stream) {
  set_last_error("");
  if (n_rows < 0 || n_cols < 0 || nnz < 0) return noalloc_fail(MERBIT_EINVAL, "negative size");
  if (!row_ptr || (n_rows > 0 && !y) || (nnz > 0 && (!col_idx || !vals || !x)))
    return noalloc_fail(MERBIT_EINVAL, "NULL pointer");
  if (n_rows + nnz >= (int64_t)INT32_MAX || n_cols >= (int64_t)INT32_MAX)
    return noalloc_fail(MERBIT_EOVERFLOW, "n_rows + nnz does not fit the int32 merge path");
  if (nnz > 0 && ((reinterpret_cast<uintptr_t>(vals) | reinterpret_cast<uintptr_t>(col_idx)) & 15))
    return noalloc_fail(MERBIT_EINVAL, "vals and col_idx must be 16-byte aligned");
  if (n_rows == 0) return MERBIT_OK;

  // schedule sizes for sigma = 14 (Sec. 4.1.1 counts)
  merbit_plan_s p;
  p.sigma = kSigmaMax;
  p.tiles_per_block = kTilesPerBlock;
  p.n_rows = n_rows;
  p.n_cols = n_cols;
  p.nnz = nnz;
  p.col = col_idx;
  const int64_t steps = n_rows + nnz;
  p.lane_num = (steps + p.sigma - 1) / p.sigma;
  p.tile_num = (steps + (int64_t)kOmega * p.sigma - 1) / ((int64_t)kOmega * p.sigma);
  p.nb = (p.tile_num + kTilesPerBlock - 1) / kTilesPerBlock;

  // carve the scratch: state | partials | tile_x | tile_y | lane_desc | rows | slots | FP64 accumulators
  size_t off[9];
  off[0] = 0;
  off[1] = off[0] + up256(sizeof(RedState));
  off[2] = off[1] + up256(sizeof(double2) * kMaxParts);
  off[3] = off[2] + up256(sizeof(uint32_t) * (size_t)(p.tile_num + 1));
  off[4] = off[3] + up256(sizeof(uint32_t) * (size_t)(p.tile_num + 1));
  off[5] = off[4] + up256(sizeof(uint32_t) * (size_t)p.lane_num);
  off[6] = off[5] + up256(sizeof(int32_t) * (size_t)(p.nb + 1));
  off[7] = off[6] + up256(sizeof(int32_t) * (size_t)(p.nb + 1));
  off[8] = off[7] + up256(sizeof(double) * (size_t)(p.nb + 1));
  if (off[8] > kNoAllocScratchBytes) {
    char msg[256];
    std::snprintf(msg, sizeof(msg),
                  "matrix too large for merbit_spmv_noalloc: it needs %zu bytes of scratch and "
                  "the library reserves %zu; use merbit_plan / merbit_spmv instead",
                  off[8], kNoAllocScratchBytes);
    return noalloc_fail(MERBIT_EINVAL, msg);
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_fail(MERBIT_ECUDA, "cudaGetDevice failed");
  if (cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return noalloc_fail(MERBIT_ECUDA, "cudaDeviceGetAttribute failed");
  p.device = dev;
  void* base = nullptr;
  if (cudaError_t e = scratch_address(dev, &base); e != cudaSuccess)
    return noalloc_fail(MERBIT_ECUDA, cudaGetErrorString(e));
  unsigned char* b = static_cast<unsigned char*>(base);
  p.red = reinterpret_cast<RedState*>(b + off[0]);
  p.part = reinterpret_cast<double2*>(b + off[1]);
  p.tile_x = reinterpret_cast<uint32_t*>(b + off[2]);
  p.tile_y = reinterpret_cast<uint32_t*>(b + off[3]);
  p.lane_desc = reinterpret_cast<uint32_t*>(b + off[4]);
  p.bnd_row = reinterpret_cast<int32_t*>(b + off[5]);
  p.bnd_slot = reinterpret_cast<int32_t*>(b + off[6]);
  p.bnd_acc = reinterpret_cast<double*>(b + off[7]);

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: the error word and the
  // boundary accumulators must start at zero
  cudaError_t e = cudaMemsetAsync(p.red, 0, sizeof(RedState), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.bnd_acc, 0, sizeof(double) * (size_t)(p.nb + 1), st);
  if (e == cudaSuccess) e = build_tiles(&p, row_ptr, st);
  if (e == cudaSuccess) e = spmv_plain_f32(&p, vals, x, y, st);
  if (e != cudaSuccess) return noalloc_fail(MERBIT_ECUDA, cudaGetErrorString(e));
  return MERBIT_OK;
}

}  // extern "C"
