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

#include "merbit_internal.cuh"

namespace merbit {
cudaError_t build_tiles(const merbit_plan_s* p, const int32_t* row_ptr, cudaStream_t st);
void set_last_error(const char* msg);   // the text merbit_last_error() returns
}  // namespace merbit

using namespace merbit;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of the scratch array in the current device's context, looked
// up on every call (a host-side lookup, no allocation).  In host code the
// array's name is only a host-side handle, so the kernels must receive this
// address instead.  Looking it up each time keeps it right after a
// cudaDeviceReset or under another context on the same device.
cudaError_t scratch_address(void** out) {
  return cudaGetSymbolAddress(out, g_noalloc_scratch);
}

// Bytes of scratch a matrix needs (the carve order of merbit_spmv_noalloc).
struct Carve {
  size_t off[9];
};

Carve carve(const merbit_plan_s& p) {
  Carve c;
  c.off[0] = 0;
  c.off[1] = c.off[0] + up256(sizeof(RedState));
  c.off[2] = c.off[1] + up256(sizeof(double2) * kMaxParts);
  c.off[3] = c.off[2] + up256(sizeof(uint32_t) * (size_t)(p.tile_num + 1));
  c.off[4] = c.off[3] + up256(sizeof(uint32_t) * (size_t)(p.tile_num + 1));
  c.off[5] = c.off[4] + up256(sizeof(uint32_t) * (size_t)p.lane_num);
  c.off[6] = c.off[5] + up256(sizeof(int32_t) * (size_t)(p.nb + 1));
  c.off[7] = c.off[6] + up256(sizeof(int32_t) * (size_t)(p.nb + 1));
  c.off[8] = c.off[7] + up256(sizeof(double) * (size_t)(p.nb + 1));
  return c;
}

// The header documents the fixed part of the requirement as 66,816 bytes.
static_assert(((sizeof(RedState) + 255) & ~size_t(255)) + sizeof(double2) * kMaxParts == 66816,
              "fixed scratch part changed: update merbit.h");

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
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 3)
    return noalloc_fail(MERBIT_EINVAL, "x and y must be 4-byte aligned");

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
  const Carve c = carve(p);
  if (c.off[8] > kNoAllocScratchBytes) {
    char msg[256];
    std::snprintf(msg, sizeof(msg),
                  "matrix too large for merbit_spmv_noalloc: it needs %zu bytes of scratch and "
                  "the library reserves %zu; use merbit_plan / merbit_spmv instead",
                  c.off[8], kNoAllocScratchBytes);
    return noalloc_fail(MERBIT_EINVAL, msg);
  }
  if (n_rows == 0) return MERBIT_OK;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_fail(MERBIT_ECUDA, "cudaGetDevice failed");
  if (cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return noalloc_fail(MERBIT_ECUDA, "cudaDeviceGetAttribute failed");
  p.device = dev;
  void* base = nullptr;
  if (cudaError_t e = scratch_address(&base); e != cudaSuccess)
    return noalloc_fail(MERBIT_ECUDA, cudaGetErrorString(e));
  unsigned char* b = static_cast<unsigned char*>(base);
  p.red = reinterpret_cast<RedState*>(b + c.off[0]);
  p.part = reinterpret_cast<double2*>(b + c.off[1]);
  p.tile_x = reinterpret_cast<uint32_t*>(b + c.off[2]);
  p.tile_y = reinterpret_cast<uint32_t*>(b + c.off[3]);
  p.lane_desc = reinterpret_cast<uint32_t*>(b + c.off[4]);
  p.bnd_row = reinterpret_cast<int32_t*>(b + c.off[5]);
  p.bnd_slot = reinterpret_cast<int32_t*>(b + c.off[6]);
  p.bnd_acc = reinterpret_cast<double*>(b + c.off[7]);

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The array keeps the previous call's contents.  The boundary accumulators and
  // the arrival count must start at zero (a call whose kernel gave up may have left
  // them set).
  // The error word at the start of the array is left alone: it is zero when
  // the library loads, a kernel that gives up on a bounded wait sets it, and
  // only merbit_spmv_noalloc_status reads and clears it.
  cudaError_t e = cudaMemsetAsync(p.bnd_acc, 0, sizeof(double) * (size_t)(p.nb + 1), st);
  // a small product is finished by the last CTA to arrive; a call whose kernel gave up
  // may have left the arrival count behind
  if (e == cudaSuccess) e = cudaMemsetAsync(&p.red->arrive, 0, sizeof(p.red->arrive), st);
  if (e == cudaSuccess) e = build_tiles(&p, row_ptr, st);
  if (e == cudaSuccess) e = spmv_plain_f32(&p, vals, x, y, st);
  if (e != cudaSuccess) return noalloc_fail(MERBIT_ECUDA, cudaGetErrorString(e));
  return MERBIT_OK;
}

merbit_status merbit_spmv_noalloc_status(void* stream) {
  set_last_error("");
  void* base = nullptr;
  if (cudaError_t e = scratch_address(&base); e != cudaSuccess)
    return noalloc_fail(MERBIT_ECUDA, cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* err = &static_cast<RedState*>(base)->err;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && h) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess && h) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return noalloc_fail(MERBIT_ECUDA, cudaGetErrorString(e));
  if (h) {
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "a merbit_spmv_noalloc kernel gave up on a bounded wait (error bits 0x%x); "
                  "the y of that call is incomplete",
                  h);
    return noalloc_fail(MERBIT_EDEVICE, msg);
  }
  return MERBIT_OK;
}

}  // extern "C"
