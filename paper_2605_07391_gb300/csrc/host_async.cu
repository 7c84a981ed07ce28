// y = A x with x and y in host memory, without waiting: consecutive calls on one plan
// overlap.  Two device staging slots alternate.  Call i uploads x into its slot on an
// upload stream, runs the product on the caller's stream once the upload's event has
// fired, and downloads y on a copy stream once the product's event has fired; so call
// i + 1's upload and call i - 1's download run while call i computes.  A slot's x is
// overwritten only after the product that last read it, and its y only after the
// download that last read it (events the upload and the caller's stream wait for).
// merbit_plan_sync waits for everything.
#include <cstdio>
#include <mutex>
#include <unordered_map>

#include "merbit_internal.cuh"

namespace merbit {
void set_last_error(const char* msg);
}  // namespace merbit

using namespace merbit;

namespace {

struct AsyncState {
  int device = 0;
  int slot = 0;
  size_t xb = 0, yb = 0;
  void* x[2] = {nullptr, nullptr};
  void* y[2] = {nullptr, nullptr};
  cudaEvent_t uploaded[2] = {nullptr, nullptr};
  cudaEvent_t kernel_done[2] = {nullptr, nullptr};
  cudaEvent_t copy_done[2] = {nullptr, nullptr};
  cudaStream_t up = nullptr;
  cudaStream_t copy = nullptr;
};

std::mutex g_mu;
std::unordered_map<const merbit_plan_s*, AsyncState*> g_state;

void free_state(AsyncState* a) {
  if (!a) return;
  if (a->up) cudaStreamSynchronize(a->up);
  if (a->copy) cudaStreamSynchronize(a->copy);
  for (int s = 0; s < 2; ++s) {
    cudaFree(a->x[s]);
    cudaFree(a->y[s]);
    if (a->uploaded[s]) cudaEventDestroy(a->uploaded[s]);
    if (a->kernel_done[s]) cudaEventDestroy(a->kernel_done[s]);
    if (a->copy_done[s]) cudaEventDestroy(a->copy_done[s]);
  }
  if (a->up) cudaStreamDestroy(a->up);
  if (a->copy) cudaStreamDestroy(a->copy);
  delete a;
}

cudaError_t get_state(const merbit_plan_s* p, size_t xb, size_t yb, AsyncState** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  AsyncState*& a = g_state[p];
  cudaError_t e = cudaSuccess;
  if (!a) {
    a = new AsyncState();
    a->device = p->device;
    e = cudaStreamCreateWithFlags(&a->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&a->up, cudaStreamNonBlocking);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
      e = cudaEventCreateWithFlags(&a->uploaded[s], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a->kernel_done[s], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a->copy_done[s], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
      // keep no half-built state: the next call starts over
      free_state(a);
      g_state.erase(p);
      *out = nullptr;
      return e;
    }
  }
  if (e == cudaSuccess && (a->xb < xb || a->yb < yb)) {
    // resize only when nothing is pending on the slots
    e = cudaStreamSynchronize(a->up);
    if (e == cudaSuccess) e = cudaStreamSynchronize(a->copy);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
      cudaFree(a->x[s]);
      cudaFree(a->y[s]);
      a->x[s] = a->y[s] = nullptr;
      e = cudaMalloc(&a->x[s], xb);
      if (e == cudaSuccess) e = cudaMalloc(&a->y[s], yb);
    }
    if (e == cudaSuccess) {
      a->xb = xb;
      a->yb = yb;
    } else {
      a->xb = a->yb = 0;
    }
  }
  *out = a;
  return e;
}

merbit_status afail(merbit_status s, const char* what, cudaError_t e) {
  char msg[256];
  std::snprintf(msg, sizeof(msg), "%s%s%s", what, e != cudaSuccess ? ": " : "",
                e != cudaSuccess ? cudaGetErrorString(e) : "");
  set_last_error(msg);
  return s;
}

}  // namespace

namespace merbit {

// Waits for the plan's pending downloads; called by merbit_plan_sync.
cudaError_t host_async_wait(const merbit_plan_s* p) {
  AsyncState* a = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_state.find(p);
    if (it == g_state.end()) return cudaSuccess;
    a = it->second;
  }
  cudaError_t e = cudaStreamSynchronize(a->up);
  if (e == cudaSuccess) e = cudaStreamSynchronize(a->copy);
  return e;
}

// Frees the plan's staging state; called by merbit_plan_destroy.
void host_async_release(const merbit_plan_s* p) {
  AsyncState* a = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_state.find(p);
    if (it == g_state.end()) return;
    a = it->second;
    g_state.erase(it);
  }
  free_state(a);
}

}  // namespace merbit

extern "C" {

merbit_status merbit_spmv_host_async(merbit_plan_t p, merbit_dtype dtype, const void* vals,
                                     const void* x_host, void* y_host, void* stream) {
  set_last_error("");
  if (!p) return afail(MERBIT_EINVAL, "plan is NULL", cudaSuccess);
  if (dtype != MERBIT_F32 && dtype != MERBIT_F64)
    return afail(MERBIT_EINVAL, "merbit_spmv_host_async: dtype must be F32 or F64", cudaSuccess);
  if ((p->n_cols > 0 && !x_host) || (p->n_rows > 0 && !y_host))
    return afail(MERBIT_EINVAL, "x_host or y_host is NULL", cudaSuccess);
  const size_t es = dtype == MERBIT_F64 ? 8 : 4;
  const size_t xb = es * (size_t)p->n_cols, yb = es * (size_t)p->n_rows;
  AsyncState* a = nullptr;
  cudaError_t e = get_state(p, std::max<size_t>(xb, 16), std::max<size_t>(yb, 16), &a);
  if (e != cudaSuccess) return afail(e == cudaErrorMemoryAllocation ? MERBIT_ENOMEM : MERBIT_ECUDA,
                                     "host staging", e);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int s = a->slot;
  a->slot ^= 1;
  // x[s] is free once the product that last read it is done; y[s] once its download is
  e = cudaStreamWaitEvent(a->up, a->kernel_done[s], 0);
  if (e == cudaSuccess && xb) e = cudaMemcpyAsync(a->x[s], x_host, xb, cudaMemcpyHostToDevice, a->up);
  if (e == cudaSuccess) e = cudaEventRecord(a->uploaded[s], a->up);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, a->uploaded[s], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, a->copy_done[s], 0);
  if (e != cudaSuccess) return afail(MERBIT_ECUDA, "upload of x", e);
  merbit_status ms = merbit_spmv_ex(p, dtype, dtype, vals, a->x[s], a->y[s], 0, stream);
  if (ms != MERBIT_OK) return ms;
  e = cudaEventRecord(a->kernel_done[s], st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(a->copy, a->kernel_done[s], 0);
  if (e == cudaSuccess && yb) e = cudaMemcpyAsync(y_host, a->y[s], yb, cudaMemcpyDeviceToHost, a->copy);
  if (e == cudaSuccess) e = cudaEventRecord(a->copy_done[s], a->copy);
  if (e != cudaSuccess) return afail(MERBIT_ECUDA, "download of y", e);
  return MERBIT_OK;
}

}  // extern "C"
