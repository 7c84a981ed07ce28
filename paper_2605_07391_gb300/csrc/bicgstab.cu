// BiCGSTAB on the MERBIT SpMV (Sec. 5.5: the second iterative workload), FP64.
//
// Unpreconditioned BiCGSTAB with shadow residual r_hat = r_0.  Per iteration:
//   K1  p = r + beta (p - omega v),  beta = (rho / rho_prev)(alpha / omega)
//   S1  v = A p            epilogue: (r_hat, v)        -> alpha = rho / (r_hat, v)
//   K2  s = r - alpha v
//   S2  t = A s            epilogue: (t, s), (t, t)    -> omega = (t, s) / (t, t)
//   K3  x += alpha p + omega s,  r = s - omega t,  (r_hat, r), (r, r) -> rho, stop test
// The scalars live in device memory and are written by the last CTA of each grid-wide
// FP64 reduction, so no step waits for the host.  The whole solve is one CUDA-graph
// launch: r_0 = b - A x_0, then a conditional while node whose body is one iteration;
// the stop test (||r||_2 <= tol ||b||_2, max_iter, or a zero denominator) ends the loop.
// Without values (an adjacency pattern, all values 1) the SpMVs read no value stream.
#include <cmath>
#include <cstdio>
#include <vector>

#include "extensions.cuh"
#include "spmv_kernel.cuh"

namespace merbit {
void set_last_error(const char* msg);
}  // namespace merbit

using namespace merbit;

namespace {

struct BicgState {
  double rho, rho_prev, alpha, omega;
  double rr, bb, tol2;
  int iter, max_iter, status;       // status: 0 running, 1 converged, 2 max_iter, 3 breakdown
  int body;                         // loop-body runs (bounds the loop on its own)
};

struct BicgVecs {
  double *x, *r, *rhat, *p, *v, *s, *t;
  const double* b;
  double* hist;                      // ||r||_2 / ||b||_2 after each iteration
  BicgState* st;
  cudaGraphConditionalHandle loop;
};

__device__ __forceinline__ bool stopped(const RedState* red) {
  return *reinterpret_cast<const volatile int*>(&red->done) != 0;
}

__device__ __forceinline__ void stop(BicgVecs w, RedState* red, int status) {
  w.st->status = status;
  red->done = 1;
  cudaGraphSetConditional(w.loop, 0);
}

// r_0 = b - A x_0 (also r_hat), rho = (r_hat, r) = ||r||^2, ||b||^2
struct EpiBicgInit {
  static constexpr bool kReduce = true;
  BicgVecs w;
  double tol;
  __device__ __forceinline__ void init() {}
  __device__ __forceinline__ bool skip(const RedState* red) const { return stopped(red); }
  __device__ __forceinline__ void put(int r, double s, double& p0, double& p1) const {
    const double bv = w.b[r];
    const double v = bv - s;
    w.r[r] = v;
    w.rhat[r] = v;
    p0 += v * v;
    p1 += bv * bv;
  }
  __device__ __forceinline__ void row(int r, double s, double& p0, double& p1) const { put(r, s, p0, p1); }
  __device__ __forceinline__ void row64(int r, double s, double& p0, double& p1) const { put(r, s, p0, p1); }
  __device__ __forceinline__ void finish(double A, double B, RedState* red) const {
    BicgState* st = w.st;
    st->rho = A;
    st->rr = A;
    st->bb = B;
    st->tol2 = tol * tol * B;
    st->rho_prev = st->alpha = st->omega = 1.0;
    st->iter = 0;
    st->status = 0;
    if (A <= st->tol2) stop(w, red, 1);
  }
};

// v = A p; alpha = rho / (r_hat, v)
struct EpiBicgV {
  static constexpr bool kReduce = true;
  BicgVecs w;
  __device__ __forceinline__ void init() {}
  __device__ __forceinline__ bool skip(const RedState* red) const { return stopped(red); }
  __device__ __forceinline__ void row(int r, double s, double& p0, double&) const {
    w.v[r] = s;
    p0 += w.rhat[r] * s;
  }
  __device__ __forceinline__ void row64(int r, double s, double& p0, double& p1) const { row(r, s, p0, p1); }
  __device__ __forceinline__ void finish(double A, double, RedState* red) const {
    if (A == 0.0) { stop(w, red, 3); return; }
    w.st->alpha = w.st->rho / A;
  }
};

// t = A s; omega = (t, s) / (t, t)
struct EpiBicgT {
  static constexpr bool kReduce = true;
  BicgVecs w;
  __device__ __forceinline__ void init() {}
  __device__ __forceinline__ bool skip(const RedState* red) const { return stopped(red); }
  __device__ __forceinline__ void row(int r, double s, double& p0, double& p1) const {
    w.t[r] = s;
    p0 += s * w.s[r];
    p1 += s * s;
  }
  __device__ __forceinline__ void row64(int r, double s, double& p0, double& p1) const { row(r, s, p0, p1); }
  __device__ __forceinline__ void finish(double A, double B, RedState*) const {
    w.st->omega = B > 0.0 ? A / B : 0.0;
  }
};

// K1: p = r + beta (p - omega v)
__global__ void __launch_bounds__(256) bicg_p_kernel(BicgVecs w, int64_t n, const RedState* red) {
  if (stopped(red)) return;
  const BicgState st = *w.st;
  const double beta = (st.rho / st.rho_prev) * (st.alpha / st.omega);
  const double om = st.omega;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    w.p[i] = w.r[i] + beta * (w.p[i] - om * w.v[i]);
}

// K2: s = r - alpha v
__global__ void __launch_bounds__(256) bicg_s_kernel(BicgVecs w, int64_t n, const RedState* red) {
  if (stopped(red)) return;
  const double alpha = w.st->alpha;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    w.s[i] = w.r[i] - alpha * w.v[i];
}

// K3: x += alpha p + omega s; r = s - omega t; (r_hat, r), (r, r); stop test
__global__ void __launch_bounds__(256) bicg_xr_kernel(BicgVecs w, int64_t n, RedState* red) {
  if (stopped(red)) return;
  const double alpha = w.st->alpha, omega = w.st->omega;
  double p0 = 0.0, p1 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double si = w.s[i];
    w.x[i] += alpha * w.p[i] + omega * si;
    const double ri = si - omega * w.t[i];
    w.r[i] = ri;
    p0 += w.rhat[i] * ri;
    p1 += ri * ri;
  }
  grid_sum2(p0, p1, red, [&](double A, double B) {
    BicgState* st = w.st;
    const int it = st->iter + 1;
    st->iter = it;
    st->rr = B;
    w.hist[it - 1] = st->bb > 0.0 ? sqrt(B / st->bb) : 0.0;
    if (B <= st->tol2) { stop(w, red, 1); return; }
    if (it >= st->max_iter) { stop(w, red, 2); return; }
    if (st->omega == 0.0 || A == 0.0 || red->err != 0) { stop(w, red, 3); return; }
    st->rho_prev = st->rho;
    st->rho = A;
  });
}

__global__ void bicg_state_kernel(BicgState* st, int max_iter, RedState* red) {
  st->max_iter = max_iter;
  st->iter = 0;
  st->status = 0;
  st->body = 0;
  for (int i = 0; i < kRedSlots; ++i) red->slot[i][0] = red->slot[i][1] = 0.0;
  red->arrive = 0u;
  red->done = 0;
  red->iters = 0;
  red->launches = 0;
}

// Last node of the loop body: whatever the reductions did, the loop ends after max_iter
// runs of the body.
__global__ void bicg_guard_kernel(BicgVecs w, RedState* red) {
  if (stopped(red)) return;
  if (++w.st->body >= w.st->max_iter) stop(w, red, 2);
}

// the product of the plan's matrix, with values or (vals == NULL) all values 1
template <typename Epi>
cudaError_t spmv64(const merbit_plan_s* p, const double* vals, const double* x, const Epi& epi,
                   cudaStream_t st) {
  if (vals) return launch_spmv<double, double, double>(p, vals, x, epi, st);
  return launch_spmv<UnitVal<double>, double, double>(p, nullptr, x, epi, st);
}

merbit_status bfail2(merbit_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

}  // namespace

extern "C" {

merbit_status merbit_bicgstab(merbit_plan_t p, const double* vals, const double* b, double* x,
                              double tol, int max_iter, int* iters_out, double* resid_out,
                              double* resid_hist, int* status_out, void* stream) {
  set_last_error("");
  if (!p) return bfail2(MERBIT_EINVAL, "plan is NULL");
  if (p->n_rows != p->n_cols) return bfail2(MERBIT_EINVAL, "BiCGSTAB needs a square plan");
  if (max_iter < 1) return bfail2(MERBIT_EINVAL, "max_iter must be >= 1");
  if (!(tol >= 0.0)) return bfail2(MERBIT_EINVAL, "tol must be >= 0");
  const int64_t n = p->n_rows;
  if (n == 0) {
    if (iters_out) *iters_out = 0;
    if (resid_out) *resid_out = 0.0;
    if (status_out) *status_out = 1;
    return MERBIT_OK;
  }
  if (!b || !x) return bfail2(MERBIT_EINVAL, "b or x is NULL");
  if (vals && (reinterpret_cast<uintptr_t>(vals) & 15))
    return bfail2(MERBIT_EINVAL, "vals must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t vb = (sizeof(double) * (size_t)n + 255) & ~size_t(255);
  const size_t sb = (sizeof(BicgState) + 255) & ~size_t(255);
  char* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, 6 * vb + sb + sizeof(double) * (size_t)max_iter);
  if (e != cudaSuccess) return bfail2(e == cudaErrorMemoryAllocation ? MERBIT_ENOMEM : MERBIT_ECUDA,
                                      "BiCGSTAB work vectors");
  BicgVecs w;
  w.x = x;
  w.b = b;
  w.r = reinterpret_cast<double*>(mem);
  w.rhat = reinterpret_cast<double*>(mem + vb);
  w.p = reinterpret_cast<double*>(mem + 2 * vb);
  w.v = reinterpret_cast<double*>(mem + 3 * vb);
  w.s = reinterpret_cast<double*>(mem + 4 * vb);
  w.t = reinterpret_cast<double*>(mem + 5 * vb);
  w.st = reinterpret_cast<BicgState*>(mem + 6 * vb);
  w.hist = reinterpret_cast<double*>(mem + 6 * vb + sb);
  const int vgrid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)p->num_sms * 8));

  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  e = cudaGraphCreate(&graph, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&w.loop, graph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  // r_0 = b - A x_0; p = v = 0; then the loop
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cap, graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  cudaGraphNodeParams cp = {};
  if (e == cudaSuccess) {
    bicg_state_kernel<<<1, 1, 0, cap>>>(w.st, max_iter, p->red);
    e = cudaMemsetAsync(w.p, 0, 2 * vb, cap);                       // p and v
    EpiBicgInit ei{};
    ei.w = w;
    ei.tol = tol;
    if (e == cudaSuccess) e = spmv64(p, vals, x, ei, cap);
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cap, &cs, nullptr, &cg, &deps, nullptr, &ndeps);
    cudaGraphNode_t cond = nullptr;
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = w.loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cond, cg, deps, nullptr, ndeps, &cp);
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cap, &cond, nullptr, 1, cudaStreamSetCaptureDependencies);
    cudaGraph_t g_out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &g_out);
    if (e == cudaSuccess) e = e2;
  }
  // the loop body: one iteration
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cap, cp.conditional.phGraph_out[0], nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    bicg_p_kernel<<<vgrid, 256, 0, cap>>>(w, n, p->red);
    EpiBicgV ev{};
    ev.w = w;
    e = spmv64(p, vals, w.p, ev, cap);
    if (e == cudaSuccess) {
      bicg_s_kernel<<<vgrid, 256, 0, cap>>>(w, n, p->red);
      EpiBicgT et{};
      et.w = w;
      e = spmv64(p, vals, w.s, et, cap);
    }
    if (e == cudaSuccess) {
      bicg_xr_kernel<<<vgrid, 256, 0, cap>>>(w, n, p->red);
      bicg_guard_kernel<<<1, 1, 0, cap>>>(w, p->red);
      e = cudaGetLastError();
    }
    cudaGraph_t g_out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &g_out);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
  BicgState hs{};
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, w.st, sizeof(BicgState), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &p->red->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && resid_hist && max_iter > 0)
    e = cudaMemcpyAsync(resid_hist, w.hist, sizeof(double) * (size_t)max_iter, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cap) cudaStreamDestroy(cap);
  cudaFree(mem);
  if (e != cudaSuccess) {
    char msg[256];
    std::snprintf(msg, sizeof(msg), "BiCGSTAB: %s", cudaGetErrorString(e));
    return bfail2(MERBIT_ECUDA, msg);
  }
  if (err) {
    cudaMemsetAsync(p->red, 0, sizeof(RedState), st);
    cudaStreamSynchronize(st);
    return bfail2(MERBIT_EDEVICE, "a kernel reported an error");
  }
  if (iters_out) *iters_out = hs.iter;
  if (resid_out) *resid_out = hs.bb > 0.0 ? std::sqrt(hs.rr / hs.bb) : std::sqrt(hs.rr);
  if (status_out) *status_out = hs.status;
  if (hs.status == 3) return bfail2(MERBIT_ENOTCONV, "BiCGSTAB broke down (a zero denominator)");
  if (hs.status != 1) return bfail2(MERBIT_ENOTCONV, "BiCGSTAB did not reach tol in max_iter iterations");
  return MERBIT_OK;
}

}  // extern "C"
