// Many graphs solved together: PageRank of G independent graphs in one CUDA-graph
// launch (the batching extension of Sec. 5.5.1).
//
// The graphs are the diagonal blocks of one block-diagonal matrix, so one MERBIT plan
// over the concatenated rows and nonzeros balances the work across graph boundaries
// exactly as it does across rows of one graph.  Per round, the SpMV kernel runs once
// over the whole matrix with an epilogue that knows each row's graph: it applies that
// graph's teleport and dangling term and leaves graphs that have converged untouched.
// A streaming pass over contiguous row ranges then forms each graph's residual
// ||pi' - pi||_1 and dangling mass (warp sums, one FP64 atomic per warp and graph), and a
// one-block check kernel closes the round: per graph, the residual against tol, the next
// dangling mass, and the stop of the device-side while loop when no graph is left.
//
// The solve is one cudaGraphLaunch: initialisation, a conditional while node whose
// body is two rounds (x -> y, then y -> x, so kernel arguments stay fixed), and a
// final copy of every graph's last iterate into the output.  The loop body holds no
// waits of its own; the SpMV's bounded mbarrier waits report through the plan's error
// word, which also ends the loop.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <vector>

#include "extensions.cuh"
#include "spmv_kernel.cuh"

namespace merbit {
void set_last_error(const char* msg);
cudaError_t build_tiles(const merbit_plan_s* p, const int32_t* row_ptr, cudaStream_t st);
cudaError_t build_dangling(merbit_plan_s* p, cudaStream_t st, unsigned long long* host_count);
}  // namespace merbit

using namespace merbit;

namespace {

// Per-solve device state besides the plan's RedState.
struct BatchState {
  int round;        // rounds completed
  int active;       // graphs not yet converged after the last round
};

__device__ __forceinline__ int graph_of(const int32_t* off, int G, int r) {
  int lo = 0, hi = G;                // off[lo] <= r < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= r) lo = mid; else hi = mid;
  }
  return lo;
}

struct BatchParams {
  const int32_t* off;        // G + 1 row offsets
  int G;
  const double* inv_n;       // 1 / n_g
  const double* D;           // dangling mass of each graph's current iterate
  const int* conv;           // updates at convergence, -1 while active
  double alpha;
};

template <typename T>
struct EpiBatchPR {
  static constexpr bool kReduce = false;
  BatchParams p;
  T* out;
  const int32_t* block_list;   // blocks touching a graph that has not converged
  const int* block_count;
  mutable int lo, hi;
  mutable bool frozen;
  mutable T a, tele;
  __device__ __forceinline__ void init() {
    lo = hi = 0;
    frozen = true;
    a = static_cast<T>(p.alpha);
    tele = T(0);
  }
  __device__ __forceinline__ bool skip(const RedState* red) const {
    return *reinterpret_cast<const volatile int*>(&red->done) != 0;
  }
  __device__ __forceinline__ void locate(int r) const {
    if (r >= lo && r < hi) return;
    const int gid = graph_of(p.off, p.G, r);
    lo = __ldg(p.off + gid);
    hi = __ldg(p.off + gid + 1);
    frozen = __ldg(p.conv + gid) >= 0;
    tele = static_cast<T>((p.alpha * __ldg(p.D + gid) + 1.0 - p.alpha) * __ldg(p.inv_n + gid));
  }
  __device__ __forceinline__ void row(int r, T s, double&, double&) const {
    locate(r);
    if (!frozen) out[r] = a * s + tele;
  }
  __device__ __forceinline__ void row64(int r, double s, double&, double&) const {
    locate(r);
    if (!frozen) out[r] = static_cast<T>(p.alpha * s + static_cast<double>(tele));
  }
  __device__ __forceinline__ void finish(double, double, RedState*) const {}
};

// The blocks of the plan whose rows touch a graph that has not converged, in increasing
// order (so the CTAs still sweep the matrix front to back and share x in L2).  A block is
// skipped only when every graph among its rows [y_bs, y_be] has converged, so a row it
// shares with a neighbouring block belongs to a converged graph that no kernel writes any
// more.  Two passes: per chunk of kCompactChunk blocks the flags and their count, then
// every chunk writes its active blocks at the offset the counts before it give.
constexpr int kCompactChunk = 2048;

__device__ __forceinline__ bool block_active(const uint32_t* tile_y, int tile_num, int64_t n,
                                             const int32_t* off, int G, const int* conv, int v) {
  const int bs = v * kTilesPerBlock;
  const int be = min(bs + kTilesPerBlock, tile_num);
  const int64_t y0 = tile_y[bs] & ~kMsb;
  int64_t y1 = tile_y[be] & ~kMsb;
  if (y1 >= n) y1 = n - 1;
  const int g0 = y0 < n ? graph_of(off, G, (int)y0) : G - 1;
  const int g1 = graph_of(off, G, (int)y1);
  for (int g = g0; g <= g1; ++g)
    if (conv[g] < 0) return true;
  return false;
}

__global__ void __launch_bounds__(256)
    batch_flags_kernel(const uint32_t* tile_y, int tile_num, int nb, int64_t n, const int32_t* off,
                       int G, const int* conv, uint8_t* flags, int* chunk_count) {
  int mine = 0;
  const int c0 = blockIdx.x * kCompactChunk;
  for (int i = threadIdx.x; i < kCompactChunk; i += blockDim.x) {
    const int v = c0 + i;
    if (v >= nb) break;
    const bool a = block_active(tile_y, tile_num, n, off, G, conv, v);
    flags[v] = a ? 1 : 0;
    mine += a;
  }
  __shared__ int sum;
  if (threadIdx.x == 0) sum = 0;
  __syncthreads();
  atomicAdd(&sum, mine);
  __syncthreads();
  if (threadIdx.x == 0) chunk_count[blockIdx.x] = sum;
}

__global__ void __launch_bounds__(256)
    batch_list_kernel(const uint8_t* flags, const int* chunk_count, int nb, int32_t* list,
                      int* count) {
  __shared__ int base;
  __shared__ int warp_tot[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    int s = 0;
    for (int c = 0; c < (int)blockIdx.x; ++c) s += chunk_count[c];
    base = s;
    if (blockIdx.x == gridDim.x - 1) *count = s + chunk_count[blockIdx.x];
  }
  __syncthreads();
  const int c0 = blockIdx.x * kCompactChunk;
  for (int r0 = 0; r0 < kCompactChunk; r0 += blockDim.x) {
    const int v = c0 + r0 + (int)threadIdx.x;
    const bool a = v < nb && flags[v];
    const unsigned m = __ballot_sync(0xffffffffu, a);
    if (lane == 0) warp_tot[warp] = __popc(m);
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (w < warp) before += warp_tot[w];
      all += warp_tot[w];
    }
    if (a) list[base + before + __popc(m & ((1u << lane) - 1u))] = v;
    __syncthreads();
    if (threadIdx.x == 0) base += all;
    __syncthreads();
  }
}

constexpr int kRowsPerWarp = 2048;

// acc[2g] += sum |y - x|, acc[2g + 1] += sum of y over dangling rows, for active graphs.
// A warp takes kRowsPerWarp consecutive rows, its lanes consecutive rows within them; a
// lane flushes its partial sums only when its rows enter another graph, and at the end
// the warp adds the lanes of each graph together before one atomic per graph.
template <typename T>
__global__ void __launch_bounds__(256)
    batch_reduce_kernel(const T* __restrict__ y, const T* __restrict__ x, const int32_t* off,
                        int G, const int* conv, const uint32_t* dang, double* acc,
                        const RedState* red, int64_t n) {
  if (*reinterpret_cast<const volatile int*>(&red->done)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c * kRowsPerWarp < n;
       c += warps) {
    const int64_t r_end = (c + 1) * kRowsPerWarp < n ? (c + 1) * kRowsPerWarp : n;
    int gid = -1, lo = 0, hi = 0;
    bool live = false;
    double p0 = 0.0, p1 = 0.0;
    for (int64_t r = c * kRowsPerWarp + lane; r < r_end; r += 32) {
      if (r < lo || r >= hi) {
        if (live && (p0 != 0.0 || p1 != 0.0)) {
          atomicAdd(acc + 2 * gid, p0);
          atomicAdd(acc + 2 * gid + 1, p1);
        }
        p0 = p1 = 0.0;
        gid = graph_of(off, G, (int)r);
        lo = off[gid];
        hi = off[gid + 1];
        live = conv[gid] < 0;
      }
      if (!live) continue;
      const T v = y[r];
      p0 += fabs(static_cast<double>(v) - static_cast<double>(x[r]));
      if (is_dangling(dang, (int)r)) p1 += static_cast<double>(v);
    }
    // lanes of the same graph together, one atomic per graph present
    const int key = live ? gid : -1;
    unsigned rem = 0xffffffffu;
    while (rem) {
      const int lead = __ffs(rem) - 1;
      const int k = __shfl_sync(0xffffffffu, key, lead);
      const unsigned grp = __ballot_sync(0xffffffffu, key == k);
      double s0 = key == k ? p0 : 0.0, s1 = key == k ? p1 : 0.0;
      s0 = warp_sum(s0);
      s1 = warp_sum(s1);
      if (lane == lead && k >= 0 && (s0 != 0.0 || s1 != 0.0)) {
        atomicAdd(acc + 2 * k, s0);
        atomicAdd(acc + 2 * k + 1, s1);
      }
      rem &= ~grp;
    }
  }
}

// x = 1/n_g on graph g's rows; D_g = n_dangling_g / n_g; every graph active.
template <typename T>
__global__ void batch_init_kernel(T* x, const int32_t* off, int G, const double* inv_n,
                                  const double* dang0, double* D, int* conv, double* acc,
                                  double* last_r, BatchState* bs, RedState* red, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int g = -1, lo = 0, hi = 0;
  T v = T(0);
  for (int64_t r = t; r < n; r += stride) {
    if (r < lo || r >= hi) {
      g = graph_of(off, G, (int)r);
      lo = off[g];
      hi = off[g + 1];
      v = static_cast<T>(inv_n[g]);
    }
    x[r] = v;
  }
  for (int64_t i = t; i < G; i += stride) {
    D[i] = dang0[i];
    conv[i] = -1;
    acc[2 * i] = 0.0;
    acc[2 * i + 1] = 0.0;
    last_r[i] = 0.0;
  }
  if (t == 0) {
    bs->round = 0;
    bs->active = G;
    red->done = 0;
    red->iters = 0;
    red->launches = 0;
  }
}

// Close one round: per active graph the residual and the next dangling mass; stop the
// loop when no graph is left, at max_iter rounds, or on a kernel error.
__global__ void __launch_bounds__(1024)
    batch_check_kernel(int G, double tol, int max_iter, double* acc, double* D, int* conv,
                       double* last_r, BatchState* bs, RedState* red,
                       cudaGraphConditionalHandle loop) {
  __shared__ int active;
  if (*reinterpret_cast<const volatile int*>(&red->done)) return;
  if (threadIdx.x == 0) active = 0;
  __syncthreads();
  const int round = bs->round + 1;
  int mine = 0;
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    if (conv[g] >= 0) continue;
    const double r = acc[2 * g];
    D[g] = acc[2 * g + 1];
    acc[2 * g] = 0.0;
    acc[2 * g + 1] = 0.0;
    last_r[g] = r;
    if (tol > 0.0 && r < tol) conv[g] = round;
    else ++mine;
  }
  atomicAdd(&active, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    bs->round = round;
    bs->active = active;
    ++red->launches;
    if (active == 0 || round >= max_iter || red->err != 0) {
      red->iters = round;
      red->done = 1;
      cudaGraphSetConditional(loop, 0);
    }
  }
}

// Graph g's last iterate is in x1 when its number of updates is odd: copy it to x0.
template <typename T>
__global__ void batch_result_kernel(T* x0, const T* x1, const int32_t* off, int G,
                                    const int* conv, const BatchState* bs, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int g = -1, lo = 0, hi = 0;
  bool odd = false;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    if (r < lo || r >= hi) {
      g = graph_of(off, G, (int)r);
      lo = off[g];
      hi = off[g + 1];
      const int upd = conv[g] >= 0 ? conv[g] : bs->round;
      odd = upd & 1;
    }
    if (odd) x0[r] = x1[r];
  }
}

// err = 1 if a nonzero of graph g's rows has a column outside graph g's range.
__global__ void batch_validate_kernel(const Geometry g, const int32_t* off, int G, int* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < g.lane_num; j += stride) {
    const int ti = (int)(j / kOmega);
    const LaneDesc d = decode_lane(g, load_desc(g, j));
    int xk = (int)__ldg(g.tile_x + ti) + d.xo;
    int row = (int)(__ldg(g.tile_y + ti) & ~kMsb) + d.yo;
    const int64_t left = (int64_t)g.steps - j * g.sigma;
    const int len = left < g.sigma ? (int)left : g.sigma;
    int gid = row < g.n_rows ? graph_of(off, G, row) : -1;
    for (int k = 0; k < len; ++k) {
      if ((d.flags >> k) & 1u) {
        ++row;
        gid = row < g.n_rows ? graph_of(off, G, row) : -1;
      } else {
        const int c = __ldg(g.col + xk);
        if (gid < 0 || c < __ldg(off + gid) || c >= __ldg(off + gid + 1)) atomicOr(err, 1);
        ++xk;
      }
    }
  }
}

// dang_cnt[g] = number of dangling vertices of graph g.
__global__ void batch_dangling_count_kernel(const uint32_t* dang, const int32_t* off, int G,
                                            int64_t n, unsigned long long* cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int g = -1, lo = 0, hi = 0;
  unsigned long long c = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    if (r < lo || r >= hi) {
      if (g >= 0 && c) atomicAdd(cnt + g, c);
      c = 0;
      g = graph_of(off, G, (int)r);
      lo = off[g];
      hi = off[g + 1];
    }
    c += is_dangling(dang, (int)r) ? 1 : 0;
  }
  if (g >= 0 && c) atomicAdd(cnt + g, c);
}

merbit_status bfail(merbit_status s, const char* fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  set_last_error(msg);
  return s;
}

int grid_rows(int64_t n, int sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8));
}

}  // namespace

struct merbit_batch_s {
  merbit_plan_t plan = nullptr;
  int G = 0;
  int64_t n = 0;
  std::vector<int64_t> off_h;
  int32_t* off = nullptr;
  double* inv_n = nullptr;
  double* dang0 = nullptr;
  double* D = nullptr;
  int* conv = nullptr;
  double* acc = nullptr;
  double* last_r = nullptr;
  BatchState* bs = nullptr;
  int32_t* blist = nullptr;      // active blocks of the current round, in order
  int* bcount = nullptr;
  uint8_t* bflags = nullptr;     // per block: touches an active graph
  int* ccount = nullptr;         // active blocks per chunk of kCompactChunk
  void* x1 = nullptr;
  size_t x1_bytes = 0;
  // the instantiated solve and what it was built for
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  merbit_dtype dt = MERBIT_F64;
  int spmv_kernel = -1;
  const int32_t* hot_list = nullptr;   // the plan's hot-column table when recorded
  const int32_t* col_hot = nullptr;
  int hot_n = -1;
  const void* vals = nullptr;
  void* pi = nullptr;
  double alpha = -1.0, tol = -1.0;
  int max_iter = -1;
};

namespace {

void free_batch(merbit_batch_s* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  merbit_plan_destroy(b->plan);
  cudaFree(b->off);
  cudaFree(b->inv_n);
  cudaFree(b->dang0);
  cudaFree(b->D);
  cudaFree(b->conv);
  cudaFree(b->acc);
  cudaFree(b->last_r);
  cudaFree(b->bs);
  cudaFree(b->blist);
  cudaFree(b->bcount);
  cudaFree(b->bflags);
  cudaFree(b->ccount);
  cudaFree(b->x1);
  delete b;
}

// Record the whole solve (init, while loop of rounds, result copy) into b->graph.
template <typename T>
cudaError_t record_solve(merbit_batch_s* b, const T* vals, T* pi, double alpha, double tol,
                         int max_iter, cudaStream_t cap) {
  merbit_plan_s* p = b->plan;
  const int sms = p->num_sms;
  cudaError_t e = cudaGraphCreate(&b->graph, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle loop;
  e = cudaGraphConditionalHandleCreate(&loop, b->graph, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  T* x0 = pi;
  T* x1 = static_cast<T*>(b->x1);
  BatchParams bp;
  bp.off = b->off;
  bp.G = b->G;
  bp.inv_n = b->inv_n;
  bp.D = b->D;
  bp.conv = b->conv;
  bp.alpha = alpha;

  // 1. initialisation, then the conditional node appended to the captured sequence
  e = cudaStreamBeginCaptureToGraph(cap, b->graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  batch_init_kernel<T><<<grid_rows(b->n, sms), 256, 0, cap>>>(x0, b->off, b->G, b->inv_n, b->dang0,
                                                             b->D, b->conv, b->acc, b->last_r,
                                                             b->bs, p->red, b->n);
  e = cudaGetLastError();
  cudaStreamCaptureStatus status;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraph_t cg = nullptr;
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cap, &status, nullptr, &cg, &deps, nullptr, &ndeps);
  cudaGraphNode_t cond_node = nullptr;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = loop;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (e == cudaSuccess) e = cudaGraphAddNode(&cond_node, cg, deps, nullptr, ndeps, &cp);
  if (e == cudaSuccess)
    e = cudaStreamUpdateCaptureDependencies(cap, &cond_node, nullptr, 1, cudaStreamSetCaptureDependencies);
  // 3. the result copy after the loop
  if (e == cudaSuccess) {
    batch_result_kernel<T><<<grid_rows(b->n, sms), 256, 0, cap>>>(x0, x1, b->off, b->G, b->conv,
                                                                 b->bs, b->n);
    e = cudaGetLastError();
  }
  cudaGraph_t done = nullptr;
  const cudaError_t e_end = cudaStreamEndCapture(cap, &done);
  if (e == cudaSuccess) e = e_end;
  if (e != cudaSuccess) return e;

  // 2. the loop body: two rounds, x0 -> x1 and x1 -> x0
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  for (int half = 0; half < 2 && e == cudaSuccess; ++half) {
    EpiBatchPR<T> epi{};
    epi.p = bp;
    epi.out = half == 0 ? x1 : x0;
    epi.block_list = b->blist;
    epi.block_count = b->bcount;
    if (p->nb > 0) {
      const int chunks = (int)((p->nb + kCompactChunk - 1) / kCompactChunk);
      batch_flags_kernel<<<chunks, 256, 0, cap>>>(p->tile_y, (int)p->tile_num, (int)p->nb, b->n,
                                                   b->off, b->G, b->conv, b->bflags, b->ccount);
      batch_list_kernel<<<chunks, 256, 0, cap>>>(b->bflags, b->ccount, (int)p->nb, b->blist,
                                                  b->bcount);
      e = cudaGetLastError();
      if (e != cudaSuccess) break;
    }
    const T* xin = half == 0 ? x0 : x1;
    e = launch_spmv<T, T, T>(p, vals, xin, epi, cap);
    if (e == cudaSuccess) {
      const int64_t warps = (b->n + kRowsPerWarp - 1) / kRowsPerWarp;
      const int rgrid = (int)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, (int64_t)sms * 8));
      batch_reduce_kernel<T><<<rgrid, 256, 0, cap>>>(epi.out, xin, b->off, b->G, b->conv,
                                                    p->dangling_bits, b->acc, p->red, b->n);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      batch_check_kernel<<<1, 1024, 0, cap>>>(b->G, tol, max_iter, b->acc, b->D, b->conv,
                                              b->last_r, b->bs, p->red, loop);
      e = cudaGetLastError();
    }
  }
  cudaGraph_t body_done = nullptr;
  const cudaError_t e_end2 = cudaStreamEndCapture(cap, &body_done);
  if (e == cudaSuccess) e = e_end2;
  return e;
}

}  // namespace

extern "C" {

merbit_status merbit_batch_plan(const int32_t* row_ptr, const int32_t* col_idx, int64_t n,
                                int64_t nnz, const int64_t* graph_offsets, int num_graphs,
                                int sigma, void* stream, merbit_batch_t* out) {
  set_last_error("");
  if (!out) return bfail(MERBIT_EINVAL, "out is NULL");
  *out = nullptr;
  if (num_graphs < 1 || !graph_offsets) return bfail(MERBIT_EINVAL, "need num_graphs >= 1 and graph_offsets");
  if (sigma > kSigmaMax) return bfail(MERBIT_EINVAL, "batches use 32-bit lane descriptors: sigma <= %d", kSigmaMax);
  if (graph_offsets[0] != 0 || graph_offsets[num_graphs] != n)
    return bfail(MERBIT_EINVAL, "graph_offsets must start at 0 and end at n");
  for (int g = 0; g < num_graphs; ++g)
    if (graph_offsets[g + 1] <= graph_offsets[g])
      return bfail(MERBIT_EINVAL, "graph %d has no vertices", g);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto* b = new merbit_batch_s();
  b->G = num_graphs;
  b->n = n;
  b->off_h.assign(graph_offsets, graph_offsets + num_graphs + 1);
  merbit_status s = merbit_plan_ex(row_ptr, col_idx, n, n, nnz, sigma, kTilesPerBlock, stream, &b->plan);
  if (s != MERBIT_OK) {
    delete b;
    return s;
  }
  merbit_plan_s* p = b->plan;
  std::vector<int32_t> off32(b->off_h.begin(), b->off_h.end());
  std::vector<double> inv_n(num_graphs);
  for (int g = 0; g < num_graphs; ++g) inv_n[g] = 1.0 / (double)(graph_offsets[g + 1] - graph_offsets[g]);
  const size_t G = (size_t)num_graphs;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** q, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(q, bytes); };
  A((void**)&b->off, sizeof(int32_t) * (G + 1));
  A((void**)&b->inv_n, sizeof(double) * G);
  A((void**)&b->dang0, sizeof(double) * G);
  A((void**)&b->D, sizeof(double) * G);
  A((void**)&b->conv, sizeof(int) * G);
  A((void**)&b->acc, sizeof(double) * 2 * G);
  A((void**)&b->last_r, sizeof(double) * G);
  A((void**)&b->bs, sizeof(BatchState));
  A((void**)&b->blist, sizeof(int32_t) * (size_t)std::max<int64_t>(p->nb, 1));
  A((void**)&b->bcount, sizeof(int));
  A((void**)&b->bflags, (size_t)std::max<int64_t>(p->nb, 1));
  A((void**)&b->ccount, sizeof(int) * (size_t)std::max<int64_t>((p->nb + kCompactChunk - 1) / kCompactChunk, 1));
  unsigned long long* cnt = nullptr;
  int* err = nullptr;
  A((void**)&cnt, sizeof(unsigned long long) * G);
  A((void**)&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->off, off32.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->inv_n, inv_n.data(), sizeof(double) * G, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * G, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  unsigned long long ndang = 0;
  if (e == cudaSuccess && p->n_dangling < 0) {
    e = build_dangling(p, st, &ndang);
    if (e == cudaSuccess) p->n_dangling = (int64_t)ndang;
  }
  if (e == cudaSuccess) {
    batch_dangling_count_kernel<<<grid_rows(n, p->num_sms), 256, 0, st>>>(p->dangling_bits, b->off,
                                                                         num_graphs, n, cnt);
    if (p->lane_num > 0)
      batch_validate_kernel<<<grid_rows(p->lane_num, p->num_sms), 256, 0, st>>>(p->geom(), b->off,
                                                                               num_graphs, err);
    e = cudaGetLastError();
  }
  std::vector<unsigned long long> cnt_h(G);
  int err_h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt_h.data(), cnt, sizeof(unsigned long long) * G, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err_h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  std::vector<double> d0(G);
  for (size_t g = 0; g < G; ++g) d0[g] = (double)cnt_h[g] * inv_n[g];
  if (e == cudaSuccess) e = cudaMemcpy(b->dang0, d0.data(), sizeof(double) * G, cudaMemcpyHostToDevice);
  cudaFree(cnt);
  cudaFree(err);
  if (e != cudaSuccess) {
    free_batch(b);
    return bfail(e == cudaErrorMemoryAllocation ? MERBIT_ENOMEM : MERBIT_ECUDA, "merbit_batch_plan: %s",
                 cudaGetErrorString(e));
  }
  if (err_h) {
    free_batch(b);
    return bfail(MERBIT_EINVAL, "the matrix is not block diagonal: a nonzero links two graphs");
  }
  *out = b;
  return MERBIT_OK;
}

merbit_status merbit_batch_pagerank(merbit_batch_t b, merbit_dtype dtype, const void* vals,
                                    double alpha, double tol, int max_iter, void* pi,
                                    int* iters, double* resid, int* rounds_out, void* stream) {
  set_last_error("");
  if (!b) return bfail(MERBIT_EINVAL, "batch is NULL");
  if (dtype != MERBIT_F32 && dtype != MERBIT_F64) return bfail(MERBIT_EINVAL, "dtype must be F32 or F64");
  if (!(alpha >= 0.0 && alpha < 1.0)) return bfail(MERBIT_EINVAL, "alpha must be in [0, 1)");
  if (max_iter < 1) return bfail(MERBIT_EINVAL, "max_iter must be >= 1");
  if (!pi || (b->plan->nnz > 0 && !vals)) return bfail(MERBIT_EINVAL, "vals or pi is NULL");
  if (b->plan->nnz > 0 && (reinterpret_cast<uintptr_t>(vals) & 15))
    return bfail(MERBIT_EINVAL, "vals must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t es = dtype == MERBIT_F64 ? 8 : 4;
  cudaError_t e = cudaSuccess;
  const bool same = b->exec && b->dt == dtype && b->vals == vals && b->pi == pi && b->alpha == alpha &&
                    b->tol == tol && b->max_iter == max_iter && b->spmv_kernel == b->plan->spmv_kernel &&
                    b->hot_list == b->plan->hot_list && b->col_hot == b->plan->col_hot &&
                    b->hot_n == b->plan->hot_n;
  if (!same) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    if (b->x1_bytes < es * (size_t)b->n) {
      cudaFree(b->x1);
      b->x1 = nullptr;
      b->x1_bytes = 0;
      e = cudaMalloc(&b->x1, es * (size_t)std::max<int64_t>(b->n, 1));
      if (e == cudaSuccess) b->x1_bytes = es * (size_t)b->n;
    }
    cudaStream_t cap = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
      e = dtype == MERBIT_F64
              ? record_solve<double>(b, static_cast<const double*>(vals), static_cast<double*>(pi), alpha, tol, max_iter, cap)
              : record_solve<float>(b, static_cast<const float*>(vals), static_cast<float*>(pi), alpha, tol, max_iter, cap);
      cudaStreamDestroy(cap);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
      if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
      b->exec = nullptr;
      return bfail(MERBIT_ECUDA, "recording the batched solve: %s", cudaGetErrorString(e));
    }
    b->dt = dtype;
    b->vals = vals;
    b->pi = pi;
    b->alpha = alpha;
    b->tol = tol;
    b->max_iter = max_iter;
    b->spmv_kernel = b->plan->spmv_kernel;
    b->hot_list = b->plan->hot_list;
    b->col_hot = b->plan->col_hot;
    b->hot_n = b->plan->hot_n;
  }
  e = cudaGraphLaunch(b->exec, st);
  std::vector<int> conv((size_t)b->G);
  BatchState bs{};
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(conv.data(), b->conv, sizeof(int) * (size_t)b->G, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bs, b->bs, sizeof(BatchState), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &b->plan->red->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && resid)
    e = cudaMemcpyAsync(resid, b->last_r, sizeof(double) * (size_t)b->G, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bfail(MERBIT_ECUDA, "batched solve: %s", cudaGetErrorString(e));
  if (err) {
    cudaMemsetAsync(b->plan->red, 0, sizeof(RedState), st);
    cudaStreamSynchronize(st);
    return bfail(MERBIT_EDEVICE, "a kernel reported error bits 0x%x", err);
  }
  int open = 0;
  for (int g = 0; g < b->G; ++g) {
    if (iters) iters[g] = conv[g] >= 0 ? conv[g] : bs.round;
    open += conv[g] < 0;
  }
  if (rounds_out) *rounds_out = bs.round;
  if (tol > 0 && open)
    return bfail(MERBIT_ENOTCONV, "%d of %d graphs did not reach tol %.3g in %d rounds", open, b->G,
                 tol, max_iter);
  return MERBIT_OK;
}

void merbit_batch_destroy(merbit_batch_t b) { free_batch(b); }

merbit_plan_t merbit_batch_get_plan(merbit_batch_t b) { return b ? b->plan : nullptr; }

}  // extern "C"
