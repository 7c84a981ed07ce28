// MERBIT SpMV kernel for sm_103a (Sec. 4.2: Algorithms MERBIT SpMV,
// tile_normal_tackle, WarpSegmentedSum) with a pluggable row epilogue.
//
// Work unit: a block of W = 8 consecutive tiles (omega*sigma merge-path steps
// each), one warp per tile, exactly as in the paper.  GB300-specific choices:
//   * persistent CTAs (grid = SMs x resident CTAs) walk the blocks with a
//     stride, with two shared-memory stages: while block v is reduced, the
//     values and column indices of the CTA's next block are already in flight
//     as two cp.async.bulk copies completing on an mbarrier (the block's
//     nonzero range is contiguous, so one bulk copy per array suffices);
//   * matrix streams use an L2 evict_first policy, the x gather an
//     evict_last policy (x is reused by every block and, in PageRank, by the
//     next launch);
//   * products overwrite the staged values (or column indices for 16-bit
//     values) in place and the block's row partial sums follow them, so one
//     stage holds W*omega*sigma + 16 elements of each array (Sec. 4.3's
//     (b+1)*sigma bound, re-derived for this layout);
//   * rows shared between blocks (the block's first and last row) are added
//     into per-row FP64 accumulators with fire-and-forget atomics; a small
//     second kernel writes those rows, clears the accumulators and finishes the
//     grid-wide FP64 reductions, so outputs are written exactly once and no
//     vector ever needs clearing between calls (the role of the paper's
//     dual-buffer commit, which resets only block-boundary rows).
#pragma once

#include <algorithm>

#include "merbit_internal.cuh"

namespace merbit {

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for an mbarrier phase with an iteration cap; false if the cap expired.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ float ld_x(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ double ld_x(const double* p, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float widen(__half v) { return __half2float(v); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ bool is_dangling(const uint32_t* bits, int r) {
  return (__ldg(bits + (r >> 5)) >> (r & 31)) & 1u;
}

__device__ __forceinline__ double read_reset(double* p) {
  return __longlong_as_double(
      static_cast<long long>(atomicExch(reinterpret_cast<unsigned long long*>(p), 0ull)));
}

// ---------------------------------------------------------------- epilogues
// row(r, s)   : complete sum s of interior row r (accumulator type)
// row64(r, s) : complete FP64 sum of a block-boundary row
// Each may add to the two FP64 reduction partials p0, p1.

template <typename XT, typename AT>
struct EpiPlain {
  static constexpr bool kReduce = false;
  XT* y;
  AT scale;
  __device__ __forceinline__ void init() {}
  __device__ __forceinline__ bool skip(const RedState*) const { return false; }
  __device__ __forceinline__ void row(int r, AT s, double&, double&) const {
    y[r] = static_cast<XT>(s * scale);
  }
  __device__ __forceinline__ void row64(int r, double s, double&, double&) const {
    y[r] = static_cast<XT>(s * static_cast<double>(scale));
  }
  __device__ __forceinline__ void finish(double, double, RedState*) const {}
};

// pi_{k+1}[r] = alpha * (P^T pi_k)[r] + (alpha D_k + 1 - alpha) / n   (Sec. 5.5.1)
template <typename T>
struct EpiPageRank {
  static constexpr bool kReduce = true;
  PRParams p;
  const T* xold;
  T a, c;
  double cd;
  __device__ __forceinline__ void init() {
    const double D = *p.d_in;
    cd = (p.alpha * D + 1.0 - p.alpha) * p.inv_n;
    a = static_cast<T>(p.alpha);
    c = static_cast<T>(cd);
  }
  __device__ __forceinline__ bool skip(const RedState* red) const {
    return *reinterpret_cast<const volatile int*>(&red->done) != 0;
  }
  __device__ __forceinline__ void put(int r, T v, double& p0, double& p1) const {
    static_cast<T*>(p.out)[r] = v;
    p0 += fabs(static_cast<double>(v) - static_cast<double>(xold[r]));
    if (is_dangling(p.dang, r)) p1 += static_cast<double>(v);
  }
  __device__ __forceinline__ void row(int r, T s, double& p0, double& p1) const {
    put(r, a * s + c, p0, p1);
  }
  __device__ __forceinline__ void row64(int r, double s, double& p0, double& p1) const {
    put(r, static_cast<T>(p.alpha * s + cd), p0, p1);
  }
  __device__ __forceinline__ void finish(double A, double B, RedState* red) const {
    p.s_out[0] = A;
    p.s_out[1] = B;
    ++red->launches;
    if (p.tol > 0.0 && A < p.tol) {
      red->iters = p.iter + 1;
      red->done = 1;
    }
  }
};

// r = (1-alpha)/n + alpha (P^T pi) + (alpha/n) D_pi - pi   (FP64)
struct EpiResid {
  static constexpr bool kReduce = true;
  ResidParams p;
  const double* pi;
  double base;
  __device__ __forceinline__ void init() {
    base = (1.0 - p.alpha) * p.inv_n + p.alpha * p.inv_n * (*p.d_in);
  }
  __device__ __forceinline__ bool skip(const RedState* red) const {
    return *reinterpret_cast<const volatile int*>(&red->done) != 0;
  }
  __device__ __forceinline__ void row64(int r, double s, double& p0, double& p1) const {
    const double rr = base + p.alpha * s - pi[r];
    const float rf = static_cast<float>(rr);
    p.rhs[r] = rf;
    p0 += fabs(rr);
    if (is_dangling(p.dang, r)) p1 += static_cast<double>(rf);
  }
  __device__ __forceinline__ void row(int r, double s, double& p0, double& p1) const {
    row64(r, s, p0, p1);
  }
  __device__ __forceinline__ void finish(double A, double B, RedState* red) const {
    p.s_out[0] = A;
    p.s_out[1] = B;
    ++red->launches;
    red->delta = p.rhs;           // the first inner iterate is r itself
    red->inner_done = 0;
    if (A < p.tol) {
      red->iters = p.iter + 1;
      red->done = 1;
    }
  }
};

// delta'[r] = alpha 2^-k (P~^T delta)[r] + (alpha/n) D_delta + rhs[r]
struct EpiSweep {
  static constexpr bool kReduce = true;
  SweepParams p;
  const float* xin;
  float as, c;
  __device__ __forceinline__ void init() {
    as = static_cast<float>(p.alpha) * p.scale;
    c = static_cast<float>(p.alpha * p.inv_n * (*p.d_in));
  }
  __device__ __forceinline__ bool skip(const RedState* red) const {
    return *reinterpret_cast<const volatile int*>(&red->done) != 0 ||
           *reinterpret_cast<const volatile int*>(&red->inner_done) != 0;
  }
  __device__ __forceinline__ void put(int r, float d, double& p0, double& p1) const {
    p.out[r] = d;
    p0 += fabs(static_cast<double>(d) - static_cast<double>(xin[r]));
    if (is_dangling(p.dang, r)) p1 += static_cast<double>(d);
  }
  __device__ __forceinline__ void row(int r, float s, double& p0, double& p1) const {
    put(r, as * s + (c + p.rhs[r]), p0, p1);
  }
  __device__ __forceinline__ void row64(int r, double s, double& p0, double& p1) const {
    put(r, static_cast<float>(static_cast<double>(as) * s) + (c + p.rhs[r]), p0, p1);
  }
  __device__ __forceinline__ void finish(double A, double B, RedState* red) const {
    p.s_out[0] = A;
    p.s_out[1] = B;
    ++red->launches;
    red->delta = p.out;
    if (A <= p.eta * (*p.rnorm)) red->inner_done = 1;
  }
};

// ---------------------------------------------------------------- kernel
//
// One persistent CTA per SM, three warp roles connected by mbarriers over a
// ring of kStages shared-memory stages (each stage holds one block of tiles):
//   producer warp (1)  : bulk copies of the block's values and column indices
//                        (full[s] completes when both have landed);
//   gather warps (4)   : one cp.async per nonzero, x[col[k]] -> xs[s][k]
//                        (gathered[s] completes when every gather has landed);
//   compute warps (8)  : one tile per warp: descriptor-driven lane scan over
//                        vals[k] * xs[k], warp segmented sum, then the block
//                        commit (empty[s] releases the stage to the producer).
// The gathers of later blocks stay in flight while earlier blocks are reduced,
// and no register holds a gathered value.

constexpr int kComputeWarps = kTilesPerBlock;
constexpr int kGatherWarps = 4;
constexpr int kComputeThreads = kComputeWarps * 32;
constexpr int kGatherThreads = kGatherWarps * 32;
constexpr int kProducerWarp = kComputeWarps + kGatherWarps;
constexpr int kCtaThreads = (kProducerWarp + 1) * 32;
constexpr int kStagePad = 32;

struct StageInfo {
  int x_bs, x_be, y_bs, y_be;   // block start / end coordinates
  int a0, end;                  // values and column indices staged for [a0, end)
};

// Both bulk-copied arrays start at a multiple of A elements, so that values and
// column indices start on 16-byte boundaries (bulk-copy rule).
template <typename VT>
__host__ __device__ constexpr int stage_align() {
  return (16 / (int)sizeof(VT)) > 4 ? 16 / (int)sizeof(VT) : 4;
}

__host__ __device__ inline size_t round128(size_t b) { return (b + 127) & ~size_t(127); }

// Stage layout: vals[cap] | col[cap] | xs[cap] | s_y[cap], cap = 256*sigma + 32.
template <typename VT, typename XT, typename AT>
struct Layout {
  size_t col_off, xs_off, sy_off, bytes;
  __host__ __device__ explicit Layout(int sigma) {
    const size_t cap = (size_t)kComputeThreads * sigma + kStagePad;
    col_off = round128(cap * sizeof(VT));
    xs_off = col_off + round128(cap * sizeof(int32_t));
    sy_off = xs_off + round128(cap * sizeof(XT));
    bytes = sy_off + round128(cap * sizeof(AT));
  }
};

// As many stages (2 or 3) as fit in 200 KB at the largest sigma.
template <typename VT, typename XT, typename AT>
__host__ __device__ constexpr int stages_for() {
  return 3 * ((size_t)kComputeThreads * kSigmaMax + kStagePad) *
                     (sizeof(VT) + sizeof(int32_t) + sizeof(XT) + sizeof(AT)) + 3 * 512 <=
                 200 * 1024
             ? 3
             : 2;
}

__device__ __forceinline__ void cp_async_gather(void* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_gather(void* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
// the mbarrier receives one arrival once all of this thread's earlier cp.async have landed
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// barrier 1 among the compute warps only
__device__ __forceinline__ void compute_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kComputeThreads) : "memory");
}
// barrier 1 among the compute warps, returning whether any of them passes true
__device__ __forceinline__ bool compute_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kComputeThreads)
      : "memory");
  return r != 0;
}

// Per-warp tile metadata, loaded one block ahead.
struct TileMeta {
  uint32_t txs, txe, tys, desc;
};

template <typename VT, typename XT, typename AT, typename Epi>
__global__ void __launch_bounds__(kCtaThreads, 1)
    merbit_spmv_kernel(const Geometry g, const VT* __restrict__ vals, const XT* __restrict__ x,
                       Epi epi) {
  constexpr int A = stage_align<VT>();
  constexpr int S = stages_for<VT, XT, AT>();
  __shared__ __align__(8) uint64_t full[S], gathered[S], empty[S];
  __shared__ StageInfo info[S];
  __shared__ double red_smem[kComputeWarps][2];
  extern __shared__ __align__(128) unsigned char dyn_smem[];

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int G = gridDim.x;
  const int v0 = blockIdx.x;
  if (epi.skip(g.red)) return;

  const Layout<VT, XT, AT> L(g.sigma);
  auto sv = [&](int s) { return reinterpret_cast<VT*>(dyn_smem + (size_t)s * L.bytes); };
  auto sc = [&](int s) { return reinterpret_cast<int32_t*>(dyn_smem + (size_t)s * L.bytes + L.col_off); };
  auto sx = [&](int s) { return reinterpret_cast<XT*>(dyn_smem + (size_t)s * L.bytes + L.xs_off); };
  auto sy = [&](int s) { return reinterpret_cast<AT*>(dyn_smem + (size_t)s * L.bytes + L.sy_off); };
  // block b of this CTA is v0 + b*G, in stage b % S for the (b / S)-th time
  auto nblocks = [&]() { return v0 < g.nb ? (g.nb - 1 - v0) / G + 1 : 0; };
  const int nbk = nblocks();

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&gathered[s], kGatherThreads);
      mbar_init(&empty[s], kComputeThreads);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kProducerWarp) {
    // ------------------------------------------------------------ producer
    if (lane != 0) return;
    const uint64_t pol_stream = policy_evict_first();
    const int nnz_a = g.nnz & ~(A - 1);
    int b = 0;
    bool ok = true;
    for (; b < nbk; ++b) {
      const int s = b % S;
      if (b >= S && !mbar_wait_bounded(&empty[s], (uint32_t)((b / S - 1) & 1))) {
        atomicOr(&g.red->err, 1);
        ok = false;
        break;
      }
      const int v = v0 + b * G;
      const int bs = v * kTilesPerBlock;
      const int be = min(bs + kTilesPerBlock, g.tile_num);
      StageInfo in;
      in.x_bs = (int)g.tile_x[bs];
      in.x_be = (int)g.tile_x[be];
      in.y_bs = (int)(g.tile_y[bs] & ~kMsb);
      in.y_be = (int)(g.tile_y[be] & ~kMsb);
      in.a0 = in.x_bs & ~(A - 1);
      in.end = max(in.a0, min((in.x_be + A - 1) & ~(A - 1), nnz_a));
      info[s] = in;
      const uint32_t cnt = (uint32_t)(in.end - in.a0);
      mbar_arrive_expect_tx(&full[s], cnt * (uint32_t)(sizeof(VT) + sizeof(int32_t)));
      if (cnt) {
        bulk_g2s(sv(s), vals + in.a0, cnt * (uint32_t)sizeof(VT), &full[s], pol_stream);
        bulk_g2s(sc(s), g.col + in.a0, cnt * 4u, &full[s], pol_stream);
      }
    }
    if (!ok) {
      // let the copies already issued land before this CTA can retire
      for (int q = max(0, b - S); q < b; ++q) mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1));
    }
    return;
  }

  if (warp >= kComputeWarps) {
    // ------------------------------------------------------------ gather warps
    const int gt = tid - kComputeThreads;
    const uint64_t pol_x = policy_evict_last();
    (void)pol_x;
    for (int b = 0; b < nbk; ++b) {
      const int s = b % S;
      if (!mbar_wait_bounded(&full[s], (uint32_t)((b / S) & 1))) {
        atomicOr(&g.red->err, 1);
        break;
      }
      const StageInfo in = info[s];
      const int32_t* col_s = sc(s);
      XT* xs = sx(s);
      const int e0 = in.x_bs - in.a0, e1 = in.x_be - in.a0;
      if (in.a0 + e1 <= in.end) {
#pragma unroll 4
        for (int e = e0 + gt; e < e1; e += kGatherThreads) cp_async_gather(xs + e, x + col_s[e]);
      } else {
        for (int e = e0 + gt; e < e1; e += kGatherThreads) {
          const int k = in.a0 + e;
          cp_async_gather(xs + e, x + (k < in.end ? col_s[e] : __ldg(g.col + k)));
        }
      }
      cp_async_arrive(&gathered[s]);
    }
    cp_async_wait_all();
    return;
  }

  // -------------------------------------------------------------- compute warps
  epi.init();
  auto meta_of = [&](int b) {
    TileMeta m{0u, 0u, 0u, 0u};
    const int v = v0 + b * G;
    const int ti = v * kTilesPerBlock + warp;
    if (b < nbk && ti < g.tile_num) {
      const uint64_t pol = policy_evict_first();
      m.txs = __ldg(g.tile_x + ti);
      m.txe = __ldg(g.tile_x + ti + 1);
      m.tys = __ldg(g.tile_y + ti);
      const int j = ti * kOmega + lane;
      if (!(m.tys & kMsb) && j < g.lane_num) m.desc = ld_stream(g.lane_desc + j, pol);
    }
    return m;
  };
  double p0 = 0.0, p1 = 0.0;
  TileMeta meta = meta_of(0);
  for (int b = 0; b < nbk; ++b) {
    const int s = b % S;
    const int v = v0 + b * G;
    const TileMeta cur = meta;
    meta = meta_of(b + 1);                       // next block's tile metadata
    const uint32_t par = (uint32_t)((b / S) & 1);
    const bool ok = mbar_wait_bounded(&gathered[s], par) && mbar_wait_bounded(&full[s], par);
    const StageInfo in = info[s];
    AT* s_y = sy(s);
    if (ok)
      for (int r = tid; r <= in.y_be - in.y_bs; r += kComputeThreads) s_y[r] = AT(0);
    if (compute_sync_or(!ok)) {
      if (tid == 0) atomicOr(&g.red->err, 1);
      return;
    }
    const VT* vs = sv(s);
    const XT* xs = sx(s);
    // a product of the block: staged index i = k - a0; the array's last values may be
    // unstaged (only in the block holding them)
    const bool tail = in.end < in.x_be;
    auto prod = [&](int i) -> AT {
      if (!tail || in.a0 + i < in.end) return static_cast<AT>(widen(vs[i])) * static_cast<AT>(xs[i]);
      // unstaged tail: the index is clamped so that steps whose product is discarded
      // (down steps, the lane's end) never read past the array
      const VT w = vals[min(in.a0 + i, g.nnz - 1)];
      return static_cast<AT>(widen(w)) * static_cast<AT>(xs[i]);
    };

    const int ti = v * kTilesPerBlock + warp;
    const int j = ti * kOmega + lane;
    if (ti < g.tile_num && cur.txs < cur.txe) {
      const int y_ws = (int)(cur.tys & ~kMsb);
      AT* syt = s_y + (y_ws - in.y_bs);
      const int i0 = (int)cur.txs - in.a0;        // staged index of the tile's first nonzero
      if (cur.tys & kMsb) {
        // single-row tile (tile_fast_tackle): plain warp reduction, no descriptor
        AT sum = AT(0);
        const int len = (int)(cur.txe - cur.txs);
#pragma unroll
        for (int q = 0; q < kSigmaMax; ++q) {
          const int k = lane + 32 * q;
          if (k < len) sum += prod(i0 + k);
        }
        for (int k = lane + 32 * kSigmaMax; k < len; k += 32) sum += prod(i0 + k);
        sum = warp_sum(sum);
        if (lane == 0) atomicAdd(syt, sum);
      } else {
        // tile_normal_tackle: sigma steps of this lane, driven by its descriptor
        const bool active = j < g.lane_num;
        const int lane_len = active ? min(g.sigma, g.steps - j * g.sigma) : 0;
        const uint32_t valid = (1u << lane_len) - 1u;
        const uint32_t dm = (cur.desc >> 18) & valid;     // down steps
        const uint32_t rm = ~(cur.desc >> 18) & valid;    // right steps
        const int y0 = active ? (int)((cur.desc >> 9) & 511u) : (g.n_rows - y_ws);
        const int il = i0 + (int)(cur.desc & 511u);       // staged index of the lane's first nonzero
        // step k consumes nonzero k - (down steps before k): the addresses follow from
        // the descriptor alone, so all loads are issued before any addition or flush
        AT pv[kSigmaMax];
#pragma unroll
        for (int k = 0; k < kSigmaMax; ++k) pv[k] = prod(il + k - __popc(dm & ((1u << k) - 1u)));
        AT sum = AT(0);
#pragma unroll
        for (int k = 0; k < kSigmaMax; ++k) {
          const int nd = __popc(dm & ((1u << k) - 1u));
          if ((dm >> k) & 1u) {
            // down step: row y0 + nd ends here; only the lane's first such row can
            // have begun in an earlier lane, so only that one needs an atomic add
            if (nd == 0) atomicAdd(syt + y0, sum);
            else syt[y0 + nd] = sum;
            sum = AT(0);
          } else if ((rm >> k) & 1u) {
            sum += pv[k];
          }
        }
        const int yo = y0 + __popc(dm);
        const bool head = lane == 0 || dm != 0u;
        // WarpSegmentedSum: segmented inclusive scan of trailing sums; heads start segments
        AT sv_ = sum;
        int f = head ? 1 : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          if (__all_sync(0xffffffffu, f)) break;
          const AT up = __shfl_up_sync(0xffffffffu, sv_, o);
          const int fu = __shfl_up_sync(0xffffffffu, f, o);
          if (lane >= o && !f) {
            sv_ += up;
            f = fu;
          }
        }
        // a head lane adds the segment that ends just before it; lane 0 takes the
        // tile's final segment (ending at lane 31)
        const int src = lane == 0 ? 31 : lane - 1;
        const AT seg = __shfl_sync(0xffffffffu, sv_, src);
        const int row = __shfl_sync(0xffffffffu, yo, src);
        if (head) atomicAdd(syt + row, seg);
      }
    }
    compute_sync();

    // block commit: interior rows complete here, boundary rows into FP64 accumulators
    for (int r = in.y_bs + 1 + tid; r < in.y_be; r += kComputeThreads)
      epi.row(r, s_y[r - in.y_bs], p0, p1);
    if (tid == 0) atomicAdd(g.bnd_acc + __ldg(g.bnd_slot + v), static_cast<double>(s_y[0]));
    if (tid == 32 && in.y_be != in.y_bs && in.y_be < g.n_rows)
      atomicAdd(g.bnd_acc + __ldg(g.bnd_slot + v + 1), static_cast<double>(s_y[in.y_be - in.y_bs]));
    mbar_arrive(&empty[s]);                     // this thread is done with stage s
  }

  if constexpr (Epi::kReduce) {
    p0 = warp_sum(p0);
    p1 = warp_sum(p1);
    if (lane == 0) {
      red_smem[warp][0] = p0;
      red_smem[warp][1] = p1;
    }
    compute_sync();
    if (tid == 0) {
      double a = 0.0, b2 = 0.0;
#pragma unroll
      for (int w = 0; w < kComputeWarps; ++w) {
        a += red_smem[w][0];
        b2 += red_smem[w][1];
      }
      g.part[blockIdx.x] = make_double2(a, b2);
    }
  }
}

// Grid-wide FP64 sums of (p0, p1) over a launch of blockDim.x <= 256 threads:
// block sums go to spread slots, and the last CTA to arrive adds the slots in a
// fixed order, clears them and calls finish(A, B).
template <typename F>
__device__ __forceinline__ void grid_sum2(double p0, double p1, RedState* red, F finish) {
  __shared__ double red_smem[8][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  p0 = warp_sum(p0);
  p1 = warp_sum(p1);
  if (lane == 0) {
    red_smem[warp][0] = p0;
    red_smem[warp][1] = p1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      a += red_smem[w][0];
      b += red_smem[w][1];
    }
    const int q = blockIdx.x % kRedSlots;
    atomicAdd(&red->slot[q][0], a);
    atomicAdd(&red->slot[q][1], b);
    __threadfence();
    if (atomicAdd(&red->arrive, 1u) + 1 == gridDim.x) {
      __threadfence();
      double A = 0.0, B = 0.0;
      for (int i = 0; i < kRedSlots; ++i) {
        A += read_reset(&red->slot[i][0]);
        B += read_reset(&red->slot[i][1]);
      }
      red->arrive = 0u;
      finish(A, B);
    }
  }
}

// Second pass: rows shared between blocks (one thread per distinct boundary
// row: the FP64 total of its accumulator goes through the epilogue, and the
// accumulator is cleared), then the grid-wide FP64 reductions: per-CTA
// partials of both kernels are summed by the last CTA of this kernel.
template <typename Epi>
__global__ void __launch_bounds__(256) merbit_finalize_kernel(const Geometry g, Epi epi,
                                                              int nparts) {
  if (epi.skip(g.red)) return;
  epi.init();
  double p0 = 0.0, p1 = 0.0;
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  for (int k = t0; k <= g.nb; k += stride) {
    if (__ldg(g.bnd_slot + k) != k) continue;
    const int r = __ldg(g.bnd_row + k);
    if (r >= g.n_rows) continue;
    const double tot = g.bnd_acc[k];
    g.bnd_acc[k] = 0.0;
    epi.row64(r, tot, p0, p1);
  }
  if constexpr (Epi::kReduce) {
    for (int i = t0; i < nparts; i += stride) {
      const double2 q = g.part[i];
      p0 += q.x;
      p1 += q.y;
    }
    grid_sum2(p0, p1, g.red, [&](double A, double B) { epi.finish(A, B, g.red); });
  }
}

template <typename VT, typename XT, typename AT, typename Epi>
cudaError_t launch_spmv(const merbit_plan_s* p, const VT* vals, const XT* x, const Epi& epi,
                        cudaStream_t st) {
  if (p->nb == 0) return cudaSuccess;
  constexpr int S = stages_for<VT, XT, AT>();
  auto kern = merbit_spmv_kernel<VT, XT, AT, Epi>;
  const size_t smem = S * Layout<VT, XT, AT>(p->sigma).bytes;
  const size_t smem_max = S * Layout<VT, XT, AT>(kSigmaMax).bytes;
  int grid = persistent_grid(reinterpret_cast<const void*>(kern), kCtaThreads, smem, smem_max,
                             p->num_sms);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  if ((int64_t)grid > p->nb) grid = (int)p->nb;
  if (grid > kMaxParts) grid = kMaxParts;
  kern<<<grid, kCtaThreads, smem, st>>>(p->geom(), vals, x, epi);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int fgrid = (int)std::min<int64_t>((p->nb + 1 + 255) / 256, (int64_t)p->num_sms * 4);
  merbit_finalize_kernel<Epi><<<fgrid, 256, 0, st>>>(p->geom(), epi, Epi::kReduce ? grid : 0);
  return cudaGetLastError();
}

}  // namespace merbit
