// MERBIT SpMV kernels for sm_103a (Sec. 4.2: Algorithms MERBIT SpMV,
// tile_normal_tackle, WarpSegmentedSum) with a pluggable row epilogue.
//
// Work unit: a block of W = 8 consecutive tiles (omega*sigma merge-path steps
// each), one warp per tile, exactly as in the paper.  GB300-specific choices:
//   * persistent CTAs (grid = SMs x resident CTAs) walk the blocks with a
//     stride; a block's values and column indices arrive in shared memory as
//     two cp.async.bulk copies completing on an mbarrier, issued ahead of use
//     (the block's nonzero range is contiguous, so one bulk copy per array
//     suffices);
//   * two block kernels share the stages and the per-tile reduction:
//     merbit_spmv_kernel (all threads gather, then all reduce; two stages) and
//     merbit_spmv_split_kernel (producer threads gather for the next blocks
//     while consumer threads reduce the current one; a ring of three or two
//     stages), which keeps the SM's gather path busy and is the default where two
//     CTAs fit per SM;
//   * matrix streams use an L2 evict_first policy, the x gather an
//     evict_last policy (x is reused by every block and, in PageRank, by the
//     next launch);
//   * products overwrite the staged values (or column indices for 16-bit
//     values) in place and the block's row partial sums follow them, so one
//     stage holds W*omega*sigma + 32 elements of each array (Sec. 4.3's
//     (b+1)*sigma bound, re-derived for this layout);
//   * rows shared between blocks (the block's first and last row) are added
//     into per-row FP64 accumulators with fire-and-forget atomics; a small
//     second kernel writes those rows, clears the accumulators and finishes the
//     grid-wide FP64 reductions, so outputs are written exactly once and no
//     vector ever needs clearing between calls (the role of the paper's
//     dual-buffer commit, which resets only block-boundary rows).
#pragma once

#include <algorithm>
#include <type_traits>
#include <utility>

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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
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
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint32_t limit = kSpinLimit) {
  for (uint32_t i = 0; i < limit; ++i)
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

// The gather of x[c] when `pred` holds; v keeps its value otherwise (no access is made).
__device__ __forceinline__ void ld_x_if(float& v, const float* p, bool pred, uint64_t pol) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t"
      "@q ld.global.nc.L2::cache_hint.f32 %0, [%1], %3;\n\t}"
      : "+f"(v)
      : "l"(p), "r"((uint32_t)pred), "l"(pol));
}

__device__ __forceinline__ void ld_x_if(double& v, const double* p, bool pred, uint64_t pol) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t"
      "@q ld.global.nc.L2::cache_hint.f64 %0, [%1], %3;\n\t}"
      : "+d"(v)
      : "l"(p), "r"((uint32_t)pred), "l"(pol));
}

// x[c] for a column c of the staged column stream.  With a hot-column table (HOT), c < 0
// names table slot ~c, whose value this CTA holds in shared memory (tab); the other
// columns are gathered from x in global memory.
template <bool HOT, typename XT>
__device__ __forceinline__ XT gather_x(int c, const XT* x, const XT* tab, uint64_t pol_x) {
  if constexpr (HOT) {
    const bool hot = c < 0;
    XT v = XT(0);
    if (hot) v = tab[~c];
    ld_x_if(v, x + c, !hot, pol_x);
    return v;
  } else {
    return ld_x(x + c, pol_x);
  }
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

// An epilogue with members block_list / block_count makes the kernel process only the
// listed blocks (*block_count of them, read at kernel start): iterative drivers use it to
// skip blocks whose rows no longer change.
template <typename E, typename = void>
struct HasBlockList : std::false_type {};
template <typename E>
struct HasBlockList<E, std::void_t<decltype(std::declval<E&>().block_list)>> : std::true_type {};

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
  double cd;
  __device__ __forceinline__ void init() {
    const double D = *p.d_in;
    cd = (p.alpha * D + 1.0 - p.alpha) * p.inv_n;
  }
  __device__ __forceinline__ bool skip(const RedState* red) const {
    return *reinterpret_cast<const volatile int*>(&red->done) != 0;
  }
  // The step is measured on the update before it is rounded to T: once an FP32 iterate
  // stops changing (each entry rounds back to itself), the rounded step reads 0 although
  // the iterate is still about one rounding away from the fixed point, and a tolerance
  // below that floor must not be reported as reached.
  __device__ __forceinline__ void put(int r, double vd, double& p0, double& p1) const {
    const T v = static_cast<T>(vd);
    static_cast<T*>(p.out)[r] = v;
    p0 += fabs(vd - static_cast<double>(xold[r]));
    if (is_dangling(p.dang, r)) p1 += static_cast<double>(v);
  }
  __device__ __forceinline__ void row(int r, T s, double& p0, double& p1) const {
    put(r, fma(p.alpha, static_cast<double>(s), cd), p0, p1);
  }
  __device__ __forceinline__ void row64(int r, double s, double& p0, double& p1) const {
    put(r, fma(p.alpha, s, cd), p0, p1);
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

struct StageInfo {
  int x_bs, x_be, y_bs, y_be;   // block start / end coordinates
  int a0v, endv;                // values staged for [a0v, endv)
  int a0c, endc;                // column indices staged for [a0c, endc)
};

// Elements of a stage: the W * omega * sigma steps of a block (its nonzeros, then its row
// sums) plus 32, since the lane scan may read up to 13 past the last product.
template <typename VT>
__host__ __device__ constexpr int stage_cap(int sigma, int W) {
  return W * kOmega * sigma + 32;
}

__host__ __device__ inline size_t round128(size_t b) { return (b + 127) & ~size_t(127); }

// A matrix whose stored values are all 1 (an adjacency pattern): no value stream is read
// and a nonzero's product is x[col].  The type has the accumulator's width, so the
// products take the place the values would have had in the stage.
template <typename AT>
struct UnitVal {
  AT pad;
};
template <typename T>
struct IsUnit : std::false_type {};
template <typename AT>
struct IsUnit<UnitVal<AT>> : std::true_type {};

// Products go where an input of the same width was staged (the values, or the pattern's
// product slots), else over the column indices (16-bit values).
template <typename VT, typename AT>
struct ProdInVals {
  static constexpr bool value = sizeof(VT) == sizeof(AT);
};

template <typename VT>
__host__ __device__ inline size_t stage_vals_bytes(int sigma, int W) {
  return round128(sizeof(VT) * (size_t)stage_cap<VT>(sigma, W));
}
template <typename VT>
__host__ __device__ inline size_t stage_col_bytes(int sigma, int W) {
  return round128(sizeof(int32_t) * (size_t)stage_cap<VT>(sigma, W));
}
template <typename VT>
__host__ __device__ inline size_t stage_bytes(int sigma, int W) {
  return stage_vals_bytes<VT>(sigma, W) + stage_col_bytes<VT>(sigma, W);
}

// A block's coordinate range: nonzeros [xb, xe) and rows [yb, ye] (the tiles'
// start coordinates of its first and one-past-last tile).
struct BlockSpan {
  int xb, xe;
  uint32_t yb, ye;
};

// The shared-memory stages of a block kernel and the bulk copies that fill them.  Stage
// s holds a block's values (none for UnitVal) and column indices; the products and the
// block's row sums later overwrite them in place.
template <typename VT, typename AT>
struct Stages {
  static constexpr int VE = 16 / (int)sizeof(VT);   // values per 16 bytes
  static constexpr bool kStageVals = !IsUnit<VT>::value;   // a value stream is copied
  const Geometry& g;
  const VT* vals;
  unsigned char* base;
  size_t svb, stb;
  int nnz_v, nnz_c;   // array ends rounded down to whole 16-byte units
  uint64_t pol;       // L2 policy of the streams

  __device__ __forceinline__ Stages(const Geometry& g_, const VT* v, unsigned char* smem, uint64_t p)
      : g(g_), vals(v), base(smem), svb(stage_vals_bytes<VT>(g_.sigma, g_.W)),
        stb(stage_bytes<VT>(g_.sigma, g_.W)),
        nnz_v(g_.nnz & ~(VE - 1)), nnz_c(g_.nnz & ~3), pol(p) {}

  __device__ __forceinline__ VT* sv(int s) const { return reinterpret_cast<VT*>(base + (size_t)s * stb); }
  __device__ __forceinline__ int32_t* sc(int s) const {
    return reinterpret_cast<int32_t*>(base + (size_t)s * stb + svb);
  }

  __device__ __forceinline__ BlockSpan span(int v) const {
    const int bs = v * g.W;
    const int be = min(bs + g.W, g.tile_num);
    return BlockSpan{(int)g.tile_x[bs], (int)g.tile_x[be], g.tile_y[bs] & ~kMsb, g.tile_y[be] & ~kMsb};
  }

  // Record the block's stage layout in *info and start its copies on bar (one thread).
  __device__ __forceinline__ void issue(int s, const BlockSpan& b, StageInfo* info, uint64_t* bar) const {
    StageInfo in;
    in.x_bs = b.xb; in.x_be = b.xe; in.y_bs = (int)b.yb; in.y_be = (int)b.ye;
    in.a0v = b.xb & ~(VE - 1);
    in.endv = max(in.a0v, min((b.xe + VE - 1) & ~(VE - 1), nnz_v));
    in.a0c = b.xb & ~3;
    in.endc = max(in.a0c, min((b.xe + 3) & ~3, nnz_c));
    *info = in;
    const uint32_t bv = kStageVals ? (uint32_t)(in.endv - in.a0v) * (uint32_t)sizeof(VT) : 0u;
    const uint32_t bc = (uint32_t)(in.endc - in.a0c) * 4u;
    mbar_arrive_expect_tx(bar, bv + bc);
    if (bv) bulk_g2s(sv(s), vals + in.a0v, bv, bar, pol);
    if (bc) bulk_g2s(sc(s), g.col_stage + in.a0c, bc, bar, pol);
  }

  // The stage's product slots (over the values, or over the column indices for 16-bit
  // values) and the nonzero index of slot 0.
  __device__ __forceinline__ AT* prod(int s, const StageInfo& in, int& pb) const {
    if constexpr (ProdInVals<VT, AT>::value) {
      pb = in.a0v;
      return reinterpret_cast<AT*>(sv(s));
    } else {
      pb = in.a0c;
      return reinterpret_cast<AT*>(sc(s));
    }
  }

  // x[col] of a staged nonzero k (gather_x: from the hot table for a tagged column when
  // HOT).  Nonzeros past the staged range read the plain column array.
  template <bool HOT, typename XT>
  __device__ __forceinline__ void gather(int s, const StageInfo& in, int k, const XT* x, const XT* tab,
                                         uint64_t pol_x, AT& xv) const {
    const int c = k < in.endc ? sc(s)[k - in.a0c] : __ldg(g.col + k);
    xv = static_cast<AT>(gather_x<HOT>(c, x, tab, pol_x));
  }
  __device__ __forceinline__ AT product(int s, const StageInfo& in, int k, AT xv) const {
    if constexpr (IsUnit<VT>::value) {
      return xv;
    } else {
      return static_cast<AT>(widen(k < in.endv ? sv(s)[k - in.a0v] : vals[k])) * xv;
    }
  }
};

// This CTA's copy of the hot-column table: tab[i] = x[hot_list[i]] for i < g.hot_n,
// loaded by all threads of the CTA at the start of a launch (the caller synchronises).
template <typename XT>
__device__ __forceinline__ void fill_hot(const Geometry& g, const XT* x, XT* tab, uint64_t pol_x) {
  for (int i = threadIdx.x; i < g.hot_n; i += blockDim.x) tab[i] = ld_x(x + __ldg(g.hot_list + i), pol_x);
}

// The blocks a CTA walks: all blocks in order, or the epilogue's list (*block_count
// entries, read at kernel start).
template <typename Epi>
struct BlockOrder {
  int n;
  const int* list = nullptr;
  __device__ __forceinline__ BlockOrder(const Geometry& g, const Epi& epi) : n(g.nb) {
    if constexpr (HasBlockList<Epi>::value) {
      n = *reinterpret_cast<const volatile int*>(epi.block_count);
      list = epi.block_list;
    }
  }
  __device__ __forceinline__ int operator()(int k) const {
    if constexpr (HasBlockList<Epi>::value) return __ldg(list + k);
    else return k;
  }
};

// A lane descriptor, streamed once per launch (L2 evict_first).
__device__ __forceinline__ uint64_t ld_desc(const Geometry& g, int j, uint64_t pol) {
  if (g.desc64) {
    unsigned long long v;
    asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;"
                 : "=l"(v)
                 : "l"(reinterpret_cast<const unsigned long long*>(g.lane_desc) + j), "l"(pol));
    return v;
  }
  return ld_stream(g.lane_desc + j, pol);
}

constexpr int kSplitThreadsMax = 512;   // the largest block of the SpMV kernels

// One warp reduces one tile of a staged block into the block's row sums (Algorithm
// tile_normal_tackle with WarpSegmentedSum; tile_fast_tackle for a tile marked as part
// of a single row).  pt: the tile's first product; sy: the row sums from the tile's first
// row y_ws on; desc: this lane's descriptor; j: this lane's global lane index.
template <typename AT>
__device__ __forceinline__ void reduce_tile(const Geometry& g, const AT* pt, AT* sy, uint32_t txs,
                                            uint32_t txe, uint32_t tys, int y_ws, uint64_t desc,
                                            int j, int lane) {
  if (tys & kMsb) {
    // single-row tile: plain warp reduction, no descriptor
    AT sum = AT(0);
    for (int k = lane; k < (int)(txe - txs); k += 32) sum += pt[k];
    sum = warp_sum(sum);
    if (lane == 0) atomicAdd(sy, sum);
    return;
  }
  const bool active = j < g.lane_num;
  const int lane_len = active ? min(g.sigma, g.steps - j * g.sigma) : 0;
  AT sum = AT(0);
  int yo;
  bool head;
  if (!g.desc64) {
    // 32-bit descriptor (sigma <= 14): the steps unrolled, each product addressed from
    // the descriptor alone (step k consumes product k - (down steps before k)), so no
    // load waits on the running sum
    const uint32_t d = (uint32_t)desc;
    const uint32_t valid = (1u << lane_len) - 1u;
    const uint32_t dm = (d >> 18) & valid;     // down steps
    const uint32_t rm = ~(d >> 18) & valid;    // right steps
    const int y0 = active ? (int)((d >> 9) & 511u) : (g.n_rows - y_ws);
    const AT* pl = pt + (int)(d & 511u);       // this lane's first product
#pragma unroll
    for (int k = 0; k < kSigmaMax; ++k) {
      const int nd = __popc(dm & ((1u << k) - 1u));
      const AT pv = pl[k - nd];
      if ((dm >> k) & 1u) {
        // down step: row y0 + nd ends here; only the lane's first such row can
        // have begun in an earlier lane, so only that one needs an atomic add
        if (nd == 0) atomicAdd(sy + y0, sum);
        else sy[y0 + nd] = sum;
        sum = AT(0);
      } else if ((rm >> k) & 1u) {
        sum += pv;
      }
    }
    yo = y0 + __popc(dm);
    head = lane == 0 || dm != 0u;
  } else {
    // 64-bit descriptor (sigma 15..42): the same walk as a loop over the lane's steps
    const uint64_t valid = lane_len >= 64 ? ~0ull : ((1ull << lane_len) - 1ull);
    const uint64_t dm = (desc >> 22) & valid;
    const int y0 = active ? (int)((desc >> 11) & 2047u) : (g.n_rows - y_ws);
    const AT* pl = pt + (int)(desc & 2047u);
    int nd = 0;
    for (int k = 0; k < lane_len; ++k) {
      if ((dm >> k) & 1ull) {
        if (nd == 0) atomicAdd(sy + y0, sum);
        else sy[y0 + nd] = sum;
        sum = AT(0);
        ++nd;
      } else {
        sum += pl[k - nd];
      }
    }
    yo = y0 + nd;
    head = lane == 0 || dm != 0ull;
  }
  // segmented inclusive scan of trailing sums; heads start segments
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
  // a head lane adds the segment that ends just before it; lane 0 takes
  // the tile's final segment (ending at lane 31)
  const int src = lane == 0 ? 31 : lane - 1;
  const AT seg = __shfl_sync(0xffffffffu, sv_, src);
  const int row = __shfl_sync(0xffffffffu, yo, src);
  if (head) atomicAdd(sy + row, seg);
}

// The second pass of a small product run by the block kernel itself: the CTA that
// finishes last (an arrival count after a fence) writes the rows shared between blocks
// and sums the per-CTA partials in a fixed order, then calls the epilogue's finish.
// Used when the product has few blocks (`g.fold`), where a second launch would cost
// more than the work; all threads of the CTA call it.
template <typename Epi>
__device__ __forceinline__ void fold_finalize(const Geometry& g, const Epi& epi) {
  __shared__ int last;
  __shared__ double fold_smem[kSplitThreadsMax / 32][2];
  const int tid = threadIdx.x;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    last = atomicAdd(&g.red->arrive, 1u) + 1 == gridDim.x;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double p0 = 0.0, p1 = 0.0;
  for (int k = tid; k <= g.nb; k += blockDim.x) {
    if (__ldg(g.bnd_slot + k) != k) continue;
    const int r = __ldg(g.bnd_row + k);
    if (r >= g.n_rows) continue;
    epi.row64(r, read_reset(g.bnd_acc + k), p0, p1);
  }
  if constexpr (Epi::kReduce) {
    for (int i = tid; i < (int)gridDim.x; i += blockDim.x) {
      const double2 q = __ldcg(g.part + i);
      p0 += q.x;
      p1 += q.y;
    }
    p0 = warp_sum(p0);
    p1 = warp_sum(p1);
    if ((tid & 31) == 0) {
      fold_smem[tid >> 5][0] = p0;
      fold_smem[tid >> 5][1] = p1;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
        a += fold_smem[w][0];
        b += fold_smem[w][1];
      }
      epi.finish(a, b, g.red);
    }
  }
  if (tid == 0) g.red->arrive = 0u;
}

template <typename VT, typename XT, typename AT, typename Epi>
__global__ void __launch_bounds__(kThreads, 3)
    merbit_spmv_kernel(const Geometry g, const VT* __restrict__ vals, const XT* __restrict__ x,
                       Epi epi) {
  static_assert(ProdInVals<VT, AT>::value || sizeof(AT) == 4, "product slot width");
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ StageInfo info[2];
  __shared__ double red_smem[kThreads / 32][2];
  extern __shared__ __align__(128) unsigned char dyn_smem[];

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int G = gridDim.x;
  if (epi.skip(g.red)) return;
  epi.init();

  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_x = policy_evict_last();
  const Stages<VT, AT> st(g, vals, dyn_smem, pol_stream);
  const BlockOrder<Epi> blk(g, epi);
  const int nbl = blk.n;

  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    if (blockIdx.x < nbl) st.issue(0, st.span(blk(blockIdx.x)), &info[0], &mbar[0]);
    if (blockIdx.x + G < nbl) st.issue(1, st.span(blk(blockIdx.x + G)), &info[1], &mbar[1]);
  }
  XT* tab = reinterpret_cast<XT*>(dyn_smem + 2 * st.stb);
  if (g.hot_n > 0) {
    fill_hot(g, x, tab, pol_x);
    __syncthreads();
  }

  double p0 = 0.0, p1 = 0.0;
  int it = 0;
  for (int kb = blockIdx.x; kb < nbl; kb += G, ++it) {
    const int v = blk(kb);
    const int s = it & 1;
    const uint32_t par = (it >> 1) & 1;

    // tile metadata of this warp's tiles (warp, warp + 8 while < W), loaded before the
    // wait to hide latency
    uint32_t txs[kMaxTpw], txe[kMaxTpw], tys[kMaxTpw];
    uint64_t desc[kMaxTpw];
#pragma unroll
    for (int t = 0; t < kMaxTpw; ++t) {
      const int wt = warp + t * kWarps;
      const int ti = v * g.W + wt;
      const int j = ti * kOmega + lane;
      txs[t] = txe[t] = tys[t] = desc[t] = 0;
      if (wt < g.W && ti < g.tile_num) {
        txs[t] = __ldg(g.tile_x + ti);
        txe[t] = __ldg(g.tile_x + ti + 1);
        tys[t] = __ldg(g.tile_y + ti);
        if (!(tys[t] & kMsb) && j < g.lane_num) desc[t] = ld_desc(g, j, pol_stream);
      }
    }
    // geometry for the copy issued at the end of this iteration
    BlockSpan next{0, 0, 0u, 0u};
    const bool refill = (tid == 0) && (kb + 2 * G < nbl);
    if (refill) next = st.span(blk(kb + 2 * G));

    const bool ok = mbar_wait_bounded(&mbar[s], par, g.wait_limit);
    if (__syncthreads_or(!ok)) {
      // expired wait: record it, let this CTA's copies land (bounded), leave
      if (tid == 0) atomicOr(&g.red->err, 1);
      mbar_wait_bounded(&mbar[s], par);
      if (kb + G < nbl) mbar_wait_bounded(&mbar[s ^ 1], ((it + 1) >> 1) & 1);
      return;
    }
    const StageInfo in = info[s];
    int pb;
    AT* prod = st.prod(s, in, pb);

    // ---- stage products val * x[col] (load_smem of Algorithm MERBIT SpMV)
    {
      const int cnt = in.x_be - in.x_bs;
      auto form_products = [&](auto hot_tag) {
        constexpr bool HOT = decltype(hot_tag)::value;
        for (int base = 0; base < cnt; base += kThreads * kSigmaMax) {
          AT xv[kSigmaMax];
#pragma unroll
          for (int u = 0; u < kSigmaMax; ++u) {
            const int e = base + tid + u * kThreads;
            xv[u] = AT(0);
            if (e < cnt) st.template gather<HOT>(s, in, in.x_bs + e, x, tab, pol_x, xv[u]);
          }
#pragma unroll
          for (int u = 0; u < kSigmaMax; ++u) {
            const int e = base + tid + u * kThreads;
            if (e < cnt) prod[in.x_bs + e - pb] = st.product(s, in, in.x_bs + e, xv[u]);
          }
        }
      };
      if (g.hot_n > 0) form_products(std::true_type{});
      else form_products(std::false_type{});
    }
    AT* s_y = prod + (in.x_be - pb);
    for (int r = tid; r <= in.y_be - in.y_bs; r += kThreads) s_y[r] = AT(0);
    __syncthreads();

    // ---- per-tile reduction (tile_fast_tackle / tile_normal_tackle + WarpSegmentedSum)
#pragma unroll
    for (int t = 0; t < kMaxTpw; ++t) {
      // a tile without products (or past the block's or the path's last tile) adds nothing
      if (txs[t] < txe[t]) {
        const int ti = v * g.W + warp + t * kWarps;
        const int y_ws = (int)(tys[t] & ~kMsb);
        reduce_tile<AT>(g, prod + ((int)txs[t] - pb), s_y + (y_ws - in.y_bs), txs[t], txe[t], tys[t], y_ws,
                        desc[t], ti * kOmega + lane, lane);
      }
    }
    __syncthreads();

    // ---- block commit: interior rows complete here, boundary rows via FP64 accumulators
    for (int r = in.y_bs + 1 + tid; r < in.y_be; r += kThreads) epi.row(r, s_y[r - in.y_bs], p0, p1);
    if (tid == 0) atomicAdd(g.bnd_acc + __ldg(g.bnd_slot + v), static_cast<double>(s_y[0]));
    if (tid == 32 && in.y_be != in.y_bs && in.y_be < g.n_rows)
      atomicAdd(g.bnd_acc + __ldg(g.bnd_slot + v + 1), static_cast<double>(s_y[in.y_be - in.y_bs]));
    // stage s is free again once every thread is past this point
    fence_proxy_async_smem();
    __syncthreads();
    if (refill) st.issue(s, next, &info[s], &mbar[s]);
  }

  if constexpr (Epi::kReduce) {
    p0 = warp_sum(p0);
    p1 = warp_sum(p1);
    if (lane == 0) {
      red_smem[warp][0] = p0;
      red_smem[warp][1] = p1;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) {
        a += red_smem[w][0];
        b += red_smem[w][1];
      }
      g.part[blockIdx.x] = make_double2(a, b);
    }
  }
  if (g.fold) fold_finalize(g, epi);
}

// ---------------------------------------------------------------- warp-specialized kernel
// The same block reduction with the x gather split off: kSplitConsumers consumer threads
// (warp w reduces tiles w and w + 8 of a block, those below W, with the
// per-tile reduction above) reduce and commit block i while kSplitProducers producer
// threads gather x and form the products of blocks i + 1 and i + 2, so the SM's
// load path stays busy through the scans instead of in per-block bursts.  Three stages
// rotate through bulk copy -> products -> reduction; block i + 3's copies are issued into
// block i's stage once its consumers are done with it.  Producers hand a stage to the
// consumers through a second mbarrier per stage (one arrival per producer warp).
constexpr int kSplitConsumers = 256;
constexpr int kSplitProducers = 256;
constexpr int kSplitThreads = kSplitConsumers + kSplitProducers;
constexpr int kSplitStages = 3;
static_assert(kSplitConsumers == kThreads, "a consumer warp takes the tiles a classic warp takes");

// barrier 1 among the consumer threads only (warps 0 .. kSplitConsumers/32 - 1)
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kSplitConsumers) : "memory");
}
__device__ __forceinline__ bool consumers_or(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred q, o;\n\tsetp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred o, 1, %2, q;\n\tselp.u32 %0, 1, 0, o;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "n"(kSplitConsumers)
      : "memory");
  return r != 0;
}

template <typename VT, typename XT, typename AT, typename Epi>
__global__ void __launch_bounds__(kSplitThreads, 2)
    merbit_spmv_split_kernel(const Geometry g, const VT* __restrict__ vals, const XT* __restrict__ x,
                          Epi epi) {
  static_assert(ProdInVals<VT, AT>::value || sizeof(AT) == 4, "product slot width");
  using St = Stages<VT, AT>;
  const int S = g.stages;                              // 2 or 3 stages in the ring
  __shared__ __align__(8) uint64_t full[kSplitStages];   // the stage's bulk copies have landed
  __shared__ __align__(8) uint64_t ready[kSplitStages];  // the stage's products are formed
  __shared__ StageInfo info[kSplitStages];
  __shared__ double red_smem[kSplitConsumers / 32][2];
  __shared__ int failed;
  extern __shared__ __align__(128) unsigned char dyn_smem[];

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int G = gridDim.x;
  if (epi.skip(g.red)) return;
  epi.init();

  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_x = policy_evict_last();
  const St st(g, vals, dyn_smem, pol_stream);
  const BlockOrder<Epi> blk(g, epi);
  const int nbl = blk.n;
  // this CTA's blocks: blk(blockIdx.x + i * G) for i < nmine
  const int nmine = (int)blockIdx.x < nbl ? (nbl - 1 - (int)blockIdx.x) / G + 1 : 0;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ready[s], kSplitProducers / 32);
    }
    failed = 0;
    fence_mbar_init();
  }
  __syncthreads();
  int issued = 0;   // blocks whose copies thread 0 has issued
  if (tid == 0) {
    for (; issued < S && issued < nmine; ++issued)
      st.issue(issued, st.span(blk(blockIdx.x + issued * G)), &info[issued], &full[issued]);
  }
  XT* tab = reinterpret_cast<XT*>(dyn_smem + S * st.stb);
  if (g.hot_n > 0) {
    fill_hot(g, x, tab, pol_x);
    __syncthreads();
  }

  if (tid >= kSplitConsumers) {
    // ---- producers: products val * x[col] of each block (load_smem), then the zeroed
    // row sums, in the stage the block was copied to
    const int pt = tid - kSplitConsumers;
    for (int i = 0; i < nmine; ++i) {
      const int s = i % S;
      // a warp gives up as a whole, so none of its lanes is left at the __syncwarp below
      const bool ok = mbar_wait_bounded(&full[s], (uint32_t)(i / S) & 1u, g.wait_limit);
      if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) {
          atomicOr(&g.red->err, 1);
          failed = 1;
        }
        break;
      }
      const StageInfo in = info[s];
      int pb;
      AT* prod = st.prod(s, in, pb);
      const int cnt = in.x_be - in.x_bs;
      // gathers in flight per thread: up to 14 (one block at sigma 14); 10 for 8-byte
      // products, which keeps them in registers (one block at sigma <= 10)
      constexpr int NB = sizeof(AT) == 8 ? 10 : kSigmaMax;
      // the plain gather or the hot-table gather, chosen once per block (uniform)
      auto form_products = [&](auto hot_tag) {
        constexpr bool HOT = decltype(hot_tag)::value;
        for (int base = 0; base < cnt; base += kSplitProducers * NB) {
          AT xv[NB];
#pragma unroll
          for (int u = 0; u < NB; ++u) {
            const int e = base + pt + u * kSplitProducers;
            xv[u] = AT(0);
            if (e < cnt) st.template gather<HOT>(s, in, in.x_bs + e, x, tab, pol_x, xv[u]);
          }
#pragma unroll
          for (int u = 0; u < NB; ++u) {
            const int e = base + pt + u * kSplitProducers;
            if (e < cnt) prod[in.x_bs + e - pb] = st.product(s, in, in.x_bs + e, xv[u]);
          }
        }
      };
      if (g.hot_n > 0) form_products(std::true_type{});
      else form_products(std::false_type{});
      AT* s_y = prod + (in.x_be - pb);
      for (int r = pt; r <= in.y_be - in.y_bs; r += kSplitProducers) s_y[r] = AT(0);
      // these generic writes precede the bulk copy that later refills the stage; one
      // arrival per warp once all its lanes have written
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ready[s]);
    }
  } else {
    // ---- consumers: per-tile reduction and block commit, as in merbit_spmv_kernel
    double p0 = 0.0, p1 = 0.0;
    for (int i = 0; i < nmine; ++i) {
      const int kb = blockIdx.x + i * G;
      const int v = blk(kb);
      const int s = i % S;
      constexpr int CW = kSplitConsumers / 32, TPW = kMaxTpw;
      uint32_t txs[TPW], txe[TPW], tys[TPW];
      uint64_t desc[TPW];
#pragma unroll
      for (int t = 0; t < TPW; ++t) {
        const int ti = v * g.W + warp + t * CW;
        const int j = ti * kOmega + lane;
        txs[t] = txe[t] = tys[t] = desc[t] = 0;
        if (warp + t * CW < g.W && ti < g.tile_num) {
          txs[t] = __ldg(g.tile_x + ti);
          txe[t] = __ldg(g.tile_x + ti + 1);
          tys[t] = __ldg(g.tile_y + ti);
          if (!(tys[t] & kMsb) && j < g.lane_num) desc[t] = ld_desc(g, j, pol_stream);
        }
      }
      BlockSpan next{0, 0, 0u, 0u};
      const bool refill = (tid == 0) && (i + S < nmine);
      if (refill) next = st.span(blk(kb + S * G));

      const bool ok = mbar_wait_bounded(&ready[s], (uint32_t)(i / S) & 1u, g.wait_limit);
      if (consumers_or(!ok)) {
        if (tid == 0) {
          atomicOr(&g.red->err, 1);
          failed = 1;
        }
        break;
      }
      const StageInfo in = info[s];
      int pb;
      AT* prod = st.prod(s, in, pb);
      AT* s_y = prod + (in.x_be - pb);
#pragma unroll
      for (int t = 0; t < TPW; ++t) {
        // a tile without products (or past the last tile) adds nothing
        if (txs[t] < txe[t]) {
          const int ti = v * g.W + warp + t * CW;
          const int y_ws = (int)(tys[t] & ~kMsb);
          reduce_tile<AT>(g, prod + ((int)txs[t] - pb), s_y + (y_ws - in.y_bs), txs[t], txe[t], tys[t],
                          y_ws, desc[t], ti * kOmega + lane, lane);
        }
      }
      consumers_sync();

      for (int r = in.y_bs + 1 + tid; r < in.y_be; r += kSplitConsumers)
        epi.row(r, s_y[r - in.y_bs], p0, p1);
      if (tid == 0) atomicAdd(g.bnd_acc + __ldg(g.bnd_slot + v), static_cast<double>(s_y[0]));
      if (tid == 32 && in.y_be != in.y_bs && in.y_be < g.n_rows)
        atomicAdd(g.bnd_acc + __ldg(g.bnd_slot + v + 1), static_cast<double>(s_y[in.y_be - in.y_bs]));
      fence_proxy_async_smem();
      consumers_sync();
      if (refill) {
        st.issue(s, next, &info[s], &full[s]);
        ++issued;
      }
    }
    if constexpr (Epi::kReduce) {
      p0 = warp_sum(p0);
      p1 = warp_sum(p1);
      if (lane == 0) {
        red_smem[warp][0] = p0;
        red_smem[warp][1] = p1;
      }
      consumers_sync();
      if (tid == 0) {
        double a = 0.0, b = 0.0;
#pragma unroll
        for (int w = 0; w < kSplitConsumers / 32; ++w) {
          a += red_smem[w][0];
          b += red_smem[w][1];
        }
        g.part[blockIdx.x] = make_double2(a, b);
      }
    }
  }
  // after a failed wait, let this CTA's copies in flight land (bounded) before it exits
  __syncthreads();
  if (tid == 0 && failed)
    for (int k = max(0, issued - S); k < issued; ++k) mbar_wait_bounded(&full[k % S], (uint32_t)(k / S) & 1u);
  // a CTA that gave up does not arrive, so no CTA finishes the product (the error bit
  // tells the host)
  if (g.fold && !failed) fold_finalize(g, epi);
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
    if (gridDim.x == 1) {
      // a single CTA holds the whole sum: no spread slots, fence or arrival count
      finish(a, b);
      return;
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

// Products of at most this many blocks are finished by the block kernel's last CTA.
constexpr int64_t kFoldMaxBlocks = 1024;

// Launch geometry of one block kernel: the plan's hot-column table is added to the
// stages' shared memory when the whole table fits without lowering the number of
// resident CTAs per SM; otherwise the launch streams the plain column array.
// L1 left beside the shared memory matters below about 60 KB: when the blocks' shared
// memory per SM crosses the second-largest carveout (196 KB on sm_100-class SMs), the driver
// takes the largest one and the x gather slows by ~40 % (measured on R-MAT-24).  The
// table is only added while the SM's shared memory stays at or below that carveout.
constexpr size_t kSharedPerSmKeepL1 = 196 * 1024;

// The automatic choice takes the three-stage ring only while two CTAs' rings stay within
// this much shared memory per SM; above it the L1 left for the x gather costs more than
// the deeper ring gains.  R-MAT-24, three vs two stages: f32 sigma 12 (149 KB per SM)
// 1.185 vs 1.194 ms, sigma 13 (161 KB) 1.164 vs 1.167, sigma 14 (174 KB) 1.175 vs 1.151;
// f64 sigma 9 (168 KB) 2.074 vs 2.093, sigma 10 (187 KB) 1.957 vs 1.951, sigma 12 (224 KB)
// 2.827 vs 1.898.
constexpr size_t kDeepRingSharedPerSm = 168 * 1024;

template <typename XT>
inline size_t add_hot_table(const merbit_plan_s* p, Geometry& g, const void* kern, size_t stages,
                            int per_sm) {
  if (p->hot_n <= 0 || !p->col_hot || per_sm <= 0) return stages;
  const size_t need = stages + ((sizeof(XT) * (size_t)p->hot_n + 15) & ~size_t(15));
  if (need > smem_room(kern, per_sm)) return stages;
  const size_t room_keep_l1 = smem_room_below(kern, per_sm, kSharedPerSmKeepL1);
  if (need > room_keep_l1 && stages <= room_keep_l1) return stages;   // the table would cost L1
  g.col_stage = p->col_hot;
  g.hot_list = p->hot_list;
  g.hot_n = p->hot_n;
  return need;
}

// Grid, dynamic shared memory and geometry (with or without the hot-column table) of the
// split kernel's launch for a plan; false if two of its CTAs do not fit on an SM (or
// none does, when `forced`).
template <typename VT, typename XT, typename AT, typename Epi>
bool split_config(const merbit_plan_s* p, Geometry& g, int& grid, size_t& smem, bool forced) {
  auto kern = merbit_spmv_split_kernel<VT, XT, AT, Epi>;
  const void* kp = reinterpret_cast<const void*>(kern);
  g.stages = p->spmv_kernel == MERBIT_KERNEL_SPLIT2 ? 2 : kSplitStages;
  if (!forced && g.stages == kSplitStages &&
      2 * kSplitStages * stage_bytes<VT>(p->sigma, p->tiles_per_block) > kDeepRingSharedPerSm)
    g.stages = 2;
  size_t stages = (size_t)g.stages * stage_bytes<VT>(p->sigma, p->tiles_per_block);
  grid = persistent_grid(kp, kSplitThreads, stages, stages, p->num_sms);
  if (!forced && grid < 2 * p->num_sms && g.stages == kSplitStages) {
    // the automatic choice: when three stages leave room for one CTA per SM only (8-byte
    // values at large sigma), a ring of two stages may still fit two
    g.stages = 2;
    stages = 2 * stage_bytes<VT>(p->sigma, p->tiles_per_block);
    grid = persistent_grid(kp, kSplitThreads, stages, stages, p->num_sms);
  }
  const size_t stages_max = stages;
  if (grid <= 0 || (!forced && grid < 2 * p->num_sms)) return false;
  smem = add_hot_table<XT>(p, g, kp, stages, grid / p->num_sms);
  if (smem != stages) grid = persistent_grid(kp, kSplitThreads, smem, std::max(smem, stages_max), p->num_sms);
  if (grid <= 0) return false;
  if ((int64_t)grid > p->nb) grid = (int)p->nb;
  if (grid > kMaxParts) grid = kMaxParts;
  return true;
}

template <typename VT, typename XT, typename AT, typename Epi>
cudaError_t launch_spmv(const merbit_plan_s* p, const VT* vals, const XT* x, const Epi& epi,
                        cudaStream_t st) {
  if (p->nb == 0) return cudaSuccess;
  // The split kernel is the default while two of its CTAs fit on an SM (measured on
  // sm_103a, R-MAT scale 21 and 24: 15-30 % faster than the classic kernel for 32- and
  // 64-bit values, 11 % for 16-bit values at sigma 14, slower with one CTA per SM).
  Geometry g = p->geom();
  // few blocks: the block kernel finishes the product itself (no second launch)
  g.fold = p->nb <= kFoldMaxBlocks;
  int grid = 0;
  bool split = false;
  const int kind = p->spmv_kernel;
  // A split kernel that was asked for but cannot hold even one CTA's stages on an SM (large
  // sigma x block size with 8-byte values) gives way to the classic kernel, whose ring
  // has two stages.
  if (kind == MERBIT_KERNEL_SPLIT || kind == MERBIT_KERNEL_SPLIT2 || kind == MERBIT_KERNEL_AUTO) {
    size_t smem = 0;
    split = split_config<VT, XT, AT, Epi>(p, g, grid, smem, kind != MERBIT_KERNEL_AUTO);
    if (split) merbit_spmv_split_kernel<VT, XT, AT, Epi><<<grid, kSplitThreads, smem, st>>>(g, vals, x, epi);
  }
  if (!split) {
    g = p->geom();
    g.fold = p->nb <= kFoldMaxBlocks;
    auto kern = merbit_spmv_kernel<VT, XT, AT, Epi>;
    const void* kp = reinterpret_cast<const void*>(kern);
    const size_t stages = 2 * stage_bytes<VT>(p->sigma, p->tiles_per_block);
    const size_t stages_max = stages;
    grid = persistent_grid(kp, kThreads, stages, stages_max, p->num_sms);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    const size_t smem = add_hot_table<XT>(p, g, kp, stages, grid / p->num_sms);
    if (smem != stages) grid = persistent_grid(kp, kThreads, smem, std::max(smem, stages_max), p->num_sms);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    if ((int64_t)grid > p->nb) grid = (int)p->nb;
    if (grid > kMaxParts) grid = kMaxParts;
    kern<<<grid, kThreads, smem, st>>>(g, vals, x, epi);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || g.fold) return e;
  const int fgrid = (int)std::min<int64_t>((p->nb + 1 + 255) / 256, (int64_t)p->num_sms * 4);
  merbit_finalize_kernel<Epi><<<fgrid, 256, 0, st>>>(g, epi, Epi::kReduce ? grid : 0);
  return cudaGetLastError();
}

}  // namespace merbit
