// MERBIT SpMM: Y = A X for a row-major X (n_cols x k) and Y (n_rows x k), f32,
// on the same plan as the SpMV (the batching extension of the hot path: k
// personalisation vectors in one pass).
//
// Work unit: the SpMV's block of 8 tiles, staged by the same two bulk copies;
// one warp per tile.  A column chunk of KC columns is split into slices of VW
// consecutive columns (VW = 4: one 16-byte load per slice); T = KC / VW
// threads cover a chunk, so the warp forms 32 / T groups.
//   1. The warp decodes its tile's lane descriptors (Sec. 4.1.1 bit_flag):
//      every down step ends a row, at the tile-relative nonzero position
//      x_off + (right steps before it); a warp scan of the down-step counts
//      lays these row ends out in shared memory in row order.
//   2. Group g takes an equal share [t0, t1) of the tile's nonzeros and the
//      row ends at positions in (t0, t1] (group 0 also those at 0).  It
//      gathers U row slices X[col[p], c..c+VW) at a time, independent of row
//      ends, then adds vals[p] * slice into the running row sum, closing a row
//      whenever the next row end is reached.
//   3. Rows that begin and end inside a group's share are written directly;
//      the first and last partial row of every share go to a small shared
//      table.  After a block barrier each group adds up the table entries of
//      the rows its own entries start; rows inside the block are written and
//      the block's first and last rows are added into per-row FP64
//      accumulators that a finalize kernel writes out and clears (the SpMV's
//      boundary-row scheme, KC values wide).
#pragma once

#include <climits>
#include <type_traits>

#include "spmv_kernel.cuh"

namespace merbit {

template <int VW> struct SpmmVec;
template <> struct SpmmVec<1> {
  using T = float;
  static __device__ __forceinline__ T zero() { return 0.f; }
  static __device__ __forceinline__ T load(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ T load_plain(const float* p) { return *p; }
  static __device__ __forceinline__ void store(float* p, const float (&a)[1]) { *p = a[0]; }
  static __device__ __forceinline__ void fma(float w, const T& x, T& s) { s = fmaf(w, x, s); }
  static __device__ __forceinline__ float get(const T& v, int) { return v; }
  static __device__ __forceinline__ T from(const float (&a)[1]) { return a[0]; }
  static __device__ __forceinline__ void add(T& s, const T& x) { s += x; }
  static __device__ __forceinline__ T shfl_up(const T& v, int d) {
    return __shfl_up_sync(0xffffffffu, v, d);
  }
};
template <> struct SpmmVec<4> {
  using T = float4;
  static __device__ __forceinline__ T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ T load(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
  }
  static __device__ __forceinline__ T load_plain(const float* p) {
    return *reinterpret_cast<const float4*>(p);
  }
  static __device__ __forceinline__ void store(float* p, const float (&a)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(a[0], a[1], a[2], a[3]);
  }
  static __device__ __forceinline__ void fma(float w, const T& x, T& s) {
    s.x = fmaf(w, x.x, s.x);
    s.y = fmaf(w, x.y, s.y);
    s.z = fmaf(w, x.z, s.z);
    s.w = fmaf(w, x.w, s.w);
  }
  static __device__ __forceinline__ float get(const T& v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
  }
  static __device__ __forceinline__ T from(const float (&a)[4]) {
    return make_float4(a[0], a[1], a[2], a[3]);
  }
  static __device__ __forceinline__ void add(T& s, const T& x) {
    s.x += x.x; s.y += x.y; s.z += x.z; s.w += x.w;
  }
  static __device__ __forceinline__ T shfl_up(const T& v, int d) {
    return make_float4(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d),
                       __shfl_up_sync(0xffffffffu, v.z, d), __shfl_up_sync(0xffffffffu, v.w, d));
  }
};

// Epilogue of the SpMM: Y[r, c..c+VW) = scale * (A X)[r, c..c+VW).  row() takes f32 row sums
// (called by the thread owning columns c..c+VW), row64 one column of a block-shared row
// summed in FP64 (finalize kernel).  A gated launch does nothing once an iterative driver
// has set the plan's stop flag (launches queued after convergence).
struct EpiSpmmPlain {
  float* y;
  int ldy;
  float scale;
  bool gated;
  __device__ __forceinline__ bool skip(const RedState* red) const {
    return gated && *reinterpret_cast<const volatile int*>(&red->done) != 0;
  }
  __device__ __forceinline__ void row(int r, int c, float s) const {
    y[(size_t)r * ldy + c] = scale * s;
  }
  __device__ __forceinline__ void row(int r, int c, const float4& s) const {
    *reinterpret_cast<float4*>(y + (size_t)r * ldy + c) =
        make_float4(scale * s.x, scale * s.y, scale * s.z, scale * s.w);
  }
  __device__ __forceinline__ void row64(int r, int c, double s) const {
    y[(size_t)r * ldy + c] = static_cast<float>(static_cast<double>(scale) * s);
  }
};

struct SpmmGeometry {
  double* acc;      // (nb + 1) x KC FP64 boundary-row accumulators of this chunk
  int kc;           // columns in this chunk (a multiple of VW)
};

// Two CTAs per SM: the register room (up to 128 per thread) keeps a whole batch of gathers
// in flight; capping registers for three CTAs per SM serialised them (k = 8: 1.04 ms vs
// 0.67 ms on R-MAT scale 22).
template <int KC, int VW, typename Epi>
__global__ void __launch_bounds__(kThreads, 2)
    merbit_spmm_kernel(const Geometry g, const SpmmGeometry sg, const float* __restrict__ vals,
                       const float* __restrict__ X, int ldx, Epi epi) {
  using V = SpmmVec<VW>;
  using VT = typename V::T;
  constexpr int T = KC / VW;                   // threads per chunk row
  constexpr int GRP = 32 / T;                  // groups per warp
  constexpr int U = VW == 4 ? (KC == 32 ? 12 : 8) : 16;   // row slices gathered per batch
  constexpr int VE = 4;
  constexpr int kEnds = kOmega * kSigmaMax;    // most row ends in one tile
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ StageInfo info[2];
  __shared__ uint16_t rend_s[kTilesPerBlock][kEnds];
  __shared__ __align__(16) float head_s[kThreads][VW];           // each thread's head partial
  __shared__ int wt_row[2][2 * kTilesPerBlock];                   // per-warp first / last runs
  __shared__ __align__(16) float wt_val[2][2 * kTilesPerBlock][KC];
  extern __shared__ __align__(128) unsigned char dyn_smem[];

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int grp = lane / T;
  const int c = (lane % T) * VW;               // first column of this thread's slice
  const bool c_ok = c < sg.kc;
  const int G = gridDim.x;
  if (epi.skip(g.red)) return;

  const size_t svb = stage_vals_bytes<float>(g.sigma, kTilesPerBlock);
  const size_t stb = stage_bytes<float>(g.sigma, kTilesPerBlock);
  auto sv = [&](int s) { return reinterpret_cast<float*>(dyn_smem + (size_t)s * stb); };
  auto sc = [&](int s) { return reinterpret_cast<int32_t*>(dyn_smem + (size_t)s * stb + svb); };
  const uint64_t pol_stream = policy_evict_first();
  const int nnz_a = g.nnz & ~(VE - 1);
  uint16_t* rend = rend_s[warp];

  auto geom_of = [&](int v, int& xb, int& xe, uint32_t& yb, uint32_t& ye) {
    const int bs = v * kTilesPerBlock;
    const int be = min(bs + kTilesPerBlock, g.tile_num);
    xb = (int)g.tile_x[bs];
    xe = (int)g.tile_x[be];
    yb = g.tile_y[bs] & ~kMsb;
    ye = g.tile_y[be] & ~kMsb;
  };
  auto issue = [&](int s, int xb, int xe, uint32_t yb, uint32_t ye) {
    StageInfo in;
    in.x_bs = xb; in.x_be = xe; in.y_bs = (int)yb; in.y_be = (int)ye;
    in.a0v = xb & ~(VE - 1);
    in.endv = max(in.a0v, min((xe + VE - 1) & ~(VE - 1), nnz_a));
    in.a0c = in.a0v;
    in.endc = in.endv;
    info[s] = in;
    const uint32_t cnt = (uint32_t)(in.endv - in.a0v);
    mbar_arrive_expect_tx(&mbar[s], cnt * 8u);
    if (cnt) {
      bulk_g2s(sv(s), vals + in.a0v, cnt * 4u, &mbar[s], pol_stream);
      bulk_g2s(sc(s), g.col + in.a0c, cnt * 4u, &mbar[s], pol_stream);
    }
  };

  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    int xb, xe; uint32_t yb, ye;
    if (blockIdx.x < g.nb) { geom_of(blockIdx.x, xb, xe, yb, ye); issue(0, xb, xe, yb, ye); }
    if (blockIdx.x + G < g.nb) { geom_of(blockIdx.x + G, xb, xe, yb, ye); issue(1, xb, xe, yb, ye); }
  }

  int it = 0;
  for (int v = blockIdx.x; v < g.nb; v += G, ++it) {
    const int s = it & 1;
    const uint32_t par = (it >> 1) & 1;
    const int ti = v * kTilesPerBlock + warp;
    const bool tile_ok = ti < g.tile_num;
    int txs = 0, ntile = 0, y_ws = 0, ndown = 0;
    if (tile_ok) {
      // 1. row ends of the tile from the lane descriptors
      txs = (int)__ldg(g.tile_x + ti);
      ntile = (int)__ldg(g.tile_x + ti + 1) - txs;
      y_ws = (int)(__ldg(g.tile_y + ti) & ~kMsb);
      const int j = ti * kOmega + lane;
      uint32_t dm = 0, xo = 0;
      if (j < g.lane_num) {
        const uint32_t d = ld_stream(g.lane_desc + j, pol_stream);
        const int len = min(g.sigma, g.steps - j * g.sigma);
        dm = (d >> 18) & ((1u << len) - 1u);
        xo = d & 511u;
      }
      const int nd = __popc(dm);
      int off = nd;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += t;
      }
      ndown = __shfl_sync(0xffffffffu, off, 31);
      off -= nd;
      for (uint32_t m = dm; m; m &= m - 1) {
        const int k = __ffs(m) - 1;
        rend[off++] = (uint16_t)(xo + k - __popc(dm & ((1u << k) - 1u)));
      }
    }
    int nxb = 0, nxe = 0; uint32_t nyb = 0, nye = 0;
    const bool refill = (tid == 0) && (v + 2 * G < g.nb);
    if (refill) geom_of(v + 2 * G, nxb, nxe, nyb, nye);

    const bool ok = mbar_wait_bounded(&mbar[s], par);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(&g.red->err, 1);
      mbar_wait_bounded(&mbar[s], par);
      if (v + G < g.nb) mbar_wait_bounded(&mbar[s ^ 1], ((it + 1) >> 1) & 1);
      return;
    }
    const StageInfo in = info[s];
    const float* vs = sv(s);
    const int32_t* cs = sc(s);
    const bool staged = in.endv >= in.x_be;      // false only in the block holding the array's tail

    // 2. group grp's share of the tile
    int head_row = -1, tail_row = -1;
    VT sum = V::zero();
    if (tile_ok) {
      const int t0 = (int)(((long long)grp * ntile) / GRP);
      const int t1 = (int)(((long long)(grp + 1) * ntile) / GRP);
      // first owned row end: the number of ends at positions <= t0 (none owned for group 0)
      auto count_le = [&](int t) {
        int lo = 0, hi = ndown;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if ((int)rend[mid] <= t) lo = mid + 1; else hi = mid;
        }
        return lo;
      };
      int q = grp == 0 ? 0 : count_le(t0);
      const int q1 = count_le(t1);
      int next = q < q1 ? (int)rend[q] : INT_MAX;
      bool first = true;
      auto close_row = [&]() {
        if (first) {                  // the row may have begun before this share
          head_row = y_ws + q;
#pragma unroll
          for (int k = 0; k < VW; ++k) head_s[tid][k] = V::get(sum, k);
          first = false;
        } else if (c_ok) {
          epi.row(y_ws + q, c, sum);  // begun and ended inside the share
        }
        sum = V::zero();
        ++q;
        next = q < q1 ? (int)rend[q] : INT_MAX;
      };
      const int ib = txs - in.a0v;    // staged index of the tile's first nonzero
      // U row slices from nonzero base on: ST = the block is fully staged, TAIL = the batch
      // may run past t1
      auto batch = [&](int base, auto st_tag, auto tail_tag) {
        constexpr bool ST = decltype(st_tag)::value;
        constexpr bool TAIL = decltype(tail_tag)::value;
        VT xv[U];
        float wv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          xv[u] = V::zero();
          wv[u] = 0.f;
          if ((!TAIL || base + u < t1) && c_ok) {
            const int i = ib + base + u;
            int cc;
            if (ST || in.a0v + i < in.endv) {
              cc = cs[i];
              wv[u] = vs[i];
            } else {
              cc = __ldg(g.col + in.a0v + i);
              wv[u] = __ldg(vals + in.a0v + i);
            }
            xv[u] = V::load(X + (size_t)cc * ldx + c);
          }
        }
        if (next < base + U) {
#pragma unroll
          for (int u = 0; u < U; ++u) {
            while (next == base + u) close_row();   // rows ending before nonzero base + u
            V::fma(wv[u], xv[u], sum);
          }
        } else {
#pragma unroll
          for (int u = 0; u < U; ++u) V::fma(wv[u], xv[u], sum);
        }
      };
      using yes = std::integral_constant<bool, true>;
      using no = std::integral_constant<bool, false>;
      int base = t0;
      if (staged) {
#pragma unroll 1
        for (; base + U <= t1; base += U) batch(base, yes{}, no{});
        if (base < t1) batch(base, yes{}, yes{});
      } else {
#pragma unroll 1
        for (; base < t1; base += U) batch(base, no{}, yes{});
      }
      while (next == t1) close_row();             // rows ending after the share's last nonzero
      if (first) {
        head_row = y_ws + q;          // no row ends in this share
      } else {
        tail_row = y_ws + q;          // the row in progress continues past the share
      }
    }
    if (tile_ok && tail_row < 0) {
#pragma unroll
      for (int k = 0; k < VW; ++k) head_s[tid][k] = V::get(sum, k);   // no row ends in the share
    }

    // 3a. the warp's shares in order: a segmented sum over the groups' runs, by shuffles.
    //     Group g holds one run (head_row) or two (head_row < tail_row); the run of its
    //     last row continues into group g + 1 when that group's head_row is the same row.
    //     OC_g = total of group g's last-row run up to g obeys OC_g = a_g + b_g * OC_{g-1},
    //     a linear recurrence scanned in log2(GRP) steps.
    int* wrow = wt_row[s];
    float (*wval)[KC] = wt_val[s];
    if (lane == 0) {
      wrow[2 * warp] = -1;
      wrow[2 * warp + 1] = -1;
    }
    __syncwarp();
    if (tile_ok) {
      VT hv;
      {
        float h[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) h[k] = head_s[tid][k];
        hv = V::from(h);
      }
      const bool single = tail_row < 0;
      const int row_out = single ? head_row : tail_row;
      const int prev_out = __shfl_up_sync(0xffffffffu, row_out, T);
      const int next_head = __shfl_down_sync(0xffffffffu, head_row, T);
      const int warp_first = __shfl_sync(0xffffffffu, head_row, 0);
      VT A = single ? hv : sum;
      int B = (single && grp > 0 && prev_out == head_row) ? 1 : 0;
#pragma unroll
      for (int d = 1; d < GRP; d <<= 1) {
        const VT Ap = V::shfl_up(A, d * T);
        const int Bp = __shfl_up_sync(0xffffffffu, B, d * T);
        if (grp >= d) {
          if (B) V::add(A, Ap);
          B &= Bp;
        }
      }
      const VT oc_prev = V::shfl_up(A, T);     // OC_{g-1}
      VT first_tot = hv;
      if (grp > 0 && prev_out == head_row) V::add(first_tot, oc_prev);
      // a finished run: boundary rows of the block go to the FP64 accumulators, the
      // warp's first run to the cross-warp table, any other row straight to Y
      auto emit = [&](int r, const VT& val, bool last_of_warp) {
        if (r >= g.n_rows || !c_ok) return;
        if (r == in.y_bs || r == in.y_be) {
          double* a = sg.acc + (size_t)__ldg(g.bnd_slot + (r == in.y_bs ? v : v + 1)) * KC + c;
#pragma unroll
          for (int k = 0; k < VW; ++k) atomicAdd(a + k, (double)V::get(val, k));
        } else if (last_of_warp || r == warp_first) {
          const int e = 2 * warp + (last_of_warp ? 1 : 0);
          if (lane % T == 0) wrow[e] = r;
#pragma unroll
          for (int k = 0; k < VW; ++k) wval[e][c + k] = V::get(val, k);
        } else {
          epi.row(r, c, val);
        }
      };
      const bool last_grp = grp == GRP - 1;
      if (!single || (!last_grp && next_head != head_row)) emit(head_row, first_tot, false);
      if (!single && !last_grp && next_head != tail_row) emit(tail_row, sum, false);
      if (last_grp) emit(row_out, single ? first_tot : sum, true);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (refill) issue(s, nxb, nxe, nyb, nye);

    // 3b. rows spread over several warps of the block (never a boundary row): the warp
    //     holding a row's first table entry adds up its entries
    if (grp == 0) {
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int e = 2 * warp + h;
        const int r = wrow[e];
        if (r < 0 || !c_ok) continue;
        int prev = e - 1;
        while (prev >= 0 && wrow[prev] < 0) --prev;
        if (prev >= 0 && wrow[prev] == r) continue;      // not the first entry of its row
        float tot[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) tot[k] = 0.f;
        for (int q = e; q < 2 * kTilesPerBlock; ++q) {
          const int rq = wrow[q];
          if (rq < 0) continue;
          if (rq != r) break;
#pragma unroll
          for (int k = 0; k < VW; ++k) tot[k] += wval[q][c + k];
        }
        epi.row(r, c, V::from(tot));
      }
    }
  }
}

// Boundary rows of the column chunk: Y[r, c] = acc[slot][c], accumulator cleared.
template <int KC, typename Epi>
__global__ void __launch_bounds__(256) merbit_spmm_finalize_kernel(const Geometry g,
                                                                   const SpmmGeometry sg, Epi epi) {
  if (epi.skip(g.red)) return;
  const int stride = gridDim.x * blockDim.x;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < (g.nb + 1) * KC; p += stride) {
    const int k = p / KC, cc = p % KC;
    if (cc >= sg.kc || __ldg(g.bnd_slot + k) != k) continue;
    const int r = __ldg(g.bnd_row + k);
    if (r >= g.n_rows) continue;
    double* a = sg.acc + (size_t)k * KC + cc;
    const double tot = *a;
    *a = 0.0;
    epi.row64(r, cc, tot);
  }
}

template <int KC, int VW, typename Epi>
cudaError_t launch_spmm(const merbit_plan_s* p, const float* vals, const float* X, int ldx,
                        const SpmmGeometry& sg, const Epi& epi, cudaStream_t st) {
  if (p->nb == 0) return cudaSuccess;
  auto kern = merbit_spmm_kernel<KC, VW, Epi>;
  const size_t smem = 2 * stage_bytes<float>(p->sigma, kTilesPerBlock);
  const size_t smem_max = 2 * stage_bytes<float>(kSigmaMax, kTilesPerBlock);
  int grid = persistent_grid(reinterpret_cast<const void*>(kern), kThreads, smem, smem_max,
                             p->num_sms);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  if ((int64_t)grid > p->nb) grid = (int)p->nb;
  kern<<<grid, kThreads, smem, st>>>(p->geom(), sg, vals, X, ldx, epi);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t work = (p->nb + 1) * KC;
  const int fgrid = (int)std::min<int64_t>((work + 255) / 256, (int64_t)p->num_sms * 8);
  merbit_spmm_finalize_kernel<KC, Epi><<<fgrid, 256, 0, st>>>(p->geom(), sg, epi);
  return cudaGetLastError();
}

}  // namespace merbit
