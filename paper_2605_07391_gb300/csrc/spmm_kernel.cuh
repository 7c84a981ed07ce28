// MERBIT SpMM: Y = A X for a row-major X (n_cols x k) and Y (n_rows x k), f32,
// on the same plan as the SpMV (the batching extension of the hot path: k
// personalisation vectors in one pass).
//
// Work unit: the SpMV's block of 8 tiles, staged by the same two bulk copies;
// one warp per tile.  A column chunk of KC columns is split into slices of VW
// consecutive columns (VW = 4: one 16-byte load per slice); T = KC / VW
// threads cover a chunk, so a warp walks L = 32 / T lanes at once and a tile's
// 32 lanes in T passes.
//   1. A thread takes one lane of the pass and one slice.  The lane descriptor
//      (Sec. 4.1.1 bit_flag) gives, for every step, whether it is a down step
//      and which nonzero a right step consumes (step k takes nonzero
//      x_off + k - (down steps before k)), so the row slices of all the lane's
//      right steps are gathered before any is used.
//   2. The steps are walked in order: a right step adds vals[p] * slice into
//      the running sum, a down step ends a row.  Rows ended after the lane's
//      first down step lie wholly inside the lane and are written to Y; the
//      lane's first ended row may have begun in earlier lanes.
//   3. Runs across lanes: the sum open after lane l obeys
//      OC_l = a_l + b_l * OC_{l-1} (a_l the lane's trailing sum, b_l = 1 when
//      the lane ends no row), a linear recurrence scanned by shuffles; the
//      first ended row of lane l totals OC_{l-1} plus the lane's head sum, and
//      the run open after a pass is carried into the next.
//   4. The tile's first row and the run open at its end go to a small shared
//      table; the last warp to finish the block (an arrival count, no block
//      barrier) adds up each row's entries and refills the block's stage.  The
//      block's first and last rows are added into per-row FP64 accumulators
//      that a finalize kernel writes out and clears (the SpMV's boundary-row
//      scheme, KC values wide).
// Single-row tiles (the tile_y mark of Sec. 4.1.2) skip the descriptors: lanes
// take every L-th nonzero and their sums are added across the warp.
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
  static __device__ __forceinline__ T shfl_xor(const T& v, int d) {
    return __shfl_xor_sync(0xffffffffu, v, d);
  }
  static __device__ __forceinline__ T shfl(const T& v, int src) {
    return __shfl_sync(0xffffffffu, v, src);
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
  static __device__ __forceinline__ T shfl_xor(const T& v, int d) {
    return make_float4(__shfl_xor_sync(0xffffffffu, v.x, d), __shfl_xor_sync(0xffffffffu, v.y, d),
                       __shfl_xor_sync(0xffffffffu, v.z, d), __shfl_xor_sync(0xffffffffu, v.w, d));
  }
  static __device__ __forceinline__ T shfl(const T& v, int src) {
    return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                       __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
  }
};

// Two 16-byte halves: a thread's slice is a whole 32-byte row of an 8-column chunk,
// read by one 32-byte load (its address must be 32-byte aligned).
struct Float8 {
  float4 a, b;
};
template <> struct SpmmVec<8> {
  using T = Float8;
  using H = SpmmVec<4>;
  static __device__ __forceinline__ T zero() { return T{H::zero(), H::zero()}; }
  static __device__ __forceinline__ T load(const float* p) {
    T v;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v.a.x), "=f"(v.a.y), "=f"(v.a.z), "=f"(v.a.w), "=f"(v.b.x), "=f"(v.b.y), "=f"(v.b.z),
          "=f"(v.b.w)
        : "l"(p));
    return v;
  }
  static __device__ __forceinline__ void fma(float w, const T& x, T& s) {
    H::fma(w, x.a, s.a);
    H::fma(w, x.b, s.b);
  }
  static __device__ __forceinline__ float get(const T& v, int i) {
    return i < 4 ? H::get(v.a, i) : H::get(v.b, i - 4);
  }
  static __device__ __forceinline__ T from(const float (&a)[8]) {
    return T{make_float4(a[0], a[1], a[2], a[3]), make_float4(a[4], a[5], a[6], a[7])};
  }
  static __device__ __forceinline__ void add(T& s, const T& x) {
    H::add(s.a, x.a);
    H::add(s.b, x.b);
  }
  static __device__ __forceinline__ T shfl_up(const T& v, int d) {
    return T{H::shfl_up(v.a, d), H::shfl_up(v.b, d)};
  }
  static __device__ __forceinline__ T shfl_xor(const T& v, int d) {
    return T{H::shfl_xor(v.a, d), H::shfl_xor(v.b, d)};
  }
  static __device__ __forceinline__ T shfl(const T& v, int src) {
    return T{H::shfl(v.a, src), H::shfl(v.b, src)};
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
  __device__ __forceinline__ void row(int r, int c, const Float8& s) const {
    row(r, c, s.a);
    row(r, c + 4, s.b);
  }
  __device__ __forceinline__ void row64(int r, int c, double s) const {
    y[(size_t)r * ldy + c] = static_cast<float>(static_cast<double>(scale) * s);
  }
};

// Depth of the SpMM's block ring.  A third stage (two CTAs per SM still fit) took the
// shared memory per SM past the point where the driver shrinks L1: k = 8 on R-MAT scale
// 22 went from 0.458 to 0.548 ms.
constexpr int kSpmmStages = 2;

struct SpmmGeometry {
  double* acc;      // (nb + 1) x KC FP64 boundary-row accumulators of this chunk
  int kc;           // columns in this chunk (a multiple of VW)
};

// Two CTAs per SM: the register room (up to 128 per thread) holds a lane's sigma row
// slices in flight.
template <int KC, int VW, typename Epi>
__global__ void __launch_bounds__(kThreads, 2)
    merbit_spmm_kernel(const Geometry g, const SpmmGeometry sg, const float* __restrict__ vals,
                       const float* __restrict__ X, int ldx, Epi epi) {
  using V = SpmmVec<VW>;
  using VT = typename V::T;
  constexpr int T = KC / VW;                   // threads per lane, one slice of VW columns each
  constexpr int L = 32 / T;                    // lanes walked at once (one pass)
  constexpr int U1 = 8;                        // row slices per round of a single-row tile
  constexpr int HB = VW == 8 ? kSigmaMax / 2 : kSigmaMax;   // steps per batch of gathers
  static_assert(kSigmaMax % HB == 0, "step batches");
  constexpr int VE = 4;
  constexpr int NE = 2 * kTilesPerBlock;       // table entries of a block: each warp's first / last run
  constexpr int S = kSpmmStages;
  __shared__ __align__(8) uint64_t mbar[S];
  __shared__ StageInfo info[S];
  __shared__ int arrive[S];                    // warps done with the stage's block
  __shared__ int wt_row[S][NE];
  __shared__ __align__(16) float wt_val[S][NE][KC];
  extern __shared__ __align__(128) unsigned char dyn_smem[];

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int gl = lane / T;                     // lane of the pass this thread walks
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
    for (int i = 0; i < S; ++i) {
      mbar_init(&mbar[i], 1);
      arrive[i] = 0;
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      const int v = blockIdx.x + i * G;
      if (v >= g.nb) break;
      int xb, xe; uint32_t yb, ye;
      geom_of(v, xb, xe, yb, ye);
      issue(i, xb, xe, yb, ye);
    }
  }

  // The warps move through the ring on their own: no block-wide barrier.  The last warp
  // to finish a block (a shared-memory arrival count) adds up the block's cross-warp table
  // and refills the stage with the block S steps ahead.
  int s = 0;
  uint32_t par = 0;
  for (int v = blockIdx.x; v < g.nb; v += G) {
    const int ti = v * kTilesPerBlock + warp;
    const bool tile_ok = ti < g.tile_num;
    // the tile's bounds and its 32 lane descriptors (one per thread), read before the
    // stage wait so that their latency hides behind it
    uint32_t txs = 0, txe = 0, tys = 0, dreg = 0;
    if (tile_ok) {
      txs = __ldg(g.tile_x + ti);
      txe = __ldg(g.tile_x + ti + 1);
      tys = __ldg(g.tile_y + ti);
      const int j = ti * kOmega + lane;
      if (j < g.lane_num) dreg = ld_stream(g.lane_desc + j, pol_stream);
    }
    const bool ok = mbar_wait_bounded(&mbar[s], par, g.wait_limit);
    if (!__all_sync(0xffffffffu, ok)) {
      // this warp gives up: it records the error and waits, with the default limit, for
      // the copies that may still be landing in the ring (this block and the next S - 1
      // of the CTA; a wait for a copy never issued simply runs out), then returns.  A
      // warp that gives up never arrives, so the other warps' waits run out in turn.
      if (lane == 0) atomicOr(&g.red->err, 1);
      int ss = s;
      uint32_t pp = par;
      for (int m = 0; m < S && v + m * G < g.nb; ++m) {
        mbar_wait_bounded(&mbar[ss], pp);
        if (++ss == S) {
          ss = 0;
          pp ^= 1u;
        }
      }
      return;
    }
    const StageInfo in = info[s];
    const float* vs = sv(s);
    const int32_t* cs = sc(s);
    int* wrow = wt_row[s];
    float (*wval)[KC] = wt_val[s];
    if (lane == 0) {
      wrow[2 * warp] = -1;
      wrow[2 * warp + 1] = -1;
    }
    __syncwarp();

    if (tile_ok) {
      const int y_ws = (int)(tys & ~kMsb);
      const int ntile = (int)(txe - txs);
      const int ib = (int)txs - in.a0v;          // staged index of the tile's first nonzero
      // a finished run of row r: block boundary rows go to the FP64 accumulators, the
      // tile's first row and its run open at the tile's end to the cross-warp table,
      // any other row straight to Y
      auto emit = [&](int r, const VT& val, bool last_of_warp) {
        if (r >= g.n_rows || !c_ok) return;
        if (r == in.y_bs || r == in.y_be) {
          double* a = sg.acc + (size_t)__ldg(g.bnd_slot + (r == in.y_bs ? v : v + 1)) * KC + c;
#pragma unroll
          for (int k = 0; k < VW; ++k) atomicAdd(a + k, (double)V::get(val, k));
        } else if (last_of_warp || r == y_ws) {
          const int e = 2 * warp + (last_of_warp ? 1 : 0);
          if (lane % T == 0) wrow[e] = r;
#pragma unroll
          for (int k = 0; k < VW; ++k) wval[e][c + k] = V::get(val, k);
        } else {
          epi.row(r, c, val);
        }
      };
      // the tile's nonzeros, ST = every one of them is staged (false only in the block
      // holding the array's last few nonzeros, which are read from global memory)
      auto walk = [&](auto st_tag) {
        constexpr bool ST = decltype(st_tag)::value;
        auto gather = [&](int idx, float& w) -> VT {
          const int i = ib + idx;
          int cc;
          if (ST || in.a0v + i < in.endv) {
            cc = cs[i];
            w = vs[i];
          } else {
            cc = __ldg(g.col + in.a0v + i);
            w = __ldg(vals + in.a0v + i);
          }
          return V::load(X + (size_t)cc * ldx + c);
        };
        if (tys & kMsb) {
          // single-row tile: every nonzero belongs to row y_ws; lane gl takes every
          // L-th one, then the lanes' sums are added across the warp
          VT sum = V::zero();
#pragma unroll 1
          for (int base = gl; base < ntile; base += L * U1) {
            VT xv[U1];
            float wv[U1];
#pragma unroll
            for (int u = 0; u < U1; ++u) {
              xv[u] = V::zero();
              wv[u] = 0.f;
              if (base + u * L < ntile && c_ok) xv[u] = gather(base + u * L, wv[u]);
            }
#pragma unroll
            for (int u = 0; u < U1; ++u) V::fma(wv[u], xv[u], sum);
          }
#pragma unroll
          for (int o = T; o < 32; o <<= 1) V::add(sum, V::shfl_xor(sum, o));
          if (gl == 0) emit(y_ws, sum, true);
          return;
        }
        // lane walk (Sec. 4.2, k values wide): T passes of L lanes; each thread issues the
        // row-slice gathers of all its lane's right steps before using any (the step ->
        // nonzero map comes from the descriptor alone), then walks the steps: a down step
        // ends a row.  A lane's first ended row may have begun in earlier lanes, so its
        // head partial joins the runs flowing in; rows ended later in the lane are whole.
        VT carry = V::zero();                    // run open after the previous pass
        int open_row = y_ws;
#pragma unroll 1
        for (int p = 0; p < T; ++p) {
          const int l = p * L + gl;
          const uint32_t d = __shfl_sync(0xffffffffu, dreg, l);
          const int j = ti * kOmega + l;
          const bool active = j < g.lane_num;
          const int len = active ? min(g.sigma, g.steps - j * g.sigma) : 0;
          const uint32_t valid = (1u << len) - 1u;
          const uint32_t dm = (d >> 18) & valid;   // down steps
          const uint32_t rm = ~(d >> 18) & valid;  // right steps
          const int xo = (int)(d & 511u);
          const int y0 = active ? (int)((d >> 9) & 511u) : (g.n_rows - y_ws);
          // right step k takes the lane's nonzero k - (down steps before k); a batch of
          // HB steps has all its slices in flight before any is used (HB = sigma_max, or
          // half of it for 32-byte slices, which would not fit the registers)
          const uint32_t rk = c_ok ? rm : 0u;
          VT sum = V::zero(), head = V::zero();
          int ndk = 0;
#pragma unroll
          for (int k0 = 0; k0 < kSigmaMax; k0 += HB) {
            VT xv[HB];
            float wv[HB];
            int nd_b = ndk;
#pragma unroll
            for (int u = 0; u < HB; ++u) {
              const int k = k0 + u;
              xv[u] = V::zero();
              wv[u] = 0.f;
              if ((rk >> k) & 1u) xv[u] = gather(xo + k - nd_b, wv[u]);
              nd_b += (int)((dm >> k) & 1u);
            }
#pragma unroll
            for (int u = 0; u < HB; ++u) {
              const int k = k0 + u;
              V::fma(wv[u], xv[u], sum);         // zero at down steps and past the lane
              if ((dm >> k) & 1u) {
                if (ndk == 0) head = sum;
                else if (c_ok) epi.row(y_ws + y0 + ndk, c, sum);
                sum = V::zero();
                ++ndk;
              }
            }
          }
          // runs across the pass's lanes: OC_l = run open after lane l obeys
          // OC_l = a_l + b_l * OC_{l-1} (a_l = the lane's trailing sum, b_l = 1 when the
          // lane ends no row), with OC_{-1} = carry; scanned in log2(L) shuffle steps
          const bool hd = dm != 0u;
          VT A = sum;
          int B = hd ? 0 : 1;
          if (gl == 0) {
            if (B) V::add(A, carry);
            B = 0;
          }
#pragma unroll
          for (int dd = 1; dd < L; dd <<= 1) {
            const VT Ap = V::shfl_up(A, dd * T);
            const int Bp = __shfl_up_sync(0xffffffffu, B, dd * T);
            if (gl >= dd) {
              if (B) V::add(A, Ap);
              B &= Bp;
            }
          }
          const VT up = V::shfl_up(A, T);
          if (hd) {
            VT tot = head;
            V::add(tot, gl == 0 ? carry : up);
            emit(y_ws + y0, tot, false);
          }
          const int src = (L - 1) * T + (lane % T);
          carry = V::shfl(A, src);
          open_row = y_ws + __shfl_sync(0xffffffffu, y0 + __popc(dm), src);
        }
        if (gl == L - 1) emit(open_row, carry, true);
      };
      if (in.endv >= in.x_be) walk(std::integral_constant<bool, true>{});
      else walk(std::integral_constant<bool, false>{});
    }
    // arrival: this warp's reads of the stage and its table entries are done
    fence_proxy_async_smem();
    __syncwarp();
    int last = 0;
    if (lane == 0) {
      __threadfence_block();
      last = atomicAdd(&arrive[s], 1) == kWarps - 1;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence_block();
      // rows spread over several warps of the block (never a boundary row): the table's
      // first entry of each row adds up the row's entries
      for (int e = gl; e < NE; e += L) {
        const int r = wrow[e];
        if (r < 0 || !c_ok) continue;
        int prev = e - 1;
        while (prev >= 0 && wrow[prev] < 0) --prev;
        if (prev >= 0 && wrow[prev] == r) continue;      // not the first entry of its row
        float tot[VW];
#pragma unroll
        for (int q = 0; q < VW; ++q) tot[q] = 0.f;
        for (int q = e; q < NE; ++q) {
          const int rq = wrow[q];
          if (rq < 0) continue;
          if (rq != r) break;
#pragma unroll
          for (int u = 0; u < VW; ++u) tot[u] += wval[q][c + u];
        }
        epi.row(r, c, V::from(tot));
      }
      __syncwarp();
      if (lane == 0) {
        arrive[s] = 0;
        const int vn = v + S * G;
        if (vn < g.nb) {
          int xb, xe; uint32_t yb, ye;
          geom_of(vn, xb, xe, yb, ye);
          issue(s, xb, xe, yb, ye);
        }
      }
    }
    if (++s == S) {
      s = 0;
      par ^= 1u;
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
  const void* kp = reinterpret_cast<const void*>(kern);
  const size_t smem = kSpmmStages * stage_bytes<float>(p->sigma, kTilesPerBlock);
  const size_t smem_max = kSpmmStages * stage_bytes<float>(kSigmaMax, kTilesPerBlock);
  int grid = persistent_grid(kp, kThreads, smem, smem_max, p->num_sms);
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
